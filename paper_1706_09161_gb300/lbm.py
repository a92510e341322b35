"""ctypes binding of liblbm_fade.so (C ABI declared in include/lbm_fade.h).

Argument marshalling only: every step of the scheme runs in the library's CUDA
kernels.  The functions keep the C names (``lbm_create``, ``lbm_step``, ...);
``Lattice`` wraps a handle for convenience.  There is no CPU fallback: if the
library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm_fade.so")

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_ERR_UNSTABLE = -4
LBM_ENOTSUP = -5
LBM_ERR_TIMEOUT = -6
LBM_ETOOBIG = -7

LBM_D2Q5, LBM_D3Q7 = 0, 1
LBM_BGK, LBM_MRT = 0, 1
LBM_FP64, LBM_FP32, LBM_FP32_BF16SPLIT, LBM_FP32_TF32SPLIT, LBM_FP32_BF16SPLIT5, LBM_FP32_BF16SPLIT6 = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "bf16split": LBM_FP32_BF16SPLIT, "tf32split": LBM_FP32_TF32SPLIT,
              "bf16x5split": LBM_FP32_BF16SPLIT5, "bf16x6split": LBM_FP32_BF16SPLIT6}
LBM_VARIANT_FG, LBM_VARIANT_CAPUTO = 0, 1
VARIANTS = {"fg": LBM_VARIANT_FG, "caputo": LBM_VARIANT_CAPUTO}


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("grid", ctypes.c_int * 3),
        ("alpha", ctypes.c_double * 3),
        ("p", ctypes.c_double * 3),
        ("g", ctypes.c_double * 3),
        ("D", ctypes.c_double * 9),
        ("u", ctypes.c_double * 3),
        ("s_free", ctypes.c_double * 3),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("C_wall", ctypes.c_double),
        ("variant", ctypes.c_int),
    ]


class lbm_walk_params(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("alpha", ctypes.c_double * 3),
        ("p", ctypes.c_double * 3),
        ("D", ctypes.c_double * 3),
        ("g", ctypes.c_double * 3),
        ("u", ctypes.c_double * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_ulonglong),
    ]


class LBMError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = f"{where}: {lbm_strerror(code)} ({code})"
        if code == LBM_ECUDA or code == LBM_ENOMEM:
            msg += f" [{lbm_last_cuda_error()}]"
        super().__init__(msg)
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1706_09161_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    sig = {
        "lbm_create": (ctypes.c_int, [P(lbm_params), dp, P(vp), vp]),
        "lbm_create_batch": (ctypes.c_int, [ctypes.c_int, P(lbm_params), P(dp), P(vp), vp]),
        "lbm_batch_size": (ctypes.c_int, [vp, P(ctypes.c_int)]),
        "lbm_batch_set_C": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lbm_set_C": (ctypes.c_int, [vp, dp]),
        "lbm_reset": (ctypes.c_int, [vp]),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_profile": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lbm_read_C": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
        "lbm_read_F": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lbm_read_f": (ctypes.c_int, [vp, dp]),
        "lbm_write_f": (ctypes.c_int, [vp, dp]),
        "lbm_state_size": (ctypes.c_longlong, [vp]),
        "lbm_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]),
        "lbm_configure": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lbm_save": (ctypes.c_int, [vp, vp, ctypes.c_longlong]),
        "lbm_load": (ctypes.c_int, [vp, vp, ctypes.c_longlong]),
        "lbm_mass": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lbm_set_mass_limit": (ctypes.c_int, [vp, ctypes.c_double]),
        "lbm_set_fields": (ctypes.c_int, [vp, dp, dp, dp]),
        "lbm_set_source": (ctypes.c_int, [vp, dp, ctypes.c_double]),
        "lbm_set_wall_values": (ctypes.c_int, [vp, dp, ctypes.c_double]),
        "lbm_set_params": (ctypes.c_int, [vp, P(lbm_params)]),
        "lbm_walk": (ctypes.c_int, [P(lbm_walk_params), ctypes.c_longlong, vp, vp, ctypes.c_longlong, ctypes.c_int,
                                    vp]),
        "lbm_walk_density": (ctypes.c_int, [P(lbm_walk_params), ctypes.c_longlong, vp, vp, P(ctypes.c_int),
                                            ctypes.c_double, vp, vp]),
        "lbm_sync": (ctypes.c_int, [vp]),
        "lbm_get_stream": (ctypes.c_int, [vp, P(vp)]),
        "lbm_launches_per_step": (ctypes.c_int, [vp, P(ctypes.c_int)]),
        "lbm_wait_check": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp]),
        "lbm_set_allocator": (ctypes.c_int, [vp, vp, vp]),
        "lbm_frac_matrix": (ctypes.c_int, [P(lbm_params), ctypes.c_int, dp]),
        "lbm_grad": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int), dp, ctypes.c_int, dp, dp]),
        "lbm_frac_matrix_grad": (ctypes.c_int, [P(lbm_params), ctypes.c_int, dp, dp]),
        "lbm_digamma": (ctypes.c_double, [ctypes.c_double]),
        "lbm_mass_static": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_longlong, vp, vp]),
        "lbm_destroy": (None, [vp]),
        "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_last_cuda_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

# Declared C entry points, re-exported under their own names.
EXPORTED = ("lbm_create", "lbm_create_batch", "lbm_batch_size", "lbm_batch_set_C", "lbm_set_C", "lbm_reset", "lbm_step", "lbm_profile", "lbm_read_C", "lbm_read_F", "lbm_read_f", "lbm_write_f", "lbm_state_size", "lbm_save", "lbm_load", "lbm_autotune", "lbm_configure",
            "lbm_mass", "lbm_set_mass_limit", "lbm_set_fields", "lbm_set_source", "lbm_set_wall_values",
            "lbm_walk", "lbm_walk_density", "lbm_sync", "lbm_get_stream", "lbm_launches_per_step", "lbm_wait_check", "lbm_set_allocator",
            "lbm_frac_matrix",
            "lbm_grad", "lbm_frac_matrix_grad", "lbm_digamma", "lbm_mass_static", "lbm_destroy", "lbm_strerror", "lbm_last_cuda_error")


def lbm_strerror(code: int) -> str:
    return _lib.lbm_strerror(int(code)).decode()


def lbm_last_cuda_error() -> str:
    return _lib.lbm_last_cuda_error().decode()


def _check(code: int, where: str) -> None:
    if code != LBM_OK:
        raise LBMError(code, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params_from_problem(pb, precision: str = "fp32") -> lbm_params:
    """Fill lbm_params from a workloads.Problem (or any object with the same attributes)."""
    prm = lbm_params()
    d = int(pb.d)
    prm.lattice = LBM_D2Q5 if d == 2 else LBM_D3Q7
    prm.collision = LBM_BGK if pb.collision == "bgk" else LBM_MRT
    prm.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for mu in range(3):
        prm.grid[mu] = int(pb.grid[mu]) if mu < d else 1
        prm.alpha[mu] = float(pb.alpha[mu]) if mu < d else 2.0
        prm.p[mu] = float(pb.p[mu]) if mu < d else 0.5
        prm.g[mu] = float(pb.g[mu]) if mu < d else 1.0
        prm.u[mu] = float(pb.u[mu]) if mu < d else 0.0
    for i in range(d):
        for j in range(d):
            prm.D[3 * i + j] = float(pb.D[i][j])
    for k, s in enumerate(getattr(pb, "s_free", ()) or ()):
        prm.s_free[k] = float(s)
    prm.dx = float(getattr(pb, "dx", 1.0))
    prm.dt = float(getattr(pb, "dt", 1.0))
    prm.C_wall = float(getattr(pb, "C_wall", 0.0))
    prm.variant = VARIANTS[getattr(pb, "variant", "fg")]
    return prm


def lbm_create(prm: lbm_params, C0: np.ndarray, stream: Optional[int] = None) -> int:
    C0 = np.ascontiguousarray(C0, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(_lib.lbm_create(ctypes.byref(prm), _dptr(C0), ctypes.byref(h), ctypes.c_void_p(stream or 0)),
           "lbm_create")
    return h.value


def lbm_create_batch(prms, C0s, stream: Optional[int] = None) -> int:
    n = len(prms)
    arr = (lbm_params * n)(*prms)
    fields = [np.ascontiguousarray(c, dtype=np.float64) for c in C0s]
    ptrs = (ctypes.POINTER(ctypes.c_double) * n)(*[_dptr(f) for f in fields])
    h = ctypes.c_void_p()
    _check(_lib.lbm_create_batch(n, arr, ptrs, ctypes.byref(h), ctypes.c_void_p(stream or 0)), "lbm_create_batch")
    return h.value


def lbm_batch_size(h: int) -> int:
    n = ctypes.c_int()
    _check(_lib.lbm_batch_size(ctypes.c_void_p(h), ctypes.byref(n)), "lbm_batch_size")
    return n.value


def lbm_batch_set_C(h: int, prob: int, C: np.ndarray) -> None:
    C = np.ascontiguousarray(C, dtype=np.float64)
    _check(_lib.lbm_batch_set_C(ctypes.c_void_p(h), int(prob), _dptr(C)), "lbm_batch_set_C")


def lbm_set_C(h: int, C: np.ndarray) -> None:
    C = np.ascontiguousarray(C, dtype=np.float64)
    _check(_lib.lbm_set_C(ctypes.c_void_p(h), _dptr(C)), "lbm_set_C")


def lbm_reset(h: int) -> None:
    _check(_lib.lbm_reset(ctypes.c_void_p(h)), "lbm_reset")


def lbm_profile(h: int, nsteps: int):
    ms = (ctypes.c_double * 2)()
    _check(_lib.lbm_profile(ctypes.c_void_p(h), int(nsteps), ms), "lbm_profile")
    return float(ms[0]), float(ms[1])


def lbm_step(h: int, nsteps: int) -> None:
    _check(_lib.lbm_step(ctypes.c_void_p(h), int(nsteps)), "lbm_step")


def lbm_read_C(h: int, prob: int, out: np.ndarray) -> np.ndarray:
    """Concentration of problem `prob` into a host float64 array."""
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(_lib.lbm_read_C(ctypes.c_void_p(h), int(prob), out.ctypes.data_as(ctypes.c_void_p), 0), "lbm_read_C")
    return out


def lbm_read_C_device(h: int, prob: int, dst_ptr: int) -> None:
    """Concentration of problem `prob` into a caller-owned device float64 array (by address)."""
    _check(_lib.lbm_read_C(ctypes.c_void_p(h), int(prob), ctypes.c_void_p(dst_ptr), 1), "lbm_read_C")


def lbm_read_F(h: int, mu: int, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(_lib.lbm_read_F(ctypes.c_void_p(h), int(mu), _dptr(out)), "lbm_read_F")
    return out


def lbm_read_f(h: int, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(_lib.lbm_read_f(ctypes.c_void_p(h), _dptr(out)), "lbm_read_f")
    return out


def lbm_autotune(h: int, nsteps: int = 64) -> str:
    """Pick the fastest launch configuration for this handle; returns its description."""
    buf = ctypes.create_string_buffer(256)
    _check(_lib.lbm_autotune(ctypes.c_void_p(h), int(nsteps), buf, len(buf)), "lbm_autotune")
    return buf.value.decode()


def lbm_configure(h: int, bn: int = 0, ks: int = 0, persist: int = 0, chunk: int = 0, fused: int = 0) -> None:
    _check(_lib.lbm_configure(ctypes.c_void_p(h), int(bn), int(ks), int(persist), int(chunk), int(fused)),
           "lbm_configure")


def lbm_state_size(h: int) -> int:
    n = int(_lib.lbm_state_size(ctypes.c_void_p(h)))
    _check(n if n < 0 else 0, "lbm_state_size")
    return n


def lbm_save(h: int) -> np.ndarray:
    """The handle's state (header + populations in the working precision) as bytes."""
    buf = np.empty(lbm_state_size(h), dtype=np.uint8)
    _check(_lib.lbm_save(ctypes.c_void_p(h), buf.ctypes.data_as(ctypes.c_void_p), buf.size), "lbm_save")
    return buf


def lbm_load(h: int, state: np.ndarray) -> None:
    state = np.ascontiguousarray(state, dtype=np.uint8)
    _check(_lib.lbm_load(ctypes.c_void_p(h), state.ctypes.data_as(ctypes.c_void_p), state.size), "lbm_load")


def lbm_write_f(h: int, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(_lib.lbm_write_f(ctypes.c_void_p(h), _dptr(f)), "lbm_write_f")


def lbm_mass(h: int, prob: int = 0) -> float:
    m = ctypes.c_double()
    _check(_lib.lbm_mass(ctypes.c_void_p(h), int(prob), ctypes.byref(m)), "lbm_mass")
    return m.value


def lbm_set_mass_limit(h: int, limit: float) -> None:
    _check(_lib.lbm_set_mass_limit(ctypes.c_void_p(h), float(limit)), "lbm_set_mass_limit")


def lbm_set_fields(h: int, D=None, g=None, u=None) -> None:
    """Spatially varying D(x) (d, d, *shape), g(x) (d, *shape), u(x) (d, *shape); None keeps
    the constant value (all None: constant coefficients again)."""
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (D, g, u)]
    ptrs = [None if a is None else _dptr(a) for a in arrs]
    _check(_lib.lbm_set_fields(ctypes.c_void_p(h), *ptrs), "lbm_set_fields")


def lbm_set_source(h: int, S=None, rate: float = 0.0) -> None:
    """S_c(x, t) = S(x) exp(rate t) (S in the field layout; None removes the source)."""
    a = None if S is None else np.ascontiguousarray(S, dtype=np.float64)
    _check(_lib.lbm_set_source(ctypes.c_void_p(h), None if a is None else _dptr(a), float(rate)), "lbm_set_source")


def lbm_set_wall_values(h: int, Cw=None, rate: float = 0.0) -> None:
    """Wall values C_w(x) exp(rate t) (field layout; None: the constant C_wall)."""
    a = None if Cw is None else np.ascontiguousarray(Cw, dtype=np.float64)
    _check(_lib.lbm_set_wall_values(ctypes.c_void_p(h), None if a is None else _dptr(a), float(rate)),
           "lbm_set_wall_values")


def lbm_set_params(h: int, prm: lbm_params) -> None:
    """New constant parameters for the handle (same lattice, collision, precision, grid, variant)."""
    _check(_lib.lbm_set_params(ctypes.c_void_p(h), ctypes.byref(prm)), "lbm_set_params")


def walk_params(d: int, alpha, p, D, g, u, lo, hi, dt: float, seed: int, precision: str = "fp32") -> lbm_walk_params:
    prm = lbm_walk_params()
    prm.d = int(d)
    prm.precision = PRECISIONS[precision]
    for mu in range(3):
        ok = mu < d
        prm.alpha[mu] = float(alpha[mu]) if ok else 2.0
        prm.p[mu] = float(p[mu]) if ok else 0.5
        prm.D[mu] = float(D[mu]) if ok else 1.0
        prm.g[mu] = float(g[mu]) if ok else 1.0
        prm.u[mu] = float(u[mu]) if ok else 0.0
        prm.lo[mu] = float(lo[mu]) if ok else 0.0
        prm.hi[mu] = float(hi[mu]) if ok else 1.0
    prm.dt = float(dt)
    prm.seed = int(seed)
    return prm


def lbm_walk(prm: lbm_walk_params, n: int, X_ptr: int, alive_ptr: int, step0: int, nsteps: int,
             stream: Optional[int] = None) -> None:
    """Advance n paths (device arrays by address: X [d][n] float64, alive uint8) by nsteps."""
    _check(_lib.lbm_walk(ctypes.byref(prm), int(n), ctypes.c_void_p(X_ptr), ctypes.c_void_p(alive_ptr), int(step0),
                         int(nsteps), ctypes.c_void_p(stream or 0)), "lbm_walk")


def lbm_walk_density(prm: lbm_walk_params, n: int, X_ptr: int, alive_ptr: int, grid, dx: float, counts_ptr: int,
                     stream: Optional[int] = None) -> None:
    g = (ctypes.c_int * 3)(*[int(v) for v in list(grid) + [1] * (3 - len(grid))])
    _check(_lib.lbm_walk_density(ctypes.byref(prm), int(n), ctypes.c_void_p(X_ptr), ctypes.c_void_p(alive_ptr), g,
                                 float(dx), ctypes.c_void_p(counts_ptr), ctypes.c_void_p(stream or 0)),
           "lbm_walk_density")


def lbm_sync(h: int) -> int:
    return int(_lib.lbm_sync(ctypes.c_void_p(h)))


def lbm_get_stream(h: int) -> int:
    s = ctypes.c_void_p()
    _check(_lib.lbm_get_stream(ctypes.c_void_p(h), ctypes.byref(s)), "lbm_get_stream")
    return s.value or 0


def lbm_launches_per_step(h: int) -> int:
    n = ctypes.c_int()
    _check(_lib.lbm_launches_per_step(ctypes.c_void_p(h), ctypes.byref(n)), "lbm_launches_per_step")
    return n.value


def lbm_frac_matrix(prm: lbm_params, mu: int) -> np.ndarray:
    side = prm.grid[mu]
    K = np.empty((side, side), dtype=np.float64)
    _check(_lib.lbm_frac_matrix(ctypes.byref(prm), int(mu), _dptr(K)), "lbm_frac_matrix")
    return K


def lbm_mass_static(x_dev: int, elem_bytes: int, n: int, sum_dev: int, stream: Optional[int] = None) -> int:
    """Return code of the static-scratch FP64 sum (the result lands in *sum_dev)."""
    return int(_lib.lbm_mass_static(ctypes.c_void_p(x_dev), int(elem_bytes), int(n), ctypes.c_void_p(sum_dev),
                                     ctypes.c_void_p(stream or 0)))


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_hook_refs = []  # callbacks stay alive for the handles created with them


def lbm_set_allocator(alloc, release, ctx: Optional[int] = None) -> None:
    """Install device-memory hooks (ctypes callbacks of the C signatures) for handles
    created from now on; (None, None) restores cudaMalloc/cudaFree."""
    alloc = _ALLOC_FN(alloc) if alloc is not None else None
    release = _FREE_FN(release) if release is not None else None
    _hook_refs.append((alloc, release))
    a = ctypes.cast(alloc, ctypes.c_void_p) if alloc is not None else None
    r = ctypes.cast(release, ctypes.c_void_p) if release is not None else None
    _check(_lib.lbm_set_allocator(a, r, ctypes.c_void_p(ctx or 0)), "lbm_set_allocator")


def use_torch_allocator(on: bool = True) -> None:
    """Handles created from now on take their device memory from PyTorch's caching
    allocator (on the handle's stream) and give it back there; off: cudaMalloc again."""
    if not on:
        lbm_set_allocator(None, None)
        return
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:  # out of memory: the library reports LBM_ENOMEM
            return None

    def release(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    lbm_set_allocator(alloc, release)


def lbm_wait_check(complete: bool, limit_us: int, stream: Optional[int] = None) -> int:
    """Return code of one bounded device-side wait on a barrier completed (LBM_OK) or
    left incomplete (LBM_ERR_TIMEOUT after limit_us microseconds)."""
    return int(_lib.lbm_wait_check(1 if complete else 0, int(limit_us), ctypes.c_void_p(stream or 0)))


def lbm_grad(h: int, snap_steps, obs: np.ndarray, ckpt_every: int, d: int):
    """(loss, grad[4d]) of the snapshot misfit; grad = dL/d[alpha, p, D_diag, u]."""
    snaps = (ctypes.c_int * len(snap_steps))(*[int(t) for t in snap_steps])
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    loss = ctypes.c_double()
    grad = np.zeros(4 * d, dtype=np.float64)
    _check(_lib.lbm_grad(ctypes.c_void_p(h), len(snap_steps), snaps, _dptr(obs), int(ckpt_every), ctypes.byref(loss),
                         _dptr(grad)), "lbm_grad")
    return loss.value, grad


def lbm_frac_matrix_grad(prm: lbm_params, mu: int):
    side = prm.grid[mu]
    da = np.empty((side, side), dtype=np.float64)
    dp_ = np.empty((side, side), dtype=np.float64)
    _check(_lib.lbm_frac_matrix_grad(ctypes.byref(prm), int(mu), _dptr(da), _dptr(dp_)), "lbm_frac_matrix_grad")
    return da, dp_


def lbm_digamma(x: float) -> float:
    return float(_lib.lbm_digamma(float(x)))


def lbm_destroy(h: int) -> None:
    _lib.lbm_destroy(ctypes.c_void_p(h))


class Lattice:
    """One FADE lattice Boltzmann problem on the GPU (owns an lbm_t handle)."""

    def __init__(self, pb, C0: np.ndarray, precision: str = "fp32", stream: Optional[int] = None):
        self.problem = pb
        self.shape = tuple(reversed(tuple(int(n) for n in pb.grid)))
        self.d = int(pb.d)
        self.Q = 2 * self.d + 1
        self.prm = params_from_problem(pb, precision)
        self.h = lbm_create(self.prm, C0, stream)

    def close(self) -> None:
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_C(self, C: np.ndarray) -> None:
        lbm_set_C(self.h, C)

    def set_params(self, pb) -> None:
        """New constant parameters from a problem of the same lattice, collision and grid;
        re-initialises from the initial concentration."""
        prm = params_from_problem(pb, self.prm.precision)
        lbm_set_params(self.h, prm)
        self.problem, self.prm = pb, prm

    def reset(self) -> None:
        lbm_reset(self.h)

    def step(self, n: int = 1) -> None:
        lbm_step(self.h, n)

    def profile(self, n: int):
        """(ms fractional operator, ms collide-stream) summed over n one-kernel-launch steps."""
        return lbm_profile(self.h, n)

    def C(self) -> np.ndarray:
        return lbm_read_C(self.h, 0, np.empty(self.shape, dtype=np.float64))

    def C_into(self, out) -> None:
        """Concentration into a CUDA float64 tensor of the field's shape (no host round trip)."""
        assert out.is_cuda and out.dtype.is_floating_point and out.element_size() == 8 and out.is_contiguous()
        assert tuple(out.shape) == self.shape
        lbm_read_C_device(self.h, 0, out.data_ptr())

    def F(self, mu: int) -> np.ndarray:
        return lbm_read_F(self.h, mu, np.empty(self.shape, dtype=np.float64))

    def f(self) -> np.ndarray:
        return lbm_read_f(self.h, np.empty((self.Q,) + self.shape, dtype=np.float64))

    def write_f(self, f: np.ndarray) -> None:
        lbm_write_f(self.h, f)

    def autotune(self, nsteps: int = 64) -> str:
        """Time the candidate launch configurations on this problem and keep the fastest."""
        return lbm_autotune(self.h, nsteps)

    def configure(self, bn: int = 0, ks: int = 0, persist: int = 0, chunk: int = 0, fused: int = 0) -> None:
        """Apply a launch configuration (operator tile width / split / persistent, chunk, fused step)."""
        lbm_configure(self.h, bn, ks, persist, chunk, fused)

    def save(self) -> np.ndarray:
        """Checkpoint: the populations, bit for bit, behind a header (lbm_save)."""
        return lbm_save(self.h)

    def load(self, state: np.ndarray) -> None:
        """Resume from a checkpoint of a handle with the same lattice, precision and grid."""
        lbm_load(self.h, state)

    def mass(self) -> float:
        return lbm_mass(self.h, 0)

    def set_fields(self, D=None, g=None, u=None) -> None:
        """Coefficients varying in space (arrays in the field layout with a leading axis per
        component); re-initialises from the initial concentration."""
        lbm_set_fields(self.h, D, g, u)

    def set_source(self, S=None, rate: float = 0.0) -> None:
        """Source S_c(x, t) = S(x) exp(rate t); re-initialises (time 0)."""
        lbm_set_source(self.h, S, rate)

    def set_wall_values(self, Cw=None, rate: float = 0.0) -> None:
        """Wall values C_w(x) exp(rate t); re-initialises (time 0)."""
        lbm_set_wall_values(self.h, Cw, rate)

    def set_mass_limit(self, limit: float) -> None:
        """Latch LBM_ERR_UNSTABLE at the next synchronising call if |mass| > limit (0: off)."""
        lbm_set_mass_limit(self.h, limit)

    def sync(self) -> None:
        _check(lbm_sync(self.h), "lbm_sync")

    def grad(self, snap_steps, obs: np.ndarray, ckpt_every: int = 100):
        """(loss, dL/d[alpha, p, D_diag, u]) of sum_k |C(t_k) - obs_k|^2 via the discrete adjoint."""
        return lbm_grad(self.h, snap_steps, obs, ckpt_every, self.d)

    @property
    def stream(self) -> int:
        return lbm_get_stream(self.h)

    @property
    def launches_per_step(self) -> int:
        return lbm_launches_per_step(self.h)


class Batch:
    """Independent problems advanced together by grouped launches (owns an lbm_t handle)."""

    def __init__(self, problems, fields, precision: str = "bf16split", stream: Optional[int] = None):
        self.problems = list(problems)
        self.shapes = [tuple(reversed(tuple(int(n) for n in pb.grid))) for pb in self.problems]
        self.h = lbm_create_batch([params_from_problem(pb, precision) for pb in self.problems], fields, stream)

    def close(self) -> None:
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self) -> int:
        return lbm_batch_size(self.h)

    def step(self, n: int = 1) -> None:
        lbm_step(self.h, n)

    def reset(self) -> None:
        lbm_reset(self.h)

    def C(self, prob: int) -> np.ndarray:
        return lbm_read_C(self.h, prob, np.empty(self.shapes[prob], dtype=np.float64))

    def C_into(self, prob: int, out) -> None:
        """Concentration of problem `prob` into a CUDA float64 tensor of its shape."""
        assert out.is_cuda and out.element_size() == 8 and out.is_contiguous()
        assert tuple(out.shape) == self.shapes[prob]
        lbm_read_C_device(self.h, prob, out.data_ptr())

    def set_C(self, prob: int, C: np.ndarray) -> None:
        lbm_batch_set_C(self.h, prob, C)

    def mass(self, prob: int) -> float:
        return lbm_mass(self.h, prob)

    def autotune(self, nsteps: int = 64) -> str:
        """Time the candidate tile rows per collide-stream block and keep the fastest."""
        return lbm_autotune(self.h, nsteps)

    def save(self) -> np.ndarray:
        """Checkpoint of every problem's populations (lbm_save)."""
        return lbm_save(self.h)

    def load(self, state: np.ndarray) -> None:
        lbm_load(self.h, state)

    def sync(self) -> None:
        _check(lbm_sync(self.h), "lbm_sync")

    def profile(self, n: int):
        return lbm_profile(self.h, n)

    @property
    def stream(self) -> int:
        return lbm_get_stream(self.h)

    @property
    def launches_per_step(self) -> int:
        return lbm_launches_per_step(self.h)


def _problem_with_theta(problem, theta):
    """Copy of `problem` whose alpha, p, diagonal D and u are taken from theta (4d values)."""
    import dataclasses
    d = int(problem.d)
    th = [float(v) for v in theta]
    D = [list(row) for row in problem.D]
    for i in range(d):
        D[i][i] = th[2 * d + i]
    return dataclasses.replace(problem, alpha=tuple(th[:d]), p=tuple(th[d:2 * d]),
                               D=tuple(tuple(r) for r in D), u=tuple(th[3 * d:4 * d]))


def snapshot_loss(problem, C0, snap_steps, obs, theta, precision: str = "fp32", ckpt_every: int = 100,
                  lattice: Optional["Lattice"] = None):
    """Differentiable L(theta) = sum_k |C(t_k) - obs_k|^2, theta = [alpha, p, D_diag, u] (torch tensor).

    Forward and gradient are one lbm_grad call (discrete adjoint on the GPU); backward
    returns the stored gradient scaled by the incoming one.  With `lattice` (a Lattice of
    this problem and C0) the handle is reused across calls (lbm_set_params); otherwise each
    call builds a handle with the current parameters.
    """
    import torch

    class _SnapshotLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            pb = _problem_with_theta(problem, th.detach().cpu().tolist())
            if lattice is not None:
                lattice.set_params(pb)
                loss, grad = lattice.grad(snap_steps, obs, ckpt_every)
            else:
                with Lattice(pb, C0, precision) as lat:
                    loss, grad = lat.grad(snap_steps, obs, ckpt_every)
            ctx.save_for_backward(torch.as_tensor(grad, dtype=th.dtype, device=th.device))
            return th.new_tensor(loss)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad

    return _SnapshotLoss.apply(theta)
