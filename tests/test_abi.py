"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, validates parameters, and builds the fractional weight matrices on the
host exactly as the FP64 oracle does (within the oracle's own rounding)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest
import torch

from oracle import lbm_oracle as O
from paper_1706_09161_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_1706_09161_gb300 import build
    build.build()
    from paper_1706_09161_gb300 import lbm
    return lbm


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for want in ("lbm_create", "lbm_step", "lbm_read_C", "lbm_mass", "lbm_destroy", "lbm_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.LIB_PATH)
    for name in _declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    for name in L.EXPORTED:
        assert name in _declared_symbols()


def test_strerror(L):
    assert L.lbm_strerror(0) == "ok"
    assert "instability" in L.lbm_strerror(L.LBM_ERR_UNSTABLE)


@pytest.mark.parametrize("side,alpha,p,g,dx", [(3, 1.5, 0.5, 1.0, 1.0), (17, 1.2, 0.3, 0.7, 0.25),
                                               (64, 1.7, 0.5, 1.0, 1.0), (101, 1.99, 0.9, 1.3, 0.02),
                                               (257, 1.05, 0.0, 1.0, 1.0), (40, 2.0, 0.4, 1.0, 1.0)])
def test_host_weight_matrix_matches_oracle(L, side, alpha, p, g, dx):
    pb = W.Problem(d=2, collision="mrt", grid=(side, 5), alpha=(alpha, 1.5), p=(p, 0.5), g=(g, 1.0),
                   D=((0.01, 0), (0, 0.01)), u=(0, 0), s_free=(1.0, 1.0), dx=dx)
    K = L.lbm_frac_matrix(L.params_from_problem(pb, "fp64"), 0)
    Ko = O.frac_matrix(alpha, p, g, side - 1, dx).numpy()
    # both sides are accurate to a few units in the last place of every entry (the oracle
    # through 40-digit differences, the library through the coefficients' binomial series)
    assert np.all(np.abs(K - Ko) <= 4e-15 * np.abs(Ko) + 1e-300)


def test_host_weight_matrix_bgk_diagonal_D(L):
    """BGK with non-spherical diagonal D: h_mu = D_mumu / max D scales g_mu (end of Section 2.2)."""
    pb = W.Problem(d=2, collision="bgk", grid=(9, 7), alpha=(1.5, 1.6), p=(0.5, 0.2), g=(1.0, 2.0),
                   D=((0.02, 0), (0, 0.005)), u=(0, 0))
    prm = L.params_from_problem(pb, "fp64")
    ops = O.Operators(pb)
    for mu in range(2):
        assert np.allclose(L.lbm_frac_matrix(prm, mu), ops.K[mu].numpy(), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("field,value", [("alpha", 1.0), ("alpha", 2.1), ("p", -0.1), ("p", 1.2), ("g", 0.0),
                                         ("dx", 0.0), ("grid", 2)])
def test_invalid_parameters_rejected(L, field, value):
    pb = W.Problem(d=2, collision="mrt", grid=(8, 8), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((0.01, 0), (0, 0.01)), u=(0, 0), s_free=(1.0, 1.0))
    prm = L.params_from_problem(pb, "fp32")
    if field in ("alpha", "p", "g"):
        getattr(prm, field)[0] = value
    elif field == "grid":
        prm.grid[0] = value
    else:
        setattr(prm, field, value)
    K = np.empty((8, 8))
    rc = L._lib.lbm_frac_matrix(ctypes.byref(prm), 0, K.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == L.LBM_EINVAL


def test_bgk_rejects_off_diagonal_D_and_mrt_rejects_non_spd(L):
    K = np.empty((8, 8))
    ptr = K.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    pb = W.Problem(d=2, collision="bgk", grid=(8, 8), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((0.01, 0.002), (0.002, 0.01)), u=(0, 0))
    assert L._lib.lbm_frac_matrix(ctypes.byref(L.params_from_problem(pb)), 0, ptr) == L.LBM_EINVAL
    pb = W.Problem(d=2, collision="mrt", grid=(8, 8), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((0.01, 0.5), (0.5, 0.01)), u=(0, 0), s_free=(1.0, 1.0))
    assert L._lib.lbm_frac_matrix(ctypes.byref(L.params_from_problem(pb)), 0, ptr) == L.LBM_EINVAL
    pb = W.Problem(d=2, collision="mrt", grid=(8, 8), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((0.01, 0.0), (0.0, 0.01)), u=(0, 0), s_free=(2.5, 1.0))
    assert L._lib.lbm_frac_matrix(ctypes.byref(L.params_from_problem(pb)), 0, ptr) == L.LBM_EINVAL


def test_digamma_closed_values_and_lgamma_slope(L):
    """psi(1) = -gamma_E, psi(2) = 1 - gamma_E, psi(1/2) = -gamma_E - 2 ln 2, and psi = (ln Gamma)'."""
    import math
    eg = 0.5772156649015329
    assert L.lbm_digamma(1.0) == pytest.approx(-eg, abs=1e-14)
    assert L.lbm_digamma(2.0) == pytest.approx(1 - eg, abs=1e-14)
    assert L.lbm_digamma(0.5) == pytest.approx(-eg - 2 * math.log(2.0), abs=1e-14)
    for x in (2.05, 2.5, 2.95, 7.3):
        h = 1e-5
        fd = (math.lgamma(x + h) - math.lgamma(x - h)) / (2 * h)
        assert L.lbm_digamma(x) == pytest.approx(fd, abs=1e-9)


@pytest.mark.parametrize("side,alpha,p,dx", [(9, 1.5, 0.3, 1.0), (40, 1.2, 0.7, 0.05), (257, 1.8, 0.5, 1.0)])
def test_host_weight_matrix_derivatives_match_oracle_autograd(L, side, alpha, p, dx):
    pb = W.Problem(d=2, collision="mrt", grid=(side, 5), alpha=(alpha, 1.5), p=(p, 0.5), g=(1.3, 1.0),
                   D=((0.01, 0), (0, 0.01)), u=(0, 0), s_free=(1.0, 1.0), dx=dx)
    da, dp = L.lbm_frac_matrix_grad(L.params_from_problem(pb, "fp64"), 0)
    a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    pp = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    K = O.frac_matrix(a, pp, 1.3, side - 1, dx)
    w = torch.tensor(np.random.default_rng(side).normal(size=(side, side)))
    (K * w).sum().backward()
    assert float((torch.tensor(da) * w).sum()) == pytest.approx(float(a.grad), rel=1e-9, abs=1e-12)
    assert float((torch.tensor(dp) * w).sum()) == pytest.approx(float(pp.grad), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("side,alpha,p,g,dx", [(3, 1.5, 0.5, 1.0, 1.0), (21, 1.7, 1.0, 1.0, 0.05),
                                               (64, 1.2, 0.3, 0.7, 0.25), (40, 2.0, 0.4, 1.0, 1.0)])
def test_host_caputo_matrix_and_derivatives_match_oracle(L, side, alpha, p, g, dx):
    """Section 3.5 variant: K~ = K - B (oracle's caputo_boundary_terms), its alpha and p
    derivatives against the oracle's autograd."""
    pb = W.Problem(d=2, collision="mrt", grid=(side, 5), alpha=(alpha, 1.5), p=(p, 0.5), g=(g, 1.0),
                   D=((0.01, 0), (0, 0.01)), u=(0, 0), s_free=(1.0, 1.0), dx=dx, variant="caputo")
    prm = L.params_from_problem(pb, "fp64")
    assert prm.variant == L.LBM_VARIANT_CAPUTO
    K = L.lbm_frac_matrix(prm, 0)
    a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    pp = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    Ko = O.frac_matrix(a, pp, g, side - 1, dx) - O.caputo_boundary_terms(a, pp, g, side - 1, dx)
    Kd = Ko.detach().numpy()
    # columns 0 and N subtract the boundary terms, so their entries may cancel: bound them
    # by the terms' size
    assert np.max(np.abs(K - Kd)) <= 4e-15 * np.max(np.abs(Kd))
    assert np.max(np.abs(K.sum(axis=1))) < 1e-12 * np.max(np.abs(K))  # constants map to 0
    if alpha < 2.0:  # x^gamma is not differentiable in gamma at gamma = 0, x = 0
        da, dp = L.lbm_frac_matrix_grad(prm, 0)
        w = torch.tensor(np.random.default_rng(side).normal(size=(side, side)))
        (Ko * w).sum().backward()
        assert float((torch.tensor(da) * w).sum()) == pytest.approx(float(a.grad), rel=1e-9, abs=1e-12)
        assert float((torch.tensor(dp) * w).sum()) == pytest.approx(float(pp.grad), rel=1e-9, abs=1e-12)


def test_unknown_variant_rejected(L):
    pb = W.Problem(d=2, collision="mrt", grid=(8, 8), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((0.01, 0), (0, 0.01)), u=(0, 0), s_free=(1.0, 1.0))
    prm = L.params_from_problem(pb, "fp64")
    prm.variant = 2
    with pytest.raises(L.LBMError):
        L.lbm_frac_matrix(prm, 0)


def test_allocator_hooks_come_in_pairs(L):
    """lbm_set_allocator: both hooks or neither (host-side check, no GPU call)."""
    with pytest.raises(L.LBMError):
        L.lbm_set_allocator(lambda n, s, c: None, None)
    with pytest.raises(L.LBMError):
        L.lbm_set_allocator(None, lambda p, c: None)
    L.lbm_set_allocator(None, None)  # restores cudaMalloc / cudaFree


def test_wait_check_validates_its_limit(L):
    """lbm_wait_check rejects limits outside [1 us, 1 s] before touching a GPU."""
    assert L.lbm_wait_check(False, 0) == L.LBM_EINVAL
    assert L.lbm_wait_check(True, -5) == L.LBM_EINVAL
    assert L.lbm_wait_check(False, 1000001) == L.LBM_EINVAL
