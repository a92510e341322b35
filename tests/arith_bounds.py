"""Error bounds derived from the arithmetic of each precision form.

The scheme is re-run on the CPU with the oracle's own stage functions, on
float32 tensors, with the fractional operator's operands rounded exactly as a
precision form rounds them (none; bf16 or tf32 hi+lo with three products, lo*lo
dropped; bf16 with the weights in three parts and C in two, five products, or
both in three parts, six products).  Its distance to the FP64 oracle is the error that arithmetic
itself makes on the problem; the GPU result must stay within a small multiple
of it, both as a relative L2 over all nodes and node by node (max |error| over
max |C|).  No GPU code is involved.
"""
import numpy as np
import torch

from oracle import lbm_oracle as O


def _round_tf32(x: torch.Tensor) -> torch.Tensor:
    """Round float32 to tf32 (10 explicit mantissa bits), ties away from zero."""
    b = x.float().contiguous().view(torch.int32)
    b = (b + 0x1000) & ~0x1FFF
    return b.view(torch.float32)


def _split(x: torch.Tensor, kind: str):
    x = x.float()
    if kind == "bf16split":
        hi = x.to(torch.bfloat16).float()
        lo = (x - hi).to(torch.bfloat16).float()
    else:
        hi = _round_tf32(x)
        lo = _round_tf32(x - hi)
    return hi, lo


def _bf16_parts(x: torch.Tensor, n: int):
    """x = p1 + p2 + ... + pn + rest, each part the bf16 rounding of what the previous left."""
    parts, r = [], x.float()
    for _ in range(n):
        p = r.to(torch.bfloat16).float()
        parts.append(p)
        r = r - p
    return parts


def _frac(K, C, mu, kind):
    if kind in ("fp32", None):
        return O.apply_along_axis(K, C, mu)
    if kind == "bf16x5split":
        k1, k2, k3 = _bf16_parts(K, 3)
        c1, c2 = _bf16_parts(C, 2)
        terms = [(k1, c1), (k1, c2), (k2, c1), (k2, c2), (k3, c1)]
        return sum(O.apply_along_axis(k, c, mu) for k, c in terms)
    if kind == "bf16x6split":
        k1, k2, k3 = _bf16_parts(K, 3)
        c1, c2, c3 = _bf16_parts(C, 3)
        terms = [(k1, c1), (k1, c2), (k2, c1), (k1, c3), (k2, c2), (k3, c1)]
        return sum(O.apply_along_axis(k, c, mu) for k, c in terms)
    Kh, Kl = _split(K, kind)
    Ch, Cl = _split(C, kind)
    return (O.apply_along_axis(Kh, Ch, mu) + O.apply_along_axis(Kh, Cl, mu) + O.apply_along_axis(Kl, Ch, mu))


def rerun(pb, C0, n, kind="fp32", fields=None):
    """Concentration after n steps with FP32 collision and the given operator rounding
    (with coefficients varying in space when `fields` is given, as the oracle takes them)."""
    ops = O.Operators(pb, fields=fields)
    Om = ops.Omega.float()
    K = [k.float() for k in ops.K]
    ops.w, ops.e, ops.u = ops.w.float(), ops.e.float(), ops.u.float()
    gf = None
    if fields:
        ops.ufield = ops.ufield.float()
        gf = ops.gfield.float()

    def frac(C):
        return [_frac(K[mu], C if gf is None else gf[mu] * C, mu, kind) for mu in range(pb.d)]

    eq = "ij...,j...->i..." if Om.dim() > 2 else "ij,j...->i..."
    C = torch.tensor(C0).float()
    f = O.equilibrium(ops, C, frac(C))
    C = f.sum(0)
    unknown = O.unknown_mask(ops)
    k = unknown.sum(0).float().clamp(min=1.0)
    for _ in range(n):
        C = f.sum(0)
        feq = O.equilibrium(ops, C, frac(C))
        fn = O.stream(ops, f - torch.einsum(eq, Om, f - feq))
        known = torch.where(unknown, torch.zeros(()), fn).sum(0)
        f = torch.where(unknown, ((float(pb.C_wall) - known) / k).unsqueeze(0).expand_as(fn), fn)
    return f.sum(0).double().numpy()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def node_err(a, b):
    """Largest error at any node, relative to the largest |value|: max|a - b| / max|b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def bound(pb, C0, n, kind="fp32", factor=10.0, floor=1e-5):
    """max(floor, factor x the error the form's arithmetic makes on this problem)."""
    ref = O.run_C(pb, C0, n).numpy()
    return max(floor, factor * rel_l2(rerun(pb, C0, n, kind), ref))


def bounds(pb, C0, n, kind="fp32", factor=6.0, floor=1e-5, C_ref=None, fields=None):
    """(relative-L2 bound, per-node bound) for the form `kind` on this problem: `factor`
    x the errors the form's own arithmetic makes when re-run on the CPU (relative L2 and
    max|C - C_ref| / max|C_ref|), never below `floor`; and the oracle's C."""
    if C_ref is not None:
        ref = C_ref
    else:
        ref = (O.run_fields_C(pb, C0, n, fields) if fields else O.run_C(pb, C0, n)).numpy()
    cpu = rerun(pb, C0, n, kind, fields)
    return (max(floor, factor * rel_l2(cpu, ref)), max(floor, factor * node_err(cpu, ref)), ref)


def assert_close(C, C_ref, l2_tol, node_tol, what=""):
    """Whole-field relative L2 AND every node (walls, corners, tile seams included):
    max|C - C_ref| <= node_tol x max|C_ref|."""
    e2, en = rel_l2(C, C_ref), node_err(C, C_ref)
    assert e2 < l2_tol, f"{what}: relative L2 {e2:.3e} >= {l2_tol:.3e}"
    assert en < node_tol, f"{what}: node error {en:.3e} (of max |C|) >= {node_tol:.3e}"


def check_form(C, pb, C0, n, kind, what="", factor=6.0):
    """C after n steps of form `kind` against the oracle, both bounds from the arithmetic."""
    l2_tol, node_tol, ref = bounds(pb, C0, n, kind, factor)
    assert_close(C, ref, l2_tol, node_tol, what)
