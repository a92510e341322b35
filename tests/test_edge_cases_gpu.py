"""GPU parity on the inputs the random cases do not reach, in every precision form:

* a constant diffusion tensor with off-diagonal entries under MRT (Section 2.3,
  Eq. (D_ab): the flux block of Lambda^-1 is the full d x d matrix D/e^2 + Id/2);
* the one-sided operators p = 0 and p = 1 (Eq. Fg: K_mu is then upper or lower
  triangular, half of the dense contraction multiplies zeros);
* alpha = 2 exactly on an axis (gamma = 0: both integrals are the identity, K = g Id,
  and the scheme is the classical ADE on that axis, Section 2.2 after Eq. CoeffA_FADE3D).

Every case checks the whole field (relative L2) and every node (max |C - C_ref| over
max |C_ref|) against the FP64 oracle: 1e-12 for FP64; for the FP32 forms 4x the error the
same arithmetic makes when re-run on the CPU, never below 1e-5.  Also: the concentration
read straight into a device array equals the host read, for single problems and batch
members, and lbm_mass takes the problem index.
"""
import dataclasses

import numpy as np
import pytest
import torch

import arith_bounds
from oracle import lbm_oracle as O
from paper_1706_09161_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORMS = ["fp64", "fp32", "bf16split", "tf32split", "bf16x5split", "bf16x6split"]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1706_09161_gb300 import build
    build.build()
    from paper_1706_09161_gb300 import lbm
    return lbm


def _check(L, pb, C0, n, form, what):
    C_ref = O.run_C(pb, C0, n).numpy()
    with L.Lattice(pb, C0, form) as lat:
        lat.step(n)
        C = lat.C()
    if form == "fp64":
        arith_bounds.assert_close(C, C_ref, 1e-12, 1e-12, what)
    else:
        l2_tol, node_tol, _ = arith_bounds.bounds(pb, C0, n, form, C_ref=C_ref)
        arith_bounds.assert_close(C, C_ref, l2_tol, node_tol, what)


# off-diagonal D: lambdabar = D / e^2 + Id / 2 stays symmetric positive definite
D_OFF_2D = ((0.02, 0.008), (0.008, 0.015))
D_OFF_3D = ((0.02, 0.006, -0.004), (0.006, 0.015, 0.003), (-0.004, 0.003, 0.012))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("grid", [(70, 65), (128, 96), (40, 21, 19), (44, 36, 33)])
def test_offdiagonal_diffusion_tensor_mrt(L, form, grid):
    rng = np.random.default_rng(501 + grid[0] + len(grid))
    d = len(grid)
    pb = dataclasses.replace(W.random_problem(rng, d, "mrt", grid), D=D_OFF_2D if d == 2 else D_OFF_3D)
    _check(L, pb, W.random_field(rng, grid), 15, form, f"off-diagonal D {grid} {form}")


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("grid", [(130, 70), (64, 48, 40)])
@pytest.mark.parametrize("p", [(0.0, 1.0, 0.0), (1.0, 0.0, 1.0)])
def test_one_sided_operators(L, form, grid, p):
    """p in {0, 1}: triangular K_mu (only I- or only I+ on each axis)."""
    rng = np.random.default_rng(601 + grid[0] + int(p[0]))
    d = len(grid)
    pb = dataclasses.replace(W.random_problem(rng, d, "mrt", grid), p=p[:d])
    C0 = W.random_field(rng, grid)
    # the operator itself, every axis
    ops = O.Operators(pb)
    F = O.fractional_terms(ops, O.concentration(O.init_populations(ops, torch.tensor(C0))))
    with L.Lattice(pb, C0, form) as lat:
        for mu in range(d):
            tol = 1e-13 if form == "fp64" else (1e-6 if form == "fp32" else 4e-5)
            assert arith_bounds.rel_l2(lat.F(mu), F[mu].numpy()) < tol, (form, mu)
    _check(L, pb, C0, 12, form, f"p={p[:d]} {grid} {form}")


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("grid", [(96, 70), (40, 36, 21)])
def test_alpha_two_exactly(L, form, grid):
    """alpha = 2 on the first axis (classical dispersion there), fractional elsewhere;
    and alpha = 2 on every axis (the classical ADE)."""
    rng = np.random.default_rng(701 + grid[0])
    d = len(grid)
    base = W.random_problem(rng, d, "mrt", grid)
    C0 = W.random_field(rng, grid)
    for alpha in [(2.0,) + tuple(base.alpha[1:]), (2.0,) * d]:
        pb = dataclasses.replace(base, alpha=alpha)
        ops = O.Operators(pb)
        # K = g Id at alpha = 2 (gamma = 0): the oracle's own closed form
        assert torch.allclose(ops.K[0], ops.g[0] * torch.eye(grid[0], dtype=torch.float64), atol=1e-15)
        _check(L, pb, C0, 12, form, f"alpha={alpha} {grid} {form}")


@pytest.mark.parametrize("form", ["fp64", "fp32", "bf16split"])
def test_read_C_into_device_array(L, form):
    rng = np.random.default_rng(801)
    pb = W.random_problem(rng, 2, "mrt", (130, 70))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, form) as lat:
        lat.step(9)
        host = lat.C()
        dev = torch.full(pb.shape, float("nan"), dtype=torch.float64, device="cuda")
        lat.C_into(dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host)
        assert lat.mass() == pytest.approx(float(host.sum()), rel=1e-12 if form == "fp64" else 1e-6)


def test_batch_read_C_into_device_array_and_mass_by_index(L):
    probs, fields, _ = W.batch64(nprob=3, sides=(64, 128), seed=21)
    with L.Batch(probs, fields, "bf16split") as b:
        b.step(5)
        for i in range(3):
            host = b.C(i)
            dev = torch.zeros(probs[i].shape, dtype=torch.float64, device="cuda")
            b.C_into(i, dev)
            torch.cuda.synchronize()
            assert np.array_equal(dev.cpu().numpy(), host)
            assert b.mass(i) == pytest.approx(float(host.sum()), rel=1e-6)
        with pytest.raises(L.LBMError):
            L.lbm_read_C(b.h, 3, np.empty(probs[0].shape))
        with pytest.raises(L.LBMError):
            L.lbm_mass(b.h, -1)
