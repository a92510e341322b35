"""The GPU discrete adjoint (lbm_grad) against the FP64 oracle's adjoint (autograd through
the plain restatement, itself pinned to central finite differences in the CPU tests).

Bounds: FP64 handles 1e-8, FP32 and split-precision handles 1e-4 (the stated gradient bar):
every component within that fraction of its family's largest component (alpha, p, D, u), and
the components above 1e-2 of it within that fraction of themselves.  BGK and MRT, 2-D and
3-D; after lbm_grad the handle holds its initial state bit for bit."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import lbm_oracle as O
from paper_1706_09161_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1706_09161_gb300 import build
    build.build()
    from paper_1706_09161_gb300 import lbm
    return lbm


def observations(pb, C0, snaps, seed, noise=1e-4):
    """Snapshots of the scheme run with perturbed parameters (oracle), plus N(0, noise^2)."""
    pb_obs = dataclasses.replace(pb, alpha=tuple(min(2.0, a + 0.04) for a in pb.alpha),
                                 p=tuple(min(1.0, max(0.0, p - 0.05)) for p in pb.p),
                                 u=tuple(0.9 * v for v in pb.u))
    ops = O.Operators(pb_obs)
    f = O.init_populations(ops, torch.tensor(C0))
    out, t = [], 0
    rng = np.random.default_rng(seed)
    for ts in snaps:
        while t < ts:
            f = O.step(ops, f)
            t += 1
        out.append(O.concentration(f).numpy() + noise * rng.normal(size=pb.shape) * C0.max())
    return np.stack(out)


def check(L, pb, C0, snaps, ckpt, precision, rtol):
    obs = observations(pb, C0, snaps, seed=len(snaps))
    loss_ref, grad_ref = O.loss_and_grad(pb, C0, snaps, torch.tensor(obs))
    grad_ref = grad_ref.numpy()
    with L.Lattice(pb, C0, precision) as lat:
        loss, grad = lat.grad(snaps, obs, ckpt)
        C_after = lat.C()
    assert loss == pytest.approx(loss_ref, rel=max(rtol, 1e-12))
    d = pb.d
    for k, fam in enumerate(("alpha", "p", "D", "u")):
        # each parameter family against its own largest component: every component within
        # rtol of that, and the components above 1e-2 of it within rtol of themselves (the
        # arithmetic's error scales with the family, not with a small component)
        a, b = grad[k * d:(k + 1) * d], grad_ref[k * d:(k + 1) * d]
        top = np.abs(b).max()
        assert np.all(np.abs(a - b) <= rtol * top), (fam, a, b)
        big = np.abs(b) > 1e-2 * top
        rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
        assert np.all(rel[big] < rtol), (fam, a, b)
    # the handle is left at its initial state, bit for bit
    with L.Lattice(pb, C0, precision) as fresh:
        assert np.array_equal(C_after, fresh.C())


@pytest.mark.parametrize("grid,snaps,ckpt", [((24, 20), [10, 20, 30], 7), ((37, 29), [0, 15, 16, 40], 10)])
def test_adjoint_fp64_2d(L, grid, snaps, ckpt):
    rng = np.random.default_rng(grid[0])
    pb = W.random_problem(rng, 2, "mrt", grid)
    check(L, pb, W.random_field(rng, grid), snaps, ckpt, "fp64", 1e-8)


def test_adjoint_fp64_3d(L):
    rng = np.random.default_rng(41)
    pb = W.random_problem(rng, 3, "mrt", (12, 10, 9))
    check(L, pb, W.random_field(rng, pb.grid), [6, 12], 5, "fp64", 1e-8)


def test_adjoint_fp32_2d(L):
    rng = np.random.default_rng(43)
    pb = W.random_problem(rng, 2, "mrt", (40, 33))
    check(L, pb, W.random_field(rng, pb.grid), [20, 40, 60], 25, "fp32", 1e-4)


def test_adjoint_inverse_workload_reduced(L):
    """The inverse-problem workload's parameters on a 64x64 grid, 300 steps, 3 snapshots,
    checkpoint every 100 (FP32 forward and adjoint)."""
    pb, C0, _ = W.inverse_256(side=64)
    check(L, pb, C0, [100, 200, 300], 100, "fp32", 1e-4)


@pytest.mark.parametrize("grid,spherical,precision,rtol", [((26, 22), False, "fp64", 1e-8),
                                                           ((26, 22), True, "fp64", 1e-8),
                                                           ((40, 33), False, "fp32", 1e-4)])
def test_adjoint_bgk_2d(L, grid, spherical, precision, rtol):
    """BGK (Omega = I / lambda, K_mu scaled by h_mu = D_mumu / max D, end of Section 2.2),
    non-spherical and spherical D (a tie: each D_mumu takes an equal part of d(max D), as
    the oracle's autograd does)."""
    rng = np.random.default_rng(grid[0] + 3 * spherical)
    pb = W.random_problem(rng, 2, "bgk", grid, spherical=spherical)
    check(L, pb, W.random_field(rng, grid), [10, 20, 30], 7, precision, rtol)


def test_adjoint_bgk_3d(L):
    rng = np.random.default_rng(53)
    pb = W.random_problem(rng, 3, "bgk", (12, 10, 9))
    check(L, pb, W.random_field(rng, pb.grid), [6, 12], 5, "fp64", 1e-8)


@pytest.mark.parametrize("form,coll", [("bf16x6split", "mrt"), ("tf32split", "bgk"), ("bf16split", "mrt")])
def test_adjoint_split_forms(L, form, coll):
    """On a split-precision handle lbm_grad returns the plain FP32 scheme's gradient (computed
    on an FP32 copy of the problem) and leaves the handle at its initial state."""
    rng = np.random.default_rng(61 + len(form))
    pb = W.random_problem(rng, 2, coll, (40, 33), spherical=(coll == "bgk"))
    check(L, pb, W.random_field(rng, pb.grid), [20, 40], 10, form, 1e-4)


def test_grad_refuses_unsupported(L):
    rng = np.random.default_rng(1)
    pb = W.random_problem(rng, 2, "mrt", (32, 32))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "fp32") as lat:
        lat.set_fields(u=np.full((2,) + pb.shape, 0.01))
        with pytest.raises(L.LBMError) as ei:
            lat.grad([5], np.zeros((1,) + pb.shape), 2)
        assert ei.value.code == L.LBM_ENOTSUP
    probs, fields, _ = W.batch64(nprob=2, sides=(64,), seed=3)
    with L.Batch(probs, fields, "fp32") as b:
        with pytest.raises(L.LBMError):
            L.lbm_grad(b.h, [5], np.zeros((1,) + probs[0].shape), 2, 2)


def test_autograd_function_fits_parameters(L):
    """snapshot_loss as a torch.autograd.Function: its gradient is lbm_grad's, and a few
    gradient steps on alpha and u reduce the misfit (parameters fitted to observed plumes)."""
    rng = np.random.default_rng(47)
    pb = W.random_problem(rng, 2, "mrt", (32, 30))
    C0 = W.random_field(rng, pb.grid)
    snaps = [10, 20]
    truth = dataclasses.replace(pb, alpha=tuple(min(2.0, a + 0.04) for a in pb.alpha), u=tuple(0.9 * v for v in pb.u))
    obs = np.stack([O.run_C(truth, C0, ts).numpy() for ts in snaps])
    d = pb.d
    theta = torch.tensor(list(pb.alpha) + list(pb.p) + [pb.D[i][i] for i in range(d)] + list(pb.u),
                         dtype=torch.float64, requires_grad=True)
    loss = L.snapshot_loss(pb, C0, snaps, obs, theta, "fp64", 5)
    loss.backward()
    _, g_ref = O.loss_and_grad(pb, C0, snaps, torch.tensor(obs))
    assert torch.allclose(theta.grad, g_ref, rtol=1e-8, atol=1e-14)
    # fit alpha and u by normalised gradient steps with backtracking
    mask = torch.zeros(4 * d, dtype=torch.float64)
    mask[:d] = 1.0
    mask[3 * d:] = 1.0
    th = theta.detach().clone()
    L0 = float(loss.detach())
    cur = L0
    # one handle for the whole fit (lbm_set_params between evaluations)
    with L.Lattice(pb, C0, "fp64") as lat:
        for _ in range(6):
            t = th.clone().requires_grad_(True)
            lt = L.snapshot_loss(pb, C0, snaps, obs, t, "fp64", 5, lattice=lat)
            lt.backward()
            # the reused handle gives what a new handle gives
            t2 = th.clone().requires_grad_(True)
            L.snapshot_loss(pb, C0, snaps, obs, t2, "fp64", 5).backward()
            assert torch.allclose(t.grad, t2.grad, rtol=1e-13, atol=0)
            step = -(t.grad * mask)
            step = step / step.abs().max() * 0.01
            for _ in range(6):
                cand = th + step
                lc = float(L.snapshot_loss(pb, C0, snaps, obs, cand, "fp64", 5, lattice=lat))
                if lc < cur:
                    th, cur = cand, lc
                    break
                step = step / 2
    assert cur < 0.5 * L0
