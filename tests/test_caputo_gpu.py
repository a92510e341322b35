"""GPU parity of the Caputo-type variant F~ (Section 3.5, Eqs. Fg2, PSRLdD-a/b, Fg22:
lbm_params.variant = LBM_VARIANT_CAPUTO) against the FP64 oracle and the section's exact
solution.  The variant changes only the weight matrices (columns 0 and N of K_mu), so every
form runs it through its usual kernels:

* every precision form on a 2D MRT problem (tiles with ragged tails) and a 3D BGK
  problem, against the oracle within the bounds its arithmetic gives (FP64: 1e-12);
* a batch whose members alternate between the two variants;
* Section 3.5's exact solution C = exp(-t) prod (x^alpha + a) (source Eq. SourceTerm_PS,
  wall values from C): the oracle to 1e-12 in FP64, second-order convergence in dx;
* a uniform state with the same wall value and no source stays uniform;
* the discrete adjoint (lbm_grad) against the oracle's autograd.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import arith_bounds
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


def _problem(seed, d, collision, grid):
    rng = np.random.default_rng(seed)
    pb = dataclasses.replace(W.random_problem(rng, d, collision, grid, spherical=(collision == "bgk")),
                             variant="caputo", C_wall=0.3)
    f0 = W.random_field(rng, grid)
    return pb, 0.3 + f0 / f0.max()  # the wall value and O(1) variations about it


@pytest.mark.parametrize("form", ["fp64", "fp32", "bf16split", "tf32split", "bf16x5split", "bf16x6split"])
def test_caputo_2d_mrt_every_form(L, form):
    pb, C0 = _problem(1701, 2, "mrt", (150, 133))
    n = 40
    with L.Lattice(pb, C0, form) as lat:
        lat.step(n)
        C = lat.C()
    if form == "fp64":
        arith_bounds.assert_close(C, O.run_C(pb, C0, n).numpy(), 1e-12, 1e-12, "caputo 2d fp64")
    else:
        arith_bounds.check_form(C, pb, C0, n, form, f"caputo 2d {form}")


@pytest.mark.parametrize("form", ["fp64", "fp32", "tf32split", "bf16x6split"])
def test_caputo_3d_bgk_every_form(L, form):
    pb, C0 = _problem(1702, 3, "bgk", (40, 36, 33))
    n = 20
    with L.Lattice(pb, C0, form) as lat:
        lat.step(n)
        C = lat.C()
    if form == "fp64":
        arith_bounds.assert_close(C, O.run_C(pb, C0, n).numpy(), 1e-12, 1e-12, "caputo 3d fp64")
    else:
        arith_bounds.check_form(C, pb, C0, n, form, f"caputo 3d {form}")


@pytest.mark.parametrize("form", ["fp32", "bf16x6split"])
def test_batch_mixes_variants(L, form):
    probs, fields = [], []
    for i in range(6):
        pb, C0 = _problem(1800 + i, 2, "mrt", (48 + 16 * i, 40 + 9 * i))
        probs.append(pb if i % 2 else dataclasses.replace(pb, variant="fg"))
        fields.append(C0)
    n = 15
    with L.Batch(probs, fields, form) as b:
        b.step(n)
        got = [b.C(i) for i in range(len(probs))]
    for i, (pb, C0) in enumerate(zip(probs, fields)):
        arith_bounds.check_form(got[i], pb, C0, n, form, f"batch member {i} {pb.variant} {form}")


def _exact_case(N, T=0.1):
    """Section 3.5: D = 1, g = 1, u = 0, p = 1 on ]0,1[^2, alpha = (1.7, 1.2), a = (0.3, 1.2)."""
    alpha, a = (1.7, 1.2), (0.3, 1.2)
    dx = 1.0 / N
    n = int(round(T / (0.5 * (1.0 / 3.0) * dx * dx)))
    dt = T / n
    x = np.arange(N + 1) * dx
    X = np.broadcast_to(x[None, :], (N + 1, N + 1))
    Y = np.broadcast_to(x[:, None], (N + 1, N + 1))
    px, py = X ** alpha[0] + a[0], Y ** alpha[1] + a[1]
    prof = np.ascontiguousarray(px * py)
    S = np.ascontiguousarray(-(prof + math.gamma(alpha[0] + 1) * py + math.gamma(alpha[1] + 1) * px))
    pb = W.Problem(d=2, collision="mrt", grid=(N + 1, N + 1), alpha=alpha, p=(1.0, 1.0), g=(1.0, 1.0),
                   D=((1.0, 0.0), (0.0, 1.0)), u=(0.0, 0.0), s_free=(1.2, 1.2), dx=dx, dt=dt, variant="caputo")
    return pb, prof, S, n, math.exp(-T) * prof


def _gpu_exact(L, N, form):
    pb, prof, S, n, exact = _exact_case(N)
    with L.Lattice(pb, prof, form) as lat:
        lat.set_source(S, -1.0)
        lat.set_wall_values(prof, -1.0)
        lat.step(n)
        return pb, prof, S, n, exact, lat.C()


def test_caputo_exact_solution_fp64(L):
    pb, prof, S, n, exact, C = _gpu_exact(L, 20, "fp64")
    ops = O.with_source_and_walls(O.Operators(pb), source=(S, -1.0), walls=(prof, -1.0))
    C_ref = O.concentration(O.run(pb, prof, n, ops)).numpy()
    arith_bounds.assert_close(C, C_ref, 1e-12, 1e-12, "caputo exact case fp64")
    assert arith_bounds.rel_l2(C, exact) < 6e-4


def test_caputo_exact_solution_converges(L):
    errs = []
    for N in (20, 40):
        *_, exact, C = _gpu_exact(L, N, "fp32")
        errs.append(arith_bounds.rel_l2(C, exact))
    assert errs[1] < 3e-4 and errs[1] < 0.4 * errs[0], errs


@pytest.mark.parametrize("form,tol", [("fp64", 1e-12), ("fp32", 3e-5), ("bf16x6split", 3e-5)])
def test_caputo_keeps_uniform_state(L, form, tol):
    pb, _ = _problem(1703, 2, "mrt", (70, 64))
    pb = dataclasses.replace(pb, u=(0.0, 0.0), C_wall=0.7)
    with L.Lattice(pb, np.full(pb.shape, 0.7), form) as lat:
        lat.step(60)
        C = lat.C()
    assert np.max(np.abs(C - 0.7)) < tol * 0.7


def test_caputo_adjoint_matches_oracle(L):
    pb, C0 = _problem(1704, 2, "mrt", (26, 22))
    snaps = [8, 20]
    rng = np.random.default_rng(5)
    obs = np.stack([O.run_C(dataclasses.replace(pb, alpha=tuple(min(2.0, a + 0.03) for a in pb.alpha)), C0, t).numpy()
                    for t in snaps]) + 1e-4 * rng.normal(size=(2,) + pb.shape)
    loss_ref, g_ref = O.loss_and_grad(pb, C0, snaps, torch.tensor(obs))
    g_ref = g_ref.numpy()
    with L.Lattice(pb, C0, "fp64") as lat:
        loss, g = lat.grad(snaps, obs, 5)
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    assert np.all(np.abs(g - g_ref)[big] < 1e-8 * np.abs(g_ref)[big]), (g, g_ref)
