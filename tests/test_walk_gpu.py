"""GPU killed stable-Levy walk (lbm_walk, lbm_walk_density) against the oracle's walk with the
same Philox4x32-10 draws (Section 3.1: Eqs. RW_STABLE, distri; the bounded-domain
subsection; Appendix A), and its density against the lattice Boltzmann oracle.

* FP64 form: every position within 1e-12 (relative to the box) of the oracle's and the same
  paths alive; a run split over launches equals one launch, bit for bit;
* FP32 form (23-bit uniforms, exact in FP32, which the oracle replays in FP64): positions of paths alive on
  both sides within 2e-5, at most 0.1% of the kill decisions different (a path that passes
  within FP32 rounding of a wall);
* the density histogram equals a histogram of the returned positions exactly, and over 4e6
  paths it matches the killed walk's lattice Boltzmann solution (marginals within 4 standard
  errors plus 2% of the peak, surviving fraction against the remaining mass).
"""
import math

import numpy as np
import pytest
import torch

from oracle import lbm_oracle as O
from oracle import levy_walk as LW
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


CASES = {2: dict(alpha=(1.5, 1.7), p=(0.3, 0.8), D=(0.1, 0.1), g=(1.0, 1.0), u=(0.05, -0.02)),
         3: dict(alpha=(1.4, 1.8, 2.0), p=(0.2, 0.6, 0.5), D=(0.08, 0.1, 0.05), g=(1.0, 1.2, 1.0),
                 u=(0.0, 0.03, -0.01))}


def _start(d, n, seed):
    rng = np.random.default_rng(seed)
    X0 = rng.normal(0.5, 0.08, size=(n, d))
    return X0, np.all((X0 > 0) & (X0 < 1), axis=1)


def _gpu_walk(L, prm, X0, alive0, splits):
    n, d = X0.shape
    X = torch.tensor(np.ascontiguousarray(X0.T), device="cuda")
    A = torch.tensor(alive0.astype(np.uint8), device="cuda")
    step = 0
    for k in splits:
        L.lbm_walk(prm, n, X.data_ptr(), A.data_ptr(), step, k)
        step += k
    torch.cuda.synchronize()
    return X.cpu().numpy().T, A.cpu().numpy().astype(bool)


@pytest.mark.parametrize("d", [2, 3])
def test_fp64_walk_matches_oracle_and_splits(L, d):
    c = CASES[d]
    dt, seed, n, nsteps = 1e-3, 31 + d, 4096, 60
    prm = L.walk_params(d, c["alpha"], c["p"], c["D"], c["g"], c["u"], (0,) * d, (1,) * d, dt, seed, "fp64")
    X0, alive0 = _start(d, n, 5 + d)
    X_ref, alive_ref = LW.killed_walk_philox(X0, alive0, c["alpha"], c["p"], c["D"], c["g"], c["u"], (0,) * d,
                                             (1,) * d, dt, seed, 0, nsteps)
    X, alive = _gpu_walk(L, prm, X0, alive0, [nsteps])
    assert np.array_equal(alive, alive_ref)
    assert np.max(np.abs(X - X_ref)) < 1e-12
    assert np.count_nonzero(alive0 & ~alive) > 0  # the walls kill some paths
    X2, alive2 = _gpu_walk(L, prm, X0, alive0, [7, 23, 30])
    assert np.array_equal(X2, X) and np.array_equal(alive2, alive)


@pytest.mark.parametrize("d", [2, 3])
def test_fp32_walk_follows_the_oracle(L, d):
    c = CASES[d]
    dt, seed, n, nsteps = 1e-3, 41 + d, 8192, 60
    prm = L.walk_params(d, c["alpha"], c["p"], c["D"], c["g"], c["u"], (0,) * d, (1,) * d, dt, seed, "fp32")
    X0, alive0 = _start(d, n, 9 + d)
    X0 = X0.astype(np.float32).astype(np.float64)  # representable in the FP32 form
    X_ref, alive_ref = LW.killed_walk_philox(X0, alive0, c["alpha"], c["p"], c["D"], c["g"], c["u"], (0,) * d,
                                             (1,) * d, dt, seed, 0, nsteps, bits=23)
    X, alive = _gpu_walk(L, prm, X0, alive0, [nsteps])
    both = alive & alive_ref
    assert np.max(np.abs(X[both] - X_ref[both])) < 2e-5
    assert np.count_nonzero(alive != alive_ref) <= max(2, n // 1000)


def test_density_histogram_and_killed_walk_solution(L):
    """The paper's check (LBM against the walk, Validations 1-2): 4e6 FP32 paths on the
    [0,1]^2 case of the oracle's own pin (dx = 1/40, lambda = 1, t = 0.25)."""
    N = 40
    dx = 1.0 / N
    alpha, p, D = (1.5, 1.7), (0.3, 0.8), (0.1, 0.1)
    dt = 0.5 * (1.0 / 3.0) * dx * dx / D[0]
    nsteps, sig = 240, 0.08
    x = np.arange(N + 1) * dx
    Xg, Yg = np.meshgrid(x, x, indexing="xy")
    C0 = W.zero_walls(np.exp(-((Xg - 0.5) ** 2 + (Yg - 0.5) ** 2) / (2 * sig * sig)) / (2 * math.pi * sig * sig))
    pb = W.Problem(d=2, collision="mrt", grid=(N + 1, N + 1), alpha=alpha, p=p, g=(1.0, 1.0),
                   D=((D[0], 0.0), (0.0, D[1])), u=(0.0, 0.0), s_free=(1.2, 1.2), dx=dx, dt=dt)
    C = O.run_C(pb, C0, nsteps).numpy()
    mass = float(C.sum()) * dx * dx
    n = 4_000_000
    prm = L.walk_params(2, alpha, p, D, (1.0, 1.0), (0.0, 0.0), (0.0, 0.0), (1.0, 1.0), dt, 2024, "fp32")
    gen = torch.Generator(device="cuda").manual_seed(7)
    X = (0.5 + sig * torch.randn((2, n), dtype=torch.float64, device="cuda", generator=gen)).contiguous()
    A = ((X > 0) & (X < 1)).all(0).to(torch.uint8).contiguous()
    L.lbm_walk(prm, n, X.data_ptr(), A.data_ptr(), 0, nsteps)
    counts = torch.zeros((N + 1) * (N + 1), dtype=torch.int32, device="cuda")
    L.lbm_walk_density(prm, n, X.data_ptr(), A.data_ptr(), (N + 1, N + 1), dx, counts.data_ptr())
    torch.cuda.synchronize()
    Xh, Ah = X.cpu().numpy(), A.cpu().numpy().astype(bool)
    # the histogram kernel counts exactly what the positions say
    k = np.floor(Xh[:, Ah] / dx + 0.5).astype(np.int64)
    inb = np.all((k >= 0) & (k <= N), axis=0)
    want = np.zeros((N + 1) * (N + 1), dtype=np.int64)
    np.add.at(want, k[1, inb] * (N + 1) + k[0, inb], 1)
    got = counts.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want)
    # and the density solves the FADE with C = 0 on the walls
    surv = float(Ah.mean())
    assert abs(surv - mass) < 4.0 * math.sqrt(surv * (1 - surv) / n) + 2e-3, (surv, mass)
    dens = got.reshape(N + 1, N + 1) / n / (dx * dx)
    for mu in range(2):
        marg_w = (dens.sum(axis=0) if mu == 0 else dens.sum(axis=1))[1:-1] * dx
        marg = (C.sum(axis=0) if mu == 0 else C.sum(axis=1))[1:-1] * dx
        se = np.sqrt(np.maximum(marg_w, 1e-3) * dx / n) / dx
        assert np.all(np.abs(marg_w - marg) < 4.0 * se + 0.02 * marg.max()), mu


def test_walk_rejects_bad_arguments(L):
    c = CASES[2]
    X = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    A = torch.ones(4, dtype=torch.uint8, device="cuda")
    good = dict(d=2, alpha=c["alpha"], p=c["p"], D=c["D"], g=c["g"], u=c["u"], lo=(0, 0), hi=(1, 1), dt=1e-3, seed=1)
    for key, val in [("alpha", (1.0, 1.5)), ("p", (1.2, 0.5)), ("D", (0.0, 0.1)), ("dt", 0.0), ("hi", (0.0, 1.0))]:
        kw = dict(good, **{key: val})
        prm = L.walk_params(**kw)
        with pytest.raises(L.LBMError):
            L.lbm_walk(prm, 4, X.data_ptr(), A.data_ptr(), 0, 5)
    prm = L.walk_params(**good)
    with pytest.raises(L.LBMError):
        L.lbm_walk(prm, 4, X.data_ptr(), A.data_ptr(), 0xffffffff, 5)
    L.lbm_walk(prm, 0, 0, 0, 0, 5)  # nothing to do
