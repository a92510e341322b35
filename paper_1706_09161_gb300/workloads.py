"""Seeded synthetic inputs for the fractional ADE lattice Boltzmann step.

This module only *generates* inputs: problem parameters and initial
concentration fields.  It holds none of the scheme's arithmetic (no weights,
no relaxation rates, no equilibrium), so that the FP64 oracle and the CUDA
path can both be fed from it without sharing any of the method's code.

Array convention: a field on a grid ``(n_1, ..., n_d)`` (nodes per axis,
walls included) is stored with axis 1 (x) fastest, i.e. a numpy array of
shape ``(n_2, n_1)`` in 2-D and ``(n_3, n_2, n_1)`` in 3-D.

The named workloads are in lattice units (dx = dt = 1) except ``varying_512`` and
``exact_e5``, which set dx = 1/(side-1) on [0,1]^2 and dt from D.

The named workloads follow the paper's validation style (Section 3: Gaussian
hills in square domains, homogeneous Dirichlet walls, alpha in ]1,2],
p in [0,1]) at the sizes of the performance study:

* ``fp64_bgk_64``        2-D D2Q5 BGK, 64x64, FP64, 200 steps
* ``mrt_aniso_512``      2-D D2Q5 MRT, 512x512, anisotropic, advected, 5000 steps
* ``mrt3d_256``          3-D D3Q7 MRT, 256^3, 2000 steps
* ``batch64``            64 independent 2-D MRT problems of uneven sizes
* ``inverse_256``        2-D MRT 256x256 with hidden parameters and noisy snapshots
* ``varying_512``        2-D MRT 512x512 on [0,1]^2 with D(x), g(x), u(x) varying in space
* ``exact_e5``           2-D MRT on ]0,1[^2 with the source, varying D(x) and time-dependent wall
                         values of Section 3.4, whose exact solution is known
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class Problem:
    """Parameters of one FADE lattice Boltzmann problem (lattice units by default).

    d          : space dimension (2 -> D2Q5, 3 -> D3Q7)
    collision  : "bgk" or "mrt"
    grid       : nodes per axis, both wall nodes included (n_1, ..., n_d)
    alpha, p, g: per-axis fractional order in ]1,2], skewness weight in [0,1],
                 positive factor g_mu (constant)
    D          : d x d diffusion tensor (row-major nested lists)
    u          : advection velocity per axis
    s_free     : MRT relaxation *rates* (inverse relaxation times) of the
                 non-conserved, non-flux moments (D2Q5: 2 values, D3Q7: 3)
    dx, dt     : space and time steps
    C_wall     : Dirichlet value imposed on every wall node
    variant    : "fg" (fractional term of Eq. Fg) or "caputo" (Caputo-type F~, Eq. Fg2)
    """

    d: int
    collision: str
    grid: Tuple[int, ...]
    alpha: Tuple[float, ...]
    p: Tuple[float, ...]
    g: Tuple[float, ...]
    D: Tuple[Tuple[float, ...], ...]
    u: Tuple[float, ...]
    s_free: Tuple[float, ...] = ()
    dx: float = 1.0
    dt: float = 1.0
    C_wall: float = 0.0
    variant: str = "fg"

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape of a field (axis 1 fastest)."""
        return tuple(reversed(self.grid))

    @property
    def nodes(self) -> int:
        return int(np.prod(self.grid))


def _diag(vals: Sequence[float]) -> Tuple[Tuple[float, ...], ...]:
    d = len(vals)
    return tuple(tuple(float(vals[i]) if i == j else 0.0 for j in range(d)) for i in range(d))


def zero_walls(C: np.ndarray) -> np.ndarray:
    """Set every boundary node of a field to zero (homogeneous Dirichlet data)."""
    C = C.copy()
    for ax in range(C.ndim):
        idx = [slice(None)] * C.ndim
        idx[ax] = 0
        C[tuple(idx)] = 0.0
        idx[ax] = -1
        C[tuple(idx)] = 0.0
    return C


def gaussian_pulse(grid: Sequence[int], sigma: float,
                   centre: Optional[Sequence[float]] = None) -> np.ndarray:
    """Gaussian hill sampled at the nodes, walls zeroed, renormalised to unit mass.

    ``centre`` is in node indices per axis (default: the middle, (n-1)/2).
    """
    grid = tuple(int(n) for n in grid)
    if centre is None:
        centre = [(n - 1) / 2.0 for n in grid]
    axes = [np.arange(n, dtype=np.float64) for n in reversed(grid)]
    mesh = np.meshgrid(*axes, indexing="ij")  # mesh[k] is the coordinate of array dim k
    r2 = np.zeros(tuple(reversed(grid)))
    for k, c in enumerate(reversed(list(centre))):
        r2 += (mesh[k] - c) ** 2
    C = np.exp(-r2 / (2.0 * sigma * sigma))
    C = zero_walls(C)
    return C / C.sum()


def square_pulse(grid: Sequence[int], width: int = 5) -> np.ndarray:
    """width^d block of equal values centred at node n//2 on every axis, unit mass."""
    C = np.zeros(tuple(reversed(tuple(grid))))
    sl = tuple(slice(n // 2 - width // 2, n // 2 - width // 2 + width) for n in reversed(tuple(grid)))
    C[sl] = 1.0
    return C / C.sum()


# --------------------------------------------------------------------------- named workloads

def fp64_bgk_64() -> Tuple[Problem, np.ndarray, int]:
    """2-D pure space-fractional diffusion, D2Q5 BGK, 64x64, FP64, 200 steps."""
    pb = Problem(d=2, collision="bgk", grid=(64, 64), alpha=(1.7, 1.7), p=(0.5, 0.5),
                 g=(1.0, 1.0), D=_diag([1e-3, 1e-3]), u=(0.0, 0.0))
    return pb, gaussian_pulse(pb.grid, 2.0), 200


def mrt_aniso_512() -> Tuple[Problem, np.ndarray, int]:
    """2-D anisotropic fractional ADE, D2Q5 MRT, 512x512, 5000 steps, 5x5 pulse."""
    rng = np.random.default_rng(2)
    s_free = tuple(float(v) for v in rng.uniform(0.8, 1.9, size=2))
    pb = Problem(d=2, collision="mrt", grid=(512, 512), alpha=(1.5, 1.8), p=(0.3, 0.7),
                 g=(1.0, 1.0), D=_diag([2e-3, 5e-4]), u=(0.05, 0.02), s_free=s_free)
    return pb, square_pulse(pb.grid, 5), 5000


def mrt3d_256(side: int = 256) -> Tuple[Problem, np.ndarray, int]:
    """3-D fractional ADE, D3Q7 MRT, side^3 (256^3 by default), 2000 steps."""
    rng = np.random.default_rng(3)
    s_free = tuple(float(v) for v in rng.uniform(0.8, 1.9, size=3))
    pb = Problem(d=3, collision="mrt", grid=(side, side, side), alpha=(1.6, 1.6, 1.9),
                 p=(0.5, 0.2, 0.8), g=(1.0, 1.0, 1.0), D=_diag([1e-3, 1e-3, 4e-4]),
                 u=(0.03, 0.0, 0.0), s_free=s_free)
    return pb, gaussian_pulse(pb.grid, 3.0), 2000


BATCH_SIDES = (128, 256, 384, 512, 768, 1024)


def batch64(nprob: int = 64, sides: Sequence[int] = BATCH_SIDES, seed: int = 4
            ) -> Tuple[List[Problem], List[np.ndarray], int]:
    """Ensemble of independent 2-D MRT problems with uneven side lengths, 1000 steps each."""
    rng = np.random.default_rng(seed)
    probs, fields = [], []
    for _ in range(nprob):
        side = int(rng.choice(np.asarray(sides)))
        alpha = tuple(float(v) for v in rng.uniform(1.2, 2.0, size=2))
        p = tuple(float(v) for v in rng.uniform(0.0, 1.0, size=2))
        Dd = [float(v) for v in rng.uniform(1e-4, 3e-3, size=2)]
        # velocity uniform in the disc |u| <= 0.08
        r = 0.08 * np.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2.0 * np.pi)
        u = (float(r * np.cos(th)), float(r * np.sin(th)))
        s_free = tuple(float(v) for v in rng.uniform(0.8, 1.9, size=2))
        sigma = float(rng.uniform(2.0, 6.0))
        margin = max(8.0, 3.0 * sigma)
        centre = [float(rng.uniform(margin, side - 1 - margin)) for _ in range(2)]
        pb = Problem(d=2, collision="mrt", grid=(side, side), alpha=alpha, p=p,
                     g=(1.0, 1.0), D=_diag(Dd), u=u, s_free=s_free)
        probs.append(pb)
        fields.append(gaussian_pulse(pb.grid, sigma, centre))
    return probs, fields, 1000


INVERSE_TRUTH = dict(alpha=(1.45, 1.75), p=(0.35, 0.65), D=(1.5e-3, 7e-4), u=(0.04, -0.01))


def inverse_256(side: int = 256, nsteps: int = 3000, nsnap: int = 10
                ) -> Tuple[Problem, np.ndarray, List[int]]:
    """Inverse problem: hidden parameters, initial Gaussian, snapshot steps.

    The observations themselves are produced by running a forward model on
    these parameters and adding ``observation_noise``.
    """
    rng = np.random.default_rng(5)
    s_free = tuple(float(v) for v in rng.uniform(0.8, 1.9, size=2))
    t = INVERSE_TRUTH
    pb = Problem(d=2, collision="mrt", grid=(side, side), alpha=t["alpha"], p=t["p"],
                 g=(1.0, 1.0), D=_diag(t["D"]), u=t["u"], s_free=s_free)
    snaps = [nsteps * (k + 1) // nsnap for k in range(nsnap)]
    return pb, gaussian_pulse(pb.grid, 3.0), snaps


def observation_noise(shape: Sequence[int], seed: int = 5, std: float = 1e-4) -> np.ndarray:
    """N(0, std^2) noise for the synthetic observations."""
    return np.random.default_rng(seed + 1000).normal(0.0, std, size=tuple(shape))


def smooth_fields(rng: np.random.Generator, grid: Sequence[int], collision: str, D0: float, g_amp: float = 0.2,
                  u_amp: float = 0.0, u0: Sequence[float] = (), offdiag: float = 0.1) -> dict:
    """Seeded smooth coefficient fields on a grid (array order = reversed grid, leading axis
    per component): diagonal D(x) = D0 (1 +- 0.5 sin), off-diagonal entries up to
    offdiag * D0 (MRT only; BGK gets a spherical D(x)), g(x) = 1 +- g_amp, u(x) = u0 +- u_amp.
    Each component is a sum of one or two plane waves with random phases and wave numbers."""
    grid = tuple(int(n) for n in grid)
    d = len(grid)
    shape = tuple(reversed(grid))
    axes = np.meshgrid(*[np.linspace(0.0, 1.0, n) for n in shape], indexing="ij")

    def wave(amp):
        k = rng.uniform(0.5, 2.0, size=d)
        return amp * np.sin(2 * np.pi * (rng.uniform() + sum(kk * x for kk, x in zip(k, axes))))

    D = np.zeros((d, d) + shape)
    for i in range(d):
        D[i, i] = D0 * (1.0 + wave(0.5))
    if collision == "mrt":
        for i in range(d):
            for j in range(i + 1, d):
                D[i, j] = D[j, i] = D0 * wave(offdiag)
    else:
        for i in range(1, d):
            D[i, i] = D[0, 0]
    g = np.stack([1.0 + wave(g_amp) for _ in range(d)])
    u = np.stack([(u0[i] if u0 else 0.0) + wave(u_amp) for i in range(d)])
    return {"D": D, "g": g, "u": u}


def varying_512(side: int = 512) -> Tuple[Problem, np.ndarray, int, dict]:
    """2-D MRT with spatially varying coefficients, side^2 nodes on [0,1]^2 (dx = 1/(side-1)):
    D(x) = 0.02 (1 +- 0.5) with off-diagonal entries, g(x) = 1 +- 0.2, u(x) = (0.1, -0.05)
    +- 0.05, alpha = (1.6, 1.8), p = (0.4, 0.6), dt such that lambda = 1 at the mean D,
    unit-mass Gaussian (sigma = 0.05) at the centre, 2000 steps (t = 0.04)."""
    rng = np.random.default_rng(6)
    dx = 1.0 / (side - 1)
    D0 = 0.02
    dt = 0.5 * (1.0 / 3.0) * dx * dx / D0
    pb = Problem(d=2, collision="mrt", grid=(side, side), alpha=(1.6, 1.8), p=(0.4, 0.6), g=(1.0, 1.0),
                 D=_diag([D0, D0]), u=(0.1, -0.05), s_free=(1.2, 1.2), dx=dx, dt=dt)
    fields = smooth_fields(rng, pb.grid, "mrt", D0, g_amp=0.2, u_amp=0.05, u0=(0.1, -0.05))
    C0 = gaussian_pulse(pb.grid, 0.05 / dx)
    return pb, C0, 2000, fields


def exact_e5(side: int = 256, T: float = 0.1, alpha=(1.5, 1.7), a=(0.4, 0.7), lam_max: float = 1.0) -> dict:
    """Section 3.4's case with a closed-form solution, on ]0,1[^2 with side^2 nodes (dx =
    1/(side-1)): p = 1, g = 1, u = 0, diagonal D_mumu(x) = x_mu^alpha_mu Gamma(a_mu + 2 -
    alpha_mu) / Gamma(a_mu + 2), source S_c = -3 exp(-t) x^a1 y^a2, initial and wall values from
    C = exp(-t) x^a1 y^a2 (Eqs. Def_D_AS, exsolFADE_3D); MRT with free rates 1.2, dt such that
    lambda <= lam_max.  These are the paper's formulas for the inputs, written out as fields.
    Returns a dict: problem, C0, nsteps, coefficient fields, source (profile, rate), walls
    (profile, rate), exact (the solution at t = nsteps dt)."""
    import math
    N = side - 1
    dx = 1.0 / N
    x = np.arange(side) * dx
    X = np.broadcast_to(x[None, :], (side, side))
    Y = np.broadcast_to(x[:, None], (side, side))
    D = np.zeros((2, 2, side, side))
    D[0, 0] = X ** alpha[0] * math.gamma(a[0] + 2 - alpha[0]) / math.gamma(a[0] + 2)
    D[1, 1] = Y ** alpha[1] * math.gamma(a[1] + 2 - alpha[1]) / math.gamma(a[1] + 2)
    dt = (lam_max - 0.5) * (1.0 / 3.0) * dx * dx / float(D.max())
    n = int(round(T / dt))
    dt = T / n
    pb = Problem(d=2, collision="mrt", grid=(side, side), alpha=tuple(alpha), p=(1.0, 1.0), g=(1.0, 1.0),
                 D=_diag([0.1, 0.1]), u=(0.0, 0.0), s_free=(1.2, 1.2), dx=dx, dt=dt)
    prof = np.ascontiguousarray(X ** a[0] * Y ** a[1])
    return dict(problem=pb, C0=prof.copy(), nsteps=n, fields={"D": D}, source=(-3.0 * prof, -1.0),
                walls=(prof, -1.0), exact=math.exp(-T) * prof)


# --------------------------------------------------------------------------- random small cases

def random_problem(rng: np.random.Generator, d: int, collision: str, grid: Sequence[int],
                   advect: bool = True, spherical: bool = False) -> Problem:
    """Random admissible problem for parity tests (alpha in [1.2,2], p in [0,1], lattice units)."""
    alpha = tuple(float(v) for v in rng.uniform(1.2, 2.0, size=d))
    p = tuple(float(v) for v in rng.uniform(0.0, 1.0, size=d))
    g = tuple(float(v) for v in rng.uniform(0.5, 1.5, size=d))
    if spherical:
        Dd = [float(rng.uniform(1e-3, 5e-2))] * d
    else:
        Dd = [float(v) for v in rng.uniform(1e-3, 5e-2, size=d)]
    u = tuple(float(v) for v in rng.uniform(-0.08, 0.08, size=d)) if advect else (0.0,) * d
    nfree = 2 if d == 2 else 3
    s_free = tuple(float(v) for v in rng.uniform(0.8, 1.9, size=nfree)) if collision == "mrt" else ()
    return Problem(d=d, collision=collision, grid=tuple(int(n) for n in grid), alpha=alpha, p=p,
                   g=g, D=_diag(Dd), u=u, s_free=s_free)


def random_field(rng: np.random.Generator, grid: Sequence[int], walls_zero: bool = True) -> np.ndarray:
    """Smooth positive random field (sum of a few Gaussians) with unit mass."""
    grid = tuple(int(n) for n in grid)
    C = np.zeros(tuple(reversed(grid)))
    for _ in range(3):
        centre = [float(rng.uniform(1, n - 2)) for n in grid]
        sigma = float(rng.uniform(1.0, max(1.5, min(grid) / 5)))
        C += rng.uniform(0.5, 1.5) * gaussian_pulse(grid, sigma, centre)
    C += 1e-3 * rng.uniform(size=C.shape)
    if walls_zero:
        C = zero_walls(C)
    return C / C.sum()
