"""Killed stable-Levy random walk: a Monte-Carlo solution of the FADE with homogeneous
Dirichlet walls, used to pin the FP64 lattice Boltzmann oracle for alpha < 2.

TEST INFRASTRUCTURE ONLY: imported by the tests (and nothing in the product path).

What it computes (Section 3.1 of Cartalade, Younsi & Neel, arXiv:1706.09161):

* Eq. (RW_STABLE): dX = u dt + D' dL, with D'_mumu = (D_mumu g_mu)^(1/alpha_mu) and the
  d components of dL independent;
* Eq. (distri): each component of dL over dt is distributed as
  (-cos(pi alpha_mu / 2) dt)^(1/alpha_mu) S(alpha_mu, beta_mu), beta_mu = 2 p_mu - 1;
* Appendix A, Eqs. (stb)-(stbb): S(alpha, beta) has the characteristic function
  exp(-|k|^alpha (1 - i beta sign(k) tan(pi alpha / 2)));
* the bounded-domain subsection of Section 3.1 (and its appendix): a sample path is
  killed at its first exit from the rectangle; the density of the surviving positions
  solves the FADE with C = 0 on the boundary.  Exits are checked after every increment
  (the paper's criterion: dt small enough that halving it no longer changes the
  histogram).

S(alpha, beta) is drawn from two independent uniforms with the algebraic formula of
Chambers, Mallows & Stuck (1976) in the form given by Weron (1996), valid for
alpha != 1: V = pi (U1 - 1/2), W = -ln U2,
B = arctan(beta tan(pi alpha/2)) / alpha, A = (1 + beta^2 tan^2(pi alpha/2))^(1/(2 alpha)),
S = A sin(alpha (V + B)) / cos(V)^(1/alpha) * (cos(V - alpha (V + B)) / W)^((1-alpha)/alpha).
The uniforms are inputs, so the same draws can be replayed.

Parity of this module is pinned in tests/test_oracle_pins.py: the sampler against the
closed-form characteristic function, the walk against the lattice Boltzmann oracle.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np


def stable_from_uniforms(alpha: float, beta: float, u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """S(alpha, beta) (characteristic function of Appendix A) from uniforms u1, u2 in ]0,1[."""
    if not (0.0 < alpha <= 2.0) or alpha == 1.0 or not (-1.0 <= beta <= 1.0):
        raise ValueError("alpha in ]0,2] \\ {1}, beta in [-1,1]")
    V = math.pi * (np.asarray(u1, dtype=np.float64) - 0.5)
    Wexp = -np.log(np.asarray(u2, dtype=np.float64))
    t = beta * math.tan(math.pi * alpha / 2.0)
    B = math.atan(t) / alpha
    A = (1.0 + t * t) ** (1.0 / (2.0 * alpha))
    return (A * np.sin(alpha * (V + B)) / np.cos(V) ** (1.0 / alpha)
            * (np.cos(V - alpha * (V + B)) / Wexp) ** ((1.0 - alpha) / alpha))


def increment_scale(alpha: float, D: float, g: float, dt: float) -> float:
    """D'_mumu (-cos(pi alpha/2) dt)^(1/alpha), D'_mumu = (D g)^(1/alpha): Eqs. (RW_STABLE), (distri)."""
    return (D * g) ** (1.0 / alpha) * (-math.cos(math.pi * alpha / 2.0) * dt) ** (1.0 / alpha)


def killed_walk(X0: np.ndarray, alpha: Sequence[float], p: Sequence[float], D: Sequence[float],
                g: Sequence[float], u: Sequence[float], lo: Sequence[float], hi: Sequence[float],
                dt: float, nsteps: int, rng: np.random.Generator) -> Tuple[np.ndarray, np.ndarray]:
    """Advance particles X0 (n x d) by nsteps increments of Eq. (RW_STABLE) in the box
    ]lo, hi[; returns (positions, alive), alive False from a path's first exit on."""
    X = np.array(X0, dtype=np.float64, copy=True)
    n, d = X.shape
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    alive = np.all((X > lo) & (X < hi), axis=1)
    for _ in range(nsteps):
        for mu in range(d):
            s = stable_from_uniforms(alpha[mu], 2.0 * p[mu] - 1.0, rng.uniform(size=n), rng.uniform(size=n))
            X[:, mu] += u[mu] * dt + increment_scale(alpha[mu], D[mu], g[mu], dt) * s
        alive &= np.all((X > lo) & (X < hi), axis=1)
    return X, alive
