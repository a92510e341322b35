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
cos V is evaluated as sin(pi (1/2 - |U1 - 1/2|)), the same value, so that it keeps its
relative accuracy as V -> +-pi/2 (where the FP64 rounding of pi (U1 - 1/2) would dominate).
The uniforms are inputs, so the same draws can be replayed.

For draws shared with another implementation the uniforms come from Philox4x32-10, the
counter-based generator of Salmon, Moraes, Dror & Shaw ("Parallel random numbers: as easy
as 1, 2, 3", SC 2011), written here from its definition: ten rounds on a 4 x 32-bit
counter with a 2 x 32-bit key; a round multiplies counter words 0 and 2 by 0xD2511F53 and
0xCD9E8D57 (64-bit products split into high and low halves), xors the high halves with
counter words 1 and 3 and the key, and permutes; the key is bumped by (0x9E3779B9,
0xBB67AE85) between rounds.  Counter of particle i, step n, call c: (i mod 2^32,
i div 2^32, n, c), key = (seed mod 2^32, seed div 2^32); call c = 0 serves axes 0 and 1,
c = 1 axis 2; axis a takes output words 2(a mod 2) and 2(a mod 2) + 1 as (U1, U2), each
mapped to ]0,1[ by (o + 1/2) 2^-32 (bits = 32) or, with 23 bits, ((o >> 9) + 1/2) 2^-23
(exactly representable in FP32, as are U - 1/2 and 1 - U).

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
    v = np.asarray(u1, dtype=np.float64) - 0.5
    V = math.pi * v
    cosV = np.sin(math.pi * (0.5 - np.abs(v)))
    Wexp = -np.log(np.asarray(u2, dtype=np.float64))
    t = beta * math.tan(math.pi * alpha / 2.0)
    B = math.atan(t) / alpha
    A = (1.0 + t * t) ** (1.0 / (2.0 * alpha))
    return (A * np.sin(alpha * (V + B)) / cosV ** (1.0 / alpha)
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


# --------------------------------------------------------------------------- Philox4x32-10

_PHILOX_M = (0xD2511F53, 0xCD9E8D57)
_PHILOX_W = (0x9E3779B9, 0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of 32-bit counter words (any shape, broadcast) and key words;
    returns the four 32-bit output words as uint64 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3)]
    k = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (k0, k1)]
    for r in range(10):
        p0 = np.uint64(_PHILOX_M[0]) * c[0]
        p1 = np.uint64(_PHILOX_M[1]) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [(hi1 ^ c[1] ^ k[0]) & _MASK32, lo1, (hi0 ^ c[3] ^ k[1]) & _MASK32, lo0]
        if r < 9:
            k = [(k[0] + np.uint64(_PHILOX_W[0])) & _MASK32, (k[1] + np.uint64(_PHILOX_W[1])) & _MASK32]
    return c


def philox_uniforms(particles: np.ndarray, step: int, axis: int, seed: int, bits: int = 32):
    """(U1, U2) of `axis` for the given particle indices at absolute step `step`."""
    i = np.asarray(particles, dtype=np.uint64)
    call = axis // 2
    out = philox4x32_10(i & _MASK32, i >> np.uint64(32), np.uint64(step), np.uint64(call),
                        np.uint64(seed) & _MASK32, np.uint64(seed) >> np.uint64(32))
    o1, o2 = out[2 * (axis % 2)], out[2 * (axis % 2) + 1]
    if bits == 23:
        return ((o1 >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23, \
               ((o2 >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23
    if bits != 32:
        raise ValueError("bits must be 32 or 23")
    return (o1.astype(np.float64) + 0.5) * 2.0 ** -32, (o2.astype(np.float64) + 0.5) * 2.0 ** -32


def killed_walk_philox(X0: np.ndarray, alive0: np.ndarray, alpha: Sequence[float], p: Sequence[float],
                       D: Sequence[float], g: Sequence[float], u: Sequence[float], lo: Sequence[float],
                       hi: Sequence[float], dt: float, seed: int, step0: int, nsteps: int, bits: int = 32
                       ) -> Tuple[np.ndarray, np.ndarray]:
    """As killed_walk, with the Philox uniforms of particle i = 0..n-1 at steps step0 ..
    step0 + nsteps - 1 (X0: n x d; alive0: the paths still alive at step0).  A killed path
    keeps the position at which it left the box."""
    X = np.array(X0, dtype=np.float64, copy=True)
    n, d = X.shape
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    alive = np.array(alive0, dtype=bool, copy=True)
    idx = np.arange(n, dtype=np.uint64)
    for j in range(nsteps):
        Y = X.copy()
        for mu in range(d):
            u1, u2 = philox_uniforms(idx, step0 + j, mu, seed, bits)
            s = stable_from_uniforms(alpha[mu], 2.0 * p[mu] - 1.0, u1, u2)
            Y[:, mu] += u[mu] * dt + increment_scale(alpha[mu], D[mu], g[mu], dt) * s
        X = np.where(alive[:, None], Y, X)
        alive &= np.all((X > lo) & (X < hi), axis=1)
    return X, alive
