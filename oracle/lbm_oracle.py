"""FP64 CPU oracle of the fractional-ADE lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY.  This module is imported by the tests, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``;
the product path (the CUDA library and its Python binding) never imports,
calls or links it, and it imports nothing from the product.

It is a plain, slow, step-by-step FP64 restatement of the scheme of
Cartalade, Younsi & Neel, "Multiple-Relaxation-Time Lattice Boltzmann scheme
for Fractional Advection-Diffusion Equation" (arXiv:1706.09161), written with
plain PyTorch CPU ops so that the discrete adjoint is available through
autograd.  Every function cites the section / equation it follows:

* lattices D2Q5 / D3Q7, weights, e^2 .......... Section 2.1, Eq. (weights_c), Fig. 1 caption
* trapezoidal product-integration weights ..... Section 2.4, Eqs. (1Dminus_discret), (c+), (c-);
                                                 the differences of powers taken in 40-digit
                                                 decimal arithmetic, then rounded to FP64
* per-axis fractional term F_mu ............... Section 2.4, Eq. (XXminus_discret); Eq. (M2_FADE_3D)
* Caputo-type variant F~ ...................... Section 3.5, Eqs. (Fg2), (PSRLdD-a/b), (Fg22),
                                                 (CoeffA_FADE3DPS)
* equilibrium ................................. Section 2.2, Eqs. (Feq), (CoeffA_FADE3D)
* BGK relaxation time from D .................. Section 2.2, Eq. (Diffusion_Coefficient_3D)
* diagonal D under BGK through h_mu ........... Section 2.2 (end)
* MRT matrices M, Lambda^-1, D <-> lambda ...... Section 2.3, Eqs. (MRT-Coll), (MatrixD2), (MatrixS), (D_ab)
* spatially varying D(x), g(x), u(x) .......... Section 1 (D and g may depend on x), Eq. (Fg) with
                                                 g_mu(x) inside the integrals, Eqs. (MatrixS), (D_ab) with
                                                 lambda_{mu nu}(x), Eq. (Feq) with u(x)
* source term w_i S_c(x, t) dt ................ Section 2.2, Eqs. (LBE_FADE), (LBE_Ket), (MRT-Coll)
* time-dependent, non-homogeneous walls ........ Section 2.5 (C_0 varies with position and time),
                                                 Section 3.4 (Eqs. Def_D_AS, exsolFADE_3D)
* streaming (push) ............................ Section 2.2, Eqs. (LBE_Ket), (Def_Translation)
* Dirichlet walls ............................. Section 2.5, Eq. (Dirichlet_BC)
* time loop ................................... Section 2.5, Algorithm 1

Readings taken where the paper is silent (the same conventions the CUDA path
implements, each written out independently):

* grid = nodes per axis including both wall nodes, n = 0..N, N = grid-1;
* the diagonal l = n of both weight matrices is 1, except at the line's first node
  for W+ (n = 0) and its last node for W- (n = N): there the integral runs over an
  empty interval (Eqs. Def_FracInt, Def_FracIntspe: ]l, x[ with x = l) and is 0 for
  alpha < 2 (at alpha = 2, I^0 is the identity and the entry stays 1);
* a wall node with k unknown incoming populations (edges, corners) gives each
  of them (C_wall - sum of the known populations) / k;
* the initial populations are the equilibrium of the initial concentration;
* BGK with a diagonal, non-spherical D: lambda is set by the largest D_mumu
  and h_mu = D_mumu / max(D) multiplies g_mu;
* MRT: ``s_free`` are relaxation *rates* 1/lambda_k of the free moments;
  lambda_0 (conserved moment) is set to 1, it has no effect;
* a source S_c(x, t) enters the step from t to t + dt at time t, added after the
  collision as w_i S_c dt; the wall values of that step are those of time t + dt
  (the populations being assigned are those of t + dt).  Both are taken in the
  separable form profile(x) exp(rate t), which covers Section 3.4's solution.

Parity of every function here is pinned by the tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, special cases).
"""
from __future__ import annotations

import decimal
import functools
import math
from typing import List, Sequence, Tuple

import torch

DT = torch.float64


# --------------------------------------------------------------------------- lattice

def lattice(d: int) -> Tuple[torch.Tensor, torch.Tensor, float]:
    """Velocity array e (d x Q, columns e_i), weights w (Q) and e^2.

    Section 2.1: D3Q7 has e_0 = 0, e_{1,2} = +-b_1, e_{3,4} = +-b_2,
    e_{5,6} = +-b_3, w_0 = 1/4, w_i = 1/8, e^2 = 1/4; D2Q5 drops e_5, e_6 and
    has w_0 = 1/3, w_i = 1/6, e^2 = 1/3 (Fig. 1 caption).
    """
    if d == 2:
        cols = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]
        w = [1 / 3] + [1 / 6] * 4
        e2 = 1 / 3
    elif d == 3:
        cols = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
        w = [1 / 4] + [1 / 8] * 6
        e2 = 1 / 4
    else:
        raise ValueError("d must be 2 or 3")
    e = torch.tensor(cols, dtype=DT).T.contiguous()
    return e, torch.tensor(w, dtype=DT), e2


def moment_matrix(d: int) -> torch.Tensor:
    """MRT change of basis M, Eq. (MatrixD2) (D3Q7 left, D2Q5 right)."""
    if d == 3:
        rows = [[1, 1, 1, 1, 1, 1, 1],
                [0, 1, -1, 0, 0, 0, 0],
                [0, 0, 0, 1, -1, 0, 0],
                [0, 0, 0, 0, 0, 1, -1],
                [6, -1, -1, -1, -1, -1, -1],
                [0, 2, 2, -1, -1, -1, -1],
                [0, 0, 0, 1, 1, -1, -1]]
    else:
        rows = [[1, 1, 1, 1, 1],
                [0, 1, -1, 0, 0],
                [0, 0, 0, 1, -1],
                [4, -1, -1, -1, -1],
                [0, 1, 1, -1, -1]]
    return torch.tensor(rows, dtype=DT)


# --------------------------------------------------------------------------- discrete fractional integrals

def _as_t(x) -> torch.Tensor:
    return x if isinstance(x, torch.Tensor) else torch.tensor(float(x), dtype=DT)


_LN_INT: List[decimal.Decimal] = []   # ln k, k = 1, 2, ..., in 40-digit decimal arithmetic


@functools.lru_cache(maxsize=256)
def _exact_coefficients(gamma: float, N: int) -> Tuple[Tuple[float, ...], Tuple[float, ...]]:
    """a[k], k = 0..N and b[m], m = 0..N of Eqs. (c+), (c-) (index 0 unused, 0), with every
    power and difference taken in 40-digit decimal arithmetic and the result rounded to FP64.

    The FP64 evaluation of a second difference of k^(g+1) cancels ~2 log10(k) digits; the
    extended precision leaves each coefficient correctly rounded (up to a unit in the last
    place), so the matrices carry no error of their own beyond FP64 rounding.
    """
    ctx = decimal.Context(prec=40)
    while len(_LN_INT) < N + 1:
        _LN_INT.append(ctx.ln(decimal.Decimal(len(_LN_INT) + 1)))
    g = decimal.Decimal(gamma)          # the binary value of gamma, exactly
    s = g + 1
    # powers k^s (k = 0..N+1) and m^g (m = 1..N); 0^s = 0 since s >= 1; integers at g = 0
    if g == 0:
        ps = [decimal.Decimal(k) for k in range(N + 2)]
        pg = [decimal.Decimal(0)] + [decimal.Decimal(1)] * N
    else:
        ps = [decimal.Decimal(0)] + [ctx.exp(ctx.multiply(s, _LN_INT[k - 1])) for k in range(1, N + 2)]
        pg = [decimal.Decimal(0)] + [ctx.exp(ctx.multiply(g, _LN_INT[m - 1])) for m in range(1, N + 1)]
    a = [0.0] + [float(ctx.add(ctx.subtract(ps[k + 1], ctx.multiply(2, ps[k])), ps[k - 1])) for k in range(1, N + 1)]
    b = [0.0] + [float(ctx.add(ctx.subtract(ctx.multiply(s, pg[m]), ps[m]), ps[m - 1])) for m in range(1, N + 1)]
    return tuple(a), tuple(b)


def weight_matrices(gamma, N: int) -> Tuple[torch.Tensor, torch.Tensor]:
    """Coefficient matrices W+[n, l] = c+_{ln}(gamma) (l <= n) and W-[n, l] = c-_{ln}(gamma, N) (l >= n).

    Eqs. (c+) and (c-), Section 2.4, for nodes n, l = 0..N:
      c+_{ln} = (1+g) n^g - n^(g+1) + (n-1)^(g+1)           l = 0
              = (n-l+1)^(g+1) - 2 (n-l)^(g+1) + (n-l-1)^(g+1)  0 < l < n
              = 1                                            l = n
      c-_{ln} = (1+g) (N-n)^g - (N-n)^(g+1) + (N-n-1)^(g+1)  l = N
              = (l-n+1)^(g+1) - 2 (l-n)^(g+1) + (l-n-1)^(g+1)  n < l < N
              = 1                                            l = n
    At n = 0 (c+) and n = N (c-) the integral is over an empty interval: the row is 0
    (Eqs. Def_FracInt, Def_FracIntspe; the end formula there would take (-1)^(g+1)), except
    at g = 0 where I^0 is the identity (Section 1) and the diagonal stays 1.
    ``gamma`` may be a tensor that requires grad.
    """
    g = _as_t(gamma)
    s = g + 1.0
    k = torch.arange(0, N + 2, dtype=DT)
    kc = torch.clamp(k, min=1.0)                      # keep pow's gradient finite at k = 0
    pw = torch.where(k > 0, torch.pow(kc, s), torch.zeros((), dtype=DT))   # k^(g+1), 0^(g+1) = 0
    # interior second differences a[k] = (k+1)^s - 2 k^s + (k-1)^s, k >= 1 (a[0] unused)
    a = torch.zeros(N + 1, dtype=DT)
    if N >= 1:
        a = torch.cat([torch.zeros(1, dtype=DT), pw[2:N + 2] - 2.0 * pw[1:N + 1] + pw[0:N]])
    # end coefficient b[m] = (1+g) m^g - m^(g+1) + (m-1)^(g+1), m >= 1 (b[0] unused)
    m = torch.arange(0, N + 1, dtype=DT)
    mc = torch.clamp(m, min=1.0)
    pw_m = pw[0:N + 1]                                       # m^(g+1)
    pw_m1 = torch.cat([torch.zeros(1, dtype=DT), pw[0:N]])   # (m-1)^(g+1)
    b = torch.where(m > 0, (1.0 + g) * torch.pow(mc, g) - pw_m + pw_m1, torch.zeros((), dtype=DT))
    # values from the extended-precision evaluation, derivatives (autograd) from the FP64
    # expressions above: a + (exact - a) has the exact value and the gradient of a
    a_ex, b_ex = _exact_coefficients(float(g.detach()), N)
    a = a + (torch.tensor(a_ex, dtype=DT) - a).detach()
    b = b + (torch.tensor(b_ex, dtype=DT) - b).detach()

    n_idx = torch.arange(N + 1).view(-1, 1).expand(N + 1, N + 1)
    l_idx = torch.arange(N + 1).view(1, -1).expand(N + 1, N + 1)
    one = torch.ones((), dtype=DT)
    zero = torch.zeros((), dtype=DT)

    a_lo = a[(n_idx - l_idx).clamp(min=0)]
    b_n = b[n_idx]
    # the end node's own entry: 0 (empty interval) for gamma > 0; I^0 = Id at gamma = 0
    end_diag = torch.where(g == 0.0, one, zero)
    Wp = torch.where(l_idx == n_idx, torch.where(n_idx > 0, one, end_diag),
                     torch.where((l_idx == 0) & (n_idx > 0), b_n,
                                 torch.where((l_idx > 0) & (l_idx < n_idx), a_lo, zero)))
    a_up = a[(l_idx - n_idx).clamp(min=0)]
    b_Nn = b[(N - n_idx).clamp(min=0)]
    Wm = torch.where(l_idx == n_idx, torch.where(n_idx < N, one, end_diag),
                     torch.where((l_idx == N) & (n_idx < N), b_Nn,
                                 torch.where((l_idx > n_idx) & (l_idx < N), a_up, zero)))
    return Wp, Wm


def frac_matrix(alpha, p, g, N: int, dx: float = 1.0) -> torch.Tensor:
    """K such that (K c)[n] = p I+^gamma(g c)(n dx) + (1-p) I-^gamma(g c)(n dx), gamma = 2 - alpha.

    Eq. (1Dminus_discret) / (XXminus_discret): I+-^gamma f(n dx) ~ dx^gamma / Gamma(2+gamma)
    * sum_l f(l dx) c+-_{ln}; the fractional term of Eq. (CoeffA_FADE3D) weights the two
    one-sided integrals of g C by p and 1 - p.  ``alpha``, ``p``, ``g`` may be tensors.
    """
    gamma = 2.0 - _as_t(alpha)
    Wp, Wm = weight_matrices(gamma, N)
    scale = _as_t(g) * torch.pow(torch.tensor(float(dx), dtype=DT), gamma) / torch.exp(torch.lgamma(2.0 + gamma))
    p = _as_t(p)
    return scale * (p * Wp + (1.0 - p) * Wm)


def caputo_boundary_terms(alpha, p, g, N: int, dx: float = 1.0) -> torch.Tensor:
    """B such that (B c)[n] = g [p c_0 (n dx)^gamma + (1-p) c_N ((N-n) dx)^gamma] / Gamma(1+gamma).

    Section 3.5, Eqs. (PSRLdD-a/b) and (Fg22): along a line from l = z_+ (node 0) to L = z_-
    (node N), I+^gamma(d/dx f) = d/dx [I+^gamma f - f(l) (x-l)^gamma / Gamma(3-alpha)] and
    likewise for I- with f(L) (L-x)^gamma; gamma = 2 - alpha, Gamma(3-alpha) = Gamma(1+gamma).
    The Caputo-type variant F~ puts the bracket in the equilibrium (Eq. CoeffA_FADE3DPS):
    F~ = (K - B) g c.
    """
    gamma = 2.0 - _as_t(alpha)
    n = torch.arange(N + 1, dtype=DT)
    den = torch.exp(torch.lgamma(1.0 + gamma))
    p = _as_t(p)
    # x^gamma at x = 0 is 0 for gamma > 0 and 1 at gamma = 0 (the bracket f - f(l) of I^0 = Id)
    at0 = torch.where(gamma == 0.0, torch.ones((), dtype=DT), torch.zeros((), dtype=DT))
    left = torch.where(n > 0, torch.pow(torch.clamp(n * dx, min=1e-300), gamma), at0)
    right = torch.where(n < N, torch.pow(torch.clamp((N - n) * dx, min=1e-300), gamma), at0)
    B = torch.zeros(N + 1, N + 1, dtype=DT)
    B[:, 0] = B[:, 0] + _as_t(g) * p * left / den
    B[:, N] = B[:, N] + _as_t(g) * (1.0 - p) * right / den
    return B


def apply_along_axis(K: torch.Tensor, C: torch.Tensor, mu: int) -> torch.Tensor:
    """(K applied along axis mu)[.., n, ..] = sum_l K[n, l] C[.., l, ..]  (Eq. XXminus_discret).

    Axis mu = 0 is x (last array dim), mu = 1 is y, mu = 2 is z.
    """
    dim = C.dim() - 1 - mu
    out = torch.tensordot(K, C, dims=([1], [dim]))   # axis moved to front
    return torch.movedim(out, 0, dim)


# --------------------------------------------------------------------------- problem -> operators

class Operators:
    """All per-problem quantities of Algorithm 1's initialisation, as FP64 tensors.

    Differentiable w.r.t. alpha, p, D (diagonal entries or full tensor) and u when they are
    passed as tensors with requires_grad.
    """

    def __init__(self, pb, alpha=None, p=None, D=None, u=None, g=None, fields=None):
        self.d = d = pb.d
        self.grid = tuple(int(n) for n in pb.grid)
        self.collision = pb.collision
        self.dx, self.dt = float(pb.dx), float(pb.dt)
        self.C_wall = float(pb.C_wall)
        self.e, self.w, self.e2 = lattice(d)
        self.Q = self.e.shape[1]
        self.alpha = _vec(alpha if alpha is not None else pb.alpha, d)
        self.p = _vec(p if p is not None else pb.p, d)
        self.g = _vec(g if g is not None else pb.g, d)
        self.u = _vec(u if u is not None else pb.u, d)
        if D is None:
            Dm = torch.tensor(pb.D, dtype=DT)
        else:
            Dm = _as_t(D) if isinstance(D, torch.Tensor) else torch.tensor(D, dtype=DT)
            if Dm.dim() == 1:
                Dm = torch.diag(Dm)
        self.D = Dm
        self.h = torch.ones(d, dtype=DT)
        self.fields = None
        self.source = None   # (S(x) tensor of the field's shape, rate): S_c(x, t) = S(x) exp(rate t)
        self.walls = None    # (C_w(x) tensor, rate): C_0(x, t) = C_w(x) exp(rate t) on the wall nodes
        if fields:
            self._set_fields(pb, fields)
            return
        self.Omega = self._collision_matrix(pb)
        self.K = [frac_matrix(self.alpha[mu], self.p[mu], self.g[mu] * self.h[mu], self.grid[mu] - 1, self.dx)
                  for mu in range(d)]
        self._caputo(pb)

    def _caputo(self, pb):
        """Section 3.5: with the Caputo-type variant F~ (pb.variant == "caputo") the operator
        along each axis is K - B (caputo_boundary_terms), g (and BGK's h) as in K."""
        self.variant = getattr(pb, "variant", "fg")
        if self.variant == "caputo":
            gfac = [1.0] * self.d if self.fields else [self.g[mu] * self.h[mu] for mu in range(self.d)]
            self.K = [self.K[mu] - caputo_boundary_terms(self.alpha[mu], self.p[mu], gfac[mu], self.grid[mu] - 1,
                                                         self.dx) for mu in range(self.d)]
        elif self.variant != "fg":
            raise ValueError("variant must be 'fg' (Eq. Fg) or 'caputo' (Eq. Fg2)")

    def _set_fields(self, pb, fields):
        """Coefficients that depend on the node (Section 1: D and g may depend on x).

        fields: dict with optional entries (numpy or torch, array order = reversed grid)
          "D": (d, d, *shape) diffusion tensor per node, "g": (d, *shape), "u": (d, *shape);
        an absent entry takes the problem's constant value at every node.
        * Eq. (Fg): F_mu = p I+^gamma(g_mu C) + (1-p) I-^gamma(g_mu C): g_mu(x) multiplies C
          inside the integrals, so K_mu is built with g = 1.
        * Eqs. (MatrixS), (D_ab): Lambda^-1(x) has the flux block D(x) dt/(e^2 dx^2) + Id/2;
          Omega(x) = M^-1 Lambda(x) M with Lambda(x) the inverse of Lambda^-1(x), node by node.
          BGK (Eq. Diffusion_Coefficient_3D with lambda(x)) needs D(x) spherical at every node.
        * Eq. (Feq): the advective part uses u(x).
        """
        d, Q, e2 = self.d, self.Q, self.e2
        shape = tuple(reversed(self.grid))
        ones = torch.ones(shape, dtype=DT)

        def get(name, const):
            v = fields.get(name)
            return torch.as_tensor(v, dtype=DT).clone() if v is not None else const
        self.Dfield = get("D", self.D.reshape(d, d, *([1] * len(shape))) * ones)
        self.gfield = get("g", self.g.reshape(d, *([1] * len(shape))) * ones)
        self.ufield = get("u", self.u.reshape(d, *([1] * len(shape))) * ones)
        ratio = self.dt / (self.dx * self.dx)
        if self.collision == "bgk":
            Dd = torch.stack([self.Dfield[i, i] for i in range(d)])
            off = self.Dfield - torch.diag_embed(Dd.movedim(0, -1)).movedim(-1, 0).movedim(-1, 0)
            if not (bool(torch.all(Dd == Dd[0])) and bool(torch.all(off == 0))):
                raise ValueError("BGK with a D field needs D(x) spherical at every node")
            lam = Dd[0] * ratio / e2 + 0.5
            self.Omega = torch.eye(Q, dtype=DT).reshape(Q, Q, *([1] * len(shape))) / lam
        else:
            s_free = list(pb.s_free)
            lam_inv = torch.zeros(shape + (Q, Q), dtype=DT)
            lam_inv[..., 0, 0] = 1.0
            lam_inv[..., 1:d + 1, 1:d + 1] = self.Dfield.movedim(0, -1).movedim(0, -1) * ratio / e2 \
                + 0.5 * torch.eye(d, dtype=DT)
            for k, sf in enumerate(s_free):
                lam_inv[..., d + 1 + k, d + 1 + k] = 1.0 / float(sf)
            Lam = torch.linalg.inv(lam_inv)
            M = moment_matrix(d)
            Om = torch.linalg.inv(M) @ Lam @ M                     # (*shape, Q, Q)
            self.Omega = Om.movedim(-1, 0).movedim(-1, 0)           # (Q, Q, *shape)
        self.K = [frac_matrix(self.alpha[mu], self.p[mu], 1.0, self.grid[mu] - 1, self.dx) for mu in range(d)]
        self.fields = True
        self._caputo(pb)

    def _collision_matrix(self, pb) -> torch.Tensor:
        """Omega such that the collision is f - Omega (f - feq).

        BGK: Omega = I / lambda with D = e^2 (lambda - 1/2) dx^2 / dt, Eq. (Diffusion_Coefficient_3D).
        MRT: Omega = M^-1 Lambda M, Eq. (MRT-Coll), with Lambda^-1 = diag(lambda_0, lambdabar,
        lambda_{d+1..Q-1}) (Eq. MatrixS) and lambdabar = D dt / (e^2 dx^2) + Id/2 (Eq. D_ab).
        """
        d, Q, e2 = self.d, self.Q, self.e2
        ratio = self.dt / (self.dx * self.dx)
        if self.collision == "bgk":
            Dd = torch.diagonal(self.D)
            if not bool(torch.all(self.D == torch.diag(Dd))):
                raise ValueError("BGK needs a diagonal D")
            Dmax = torch.max(Dd)
            lam = Dmax * ratio / e2 + 0.5
            self.h = Dd / Dmax                       # diagonal non-spherical D (end of Section 2.2)
            self.lam = lam
            return torch.eye(Q, dtype=DT) / lam
        if self.collision != "mrt":
            raise ValueError("collision must be 'bgk' or 'mrt'")
        s_free = list(pb.s_free)
        if len(s_free) != Q - d - 1:
            raise ValueError("MRT needs Q-d-1 free rates")
        lam_inv = torch.zeros(Q, Q, dtype=DT)
        lam_inv[0, 0] = 1.0
        lam_inv[1:d + 1, 1:d + 1] = self.D * ratio / e2 + 0.5 * torch.eye(d, dtype=DT)
        for k, s in enumerate(s_free):
            lam_inv[d + 1 + k, d + 1 + k] = 1.0 / float(s)
        Lam = torch.linalg.inv(lam_inv)
        M = moment_matrix(d)
        return torch.linalg.inv(M) @ Lam @ M


def _vec(x, d) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(DT).reshape(d)
    return torch.tensor([float(v) for v in x], dtype=DT)


# --------------------------------------------------------------------------- the time step

def fractional_terms(ops: Operators, C: torch.Tensor) -> List[torch.Tensor]:
    """F_mu = p_mu I+^{2-alpha_mu}(g_mu C) + (1-p_mu) I-^{2-alpha_mu}(g_mu C), the fractional terms of Algorithm 1's time step."""
    if ops.fields:
        return [apply_along_axis(ops.K[mu], ops.gfield[mu] * C, mu) for mu in range(ops.d)]
    return [apply_along_axis(ops.K[mu], C, mu) for mu in range(ops.d)]


def equilibrium(ops: Operators, C: torch.Tensor, F: Sequence[torch.Tensor]) -> torch.Tensor:
    """|feq> = |A> + (C/e^2)(dt/dx) u_mu |e_mu w>, Eqs. (Feq) and (CoeffA_FADE3D).

    A_0 = C - w_0 sum_mu F_mu,  A_{2mu-1} = A_{2mu} = w_i F_mu.
    """
    Q, d = ops.Q, ops.d
    sumF = sum(F)
    A = [C - ops.w[0] * sumF]
    for mu in range(d):
        A.append(ops.w[2 * mu + 1] * F[mu])
        A.append(ops.w[2 * mu + 2] * F[mu])
    adv_scale = (ops.dt / ops.dx) / ops.e2
    feq = []
    u = ops.ufield if ops.fields else ops.u
    for i in range(Q):
        ue = sum(u[mu] * ops.e[mu, i] for mu in range(d))
        feq.append(A[i] + adv_scale * C * ue * ops.w[i])
    return torch.stack(feq)


def collide(ops: Operators, f: torch.Tensor, feq: torch.Tensor) -> torch.Tensor:
    """Right-hand side of Eq. (LBE_Ket) / (MRT-Coll) without source: f - Omega (f - feq),
    with Omega(x) node by node when the coefficients vary in space."""
    if ops.Omega.dim() > 2:
        return f - torch.einsum("ij...,j...->i...", ops.Omega, f - feq)
    return f - torch.einsum("ij,j...->i...", ops.Omega, f - feq)


def _shift(x: torch.Tensor, dim: int, s: int) -> torch.Tensor:
    """y[.., k + s, ..] = x[.., k, ..]; entries with no source node are 0."""
    y = torch.zeros_like(x)
    n = x.shape[dim]
    src = [slice(None)] * x.dim()
    dst = [slice(None)] * x.dim()
    if s > 0:
        src[dim] = slice(0, n - s)
        dst[dim] = slice(s, n)
    else:
        src[dim] = slice(-s, n)
        dst[dim] = slice(0, n + s)
    y[tuple(dst)] = x[tuple(src)]
    return y


def _axis_of(ops: "Operators", i: int) -> Tuple[int, int]:
    """(mu, sign) of the moving velocity e_i = sign * b_mu."""
    col = ops.e[:, i]
    mu = int(torch.nonzero(col).flatten()[0])
    return mu, int(col[mu])


def unknown_mask(ops: "Operators") -> torch.Tensor:
    """unknown[i, x] is True where x - e_i lies outside the domain (Section 2.5)."""
    shape = tuple(reversed(ops.grid))
    m = torch.zeros((ops.Q,) + shape, dtype=torch.bool)
    for i in range(1, ops.Q):
        mu, s = _axis_of(ops, i)
        dim = len(shape) - 1 - mu
        idx = [slice(None)] * len(shape)
        idx[dim] = 0 if s > 0 else shape[dim] - 1
        m[(i,) + tuple(idx)] = True
    return m


def stream(ops: Operators, fstar: torch.Tensor) -> torch.Tensor:
    """Push translation of Eq. (Def_Translation): f_i(x + e_i dx, t+dt) = f*_i(x, t).

    Populations that leave the domain are dropped; populations whose source
    node lies outside are set to 0 here and assigned by ``dirichlet``.
    """
    out = [fstar[0]]
    for i in range(1, ops.Q):
        mu, s = _axis_of(ops, i)
        out.append(_shift(fstar[i], fstar.dim() - 2 - mu, s))
    return torch.stack(out)


def dirichlet(ops: Operators, f: torch.Tensor, t: float = 0.0) -> torch.Tensor:
    """Eq. (Dirichlet_BC): unknown inward populations f_b = C0 - sum_{i != b} f_i.

    With k > 1 unknowns at a node (edges, corners) each gets (C0 - sum of known)/k.
    C0 is the constant C_wall, or C_w(x) exp(rate t) at time t when the wall values vary
    with position and time (Section 2.5).
    """
    unknown = unknown_mask(ops)
    known_sum = torch.where(unknown, torch.zeros((), dtype=DT), f).sum(0)
    k = unknown.sum(0).to(DT)
    C0 = ops.C_wall
    if ops.walls is not None:
        Cw, rate = ops.walls
        C0 = Cw * math.exp(rate * t)
    fill = (C0 - known_sum) / torch.clamp(k, min=1.0)
    return torch.where(unknown, fill.unsqueeze(0).expand_as(f), f)


def source_term(ops: Operators, t: float) -> torch.Tensor:
    """|w> S_c(x, t) dt of Eqs. (LBE_Ket) / (MRT-Coll), S_c(x, t) = S(x) exp(rate t)."""
    S, rate = ops.source
    St = S * math.exp(rate * t) * ops.dt
    return torch.stack([ops.w[i] * St for i in range(ops.Q)])


def concentration(f: torch.Tensor) -> torch.Tensor:
    """C = <1|f>, the moment of Algorithm 1's time step."""
    return f.sum(0)


def init_populations(ops: Operators, C0: torch.Tensor) -> torch.Tensor:
    """Initial populations: the equilibrium of the initial concentration."""
    return equilibrium(ops, C0, fractional_terms(ops, C0))


def step(ops: Operators, f: torch.Tensor, n: int = 0) -> torch.Tensor:
    """One pass of Algorithm 1's time loop from populations f(t) to f(t+dt),
    t = n dt (the time matters only for a source or wall values that depend on it)."""
    C = concentration(f)
    F = fractional_terms(ops, C)                 # fractional terms
    feq = equilibrium(ops, C, F)                 # equilibrium
    fstar = collide(ops, f, feq)                 # collision
    if ops.source is not None:
        fstar = fstar + source_term(ops, n * ops.dt)
    fnew = stream(ops, fstar)                    # streaming
    fnew = dirichlet(ops, fnew, (n + 1) * ops.dt)  # walls
    return fnew                                  # moment: C = concentration(fnew)


def run_fields_C(pb, C0, nsteps: int, fields) -> torch.Tensor:
    """C after nsteps with spatially varying coefficients (see Operators._set_fields)."""
    return concentration(run(pb, C0, nsteps, Operators(pb, fields=fields)))


def run(pb, C0, nsteps: int, ops: Operators = None) -> torch.Tensor:
    """Populations after ``nsteps`` steps from f(0) = feq(C0)."""
    ops = ops or Operators(pb)
    f = init_populations(ops, _field(C0))
    for n in range(nsteps):
        f = step(ops, f, n)
    return f


def with_source_and_walls(ops: Operators, source=None, walls=None) -> Operators:
    """Attach S_c(x, t) = S(x) exp(rate t) (source = (S, rate)) and wall values
    C_w(x) exp(rate t) (walls = (C_w, rate)); arrays in the field's shape."""
    if source is not None:
        ops.source = (torch.as_tensor(source[0], dtype=DT), float(source[1]))
    if walls is not None:
        ops.walls = (torch.as_tensor(walls[0], dtype=DT), float(walls[1]))
    return ops


def run_C(pb, C0, nsteps: int) -> torch.Tensor:
    return concentration(run(pb, C0, nsteps))


def _field(C0) -> torch.Tensor:
    if isinstance(C0, torch.Tensor):
        return C0.to(DT)
    return torch.as_tensor(C0, dtype=DT)


# --------------------------------------------------------------------------- inverse problem (adjoint)

def snapshot_loss(pb, C0, snap_steps: Sequence[int], obs: torch.Tensor, alpha, p, Ddiag, u) -> torch.Tensor:
    """L = sum_k sum_x (C(x, t_k) - obs_k(x))^2 for the scheme run with (alpha, p, diag D, u).

    The gradient of this FP64 loss by autograd is the exact discrete adjoint of the
    scheme (every stage above is differentiable in the parameters).
    """
    ops = Operators(pb, alpha=alpha, p=p, D=torch.diag(Ddiag), u=u)
    f = init_populations(ops, _field(C0))
    loss = torch.zeros((), dtype=DT)
    t = 0
    for k, ts in enumerate(snap_steps):
        while t < ts:
            f = step(ops, f)
            t += 1
        r = concentration(f) - obs[k]
        loss = loss + (r * r).sum()
    return loss


def loss_and_grad(pb, C0, snap_steps, obs) -> Tuple[float, torch.Tensor]:
    """Loss and its gradient w.r.t. theta = [alpha_1..d, p_1..d, D_11..D_dd, u_1..d] (FP64 autograd)."""
    d = pb.d
    alpha = torch.tensor(pb.alpha, dtype=DT, requires_grad=True)
    p = torch.tensor(pb.p, dtype=DT, requires_grad=True)
    Dd = torch.tensor([pb.D[i][i] for i in range(d)], dtype=DT, requires_grad=True)
    u = torch.tensor(pb.u, dtype=DT, requires_grad=True)
    obs_t = torch.as_tensor(obs, dtype=DT)
    loss = snapshot_loss(pb, C0, snap_steps, obs_t, alpha, p, Dd, u)
    loss.backward()
    grad = torch.cat([alpha.grad, p.grad, Dd.grad, u.grad])
    return float(loss.detach()), grad
