"""GPU parity of the tensor-core (tcgen05) split-precision forms against the FP64 oracle.

The fractional operator runs as a split-precision GEMM (bf16 or tf32 hi+lo parts,
three products; bf16 weights in three parts and C in two, five products; both in three
bf16 parts, six products; FP32 accumulation over short chains).  Bounds: the operator
alone is compared with a fixed relative-L2 bound from the split's rounding (bf16: 2^-16
per part, tf32: 2^-22; the five-product form is limited by C's two parts, the six-product
form carries FP32's precision); whole steps use ``arith_bounds.bounds``: 6x the error the
same arithmetic makes when re-run on the CPU, never below 1e-5, as a relative L2 and node
by node.
Sizes cover one and several 128-line / 64-column tiles, ragged tails, the
minimum grid, and the 512x512 workload; the two largest 3-D grids have enough
tiles for the persistent kernel (one with F rows that TMA cannot store, n0 % 4 != 0).
"""
import numpy as np
import pytest
import torch

import arith_bounds
from oracle import lbm_oracle as O
from paper_1706_09161_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F_TOL = {"bf16split": 4e-5, "tf32split": 2e-6, "bf16x5split": 2e-5, "bf16x6split": 2e-6}


def f_tol(kind: str, side: int) -> float:
    """Relative-L2 bound of the split operator along a line of `side` nodes.

    The fixed part covers the split itself (the dropped lo*lo product and the
    rounding of the parts); the FP32 accumulation of `side` non-negative products
    adds about sqrt(side) roundings of up to 2^-23 each (tensor-core accumulation is
    not assumed to round to nearest), counted twice.
    """
    return max(F_TOL[kind], 2.0 * np.sqrt(side) * 2.0 ** -23)
KINDS = ["bf16split", "tf32split", "bf16x5split", "bf16x6split"]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1706_09161_gb300 import build
    build.build()
    from paper_1706_09161_gb300 import lbm
    return lbm


rel_l2 = arith_bounds.rel_l2

GRIDS = [(3, 3), (37, 29), (130, 70), (200, 131), (19, 13, 11), (40, 9, 6), (131, 20, 9), (256, 64, 64),
         (130, 129, 70)]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("grid", GRIDS)
def test_tc_fractional_terms(L, kind, grid):
    """Fractional terms (Section 2.4) on the tensor cores, every axis."""
    rng = np.random.default_rng(31 + grid[0] + len(grid))
    d = len(grid)
    pb = W.random_problem(rng, d, "mrt", grid)
    C0 = W.random_field(rng, grid)
    ops = O.Operators(pb)
    C = O.concentration(O.init_populations(ops, torch.tensor(C0)))
    F = O.fractional_terms(ops, C)
    with L.Lattice(pb, C0, kind) as lat:
        for mu in range(d):
            assert rel_l2(lat.F(mu), F[mu].numpy()) < f_tol(kind, grid[mu]), f"axis {mu}"


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("grid", [(37, 29), (130, 70), (19, 13, 11), (130, 129, 70), (44, 21, 37)])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
def test_tc_steps_match_oracle(L, kind, grid, collision):
    rng = np.random.default_rng(53 + grid[0])
    pb = W.random_problem(rng, len(grid), collision, grid, spherical=(collision == "bgk"))
    C0 = W.random_field(rng, grid)
    n = 12
    C_ref = O.run_C(pb, C0, n).numpy()
    with L.Lattice(pb, C0, kind) as lat:
        lat.step(n)
        C = lat.C()
    l2_tol, node_tol, _ = arith_bounds.bounds(pb, C0, n, kind, C_ref=C_ref)
    arith_bounds.assert_close(C, C_ref, l2_tol, node_tol, f"{grid} {collision} {kind}")


@pytest.mark.parametrize("kind", KINDS)
def test_tc_config_mrt_512_full_size(L, kind):
    """512x512 anisotropic MRT workload, full size, the benchmark's launch configuration,
    first 60 steps against the oracle."""
    pb, C0, _ = W.mrt_aniso_512()
    n = 60
    C_ref = O.run_C(pb, C0, n).numpy()
    with L.Lattice(pb, C0, kind) as lat:
        lat.step(n)
        C = lat.C()
    l2_tol, node_tol, _ = arith_bounds.bounds(pb, C0, n, kind, C_ref=C_ref)
    arith_bounds.assert_close(C, C_ref, l2_tol, node_tol, f"mrt_aniso_512 {kind}")


def test_tc_config_mrt3d_256_full_size(L):
    """256^3 D3Q7 MRT workload at full size (bf16 split), first 2 steps against the oracle."""
    pb, C0, _ = W.mrt3d_256()
    n = 2
    C_ref = O.run_C(pb, C0, n).numpy()
    with L.Lattice(pb, C0, "bf16split") as lat:
        lat.step(n)
        C = lat.C()
        assert rel_l2(C, C_ref) < 1e-5
        assert lat.mass() == pytest.approx(float(C_ref.sum()), rel=1e-5)


def test_tc_graph_replay_deterministic(L):
    rng = np.random.default_rng(77)
    pb = W.random_problem(rng, 2, "mrt", (150, 140))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "bf16split") as a, L.Lattice(pb, C0, "bf16split") as b:
        a.step(135)  # one 128-step graph replay and single launches
        for _ in range(135):
            b.step(1)
        assert np.array_equal(a.C(), b.C())
        assert L.lbm_sync(a.h) == 0


def test_tf32split_config_mrt3d_256_full_size(L):
    """The 256^3 workload with the tf32 split (its stated form), first 2 steps."""
    pb, C0, _ = W.mrt3d_256()
    C_ref = O.run_C(pb, C0, 2).numpy()
    with L.Lattice(pb, C0, "tf32split") as lat:
        lat.step(2)
        assert rel_l2(lat.C(), C_ref) < 1e-5


# ---------------------------------------------------------------- launch configurations

def _plans(L, pb, kind):
    """Every operator plan lbm_autotune may pick for this problem."""
    BK = 32 if kind == "tf32split" else 64
    five = kind in ("bf16x5split", "bf16x6split")  # three weight parts: 64- or 128-column tiles only
    kbmin = min((n + BK - 1) // BK for n in pb.grid)
    out = []
    for bn in (64, 128, 256):
        for ks in (1, 2, 4, 8):
            if (bn == 256 and (ks != 1 or five)) or ks > kbmin:
                continue
            out.append((bn, ks, 0))
    out.append((128, 1, 1))
    if not five:
        out.append((256, 1, 1))
    return out


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("grid", [(130, 70), (200, 131), (44, 21, 37), (40, 9, 6)])
def test_every_operator_plan_matches_oracle(L, kind, grid):
    """Each tile width / contraction split / persistent choice gives the oracle's F."""
    rng = np.random.default_rng(71 + grid[0] + len(grid))
    d = len(grid)
    pb = W.random_problem(rng, d, "mrt", grid)
    C0 = W.random_field(rng, grid)
    ops = O.Operators(pb)
    F = O.fractional_terms(ops, O.concentration(O.init_populations(ops, torch.tensor(C0))))
    with L.Lattice(pb, C0, kind) as lat:
        for bn, ks, persist in _plans(L, pb, kind):
            lat.configure(bn, ks, persist)
            for mu in range(d):
                assert rel_l2(lat.F(mu), F[mu].numpy()) < f_tol(kind, grid[mu]), (bn, ks, persist, mu)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("grid", [(130, 70), (44, 21, 37)])
def test_autotune_restores_state_and_keeps_parity(L, kind, grid):
    rng = np.random.default_rng(81 + grid[0])
    pb = W.random_problem(rng, len(grid), "mrt", grid)
    C0 = W.random_field(rng, grid)
    n = 12
    C_ref = O.run_C(pb, C0, n).numpy()
    with L.Lattice(pb, C0, kind) as lat:
        lat.step(4)
        f0 = lat.f()
        desc = lat.autotune(8)
        assert desc
        assert np.array_equal(lat.f(), f0)
        lat.step(n - 4)
        C = lat.C()
    l2_tol, node_tol, _ = arith_bounds.bounds(pb, C0, n, kind, C_ref=C_ref)
    arith_bounds.assert_close(C, C_ref, l2_tol, node_tol, f"autotuned {kind}")


# ---------------------------------------------------------------- fused step (one cooperative launch)

FUSED_PLANS = [(64, 2), (64, 4), (128, 2), (128, 4)]


@pytest.mark.parametrize("grid", [(200, 132), (44, 29), (512, 512)])
@pytest.mark.parametrize("plan", FUSED_PLANS)
def test_fused_step_equals_two_kernel_step(L, grid, plan):
    """The fused step does the two-kernel step's arithmetic: identical populations,
    including odd step counts (buffer parity inside the launch)."""
    bn, ks = plan
    rng = np.random.default_rng(97 + grid[0])
    pb = W.random_problem(rng, 2, "mrt", grid)
    C0 = W.random_field(rng, grid)
    BK = 64
    if ks > min((n + BK - 1) // BK for n in grid):
        pytest.skip("split larger than the contraction blocks")
    with L.Lattice(pb, C0, "bf16split") as a, L.Lattice(pb, C0, "bf16split") as b:
        a.configure(bn, ks, 0, 0, 0)
        b.configure(bn, ks, 0, 0, 1)
        for n in (7, 33):
            a.step(n)
            b.step(n)
            assert np.array_equal(a.f(), b.f()), (plan, n)
        a.sync()
        b.sync()


def test_fused_step_matches_oracle_full_size(L):
    pb, C0, _ = W.mrt_aniso_512()
    n = 60
    C_ref = O.run_C(pb, C0, n).numpy()
    with L.Lattice(pb, C0, "bf16split") as lat:
        lat.configure(128, 4, 0, 0, 1)
        lat.step(n)
        C = lat.C()
    l2_tol, node_tol, _ = arith_bounds.bounds(pb, C0, n, "bf16split", C_ref=C_ref)
    arith_bounds.assert_close(C, C_ref, l2_tol, node_tol, "fused step")


def test_configure_rejects_uncovered_plans(L):
    rng = np.random.default_rng(99)
    pb = W.random_problem(rng, 2, "mrt", (130, 70))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "bf16split") as lat:
        for bn, ks, persist, fused in [(96, 1, 0, 0), (128, 3, 0, 0), (256, 2, 0, 0), (64, 1, 1, 0),
                                       (128, 16, 0, 0), (128, 2, 0, 1)]:
            # (128, 2, fused): 130 % 4 != 0, no TMA window for the fused step
            with pytest.raises(L.LBMError):
                lat.configure(bn, ks, persist, 0, fused)
        lat.configure(128, 1, 0, 0, 0)  # a covered plan still applies afterwards
        F = lat.F(0)
        assert np.isfinite(F).all()
    with L.Lattice(pb, C0, "fp32") as lat:
        with pytest.raises(L.LBMError):
            lat.configure(128, 1, 0, 0, 0)  # no tensor-core operator
        lat.configure(0, 0, 0, 3, 0)       # a collide-stream chunk is fine
        lat.step(2)


# ---------------------------------------------------------------- tf32 transposed operands

def _step_resplit(lat, n):
    """n steps, re-splitting C from the populations after each one (lbm_load rebuilds
    every operand copy of C): the reference for operand copies written by the march."""
    for _ in range(n):
        lat.step(1)
        lat.load(lat.save())


@pytest.mark.parametrize("grid", [(44, 21, 37), (64, 70, 66), (64, 70), (96, 45)])
def test_tf32_transposed_operands_written_by_the_march(L, grid):
    """The TMA-fed marches write the y- (and z-) contiguous tf32 copies of C themselves.
    Stepping on them is identical, bit for bit, to stepping on copies rebuilt from C
    after every step, for every chunking of the march (z chunks per tile column, or tile
    rows per block; aligned or not to the four-plane groups of the z copy)."""
    rng = np.random.default_rng(113 + grid[0] + len(grid))
    pb = W.random_problem(rng, len(grid), "mrt", grid)
    C0 = W.random_field(rng, grid)
    n = 9
    with L.Lattice(pb, C0, "tf32split") as ref:
        ref.configure(128, 1, 0, 0, 0)
        _step_resplit(ref, n)
        f_ref = ref.f()
    for chunk in (0, 1, 2, 3, 5):
        with L.Lattice(pb, C0, "tf32split") as lat:
            lat.configure(128, 1, 0, chunk, 0)
            lat.step(n)
            assert np.array_equal(lat.f(), f_ref), chunk
            C = lat.C()
    C_ref = O.run_C(pb, C0, n).numpy()
    assert rel_l2(C, C_ref) < arith_bounds.bound(pb, C0, n, "tf32split")


def test_tf32_plan_switch_keeps_operands_current(L):
    """3-D: a contraction split moves the step between the TMA-fed march (which writes
    the transposed copies) and the plain march (copies rebuilt before the operator);
    switching plans mid-run leaves no stale copy."""
    grid = (64, 70, 66)
    rng = np.random.default_rng(127)
    pb = W.random_problem(rng, 3, "mrt", grid)
    C0 = W.random_field(rng, grid)
    plans = [(128, 2), (128, 1), (128, 2), (128, 1)]
    with L.Lattice(pb, C0, "tf32split") as a, L.Lattice(pb, C0, "tf32split") as b:
        for bn, ks in plans:
            a.configure(bn, ks, 0, 0, 0)
            b.configure(bn, ks, 0, 0, 0)
            a.step(3)
            _step_resplit(b, 3)
            assert np.array_equal(a.f(), b.f()), (bn, ks)
        C = a.C()
    C_ref = O.run_C(pb, C0, 3 * len(plans)).numpy()
    assert rel_l2(C, C_ref) < arith_bounds.bound(pb, C0, 3 * len(plans), "tf32split")


# ---------------------------------------------------------------- five-product bf16 form

def test_bf16x5_rejects_plans_it_does_not_cover(L):
    rng = np.random.default_rng(131)
    pb = W.random_problem(rng, 2, "mrt", (520, 136))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "bf16x5split") as lat:
        for bn, ks, persist in [(256, 1, 0), (256, 1, 1), (64, 1, 1)]:
            with pytest.raises(L.LBMError):
                lat.configure(bn, ks, persist, 0, 0)
        with pytest.raises(L.LBMError):
            lat.configure(128, 2, 0, 0, 1)  # no fused step for this form
        for bn, ks, persist in [(64, 2, 0), (128, 1, 1)]:
            lat.configure(bn, ks, persist, 0, 0)
            F = O.fractional_terms(O.Operators(pb), torch.tensor(lat.C()))
            assert rel_l2(lat.F(1), F[1].numpy()) < f_tol("bf16x5split", pb.grid[1]), (bn, ks, persist)


@pytest.mark.parametrize("kind", ["bf16split", "bf16x5split", "bf16x6split"])
def test_batch_forms_match_single_problem_handles(L, kind):
    """Grouped launches (persistent operator over every member's tiles, accumulator
    regions, three weight parts for the five-product form) give the populations of one
    persistent-plan handle per problem, bit for bit."""
    probs, fields, _ = W.batch64(nprob=4, sides=(128, 256, 384), seed=23)
    with L.Batch(probs, fields, kind) as b:
        b.step(21)
        got = [b.C(i) for i in range(len(probs))]
    for i, (pb, C0) in enumerate(zip(probs, fields)):
        with L.Lattice(pb, C0, kind) as lat:
            lat.configure(128, 1, 1)
            lat.reset()
            lat.step(21)
            assert np.array_equal(lat.C(), got[i]), i
