"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 over all nodes): 1e-12 for the FP64 path; for the FP32
collision forms 1e-5 on the named workloads and, on random cases, the bound
``fp32_tol`` derived from the FP32 arithmetic and the problem's conditioning.  Sizes span several CTA tiles (32x8 in 2-D, 32x4x2 in
3-D) and GEMM tiles (64x64) with ragged tails, plus the minimum grid of 3
nodes per axis.
"""
import dataclasses

import numpy as np
import pytest
import torch

import arith_bounds
from oracle import lbm_oracle as O
from paper_1706_09161_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1706_09161_gb300 import build
    build.build()
    from paper_1706_09161_gb300 import lbm
    return lbm


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fp32_tol(pb, C0, n):
    """Relative-L2 bound for the FP32 forms on random cases: 10x the error that FP32
    arithmetic itself makes on the same problem (problems with F >> C, alpha near 1,
    cancel strongly in the rest population), never below 1e-5."""
    return arith_bounds.bound(pb, C0, n, "fp32")


def oracle_run(pb, C0, n):
    ops = O.Operators(pb)
    f = O.init_populations(ops, torch.tensor(C0))
    for _ in range(n):
        f = O.step(ops, f)
    return f.numpy(), O.concentration(f).numpy()


# (44, 29): n0 % 4 == 0, the FP32 form runs the TMA-fed 2-D march on ragged tiles
GRIDS_2D = [(3, 3), (37, 29), (70, 65), (129, 17), (44, 29)]
# (40, 9, 6) and (44, 21, 37) have n0 % 4 == 0: the FP32 form runs the TMA-fed march
# (ragged x and y tiles, several z chunks for the latter)
GRIDS_3D = [(3, 3, 3), (19, 13, 11), (40, 9, 6), (44, 21, 37)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("grid", GRIDS_2D + GRIDS_3D)
def test_fractional_terms(L, precision, grid):
    """Fractional terms (Section 2.4): F_mu of the initial concentration."""
    rng = np.random.default_rng(len(grid) * 100 + grid[0])
    d = len(grid)
    pb = W.random_problem(rng, d, "mrt", grid)
    C0 = W.random_field(rng, grid)
    ops = O.Operators(pb)
    C = O.concentration(O.init_populations(ops, torch.tensor(C0)))
    F = O.fractional_terms(ops, C)
    with L.Lattice(pb, C0, precision) as lat:
        for mu in range(d):
            got = lat.F(mu)
            assert rel_l2(got, F[mu].numpy()) < (1e-13 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
@pytest.mark.parametrize("grid", GRIDS_2D + GRIDS_3D)
def test_steps_match_oracle(L, precision, collision, grid):
    """Algorithm 1's time step, 12 steps: concentration and populations."""
    rng = np.random.default_rng(7 + len(grid) * 10 + grid[0])
    d = len(grid)
    pb = W.random_problem(rng, d, collision, grid, spherical=(collision == "bgk"))
    C0 = W.random_field(rng, grid)
    n = 12
    f_ref, C_ref = oracle_run(pb, C0, n)
    with L.Lattice(pb, C0, precision) as lat:
        lat.step(n)
        C = lat.C()
        f = lat.f()
    if precision == "fp64":
        tol = TOL["fp64"]
        arith_bounds.assert_close(C, C_ref, tol, tol, f"{grid} {collision} fp64")
    else:
        tol, node_tol, _ = arith_bounds.bounds(pb, C0, n, "fp32", C_ref=C_ref)
        arith_bounds.assert_close(C, C_ref, tol, node_tol, f"{grid} {collision} fp32")
    assert rel_l2(f, f_ref) < tol * 10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonzero_wall_value_and_corners(L, precision):
    """Eq. (Dirichlet_BC) with C_wall != 0: wall nodes hold C_wall, corners included."""
    rng = np.random.default_rng(11)
    for grid in [(21, 10), (11, 9, 7)]:
        pb = dataclasses.replace(W.random_problem(rng, len(grid), "mrt", grid), C_wall=0.03)
        C0 = W.random_field(rng, grid)
        _, C_ref = oracle_run(pb, C0, 9)
        with L.Lattice(pb, C0, precision) as lat:
            lat.step(9)
            C = lat.C()
        if precision == "fp64":
            arith_bounds.assert_close(C, C_ref, TOL["fp64"], TOL["fp64"], f"{grid} fp64")
        else:
            arith_bounds.check_form(C, pb, C0, 9, "fp32", f"{grid} fp32")
        mask = np.ones_like(C, dtype=bool)
        mask[tuple(slice(1, -1) for _ in grid)] = False
        assert np.max(np.abs(C[mask] - 0.03)) < (1e-15 if precision == "fp64" else 1e-8)


def test_config_fp64_bgk_64(L):
    """2-D BGK 64x64 FP64, alpha = 1.7, 200 steps: 1e-12 relative L2 to the oracle."""
    pb, C0, n = W.fp64_bgk_64()
    _, C_ref = oracle_run(pb, C0, n)
    with L.Lattice(pb, C0, "fp64") as lat:
        lat.step(n)
        C = lat.C()
        mass = lat.mass()
    arith_bounds.assert_close(C, C_ref, 1e-12, 1e-12, "fp64_bgk_64")
    assert mass == pytest.approx(float(C_ref.sum()), rel=1e-12)


def test_config_mrt_512_full_size_prefix(L):
    """The 512x512 anisotropic MRT workload at full size, in the launch configuration the
    benchmark times, against the oracle over its first 60 steps (FP32 collision)."""
    pb, C0, _ = W.mrt_aniso_512()
    n = 60
    _, C_ref = oracle_run(pb, C0, n)
    with L.Lattice(pb, C0, "fp32") as lat:
        lat.step(n)
        C = lat.C()
    arith_bounds.assert_close(C, C_ref, 1e-5, 1e-5, "mrt_aniso_512 fp32")


def test_graph_replay_equals_single_steps(L):
    """Graph-captured replay (128-step graphs) and one-step launches give identical results."""
    rng = np.random.default_rng(5)
    pb = W.random_problem(rng, 2, "mrt", (50, 45))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "fp32") as a, L.Lattice(pb, C0, "fp32") as b:
        a.step(263)
        for _ in range(263):
            b.step(1)
        assert np.array_equal(a.C(), b.C())


def test_mrt_equal_rates_equals_bgk_on_gpu(L):
    pb = W.Problem(d=2, collision="bgk", grid=(40, 33), alpha=(1.4, 1.8), p=(0.2, 0.6), g=(1, 1),
                   D=((0.02, 0), (0, 0.02)), u=(0.03, -0.02))
    lam = 0.02 * 3 + 0.5
    pbm = dataclasses.replace(pb, collision="mrt", s_free=(1 / lam, 1 / lam))
    C0 = W.random_field(np.random.default_rng(3), pb.grid)
    with L.Lattice(pb, C0, "fp64") as a, L.Lattice(pbm, C0, "fp64") as b:
        a.step(20)
        b.step(20)
        assert rel_l2(a.C(), b.C()) < 1e-13


def test_mass_reduction(L):
    rng = np.random.default_rng(9)
    pb = W.random_problem(rng, 3, "mrt", (33, 17, 9))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "fp64") as lat:
        lat.step(5)
        C = lat.C()
        assert lat.mass() == pytest.approx(float(C.sum()), rel=1e-14)


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-12), ("fp32", 1e-6), ("bf16split", 1e-6)])
@pytest.mark.parametrize("grid", [(130, 70), (64, 48, 40), (37, 29)])
def test_mass_of_every_step_from_the_collide_stream_partials(L, precision, rel, grid):
    """Algorithm 1's moment: the FP64 mass the collide-stream kernel leaves as block
    partials after each step equals the oracle's sum of C (FP64 path 1e-12, FP32 paths
    1e-6, on a well-conditioned problem: alpha >= 1.5, D >= 0.02, where FP32 C itself stays
    within 1e-6), and the sum of the C the step wrote (same values, summed on the host)."""
    rng = np.random.default_rng(140 + grid[0] + len(grid))
    pb = W.random_problem(rng, len(grid), "mrt", grid)
    d = len(grid)
    pb = dataclasses.replace(pb, alpha=tuple(1.5 + 0.5 * (a - 1.2) / 0.8 for a in pb.alpha),
                             D=tuple(tuple(0.02 + 0.5 * v if i == j else 0.0 for j, v in enumerate(row))
                                     for i, row in enumerate(pb.D)))
    C0 = W.random_field(rng, grid)
    ops = O.Operators(pb)
    f = O.init_populations(ops, torch.tensor(C0))
    with L.Lattice(pb, C0, precision) as lat:
        assert lat.mass() == pytest.approx(float(O.concentration(f).sum()), rel=rel)  # no step yet
        for t in range(1, 31):
            f = O.step(ops, f)
            lat.step(1)
            m = lat.mass()
            assert m == pytest.approx(float(O.concentration(f).sum()), rel=rel), t
            if t % 10 == 0:
                assert m == pytest.approx(float(lat.C().sum()), rel=1e-13), t
        lat.step(200)  # graph replay: the partials of the last replayed step
        assert lat.mass() == pytest.approx(float(lat.C().sum()), rel=1e-13)


def test_mass_of_batch_members_and_fused_step(L):
    probs, fields, _ = W.batch64(nprob=5, sides=(64, 130, 256), seed=33)
    with L.Batch(probs, fields, "bf16split") as b:
        b.step(17)
        for i in range(5):
            assert b.mass(i) == pytest.approx(float(b.C(i).sum()), rel=1e-9), i
    pb, C0, _ = W.mrt_aniso_512()
    with L.Lattice(pb, C0, "bf16split") as lat:
        lat.configure(128, 4, 0, 0, 1)  # the fused step: one partial per collide-stream item
        lat.step(33)
        assert lat.mass() == pytest.approx(float(lat.C().sum()), rel=1e-9)


def test_mass_limit_latches_instability(L):
    """A mass limit turns a run whose mass leaves [-limit, limit] into LBM_ERR_UNSTABLE at
    the next synchronising call (before any value turns non-finite)."""
    pb = W.Problem(d=2, collision="bgk", grid=(48, 24), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((1e-3, 0), (0, 1e-3)), u=(0.6, 0.0))
    with L.Lattice(pb, W.gaussian_pulse(pb.grid, 2.0), "fp32") as lat:
        lat.set_mass_limit(10.0)  # unit initial mass
        lat.step(20)
        assert L.lbm_sync(lat.h) == L.LBM_OK
        lat.step(60)
        m = lat.mass() if L.lbm_sync(lat.h) == L.LBM_OK else None
        # this E4-style run grows fast: by 80 steps its mass is far above 10
        assert m is None
        with pytest.raises(L.LBMError):
            lat.C()
        lat.reset()
        assert L.lbm_sync(lat.h) == L.LBM_OK
        with pytest.raises(L.LBMError):
            lat.set_mass_limit(-1.0)


def test_write_read_populations_and_set_C(L):
    rng = np.random.default_rng(12)
    pb = W.random_problem(rng, 2, "bgk", (23, 19), spherical=True)
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "fp64") as lat:
        f = rng.uniform(0, 0.1, size=(5,) + pb.shape)
        lat.write_f(f)
        assert np.array_equal(lat.f(), f)
        assert np.allclose(lat.C(), f.sum(0), rtol=1e-15, atol=1e-17)
        lat.set_C(C0)
        f_ref, _ = oracle_run(pb, C0, 0)
        assert rel_l2(lat.f(), f_ref) < 1e-14


def test_unstable_run_reports_error(L):
    """BGK at lambda ~ 1/2 with strong advection overflows FP32 within ~150 steps
    (E4-style instability, Section 3.3); the non-finite concentration is latched and
    returned by the next synchronising call."""
    pb = W.Problem(d=2, collision="bgk", grid=(48, 24), alpha=(1.5, 1.5), p=(0.5, 0.5), g=(1, 1),
                   D=((1e-3, 0), (0, 1e-3)), u=(0.6, 0.0))
    with L.Lattice(pb, W.gaussian_pulse(pb.grid, 2.0), "fp32") as lat:
        lat.step(400)
        assert L.lbm_sync(lat.h) == L.LBM_ERR_UNSTABLE
        with pytest.raises(L.LBMError):
            lat.C()
        lat.reset()  # a restart clears the latched error
        assert L.lbm_sync(lat.h) == L.LBM_OK


def test_zero_steps_is_noop(L):
    rng = np.random.default_rng(1)
    pb = W.random_problem(rng, 2, "mrt", (10, 10))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, "fp64") as lat:
        before = lat.f()
        lat.step(0)
        assert np.array_equal(lat.f(), before)


# ---------------------------------------------------------------- checkpoint / resume

@pytest.mark.parametrize("kind", ["fp64", "fp32", "bf16split", "tf32split", "bf16x5split", "bf16x6split"])
def test_save_load_resumes_bit_exact(L, kind):
    """Saving, stepping k times, loading and stepping k times again gives the same f."""
    rng = np.random.default_rng(91)
    pb = W.random_problem(rng, 2, "mrt", (130, 70))
    C0 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C0, kind) as lat:
        lat.step(7)
        state = lat.save()
        lat.step(140)  # graph replay and single launches
        f_a = lat.f()
        lat.load(state)
        lat.step(140)
        f_b = lat.f()
    assert np.array_equal(f_a, f_b)


def test_load_rejects_other_handles(L):
    rng = np.random.default_rng(92)
    pb = W.random_problem(rng, 2, "mrt", (37, 29))
    pb3 = W.random_problem(rng, 3, "mrt", (19, 13, 11))
    with L.Lattice(pb, W.random_field(rng, pb.grid), "fp32") as a, \
            L.Lattice(pb3, W.random_field(rng, pb3.grid), "fp32") as b, \
            L.Lattice(pb, W.random_field(rng, pb.grid), "fp64") as c:
        s = a.save()
        for other in (b, c):
            with pytest.raises(L.LBMError):
                other.load(s)
        with pytest.raises(L.LBMError):
            a.load(s[:-1])  # truncated
        a.load(s)


def test_write_f_refreshes_split_operands(L):
    """write_f on a tensor-core handle feeds the next step's operator the new C."""
    rng = np.random.default_rng(93)
    pb = W.random_problem(rng, 2, "mrt", (130, 70))
    C0 = W.random_field(rng, pb.grid)
    C1 = W.random_field(rng, pb.grid)
    with L.Lattice(pb, C1, "bf16split") as src:
        f1 = src.f()
    with L.Lattice(pb, C0, "bf16split") as lat, L.Lattice(pb, C1, "bf16split") as ref:
        lat.step(3)
        lat.write_f(f1)
        lat.step(5)
        ref.step(5)
        assert np.array_equal(lat.f(), ref.f())


# ---------------------------------------------------------------- FP32 SIMT contraction split

@pytest.mark.parametrize("grid", [(130, 70), (64, 48, 40)])
def test_fp32_contraction_split_matches_oracle(L, grid):
    """Every contraction split of the FP32 SIMT operator (partial sums added by the
    consumers) gives the oracle's F and steps, also when the split changes mid-run."""
    rng = np.random.default_rng(161 + len(grid))
    pb = W.random_problem(rng, len(grid), "mrt", grid)
    C0 = W.random_field(rng, grid)
    ops = O.Operators(pb)
    F = O.fractional_terms(ops, O.concentration(O.init_populations(ops, torch.tensor(C0))))
    n = 6
    C_ref = O.run_C(pb, C0, 2 * n).numpy()
    kbmin = min((s + 31) // 32 for s in grid)
    for ks in (1, 2, 4, 8):
        if ks > kbmin:
            with L.Lattice(pb, C0, "fp32") as lat:
                with pytest.raises(L.LBMError):
                    lat.configure(0, ks)
            continue
        with L.Lattice(pb, C0, "fp32") as lat:
            lat.configure(0, ks)
            for mu in range(len(grid)):
                assert rel_l2(lat.F(mu), F[mu].numpy()) < 1e-6, (ks, mu)
            lat.step(n)
            lat.configure(0, 1 if ks > 1 else min(2, kbmin))
            lat.step(n)
            arith_bounds.check_form(lat.C(), pb, C0, 2 * n, "fp32", f"split {ks}")


@pytest.mark.parametrize("precision", ["fp32", "bf16x6split", "tf32split"])
def test_set_params_equals_a_new_handle(L, precision):
    """lbm_set_params rebuilds weights and collision constants in place: the run equals a new
    handle's bit for bit (also with a coefficient field kept); inadmissible parameters leave
    the handle as it was; a different grid or precision is refused."""
    rng = np.random.default_rng(1201)
    pa = W.random_problem(rng, 2, "mrt", (64, 56))
    pb_ = dataclasses.replace(W.random_problem(rng, 2, "mrt", (64, 56)), s_free=pa.s_free)
    C0 = W.random_field(rng, pa.grid)
    with L.Lattice(pb_, C0, precision) as ref:
        ref.step(30)
        C_b = ref.C()
    with L.Lattice(pa, C0, precision) as ref:
        ref.step(30)
        C_a = ref.C()
    with L.Lattice(pa, C0, precision) as lat:
        lat.step(7)
        lat.set_params(pb_)
        lat.step(30)
        assert np.array_equal(lat.C(), C_b)
        with pytest.raises(L.LBMError):
            lat.set_params(dataclasses.replace(pa, alpha=(2.5, 1.5)))
        lat.set_params(pa)
        lat.step(30)
        assert np.array_equal(lat.C(), C_a)
        with pytest.raises(L.LBMError):
            L.lbm_set_params(lat.h, L.params_from_problem(dataclasses.replace(pa, grid=(64, 48)), precision))
        with pytest.raises(L.LBMError):
            L.lbm_set_params(lat.h, L.params_from_problem(pa, "fp64"))
    u = np.full((2,) + pa.shape, 0.01)
    with L.Lattice(pb_, C0, precision) as ref:
        ref.set_fields(u=u)
        ref.step(20)
        C_bu = ref.C()
    with L.Lattice(pa, C0, precision) as lat:
        lat.set_fields(u=u)
        lat.set_params(pb_)
        lat.step(20)
        assert np.array_equal(lat.C(), C_bu)
