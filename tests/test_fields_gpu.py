"""GPU parity of the coefficients that vary in space (lbm_set_fields) against the FP64
oracle's field form: D(x) (with off-diagonal entries under MRT, spherical under BGK),
g(x) inside the integrals, u(x) in the equilibrium (Section 1; Eqs. Fg, MatrixS, D_ab,
Feq with x-dependent coefficients).  FP64: 1e-12 relative L2 and node by node; FP32: 6x
the error of the same FP32 arithmetic re-run on the CPU, never below 1e-5."""
import dataclasses
import functools

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


def _case(coll, grid, seed):
    rng = np.random.default_rng(seed)
    pb = W.random_problem(rng, len(grid), coll, grid, spherical=(coll == "bgk"))
    pb = dataclasses.replace(pb, alpha=tuple(1.5 + 0.5 * (a - 1.2) / 0.8 for a in pb.alpha))
    fields = W.smooth_fields(rng, grid, coll, D0=0.03, g_amp=0.2, u_amp=0.03)
    return pb, W.random_field(rng, grid), fields


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("coll", ["mrt", "bgk"])
@pytest.mark.parametrize("grid", [(37, 29), (70, 65), (19, 13, 11), (40, 21, 19)])
def test_fields_match_oracle(L, precision, coll, grid):
    pb, C0, fields = _case(coll, grid, 900 + grid[0] + len(grid))
    n = 12
    C_ref = O.run_fields_C(pb, C0, n, fields).numpy()
    with L.Lattice(pb, C0, precision) as lat:
        lat.set_fields(**fields)
        lat.step(n)
        C = lat.C()
        assert lat.mass() == pytest.approx(float(C.sum()), rel=1e-13)
    if precision == "fp64":
        arith_bounds.assert_close(C, C_ref, 1e-12, 1e-12, f"fields {grid} {coll} fp64")
    else:
        l2, node, _ = arith_bounds.bounds(pb, C0, n, "fp32", C_ref=C_ref, fields=fields)
        arith_bounds.assert_close(C, C_ref, l2, node, f"fields {grid} {coll} fp32")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fields_fractional_terms_and_graph_replay(L, precision):
    """F_mu of the initial C with g(x) inside the integrals; 140 steps by graph replay equal
    140 single launches bit for bit."""
    pb, C0, fields = _case("mrt", (70, 65), 951)
    ops = O.Operators(pb, fields=fields)
    F = O.fractional_terms(ops, O.concentration(O.init_populations(ops, torch.tensor(C0))))
    with L.Lattice(pb, C0, precision) as a, L.Lattice(pb, C0, precision) as b:
        a.set_fields(**fields)
        b.set_fields(**fields)
        for mu in range(2):
            assert arith_bounds.rel_l2(a.F(mu), F[mu].numpy()) < (1e-13 if precision == "fp64" else 1e-6)
        a.step(140)
        for _ in range(140):
            b.step(1)
        assert np.array_equal(a.f(), b.f())


def test_constant_fields_and_switching_back(L):
    """Fields equal to the constants give the constant-coefficient run (FP64, to rounding);
    all-NULL returns to the constant path exactly."""
    rng = np.random.default_rng(961)
    pb = W.random_problem(rng, 2, "mrt", (64, 48))
    C0 = W.random_field(rng, pb.grid)
    shape = pb.shape
    ones = np.ones(shape)
    const = {"D": np.array(pb.D).reshape(2, 2, 1, 1) * ones, "g": np.array(pb.g).reshape(2, 1, 1) * ones,
             "u": np.array(pb.u).reshape(2, 1, 1) * ones}
    with L.Lattice(pb, C0, "fp64") as a, L.Lattice(pb, C0, "fp64") as b:
        a.step(20)
        b.set_fields(**const)
        b.step(20)
        arith_bounds.assert_close(b.C(), a.C(), 1e-13, 1e-13, "constant fields")
        b.set_fields()
        b.step(20)
        a.reset()
        a.step(20)
        assert np.array_equal(a.C(), b.C())


def test_piecewise_constant_regions(L):
    """Two regions of different D, g, u (alpha = 2) against the oracle (FP64 1e-12)."""
    nx, ny = 128, 64
    pb = W.Problem(d=2, collision="mrt", grid=(nx, ny), alpha=(2.0, 1.7), p=(0.5, 0.3), g=(1, 1),
                   D=((0.03, 0), (0, 0.03)), u=(0.0, 0.0), s_free=(1.1, 1.3))
    right = (np.arange(nx) >= nx // 2)[None, :] * np.ones((ny, 1), dtype=bool)
    D = np.zeros((2, 2, ny, nx))
    D[0, 0] = np.where(right, 0.02, 0.04)
    D[1, 1] = np.where(right, 0.05, 0.02)
    fields = {"D": D, "g": np.stack([np.where(right, 1.5, 1.0), np.where(right, 1.0, 1.5)]),
              "u": np.stack([np.where(right, -0.02, 0.03), np.where(right, 0.03, -0.02)])}
    C0 = W.random_field(np.random.default_rng(971), pb.grid)
    C_ref = O.run_fields_C(pb, C0, 60, fields).numpy()
    with L.Lattice(pb, C0, "fp64") as lat:
        lat.set_fields(**fields)
        lat.step(60)
        arith_bounds.assert_close(lat.C(), C_ref, 1e-12, 1e-12, "two regions")


@pytest.mark.parametrize("form", ["bf16x6split", "bf16x5split", "bf16split", "tf32split"])
@pytest.mark.parametrize("grid", [(70, 65), (40, 21, 19)])
def test_fields_tensor_core_forms(L, form, grid):
    """D(x), u(x) and g(x) (operands g_mu(x) C per axis, K_mu without g: bf16 parts, or for
    tf32 the FP32 product split into hi + lo on chip) with the tensor-core operator.  Within
    6x the same arithmetic re-run on the CPU, the fused mass equal to the sum of C."""
    pb, C0, fields = _case("mrt", grid, 960 + grid[0] + len(grid))
    n = 12
    C_ref = O.run_fields_C(pb, C0, n, fields).numpy()
    with L.Lattice(pb, C0, form) as lat:
        lat.set_fields(**fields)
        lat.step(n)
        C = lat.C()
        assert lat.mass() == pytest.approx(float(C.sum()), rel=1e-13)
    l2, node, _ = arith_bounds.bounds(pb, C0, n, form, C_ref=C_ref, fields=fields)
    arith_bounds.assert_close(C, C_ref, l2, node, f"fields {grid} {form}")


def test_fields_reject_invalid_input(L):
    rng = np.random.default_rng(981)
    pb = W.random_problem(rng, 2, "bgk", (30, 20), spherical=True)
    C0 = W.random_field(rng, pb.grid)
    f = W.smooth_fields(rng, pb.grid, "mrt", 0.03)  # not spherical
    with L.Lattice(pb, C0, "fp32") as lat:
        with pytest.raises(L.LBMError):
            lat.set_fields(D=f["D"])
        bad = np.array(f["g"])
        bad[0, 3, 4] = 0.0
        with pytest.raises(L.LBMError):
            lat.set_fields(g=bad)
        lat.set_fields(g=f["g"])  # g alone is fine under BGK with a spherical constant D
        with pytest.raises(L.LBMError) as ei:
            lat.grad([2], np.zeros((1,) + pb.shape), 1)
        assert ei.value.code == L.LBM_ENOTSUP
    pbm = W.random_problem(rng, 2, "mrt", (30, 20))
    D = W.smooth_fields(rng, pbm.grid, "mrt", 0.03)["D"]
    D[0, 1, 5, 5] = D[1, 0, 5, 5] = 10.0  # lambdabar not positive definite there
    with L.Lattice(pbm, C0, "fp64") as lat:
        with pytest.raises(L.LBMError):
            lat.set_fields(D=D)


@pytest.mark.parametrize("form,grid", [("bf16x6split", (70, 65)), ("tf32split", (70, 65)), ("tf32split", (36, 29, 23))])
def test_g_field_on_and_off_tensor_core(L, form, grid):
    """Switching g(x) on re-splits K without g and takes the operands per axis from
    g_mu(x) C; switching it off restores the constant run bit for bit."""
    pb, C0, fields = _case("mrt", grid, 977)
    with L.Lattice(pb, C0, form) as ref:
        ref.step(20)
        C_const = ref.C()
    with L.Lattice(pb, C0, form) as lat:
        lat.set_fields(g=fields["g"])
        lat.step(20)
        C_g = lat.C()
        lat.set_fields()
        lat.step(20)
        assert np.array_equal(lat.C(), C_const)
    C_ref = O.run_fields_C(pb, C0, 20, {"g": fields["g"]}).numpy()
    l2, node, _ = arith_bounds.bounds(pb, C0, 20, form, C_ref=C_ref, fields={"g": fields["g"]})
    arith_bounds.assert_close(C_g, C_ref, l2, node, f"g(x) {form} {grid}")


@functools.lru_cache(maxsize=1)
def _varying_512_ref(n):
    pb, C0, _, fields = W.varying_512()
    return O.run_fields_C(pb, C0, n, fields).numpy()


@pytest.mark.parametrize("form", ["fp32", "bf16x6split", "tf32split"])
def test_varying_512_workload(L, form):
    """The 512^2 workload with varying D(x), g(x), u(x) (bench entry), first 200 steps, in the
    plain FP32 form and in both tensor-core forms that carry g(x) per axis."""
    pb, C0, _, fields = W.varying_512()
    n = 200
    C_ref = _varying_512_ref(n)
    with L.Lattice(pb, C0, form) as lat:
        lat.set_fields(**fields)
        lat.step(n)
        arith_bounds.assert_close(lat.C(), C_ref, 1e-5, 1e-5, f"varying_512 {form}")
