"""Batched ensembles: independent problems advanced by grouped launches, each checked
against the FP64 oracle run on its own.  Bounds as in the single-problem tests."""
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


rel_l2 = arith_bounds.rel_l2


@pytest.mark.parametrize("precision", ["bf16split", "fp32"])
def test_small_uneven_batch(L, precision):
    probs, fields, _ = W.batch64(nprob=7, sides=(37, 64, 130, 200), seed=11)
    n = 12
    with L.Batch(probs, fields, precision) as b:
        assert len(b) == 7
        b.step(n)
        for i, (pb, C0) in enumerate(zip(probs, fields)):
            C_ref = O.run_C(pb, C0, n).numpy()
            tol = arith_bounds.bound(pb, C0, n, precision)
            assert rel_l2(b.C(i), C_ref) < tol, f"problem {i} side {pb.grid}"
            # members with alpha near 1 on long lines are ill-conditioned (their own FP32
            # arithmetic errs by percent after a few steps): mass within the same bound
            assert b.mass(i) == pytest.approx(float(C_ref.sum()), rel=max(1e-4, tol))


def test_batch_equals_single_problem_handles(L):
    """Grouped launches give the same populations as one handle per problem with the
    same tile shape (128 columns, no split)."""
    probs, fields, _ = W.batch64(nprob=4, sides=(128, 256), seed=12)
    with L.Batch(probs, fields, "fp32") as b:
        b.step(40)
        got = [b.C(i) for i in range(len(probs))]
    for i, (pb, C0) in enumerate(zip(probs, fields)):
        with L.Lattice(pb, C0, "fp32") as lat:
            lat.configure(0, 1)  # single FP32 problems split the contraction by default
            lat.reset()          # initial populations from the unsplit operator too
            lat.step(40)
            assert np.array_equal(lat.C(), got[i])


def test_batch64_workload_prefix(L):
    """The 64-problem workload (sides 128..1024) at full size, first 3 steps, a sample
    of its problems against the oracle."""
    probs, fields, _ = W.batch64()
    n = 3
    with L.Batch(probs, fields, "bf16split") as b:
        b.step(n)
        for i in (0, 17, 41, 63):
            C_ref = O.run_C(probs[i], fields[i], n).numpy()
            assert rel_l2(b.C(i), C_ref) < arith_bounds.bound(probs[i], fields[i], n, "bf16split")
        assert L.lbm_sync(b.h) == 0


def test_batch_rejects_mixed_collisions(L):
    probs, fields, _ = W.batch64(nprob=2, sides=(64,), seed=3)
    import dataclasses
    probs[1] = dataclasses.replace(probs[1], collision="bgk", s_free=(),
                                   D=((probs[1].D[0][0], 0.0), (0.0, probs[1].D[0][0])))
    with pytest.raises(L.LBMError) as ei:
        L.Batch(probs, fields, "bf16split")
    assert ei.value.code == L.LBM_EINVAL


@pytest.mark.parametrize("precision", ["fp32", "bf16split"])
def test_batch_save_load_resumes_bit_exact(L, precision):
    probs, fields, _ = W.batch64(nprob=5, sides=(37, 128, 200), seed=13)
    with L.Batch(probs, fields, precision) as b:
        b.step(3)
        state = b.save()
        b.step(35)
        C_a = [b.C(i) for i in range(len(probs))]
        b.load(state)
        b.step(35)
        C_b = [b.C(i) for i in range(len(probs))]
    for a, c in zip(C_a, C_b):
        assert np.array_equal(a, c)


def test_batch_autotune_restores_state(L):
    probs, fields, _ = W.batch64(nprob=5, sides=(37, 128, 200), seed=14)
    with L.Batch(probs, fields, "bf16split") as b, L.Batch(probs, fields, "bf16split") as ref:
        b.step(3)
        ref.step(3)
        desc = b.autotune(8)
        assert "chunk" in desc
        b.step(20)
        ref.step(20)
        for i in range(len(probs)):
            assert np.array_equal(b.C(i), ref.C(i))
