"""The bounded device-side wait behind LBM_ERR_TIMEOUT, exercised without a fault.

A barrier phase that nothing completes makes the library's wait give up after its
limit: the call returns LBM_ERR_TIMEOUT promptly, the CUDA context stays usable, and
a lattice created afterwards still matches the oracle.
"""
import time

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


def test_completed_phase_returns_ok(L):
    assert L.lbm_wait_check(True, 1000) == L.LBM_OK


def test_incomplete_phase_times_out_and_context_survives(L):
    t0 = time.perf_counter()
    rc = L.lbm_wait_check(False, 5000)
    dt = time.perf_counter() - t0
    assert rc == L.LBM_ERR_TIMEOUT
    assert dt < 2.0
    assert L.lbm_wait_check(True, 1000) == L.LBM_OK
    rng = np.random.default_rng(141)
    pb = W.random_problem(rng, 2, "mrt", (64, 48))
    C0 = W.random_field(rng, pb.grid)
    n = 8
    with L.Lattice(pb, C0, "bf16split") as lat:
        lat.step(n)
        C = lat.C()
    assert arith_bounds.rel_l2(C, O.run_C(pb, C0, n).numpy()) < arith_bounds.bound(pb, C0, n, "bf16split")


def test_limit_is_validated(L):
    assert L.lbm_wait_check(False, 0) == L.LBM_EINVAL
    assert L.lbm_wait_check(False, 2000000) == L.LBM_EINVAL
