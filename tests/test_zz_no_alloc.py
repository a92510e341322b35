"""The static-scratch mass reduction (lbm_mass_static), checked against lbm_mass.

lbm_mass_static serves callers that cannot allocate device memory (plug-ins of a
host framework that owns all GPU memory, code that must not let an allocation
synchronise the device): it keeps its partial sums in a static device array.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("precision,dtype", [("fp32", torch.float32), ("fp64", torch.float64)])
def test_static_scratch_sum_matches_lbm_mass_twice(L, precision, dtype):
    rng = np.random.default_rng(99)
    pb = W.random_problem(rng, 2, "mrt", (300, 257))
    C0 = W.random_field(rng, pb.grid)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with L.Lattice(pb, C0, precision) as lat:
        for call in range(2):  # two calls in a row share the static array
            lat.step(7 + call)
            want = lat.mass()                     # existing entry point (handle scratch)
            C = torch.tensor(lat.C(), dtype=dtype, device="cuda")  # same values, caller-owned memory
            torch.cuda.synchronize()
            rc = L.lbm_mass_static(C.data_ptr(), C.element_size(), C.numel(), out.data_ptr(), None)
            assert rc == L.LBM_OK
            torch.cuda.synchronize()
            got = float(out.item())
            assert got == pytest.approx(want, rel=1e-13, abs=1e-300)


def test_static_scratch_at_its_capacity(L):
    """n = 67,108,864 FP32 values (256 MiB): every one of the 65,536 partials is used,
    the last one included.  Values k/1024 (k = i mod 1024) and a marker in the last
    element make every partial sum exact in FP64, so the result is compared exactly;
    two calls in a row give the same value."""
    n = 67_108_864
    x = (torch.arange(n, device="cuda", dtype=torch.int64) % 1024).to(torch.float32) / 1024.0
    x[-1] = 4096.0  # replaces 1023/1024 in the last partial
    want = (n // 1024) * (1023 * 1024 / 2) / 1024.0 - 1023.0 / 1024.0 + 4096.0
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.cuda.synchronize()
        assert L.lbm_mass_static(x.data_ptr(), 4, n, out.data_ptr(), None) == L.LBM_OK
        torch.cuda.synchronize()
        assert float(out.item()) == want
    del x


def test_static_scratch_rejects_oversize_and_bad_arguments(L):
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert L.lbm_mass_static(x.data_ptr(), 4, 67_108_865, out.data_ptr(), None) == L.LBM_ETOOBIG
    assert L.lbm_mass_static(x.data_ptr(), 2, 16, out.data_ptr(), None) == L.LBM_EINVAL
    assert L.lbm_mass_static(x.data_ptr(), 4, -1, out.data_ptr(), None) == L.LBM_EINVAL
    assert L.lbm_mass_static(0, 4, 16, out.data_ptr(), None) == L.LBM_EINVAL
    assert L.lbm_mass_static(x.data_ptr(), 4, 0, out.data_ptr(), None) == L.LBM_OK
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
