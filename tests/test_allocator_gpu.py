"""Device memory lent by the host framework: PyTorch's caching allocator serves every
buffer a handle owns (lbm_set_allocator), the results are unchanged, and all of it goes
back when the handle (or the gradient's scratch) is done with it."""
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


@pytest.mark.parametrize("kind", ["bf16split", "tf32split", "fp32"])
def test_torch_allocator_serves_a_handle(L, kind):
    rng = np.random.default_rng(151)
    grid = (96, 40, 36) if kind == "tf32split" else (130, 70)
    pb = W.random_problem(rng, len(grid), "mrt", grid)
    C0 = W.random_field(rng, grid)
    n = 6
    nodes = int(np.prod(grid))
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    L.use_torch_allocator(True)
    try:
        with L.Lattice(pb, C0, kind) as lat:
            held = torch.cuda.memory_allocated() - base
            assert held >= 2 * lat.Q * nodes * 4  # at least the two population buffers
            lat.step(n)
            C = lat.C()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        L.use_torch_allocator(False)
    assert arith_bounds.rel_l2(C, O.run_C(pb, C0, n).numpy()) < arith_bounds.bound(pb, C0, n, kind)


def test_torch_allocator_serves_batches_and_gradients(L):
    rng = np.random.default_rng(152)
    probs = [W.random_problem(rng, 2, "mrt", g) for g in [(64, 64), (128, 96)]]
    fields = [W.random_field(rng, pb.grid) for pb in probs]
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    L.use_torch_allocator(True)
    try:
        with L.Batch(probs, fields, "bf16split") as b:
            assert torch.cuda.memory_allocated() > base
            b.step(4)
        pb = W.random_problem(rng, 2, "mrt", (40, 32))
        C0 = W.random_field(rng, pb.grid)
        with L.Lattice(pb, C0, "fp32") as lat:
            obs = np.zeros((2,) + lat.shape)
            loss, grad = lat.grad([4, 8], obs, 4)
            assert np.isfinite(loss) and np.all(np.isfinite(grad))
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        L.use_torch_allocator(False)


def test_hooks_must_come_in_pairs(L):
    with pytest.raises(L.LBMError):
        L.lbm_set_allocator(lambda n, s, c: None, None)
