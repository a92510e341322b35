"""bench.py's multi-GPU aggregation (one independent replica per rank; the workload does
not shard): value = all ranks' lattice updates / the slowest rank's time.  Run as two
gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    value, t = bench.job_value(local_ms, 1e6, world, dist, "cpu")
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, t = res[r]
        assert t == pytest.approx(200.0)
        assert value == pytest.approx(world * 1e6 / 0.2 / 1e6)


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.job_value(50.0, 2e6, 1)
    assert t == 50.0 and value == pytest.approx(40.0)
