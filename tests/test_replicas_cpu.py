"""bench.py's multi-GPU aggregation and the batch partition, run as two gloo ranks on the
CPU.  A single lattice does not shard (one independent replica per rank); the batch of
independent problems is partitioned: each rank takes a cost-balanced subset, with no
collective on the data path.  value = all ranks' lattice updates / the slowest rank's
time."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


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
    import bench
    value, t = bench.job_value(50.0, 2e6, 1)
    assert t == 50.0 and value == pytest.approx(40.0)


def _partition_rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1706_09161_gb300 import workloads as W
    probs, _, nlbm = W.batch64()
    mine = bench.partition(probs, world)[rank]
    units = sum(probs[i].nodes for i in mine) * nlbm
    # a stand-in time proportional to the rank's modelled cost
    local_ms = 1e-6 * sum(bench.problem_cost(probs[i]) for i in mine)
    value, t = bench.job_value(local_ms, units, world, dist, "cpu")
    out[rank] = (mine, units, local_ms, value, t)
    dist.destroy_process_group()


def test_batch_partition_two_ranks():
    import bench
    from paper_1706_09161_gb300 import workloads as W
    probs, _, nlbm = W.batch64()
    world = 2
    port = 30500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_partition_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every problem on exactly one rank
    owned = sorted(i for r in range(world) for i in res[r][0])
    assert owned == list(range(len(probs)))
    # the job counts every rank's updates over the slowest rank's time
    total_units = sum(res[r][1] for r in range(world))
    assert total_units == sum(pb.nodes for pb in probs) * nlbm
    t_max = max(res[r][2] for r in range(world))
    for r in range(world):
        value, t = res[r][3], res[r][4]
        assert t == pytest.approx(t_max)
        assert value == pytest.approx(total_units / (t_max * 1e-3) / 1e6)
    # cost balance: within the largest single problem's cost of the even share
    costs = [sum(bench.problem_cost(probs[i]) for i in res[r][0]) for r in range(world)]
    biggest = max(bench.problem_cost(pb) for pb in probs)
    assert max(costs) - min(costs) <= biggest


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_and_balances(world):
    import bench
    from paper_1706_09161_gb300 import workloads as W
    probs, _, _ = W.batch64()
    parts = bench.partition(probs, world)
    assert len(parts) == world
    assert sorted(i for p in parts for i in p) == list(range(len(probs)))
    assert parts == bench.partition(probs, world)  # deterministic
    loads = [sum(bench.problem_cost(probs[i]) for i in p) for p in parts]
    biggest = max(bench.problem_cost(pb) for pb in probs)
    assert max(loads) <= sum(loads) / world + biggest
