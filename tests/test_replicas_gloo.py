"""Multi-GPU runs of bench.py are independent replicas (no collective on the
data path); their numbers are combined as the slowest rank's time and the
summed iterations.  The batched workload is sharded by expected work over
the ranks instead, each rank solving its own LPs.  Checked here with two
gloo ranks on the CPU."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    ms, it = bench.aggregate_replicas(10.0 + 5.0 * rank, 100 + rank, dist)
    out[rank] = (ms, it)
    # a sharded batch: rank r solved its share in 3 + r seconds
    work = [float(w) for w in range(1, 41)]
    mine = bench.batch_shard(work, rank, world)
    out[("batch", rank)] = bench.aggregate_batch(3.0 + rank, len(mine) - rank, 1000 * (rank + 1), len(mine), dist)
    out[("shard", rank)] = mine
    dist.destroy_process_group()


def test_two_gloo_replicas_take_max_time_and_sum_iterations():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 201.0)
    # both ranks see the slowest time and the summed counts of the whole batch
    assert out[("batch", 0)] == out[("batch", 1)] == (4.0, 39, 3000, 40)
    assert sorted(out[("shard", 0)] + out[("shard", 1)]) == list(range(40))


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_replicas(3.5, 7) == (3.5, 7.0)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_batch_shard_is_a_balanced_partition(world):
    """Every LP on exactly one rank; the snake deal keeps each rank's expected
    work within one LP of the others'."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    work = np.random.default_rng(world).lognormal(0.0, 1.5, 1000)
    parts = [bench.batch_shard(work, r, world) for r in range(world)]
    assert sorted(sum(parts, [])) == list(range(1000))
    loads = [work[p].sum() for p in parts]
    assert max(loads) - min(loads) <= work.max()
    assert all(bench.batch_shard(work, r, world) == parts[r] for r in range(world))
