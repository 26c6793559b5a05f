"""Multi-GPU runs of bench.py are independent replicas (no collective on the
data path); their numbers are combined as the slowest rank's time and the
summed iterations.  Checked here with two gloo ranks on the CPU."""

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


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_replicas(3.5, 7) == (3.5, 7.0)
