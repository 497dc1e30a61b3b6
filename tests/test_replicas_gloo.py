"""The N > 1 path of bench.py on CPU: world size 2 over gloo.

The step does not shard (replicas only); the benchmark's only collective is
the max-over-ranks reduction of the timers, and the whole-job value counts
every rank's steps.  Each rank here reports a different time; both must see
the maximum and the same value.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world)
    val = bench.replica_value(10, world, ms)
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, val in out:
        assert ms == 150.0
        assert val == pytest.approx(2 * 10 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_value(4, 1, 2000.0) == pytest.approx(2.0)
