"""The multi-replica host logic of bench.py on CPU: two gloo ranks, each with its
own step time, agree on the slowest time and on the whole-job throughput (all
ranks' local solves over that time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, world)       # rank 1 is the slow one
    rate = bench.aggregate_rate(143356, world, t)
    out[rank] = (t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_units_add_up():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        t, rate = out[r]
        assert t == 2.5
        assert rate == pytest.approx(2 * 143356 / 2.5)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.aggregate_rate(10, 1, 2.0) == 5.0
