"""The multi-rank arithmetic of bench.py (independent replicas, one per GPU): the slowest rank's
time is taken with an all-reduce and the whole-job rate counts every rank's units.  Runs two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.reduce_max(100.0 + 50.0 * rank, world)
    out[rank] = (slowest, bench.whole_job_rate(3, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        slowest, rate = res[r]
        assert slowest == 150.0
        assert rate == pytest.approx(3 * 2 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.whole_job_rate(5, 1, 1000.0) == pytest.approx(5.0)
