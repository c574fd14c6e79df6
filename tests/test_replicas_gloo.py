"""Replica aggregation of bench.py on two CPU ranks (gloo): the job time is
the slowest rank's, and the whole-job rate counts every rank's solves.
The path has no data-path collective (independent problems per rank)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    total = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    rate = bench.whole_job_rate(world, 4, total)
    out[rank] = (total, rate)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        total, rate = out[r]
        assert total == pytest.approx(150.0)
        assert rate == pytest.approx(2 * 4 / 0.150)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.whole_job_rate(1, 5, 500.0) == pytest.approx(10.0)
