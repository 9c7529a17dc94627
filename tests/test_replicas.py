"""The multi-GPU form is replicas only: every rank runs the whole path on its
own data, and the ranks meet only to take the slowest rank's time.  This
checks that host logic with two gloo processes on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, world, None)
    rate = bench.whole_job_rate(1000, world, slowest)
    dist.barrier()
    out[rank] = (slowest, rate)
    dist.destroy_process_group()


def test_two_replicas_report_slowest_rank_and_total_rate():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    slowest, rate = out[0]
    assert slowest == 15.0
    assert rate == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 1, 1000.0) == 10.0
