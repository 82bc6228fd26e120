"""The multi-process path of bench.py on CPU: world_size-2 gloo ranks (one process per GPU on
a GPU node; here CPU processes).  The path shards as replicas (no data exchange): each rank
times its own work and the job's time is the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_whole_job_value_is_weak_scaling():
    # each rank verifies the whole step; the job's rate counts every rank's pairs
    assert bench.whole_job_value(1000, 10, 1, 2.0) == 5000.0
    assert bench.whole_job_value(1000, 10, 4, 2.0) == 20000.0
    assert bench.max_over_ranks(3.5, 1) == 3.5
