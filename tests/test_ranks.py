"""The multi-process path of bench.py on CPU: world_size-2 gloo ranks (one process per GPU on
a GPU node; here CPU processes).  Candidate pairs are independent, so the path shards with no
data exchange: every batch is split into contiguous probe ranges, one per rank, each rank times
its own work and the job's time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import synth


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


def _share_main(rank, world, port, out):
    """One rank: its probe ranges of a few seeded batches, gathered on every rank over gloo."""
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batches = _batches()
        mine = bench.rank_share(batches, rank, world)
        # each rank's (probe, candidate) pairs, gathered as flat int64 keys
        keys = []
        for (_, _, _, pr, co, ci) in mine:
            keys.append(np.repeat(pr.astype(np.int64), np.diff(co.astype(np.int64))) * (1 << 32)
                        + ci.astype(np.int64))
        flat = torch.from_numpy(np.concatenate(keys)) if keys else torch.zeros(0, dtype=torch.int64)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([len(flat)], dtype=torch.int64))
        width = max(int(n.item()) for n in sizes)  # gloo gathers equal sizes: pad, then trim
        padded = torch.full((width,), -1, dtype=torch.int64)
        padded[:len(flat)] = flat
        bufs = [torch.zeros(width, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(bufs, padded)
        out[rank] = [b[:int(n.item())].numpy().tolist() for b, n in zip(bufs, sizes)]
    finally:
        dist.destroy_process_group()


def _batches():
    out = []
    for seed, probes, per in ((3, 200, 40), (4, 1, 7), (5, 0, 5), (6, 50, 0)):
        b = synth.random_batch(seed, 300, 300, probes, per)
        out.append((0, 3, 5, b.probe_ids, b.cand_offsets, b.cand_ids))
    return out


def test_rank_share_tiles_every_batch_gloo_two_ranks():
    """The two ranks' probe ranges of every batch (including one-probe, empty and candidate-free
    batches) hold every candidate exactly once: the multiset union equals the whole batch."""
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_share_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        got = dict(out)
    assert got[0] == got[1]
    union = sorted(got[0][0] + got[0][1])
    want = []
    for (_, _, _, pr, co, ci) in _batches():
        want += (np.repeat(pr.astype(np.int64), np.diff(co.astype(np.int64))) * (1 << 32)
                 + ci.astype(np.int64)).tolist()
    assert union == sorted(want)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_rank_share_is_a_partition(world):
    batches = _batches()
    total = [0] * len(batches)
    for r in range(world):
        for i, (_, _, _, pr, co, ci) in enumerate(bench.rank_share(batches, r, world)):
            assert len(co) == len(pr) + 1 and int(co[0]) == 0 and int(co[-1]) == len(ci)
            total[i] += len(ci)
    assert total == [len(b[5]) for b in batches]


def test_whole_job_value_counts_every_ranks_pairs():
    # the ranks share the step's pairs; the job's rate is all pairs over the slowest rank's time
    assert bench.whole_job_value(1000, 10, 2.0) == 5000.0
    assert bench.max_over_ranks(3.5, 1) == 3.5
