"""Batched instances: several independent joins verified in one launch.

Each instance of a multi launch (plain and CUDA-graph replays) must return
exactly what it returns alone, which the other parity tests tie to the
oracle; the uneven-instance workload is also compared with the oracle's
AllPairs join directly.
"""
import numpy as np
import pytest

import oracle
import synth

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    _build.build()
    h = ssj.ssj_create(0)
    yield h
    ssj.ssj_destroy(h)


def _dev(b, dev):
    import torch
    return (torch.from_numpy(b.probe_ids.astype(np.int32)).to(dev),
            torch.from_numpy(b.cand_offsets.astype(np.int64)).to(dev),
            torch.from_numpy(b.cand_ids.astype(np.int32)).to(dev))


def _run_multi(ctx, cases, graph_reps=0, tune=None):
    """cases: list of (R, S, p, q, Batch, flags).  Returns per-instance sorted triples for the
    plain launch and for each graph replay.  tune: a list that receives the autotuner's report,
    if the launch is to be autotuned first."""
    import torch
    dev = torch.device("cuda:0")
    keep, dbs, outs, caps = [], [], [], []
    for R, S, p, q, b, fl in cases:
        t = _dev(b, dev)
        keep.append(t)
        dbs.append(ssj.DeviceBatch(R, S, p, q, *t, b.n_cands, flags=fl, n_probes=b.n_probes))
        cap = max(b.n_cands, 1)
        outs.append(torch.zeros(3 * cap, dtype=torch.int32, device=dev))
        caps.append(cap)
    counts = torch.zeros(len(cases), dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    m = ssj.ssj_multi_create(ctx, dbs, outs, caps, counts)
    results = []
    try:
        if tune is not None:
            ssj.ssj_multi_graph_launch(ctx, m)  # a graph captured before tuning is replaced
            tune.append(ssj.ssj_multi_autotune(ctx, m, reps=3))
        for rep in range(1 + graph_reps):
            for o in outs:
                o.zero_()
            torch.cuda.synchronize()
            if rep == 0:
                ssj.ssj_multi_launch(ctx, m)
            else:
                ssj.ssj_multi_graph_launch(ctx, m)
            assert ssj.ssj_device_error(ctx) == 0
            n = counts.cpu().numpy()
            res = []
            for i, o in enumerate(outs):
                if cases[i][5] & ssj.SSJ_COUNT_ONLY:
                    res.append(int(n[i]))
                else:
                    tr = o[:3 * int(n[i])].view(-1, 3).cpu().numpy().astype(np.uint32)
                    res.append(oracle.sort_triples(tr))
            results.append(res)
    finally:
        ssj.ssj_multi_destroy(ctx, m)
    return results


def _alone(ctx, R, S, p, q, b, fl):
    if fl & ssj.SSJ_COUNT_ONLY:
        return ssj.ssj_verify_batch(ctx, R, S, p, q, b.probe_ids, b.cand_offsets, b.cand_ids, flags=fl)
    return ssj.triples_to_array(ssj.ssj_verify_batch(ctx, R, S, p, q, b.probe_ids, b.cand_offsets, b.cand_ids,
                                                     flags=fl))


@pytest.mark.parametrize("policy", [0, 1, 24])
def test_multi_mixed_instances_equal_their_single_launches(ctx, policy):
    """Ten instances of different collections, thresholds and flags in one launch (their chunks
    mix in the short-pair phase) equal their single launches, at several short-pair refill thresholds."""
    spec = synth.tiny_self_join(n=600)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c_tiny = synth.collection(spec)
    c_short = synth.collection(synth.short_sets(n=15_000))
    spec_l = synth.long_sets(n=600)
    spec_l.plant_frac, spec_l.plant_edits = 0.3, 10
    c_long = synth.collection(spec_l)
    cR = synth.collection(synth.tiny_self_join(seed=7, n=300))
    h_tiny, h_short, h_long, hR = (ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
                                   for c in (c_tiny, c_short, c_long, cR))
    fb = lambda c, p, q: synth.Batch(*ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=4))
    empty = synth.Batch(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint32))
    cases = [
        (h_tiny, h_tiny, 1, 2, synth.all_pairs_batch(c_tiny.n), 0),
        (h_short, h_short, 3, 5, fb(c_short, 3, 5), 0),
        (h_short, h_short, 9, 10, fb(c_short, 9, 10), 0),
        (h_long, h_long, 3, 5, fb(c_long, 3, 5), 0),
        (h_tiny, h_tiny, 4, 5, synth.all_pairs_batch(c_tiny.n), ssj.SSJ_FORCE_WARP),
        (h_long, h_long, 4, 5, fb(c_long, 4, 5), ssj.SSJ_FORCE_BLOCK),
        (h_tiny, h_tiny, 1, 3, synth.all_pairs_batch(c_tiny.n), ssj.SSJ_COUNT_ONLY),
        (h_tiny, h_tiny, 1, 2, empty, 0),
        (hR, h_tiny, 1, 3, synth.random_batch(3, cR.n, c_tiny.n, 500, 30), 0),
        (h_short, h_short, 7, 10, fb(c_short, 7, 10), ssj.SSJ_EMIT_ALL),
    ]
    want = [_alone(ctx, *cs) for cs in cases]
    ssj.ssj_set_short_pairs(ctx, policy)
    try:
        for res in _run_multi(ctx, cases, graph_reps=2):
            for i, (got, w) in enumerate(zip(res, want)):
                if isinstance(w, int):
                    assert got == w, i
                else:
                    assert np.array_equal(got, w), (i, len(got), len(w))
    finally:
        ssj.ssj_set_short_pairs(ctx, 0)
    for h in (h_tiny, h_short, h_long, hR):
        ssj.ssj_unload_collection(ctx, h)


def test_uneven_instances_scaled_match_oracle(ctx):
    """Sixteen uneven self-join instances (sizes, skews and thresholds drawn as in the batched
    workload, scaled down) in one launch, each against the oracle's AllPairs join."""
    specs = synth.uneven_instances(count=16, n_lo=200, n_hi=3000, mean_lo=5, mean_hi=150)
    cases, wants, handles = [], [], []
    for ins in specs:
        ins.coll.plant_frac, ins.coll.plant_edits = 0.1, 1
        c = synth.collection(ins.coll)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
        handles.append(h)
        b = synth.Batch(*ssj.feeder_all(c.offsets, c.tokens, ins.p, ins.q, n_threads=4))
        cases.append((h, h, ins.p, ins.q, b, 0))
        wants.append(oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, ins.p, ins.q)[0]))
    res = _run_multi(ctx, cases, graph_reps=1)
    for r in res:
        for i, (got, w) in enumerate(zip(r, wants)):
            assert np.array_equal(got, w), (i, len(got), len(w))
    assert sum(len(w) for w in wants) > 0
    for h in handles:
        ssj.ssj_unload_collection(ctx, h)


def test_uneven_instances_full_size_match_oracle(ctx):
    """The full batched workload: 256 uneven self-joins (n log-uniform 500..50,000, mean set size
    log-uniform 5..500, Zipf s in [0.6, 1.2], t over 0.6..0.95; several hundred million candidates
    in all) in one launch and in a CUDA-graph replay; every instance's sorted (r, s, overlap) list
    equals the oracle's on the same feeder batch (the oracle split over probe ranges on every host
    core)."""
    import torch
    dev = torch.device("cuda:0")
    specs = synth.uneven_instances()
    assert len(specs) == 256
    handles, keep, dbs, outs, caps, wants = [], [], [], [], [], []
    total = 0
    for ins in specs:
        c = synth.collection(ins.coll)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
        handles.append(h)
        b = synth.Batch(*ssj.feeder_all(c.offsets, c.tokens, ins.p, ins.q, n_threads=16))
        total += b.n_cands
        want = oracle.sort_triples(oracle.verify_batch_threads(c.offsets, c.tokens, c.offsets, c.tokens, True,
                                                               ins.p, ins.q, b.probe_ids, b.cand_offsets,
                                                               b.cand_ids))
        wants.append(want)
        t = _dev(b, dev)
        keep.append(t)
        dbs.append(ssj.DeviceBatch(h, h, ins.p, ins.q, *t, b.n_cands, n_probes=b.n_probes))
        cap = len(want) + 1024
        outs.append(torch.zeros(3 * cap, dtype=torch.int32, device=dev))
        caps.append(cap)
    assert total > 300_000_000
    assert sum(len(w) for w in wants) > 0
    counts = torch.zeros(len(specs), dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    m = ssj.ssj_multi_create(ctx, dbs, outs, caps, counts)
    try:
        for rep in range(2):
            for o in outs:
                o.zero_()
            counts.zero_()
            torch.cuda.synchronize()
            if rep == 0:
                ssj.ssj_multi_launch(ctx, m)
            else:
                ssj.ssj_multi_graph_launch(ctx, m)
            torch.cuda.synchronize()
            assert ssj.ssj_device_error(ctx) == 0
            n = counts.cpu().numpy()
            for i, (o, w) in enumerate(zip(outs, wants)):
                assert int(n[i]) == len(w), (rep, i, int(n[i]), len(w))
                got = oracle.sort_triples(o[:3 * int(n[i])].view(-1, 3).cpu().numpy().astype(np.uint32))
                assert np.array_equal(got, w), (rep, i)
    finally:
        ssj.ssj_multi_destroy(ctx, m)
        for h in handles:
            ssj.ssj_unload_collection(ctx, h)


def test_multi_keeps_collections_loaded(ctx):
    import torch
    c = synth.collection(synth.tiny_self_join(n=100))
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    b = synth.all_pairs_batch(c.n)
    t = _dev(b, torch.device("cuda:0"))
    out = torch.zeros(3 * b.n_cands, dtype=torch.int32, device="cuda:0")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    m = ssj.ssj_multi_create(ctx, [ssj.DeviceBatch(h, h, 1, 2, *t, b.n_cands)], [out], [b.n_cands], cnt)
    with pytest.raises(ssj.SsjError) as ei:
        ssj.ssj_unload_collection(ctx, h)
    assert ei.value.status == ssj.SSJ_EBUSY
    ssj.ssj_multi_destroy(ctx, m)
    ssj.ssj_unload_collection(ctx, h)


def test_autotuned_launch_matches_oracle(ctx):
    """The autotuner times thread/warp/block bin boundaries and block sizes; whatever it picks,
    plain and graph launches afterwards return the oracle's join for every instance."""
    specs = synth.uneven_instances(count=12, seed=77, n_lo=300, n_hi=4000, mean_lo=5, mean_hi=400)
    cases, wants, handles = [], [], []
    for ins in specs:
        ins.coll.plant_frac, ins.coll.plant_edits = 0.1, 1
        c = synth.collection(ins.coll)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
        handles.append(h)
        b = synth.Batch(*ssj.feeder_all(c.offsets, c.tokens, ins.p, ins.q, n_threads=4))
        cases.append((h, h, ins.p, ins.q, b, 0))
        wants.append(oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, ins.p, ins.q)[0]))
    rep = []
    res = _run_multi(ctx, cases, graph_reps=1, tune=rep)
    (t,) = rep
    assert t["block_threads"] & ~(ssj.SSJ_WIDE_REGISTERS | ssj.SSJ_BULK_STAGING) in (128, 256, 512)
    assert t["thread_max_key"] in (32, 64, 128, 256, 512, 1024, 2048, 4096)
    assert t["warp_max_key"] >= t["thread_max_key"]
    assert t["drain_min_live"] in (8, 12, 16, 20, 24)
    assert t["index_min_cands"] in (0, 32, 64, 128, 256, 512, 1024, 4096)
    assert t["settings_tried"] >= 3 and 0 < t["best_ms"] <= t["initial_ms"]
    for r in res:
        for i, (got, w) in enumerate(zip(r, wants)):
            assert np.array_equal(got, w), (i, len(got), len(w))
    for h in handles:
        ssj.ssj_unload_collection(ctx, h)


def test_read_bandwidth_probe(ctx):
    l2 = ssj.ssj_read_bandwidth(ctx, 32 << 20, 20)
    hbm = ssj.ssj_read_bandwidth(ctx, 2 << 30, 3)
    assert l2 > 100 and hbm > 100
    with pytest.raises(ssj.SsjError):
        ssj.ssj_read_bandwidth(ctx, 8, 1)


@pytest.mark.parametrize("tmax,lmax,wmax,bt", [(4096, 1, 4096, 256), (32, 1, 256, 128), (32, 1, 256, 512),
                                               (128, 1, 1024, 128), (512, 1, 0xFFFFFFFF, 512),
                                               (1 << 30, 1, 1 << 30, 128), (64, 2048, 2048, 256),
                                               (256, 1024, 4096, 128), (32, 4096, 256, 512),
                                               (2048, 1, 4096, 256 | 0x10000), (32, 256, 256, 512 | 0x10000),
                                               (128, 1024, 1024, 128 | 0x10000)])
def test_bins_and_block_sizes_match_oracle(ctx, tmax, lmax, wmax, bt):
    """Every bin boundary and block size the autotuner may pick gives the oracle's result, on
    sets long enough to reach all three granularities."""
    spec = synth.long_sets(n=1200)
    spec.plant_frac, spec.plant_edits = 0.3, 10
    c = synth.collection(spec)
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    try:
        ssj.ssj_set_granularity(ctx, tmax, lmax, wmax, bt)
        for p, q in ((3, 5), (4, 5)):
            pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=4)
            got = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, p, q, pr, co, ci))
            want = oracle.sort_triples(oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, p, q,
                                                           pr, co, ci))
            assert np.array_equal(got, want), (p, q, len(got), len(want))
            assert len(want) > 0
    finally:
        ssj.ssj_set_granularity(ctx, 128, 2048, 2048, 256)
        ssj.ssj_unload_collection(ctx, h)


def test_verify_batches_host_equals_single_calls(ctx):
    """ssj_verify_batches (host batches, one launch) returns for every batch what the single
    synchronous call returns; a too-small capacity answers SSJ_ENOMEM with the true counts."""
    spec = synth.tiny_self_join(seed=31, n=600)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    short = synth.collection(synth.short_sets(n=10_000))
    cR = synth.collection(synth.tiny_self_join(seed=32, n=300))
    h, hs, hR = (ssj.ssj_load_collection(ctx, x.offsets, x.tokens) for x in (c, short, cR))
    ap = synth.all_pairs_batch(c.n)
    fb = synth.Batch(*ssj.feeder_all(short.offsets, short.tokens, 3, 5, n_threads=4))
    rb = synth.random_batch(5, cR.n, c.n, 200, 40)
    empty = synth.Batch(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint32))
    arrs = lambda b: (b.probe_ids, b.cand_offsets, b.cand_ids)
    batches = [(h, h, 4, 5, *arrs(ap), 0), (h, h, 3, 5, *arrs(ap), ssj.SSJ_SIM_COSINE | ssj.SSJ_SORTED),
               (hs, hs, 3, 5, *arrs(fb), 0), (hR, h, 1, 3, *arrs(rb), 0),
               (h, h, 1, 2, *arrs(ap), ssj.SSJ_COUNT_ONLY), (h, h, 1, 2, *arrs(empty), 0),
               (h, h, 7, 1, *arrs(ap), ssj.SSJ_SIM_OVERLAP)]
    try:
        got = ssj.ssj_verify_batches(ctx, batches)
        for i, (R, S, p, q, pr, co, ci, fl) in enumerate(batches):
            want = ssj.ssj_verify_batch(ctx, R, S, p, q, pr, co, ci, flags=fl)
            if fl & ssj.SSJ_COUNT_ONLY:
                assert got[i] == want, i
            else:
                assert np.array_equal(ssj.triples_to_array(got[i]), ssj.triples_to_array(want)), i
                if fl & ssj.SSJ_SORTED:
                    assert np.array_equal(ssj.triples_to_array(got[i]),
                                          np.stack([got[i]["r"], got[i]["s"], got[i]["overlap"]], 1)), i
        n0 = len(got[0])
        assert n0 > 1
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_verify_batches(ctx, batches[:1], caps=[n0 - 1])
        assert ei.value.status == ssj.SSJ_ENOMEM
    finally:
        for x in (h, hs, hR):
            ssj.ssj_unload_collection(ctx, x)


def test_verify_batches_host_direct_equals_copies(ctx):
    """SSJ_HOST_DIRECT: kernels reading pinned host inputs directly give the results of the copying
    path; pageable inputs under the flag are copied as usual."""
    import torch
    c = synth.collection(synth.short_sets(n=20_000))
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    pinned = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    try:
        batches = []
        for p, q in [(3, 5), (4, 5)]:
            pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=4)
            batches.append((h, h, p, q, pinned(pr), pinned(co), pinned(ci), 0))
            batches.append((h, h, p, q, pr, co, ci, 0))  # pageable
        want = ssj.ssj_verify_batches(ctx, batches)
        got = ssj.ssj_verify_batches(ctx, [b[:7] + (ssj.SSJ_HOST_DIRECT | ssj.SSJ_FORCE_WARP * (i % 2),)
                                           for i, b in enumerate(batches)])
        for g, w in zip(got, want):
            assert np.array_equal(ssj.triples_to_array(g), ssj.triples_to_array(w))
    finally:
        ssj.ssj_unload_collection(ctx, h)


def test_verify_batches_large_batch_caps_and_host_direct(ctx):
    """A batch of about 2M candidates with others in one call: results equal the single call's,
    with SSJ_HOST_DIRECT too, and a too-small capacity answers SSJ_ENOMEM."""
    import torch
    spec = synth.tiny_self_join(seed=2024, n=2000)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    short = synth.collection(synth.short_sets(n=15_000))
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    hs = ssj.ssj_load_collection(ctx, short.offsets, short.tokens)
    pinned = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    try:
        ap = synth.all_pairs_batch(c.n)
        assert ap.n_cands > (1 << 20)
        fb = synth.Batch(*ssj.feeder_all(short.offsets, short.tokens, 3, 5, n_threads=4))
        arrs = [pinned(x) for x in (ap.probe_ids, ap.cand_offsets, ap.cand_ids)]
        batches = [(hs, hs, 3, 5, fb.probe_ids, fb.cand_offsets, fb.cand_ids, 0), (h, h, 1, 2, *arrs, 0),
                   (h, h, 3, 5, *arrs, ssj.SSJ_SIM_COSINE)]
        want = [ssj.triples_to_array(ssj.ssj_verify_batch(ctx, *b[:7], flags=b[7])) for b in batches]
        for extra in (0, ssj.SSJ_HOST_DIRECT):
            got = ssj.ssj_verify_batches(ctx, [b[:7] + (b[7] | extra,) for b in batches])
            for g, w in zip(got, want):
                assert np.array_equal(ssj.triples_to_array(g), w)
        assert len(want[1]) > 100
        cap = len(want[1]) - 7
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_verify_batches(ctx, batches[1:2], caps=[cap])
        assert ei.value.status == ssj.SSJ_ENOMEM
    finally:
        ssj.ssj_unload_collection(ctx, h)
        ssj.ssj_unload_collection(ctx, hs)
