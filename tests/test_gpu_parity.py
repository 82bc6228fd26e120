"""GPU parity: the CUDA verification path against the CPU oracle.

Every comparison is bit-exact on sorted (r, s, overlap) triples: the join
result is unique, only its order is free.  Inputs come from the seeded
generators in synth/, never from the CUDA path.
"""
import numpy as np
import pytest

import oracle
import synth

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build

pytestmark = pytest.mark.gpu

GRANULARITIES = [0, ssj.SSJ_FORCE_THREAD, ssj.SSJ_FORCE_LANE, ssj.SSJ_FORCE_WARP, ssj.SSJ_FORCE_BLOCK,
                 ssj.SSJ_FORCE_INDEX]
T_ALL = [(19, 20), (9, 10), (17, 20), (4, 5), (3, 4), (7, 10), (13, 20), (3, 5)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    h = ssj.ssj_create(0)
    yield h
    ssj.ssj_destroy(h)


def load(ctx, c, flags=ssj.SSJ_VALIDATE):
    return ssj.ssj_load_collection(ctx, c.offsets, c.tokens, flags)


def gpu(ctx, R, S, p, q, b, flags=0):
    res = ssj.ssj_verify_batch(ctx, R, S, p, q, b.probe_ids, b.cand_offsets, b.cand_ids, flags=flags)
    return ssj.triples_to_array(res)


def ora(cR, cS, self_join, p, q, b, flags=oracle.EARLY):
    return oracle.sort_triples(oracle.verify_batch(cR.offsets, cR.tokens, cS.offsets, cS.tokens, self_join, p, q,
                                                   b.probe_ids, b.cand_offsets, b.cand_ids, flags=flags))


def planted_tiny(n=1000, frac=0.1, edits=2, seed=1001):
    spec = synth.tiny_self_join(seed=seed, n=n)
    spec.plant_frac, spec.plant_edits = frac, edits
    return synth.collection(spec)


def feeder_batch(c, p, q, threads=8):
    pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=threads)
    return synth.Batch(pr, co, ci)


# ----------------------------------------------------------------- tiny, all pairs

@pytest.mark.parametrize("gran", GRANULARITIES)
def test_tiny_all_pairs_planted_matches_bruteforce(ctx, gran):
    c = planted_tiny()
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    assert b.n_cands == 499_500
    for p, q in [(4, 5), (3, 5), (9, 10), (1, 1), (1, 10)]:
        want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q))
        got = gpu(ctx, h, h, p, q, b, gran)
        assert np.array_equal(got, want), (gran, p, q, len(got), len(want))
    ssj.ssj_unload_collection(ctx, h)


@pytest.mark.parametrize("gran", GRANULARITIES)
def test_tiny_every_overlap_matches(ctx, gran):
    """SSJ_EMIT_ALL: all 499,500 overlaps of the tiny workload, element by element."""
    c = synth.collection(synth.tiny_self_join())
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    want = ora(c, c, True, 4, 5, b, flags=oracle.EMIT_ALL)
    got = gpu(ctx, h, h, 4, 5, b, ssj.SSJ_EMIT_ALL | gran)
    assert len(got) == 499_500
    assert np.array_equal(got, want)
    ssj.ssj_unload_collection(ctx, h)


# ----------------------------------------------------------------- prefix-filter workloads

@pytest.mark.parametrize("renumber", [False, True])
def test_short_sets_scaled_all_thresholds(ctx, renumber):
    c = synth.collection(synth.short_sets(n=20_000))
    h = load(ctx, c, ssj.SSJ_VALIDATE | (ssj.SSJ_RENUMBER_BY_FREQ if renumber else 0))
    for p, q in [(9, 10), (4, 5), (7, 10), (3, 5)]:
        b = feeder_batch(c, p, q)
        want, _ = oracle.allpairs_self(c.offsets, c.tokens, p, q)
        want = oracle.sort_triples(want)
        assert np.array_equal(ora(c, c, True, p, q, b), want)
        for gran in GRANULARITIES:
            assert np.array_equal(gpu(ctx, h, h, p, q, b, gran), want), (p, q, gran)
    ssj.ssj_unload_collection(ctx, h)


def test_long_sets_scaled(ctx):
    c = synth.collection(synth.long_sets(n=1500))
    h = load(ctx, c)
    for p, q in [(3, 5), (4, 5)]:
        b = feeder_batch(c, p, q)
        want = oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, p, q)[0])
        for gran in GRANULARITIES:
            assert np.array_equal(gpu(ctx, h, h, p, q, b, gran), want), (p, q, gran)
        every = ora(c, c, True, p, q, b, flags=oracle.EMIT_ALL)
        for gran in GRANULARITIES:
            assert np.array_equal(gpu(ctx, h, h, p, q, b, ssj.SSJ_EMIT_ALL | gran), every), gran
    ssj.ssj_unload_collection(ctx, h)


def test_planted_long_sets_many_survivors(ctx):
    spec = synth.long_sets(n=800)
    spec.plant_frac, spec.plant_edits = 0.3, 20
    c = synth.collection(spec)
    h = load(ctx, c)
    b = feeder_batch(c, 3, 5)
    want = oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, 3, 5)[0])
    assert len(want) >= 10
    for gran in GRANULARITIES:
        assert np.array_equal(gpu(ctx, h, h, 3, 5, b, gran), want)
    ssj.ssj_unload_collection(ctx, h)


POLICIES = [1, 8, 24]


@pytest.mark.parametrize("bt", [256, 128 | ssj.SSJ_WIDE_REGISTERS, 512 | ssj.SSJ_WIDE_REGISTERS])
@pytest.mark.parametrize("policy", POLICIES)
def test_short_pair_policies(ctx, policy, bt):
    """Every short-pair refill threshold gives the oracle's join: tiny
    all pairs (also every overlap), scaled short and long sets, thread bin for all probes."""
    ssj.ssj_set_granularity(ctx, 1 << 30, 1, 1 << 30, bt)
    ssj.ssj_set_short_pairs(ctx, policy)
    try:
        c = planted_tiny(n=900)
        h = load(ctx, c)
        b = synth.all_pairs_batch(c.n)
        for p, q in [(4, 5), (3, 5)]:
            assert np.array_equal(gpu(ctx, h, h, p, q, b), ora(c, c, True, p, q, b)), (p, q)
        every = ora(c, c, True, 3, 5, b, flags=oracle.EMIT_ALL)
        assert np.array_equal(gpu(ctx, h, h, 3, 5, b, ssj.SSJ_EMIT_ALL), every)
        ssj.ssj_unload_collection(ctx, h)
        for spec, ths in ((synth.short_sets(n=20_000), [(9, 10), (7, 10), (3, 5)]),
                          (synth.long_sets(n=1200), [(3, 5), (4, 5)])):
            spec.plant_frac, spec.plant_edits = 0.2, 3
            c = synth.collection(spec)
            h = load(ctx, c, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
            for p, q in ths:
                b = feeder_batch(c, p, q)
                want = oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, p, q)[0])
                assert len(want) > 0
                assert np.array_equal(gpu(ctx, h, h, p, q, b), want), (p, q, len(want))
            ssj.ssj_unload_collection(ctx, h)
    finally:
        ssj.ssj_set_granularity(ctx, 128, 2048, 2048, 256)
        ssj.ssj_set_short_pairs(ctx, 0)


# ----------------------------------------------------------------- arbitrary batches

@pytest.mark.parametrize("seed", range(3))
def test_random_batches_self_and_rs(ctx, seed):
    cR = planted_tiny(n=700, frac=0.3, edits=1, seed=50 + seed)
    cS = planted_tiny(n=500, frac=0.3, edits=1, seed=80 + seed)
    hR, hS = load(ctx, cR), load(ctx, cS)
    b = synth.random_batch(seed, cR.n, cR.n, 3000, 40)
    b2 = synth.random_batch(seed + 100, cR.n, cS.n, 3000, 40)
    for p, q in [(1, 10), (1, 3), (3, 5)]:
        for gran in GRANULARITIES:
            assert np.array_equal(gpu(ctx, hR, hR, p, q, b, gran), ora(cR, cR, True, p, q, b))
            assert np.array_equal(gpu(ctx, hR, hS, p, q, b2, gran), ora(cR, cS, False, p, q, b2))
            assert np.array_equal(gpu(ctx, hR, hS, p, q, b2, gran | ssj.SSJ_EMIT_ALL),
                                  ora(cR, cS, False, p, q, b2, flags=oracle.EMIT_ALL))
    ssj.ssj_unload_collection(ctx, hR)
    ssj.ssj_unload_collection(ctx, hS)


def test_edge_sets_and_sizes(ctx):
    rng = np.random.default_rng(5)
    sets = [[], [7], [7], [1, 2, 3], [1, 2, 3], list(range(0, 6000, 2)), list(range(0, 6000, 2)),
            list(range(0, 5000, 2)) + [5001], list(range(1, 4000, 3)), list(range(100, 400)),
            list(range(100, 399)) + [1000]]
    for k in (31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 1023, 1024, 1025, 2047, 2048, 2049, 4093, 4100):
        base = np.sort(rng.choice(20_000, size=k, replace=False))
        other = base.copy()
        other[rng.integers(0, k)] = 20_001 + k
        sets.append(base.tolist())
        sets.append(np.unique(other).tolist())
    c = synth.from_lists(sets)
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    for p, q in [(1, 1), (9, 10), (1, 2), (1, 100)]:
        want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q))
        for gran in GRANULARITIES:
            assert np.array_equal(gpu(ctx, h, h, p, q, b, gran), want), (p, q, gran)
    every = ora(c, c, True, 1, 2, b, flags=oracle.EMIT_ALL)
    for gran in GRANULARITIES:
        assert np.array_equal(gpu(ctx, h, h, 1, 2, b, ssj.SSJ_EMIT_ALL | gran), every)
    ssj.ssj_unload_collection(ctx, h)


def test_set_tails_and_extreme_token_values(ctx):
    """Every tail shape of the last 16-byte block (lengths 1..13), the last token of a set equal to
    a token inside another set's block, and token values 0 and 2^32 - 1 (the padding repeats a
    set's last token, so no value is reserved)."""
    top = 0xFFFFFFFF
    rng = np.random.default_rng(11)
    sets = [[0], [top], [0, top], [top - 1, top], [5], [5, 6, 7, 8, 9], [1, 5, 9], [9], [4, 5, 6, 7],
            [4, 5, 6, 7, 8], [1, 2, 3, 4, 5, 6, 7, 8, 9], [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12],
            [3, 1 << 31, top], [1 << 31, top]]
    for n in range(1, 14):
        base = np.sort(rng.choice(40, size=n, replace=False)).tolist()
        sets.append(base)
        sets.append(sorted(set(base[:-1] + [top - n])))
        sets.append(sorted(set(base + [base[-1] + 1])) if base[-1] + 1 < 40 else base[:-1] + [41])
    c = synth.from_lists(sets)
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    try:
        for p, q in [(1, 1), (4, 5), (1, 2), (1, 100)]:
            want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q))
            assert len(want) > 0
            for gran in GRANULARITIES:
                assert np.array_equal(gpu(ctx, h, h, p, q, b, gran), want), (p, q, gran)
        every = ora(c, c, True, 1, 2, b, flags=oracle.EMIT_ALL)
        for gran in GRANULARITIES:
            assert np.array_equal(gpu(ctx, h, h, 1, 2, b, ssj.SSJ_EMIT_ALL | gran), every), gran
    finally:
        ssj.ssj_unload_collection(ctx, h)


def test_index_items_where_token_values_fit(ctx):
    """Index items hold the probe as a bitmap over token values, so they run only where every
    token value of the launch fits the bitmap: renumbered collections, or collections whose raw
    values are small.  Each workload here fits; it is checked with SSJ_FORCE_INDEX, with index
    items chosen by the candidate threshold (every probe: threshold 1), and with SSJ_EMIT_ALL
    (every overlap), against the oracle: planted all-pairs and long-set collections renumbered,
    empty / one-token / long edge sets and every tail shape with small raw values, and R x S
    batches between two collections of small raw values."""
    rng = np.random.default_rng(21)
    work = []
    c = planted_tiny(n=900)
    work.append((c, c, True, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ, synth.all_pairs_batch(c.n),
                 [(4, 5), (3, 5), (1, 10)]))
    spec = synth.long_sets(n=1500)
    spec.plant_frac, spec.plant_edits = 0.3, 20
    c = synth.collection(spec)
    work.append((c, c, True, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ, feeder_batch(c, 3, 5), [(3, 5), (4, 5)]))
    sets = [[], [7], [7], [1, 2, 3], [1, 2, 3], list(range(0, 6000, 2)), list(range(0, 6000, 2)),
            list(range(0, 5000, 2)) + [5001], list(range(1, 4000, 3)), list(range(100, 400)),
            list(range(100, 399)) + [1000], [0], [0, 1], [31, 32], [31], [32, 33, 63, 64, 65]]
    for n in range(1, 14):
        base = np.sort(rng.choice(40, size=n, replace=False)).tolist()
        sets.append(base)
        sets.append(sorted(set(base[:-1] + [60_000 - n])))
        sets.append(sorted(set(base + [base[-1] + 1])) if base[-1] + 1 < 40 else base[:-1] + [41])
    for k in (31, 33, 127, 129, 1023, 1025, 4093):
        base = np.sort(rng.choice(20_000, size=k, replace=False))
        other = base.copy()
        other[rng.integers(0, k)] = 20_001 + k
        sets.append(base.tolist())
        sets.append(np.unique(other).tolist())
    c = synth.from_lists(sets)
    work.append((c, c, True, ssj.SSJ_VALIDATE, synth.all_pairs_batch(c.n), [(1, 1), (9, 10), (1, 2), (1, 100)]))
    small = lambda n, seed: synth.from_lists(
        [np.unique(np.random.default_rng(seed + i).integers(0, 3000, size=int(k))).tolist()
         for i, k in enumerate(np.random.default_rng(seed).integers(1, 120, size=n))])
    cR, cS = small(400, 1000), small(300, 5000)
    work.append((cR, cS, False, ssj.SSJ_VALIDATE, synth.random_batch(9, cR.n, cS.n, 2000, 60),
                 [(1, 10), (1, 3), (3, 5)]))
    for cR, cS, selfj, lf, b, ths in work:
        hR = load(ctx, cR, lf)
        hS = hR if selfj else load(ctx, cS, lf)
        try:
            for p, q in ths:
                want = ora(cR, cS, selfj, p, q, b)
                assert np.array_equal(gpu(ctx, hR, hS, p, q, b, ssj.SSJ_FORCE_INDEX), want), (p, q)
                ssj.ssj_set_index_items(ctx, 1)
                try:
                    assert np.array_equal(gpu(ctx, hR, hS, p, q, b), want), (p, q)
                finally:
                    ssj.ssj_set_index_items(ctx, 256)
            p, q = ths[0]
            every = ora(cR, cS, selfj, p, q, b, flags=oracle.EMIT_ALL)
            assert np.array_equal(gpu(ctx, hR, hS, p, q, b, ssj.SSJ_FORCE_INDEX | ssj.SSJ_EMIT_ALL), every)
            assert ssj.ssj_device_error(ctx) == 0
        finally:
            ssj.ssj_unload_collection(ctx, hR)
            if not selfj:
                ssj.ssj_unload_collection(ctx, hS)


@pytest.mark.parametrize("bt", [256 | ssj.SSJ_BULK_STAGING, 512 | ssj.SSJ_BULK_STAGING,
                                128 | ssj.SSJ_WIDE_REGISTERS | ssj.SSJ_BULK_STAGING])
def test_bulk_staging_block_and_warp_items(ctx, bt):
    """Thread-block and warp items with their sets staged by bulk copies (SSJ_BULK_STAGING): long
    sets (raw and renumbered) at two thresholds, every overlap (SSJ_EMIT_ALL), and edge sets whose
    lengths straddle the whole-set buffers (sets of up to 6,000 tokens take the windowed path),
    against the oracle."""
    ssj.ssj_set_granularity(ctx, 0, 0, 0, bt)
    try:
        spec = synth.long_sets(n=1500)
        spec.plant_frac, spec.plant_edits = 0.3, 20
        c = synth.collection(spec)
        for lf in (ssj.SSJ_VALIDATE, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ):
            h = load(ctx, c, lf)
            for p, q in [(3, 5), (4, 5)]:
                b = feeder_batch(c, p, q)
                want = ora(c, c, True, p, q, b)
                assert len(want) > 0
                for gran in (ssj.SSJ_FORCE_BLOCK, ssj.SSJ_FORCE_WARP, ssj.SSJ_FORCE_LANE, 0):
                    assert np.array_equal(gpu(ctx, h, h, p, q, b, gran), want), (lf, p, q, gran)
            every = ora(c, c, True, 3, 5, b, flags=oracle.EMIT_ALL)
            for gran in (ssj.SSJ_FORCE_BLOCK, ssj.SSJ_FORCE_WARP):
                assert np.array_equal(gpu(ctx, h, h, 3, 5, b, gran | ssj.SSJ_EMIT_ALL), every), gran
            assert ssj.ssj_device_error(ctx) == 0
            ssj.ssj_unload_collection(ctx, h)
        rng = np.random.default_rng(31)
        sets = [[], [7], [7, 9], list(range(0, 6000, 2)), list(range(0, 6000, 2)), list(range(1, 6000, 3))]
        for k in (1, 3, 4, 5, 255, 256, 257, 1019, 1020, 1021, 2043, 2044, 2045, 2061, 4091, 4092, 4093):
            base = np.sort(rng.choice(12_000, size=k, replace=False))
            other = base.copy()
            other[rng.integers(0, k)] = 12_001 + k
            sets.append(base.tolist())
            sets.append(np.unique(other).tolist())
        c = synth.from_lists(sets)
        h = load(ctx, c)
        b = synth.all_pairs_batch(c.n)
        for p, q in [(1, 1), (9, 10), (1, 3)]:
            want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q))
            for gran in (ssj.SSJ_FORCE_BLOCK, ssj.SSJ_FORCE_WARP):
                assert np.array_equal(gpu(ctx, h, h, p, q, b, gran), want), (p, q, gran)
        every = ora(c, c, True, 1, 3, b, flags=oracle.EMIT_ALL)
        for gran in (ssj.SSJ_FORCE_BLOCK, ssj.SSJ_FORCE_WARP):
            assert np.array_equal(gpu(ctx, h, h, 1, 3, b, gran | ssj.SSJ_EMIT_ALL), every), gran
        assert ssj.ssj_device_error(ctx) == 0
        ssj.ssj_unload_collection(ctx, h)
    finally:
        ssj.ssj_set_granularity(ctx, 0, 0, 0, 256)


def test_pinned_collections_match_oracle():
    """Collections loaded with SSJ_PIN_L2 (the context's persisting-L2 set-aside raised, a
    persisting window on every launch that reads them) give the oracle's join through the
    synchronous call and a batched launch; unloading the pinned collections restores the
    set-aside and the context keeps working."""
    import torch
    pctx = ssj.ssj_create(0)
    try:
        spec = synth.long_sets(n=3000)
        spec.plant_frac, spec.plant_edits = 0.3, 20
        cl = synth.collection(spec)
        spec_s = synth.short_sets(n=30_000)
        spec_s.plant_frac, spec_s.plant_edits = 0.2, 2
        cs = synth.collection(spec_s)
        fl = ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ | ssj.SSJ_PIN_L2
        hl, hs = load(pctx, cl, fl), load(pctx, cs, fl)
        bl, bs = feeder_batch(cl, 3, 5), feeder_batch(cs, 7, 10)
        wl = oracle.sort_triples(oracle.allpairs_self(cl.offsets, cl.tokens, 3, 5)[0])
        ws = oracle.sort_triples(oracle.allpairs_self(cs.offsets, cs.tokens, 7, 10)[0])
        assert len(wl) > 0 and len(ws) > 0
        for gran in (0, ssj.SSJ_FORCE_INDEX, ssj.SSJ_FORCE_THREAD):
            assert np.array_equal(gpu(pctx, hl, hl, 3, 5, bl, gran), wl), gran
            assert np.array_equal(gpu(pctx, hs, hs, 7, 10, bs, gran), ws), gran
        res = ssj.ssj_verify_batches(pctx, [(hl, hl, 3, 5, bl.probe_ids, bl.cand_offsets, bl.cand_ids, 0),
                                            (hs, hs, 7, 10, bs.probe_ids, bs.cand_offsets, bs.cand_ids, 0)])
        assert np.array_equal(ssj.triples_to_array(res[0]), wl)
        assert np.array_equal(ssj.triples_to_array(res[1]), ws)
        assert ssj.ssj_device_error(pctx) == 0
        ssj.ssj_unload_collection(pctx, hl)
        ssj.ssj_unload_collection(pctx, hs)
        h2 = load(pctx, cs)  # not pinned, after the set-aside was restored
        assert np.array_equal(gpu(pctx, h2, h2, 7, 10, bs), ws)
        torch.cuda.synchronize()
    finally:
        ssj.ssj_destroy(pctx)


def test_empty_and_degenerate_batches(ctx):
    c = planted_tiny(n=50)
    h = load(ctx, c)
    empty = synth.Batch(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint32))
    assert len(gpu(ctx, h, h, 1, 2, empty)) == 0
    zero_c = synth.Batch(np.arange(5, dtype=np.uint32), np.zeros(6, np.uint64), np.zeros(0, np.uint32))
    assert len(gpu(ctx, h, h, 1, 2, zero_c)) == 0
    # only self pairs
    selfb = synth.Batch(np.arange(10, dtype=np.uint32), np.arange(11, dtype=np.uint64), np.arange(10, dtype=np.uint32))
    assert len(gpu(ctx, h, h, 1, 100, selfb)) == 0
    # many probes with zero candidates around a few with many (chunks span many probes)
    k = 200
    counts = np.zeros(k, dtype=np.int64)
    counts[[3, 77, 150]] = [40, 1, 33]
    offs = np.zeros(k + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(counts)
    cands = np.random.default_rng(1).integers(0, c.n, size=int(offs[-1])).astype(np.uint32)
    b = synth.Batch(np.random.default_rng(2).integers(0, c.n, size=k).astype(np.uint32), offs, cands)
    for gran in GRANULARITIES:
        assert np.array_equal(gpu(ctx, h, h, 1, 50, b, gran | ssj.SSJ_EMIT_ALL),
                              ora(c, c, True, 1, 50, b, flags=oracle.EMIT_ALL))
    ssj.ssj_unload_collection(ctx, h)


# ----------------------------------------------------------------- API behaviour

def test_count_only_sorted_and_capacity(ctx):
    c = planted_tiny(n=600, frac=0.3)
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, 1, 2))
    n = ssj.ssj_verify_batch(ctx, h, h, 1, 2, b.probe_ids, b.cand_offsets, b.cand_ids, flags=ssj.SSJ_COUNT_ONLY)
    assert n == len(want)
    res = ssj.ssj_verify_batch(ctx, h, h, 1, 2, b.probe_ids, b.cand_offsets, b.cand_ids, flags=ssj.SSJ_SORTED)
    arr = np.stack([res["r"], res["s"], res["overlap"]], axis=1)
    assert np.array_equal(arr, want)  # already in (r, s) order
    with pytest.raises(ssj.SsjError) as ei:
        ssj.ssj_verify_batch(ctx, h, h, 1, 2, b.probe_ids, b.cand_offsets, b.cand_ids, cap=len(want) - 1)
    assert ei.value.status == ssj.SSJ_ENOMEM
    ssj.ssj_unload_collection(ctx, h)


def test_invalid_inputs_are_rejected(ctx):
    c = planted_tiny(n=30)
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    for args in [(0, 2), (3, 2), (1, 2 ** 31)]:
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_verify_batch(ctx, h, h, *args, b.probe_ids, b.cand_offsets, b.cand_ids)
        assert ei.value.status == ssj.SSJ_EINVAL
    bad = b.cand_ids.copy()
    bad[5] = c.n
    with pytest.raises(ssj.SsjError):
        ssj.ssj_verify_batch(ctx, h, h, 1, 2, b.probe_ids, b.cand_offsets, bad)
    with pytest.raises(ssj.SsjError):
        ssj.ssj_verify_batch(ctx, h, 999, 1, 2, b.probe_ids, b.cand_offsets, b.cand_ids)
    unsorted = synth.from_lists([[3, 1]])
    with pytest.raises(ssj.SsjError):
        ssj.ssj_load_collection(ctx, unsorted.offsets, unsorted.tokens, ssj.SSJ_VALIDATE)
    hr = load(ctx, c, ssj.SSJ_RENUMBER_BY_FREQ)
    with pytest.raises(ssj.SsjError):
        ssj.ssj_verify_batch(ctx, h, hr, 1, 2, b.probe_ids, b.cand_offsets, b.cand_ids)
    assert ssj.ssj_collection_info(ctx, h) == (c.n, len(c.tokens))
    ssj.ssj_unload_collection(ctx, h)
    ssj.ssj_unload_collection(ctx, hr)


def test_device_pointers_sync_and_async(ctx):
    import torch
    c = planted_tiny(n=900, frac=0.2)
    h = load(ctx, c)
    b = synth.all_pairs_batch(c.n)
    want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, 3, 5))
    dev = torch.device("cuda:0")
    pr = torch.from_numpy(b.probe_ids.astype(np.int32)).to(dev)
    co = torch.from_numpy(b.cand_offsets.astype(np.int64)).to(dev)
    ci = torch.from_numpy(b.cand_ids.astype(np.int32)).to(dev)
    cap = 100_000
    out = torch.zeros(cap * 3, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()  # the library works on its own stream
    n = ssj.ssj_verify_batch(ctx, h, h, 3, 5, pr, co, ci, flags=ssj.SSJ_DEVICE_PTRS, out=out, cap=cap,
                             n_cands=b.n_cands)
    got = out[:3 * n].view(-1, 3).cpu().numpy().astype(np.uint32)
    assert np.array_equal(oracle.sort_triples(got), want)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    ssj.ssj_reserve(ctx, b.n_probes, b.n_cands)
    with torch.cuda.stream(stream):
        out.zero_()
        ssj.ssj_verify_batch_async(ctx, h, h, 3, 5, pr, co, ci, b.n_cands, out, cap, cnt,
                                   stream=stream.cuda_stream)
    stream.synchronize()
    n2 = int(cnt.item())
    got2 = out[:3 * n2].view(-1, 3).cpu().numpy().astype(np.uint32)
    assert np.array_equal(oracle.sort_triples(got2), want)
    assert ssj.ssj_device_error(ctx) == 0
    # a bad candidate id is caught on the device and reported
    ci_bad = ci.clone()
    ci_bad[17] = c.n + 5
    torch.cuda.synchronize()
    ssj.ssj_verify_batch_async(ctx, h, h, 3, 5, pr, co, ci_bad, b.n_cands, out, cap, cnt)
    assert ssj.ssj_device_error(ctx) & 2
    ssj.ssj_unload_collection(ctx, h)


def test_serving_results_alone_equal_results_in_the_mix(ctx):
    """Continuous batching: batches admitted together give what each gives alone."""
    c = synth.collection(synth.short_sets(n=30_000))
    h = load(ctx, c)
    batches = []
    for p, q in [(9, 10), (4, 5), (7, 10), (3, 5)]:
        b = feeder_batch(c, p, q)
        # split into uneven pieces
        cuts = [0, b.n_probes // 7, b.n_probes // 2, b.n_probes]
        for a, z in zip(cuts[:-1], cuts[1:]):
            o = b.cand_offsets[a:z + 1]
            batches.append(((p, q), synth.Batch(b.probe_ids[a:z], o - o[0], b.cand_ids[int(o[0]):int(o[-1])])))
    alone = [gpu(ctx, h, h, p, q, bb) for (p, q), bb in batches]
    sctx = ssj.ssj_create(0, mem_budget_bytes=256 << 20, max_inflight=3)
    try:
        hs = load(sctx, c)
        pending, done = {}, {}
        queue = list(enumerate(batches))
        while queue or pending:
            while queue:
                i, ((p, q), bb) = queue[0]
                t = ssj.ssj_submit(sctx, hs, hs, p, q, bb.probe_ids, bb.cand_offsets, bb.cand_ids)
                if t is None:
                    break
                pending[t] = i
                queue.pop(0)
            for t in list(pending):
                if ssj.ssj_poll(sctx, t, 1):
                    done[pending.pop(t)] = ssj.triples_to_array(ssj.ssj_results(sctx, t))
        for i, want in enumerate(alone):
            assert np.array_equal(done[i], want), i
    finally:
        ssj.ssj_destroy(sctx)
    ssj.ssj_unload_collection(ctx, h)


# ----------------------------------------------------------------- full-size workloads

def test_full_short_sets_all_thresholds(ctx):
    """200,000 short sets (the bench workload), every threshold, exact result sets."""
    c = synth.collection(synth.short_sets())
    h = load(ctx, c, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
    for p, q in [(9, 10), (4, 5), (7, 10), (3, 5)]:
        b = feeder_batch(c, p, q)
        want = oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, p, q)[0])
        assert np.array_equal(gpu(ctx, h, h, p, q, b), want), (p, q)
    ssj.ssj_unload_collection(ctx, h)


def _exact_against_threaded_oracle(ctx, c, h, p, q, b, flags=0):
    """GPU triples of one batch against the oracle's over the same batch (split over probe ranges
    on every host core), element by element; returns the oracle's sorted triples."""
    want = oracle.sort_triples(oracle.verify_batch_threads(c.offsets, c.tokens, c.offsets, c.tokens, True, p, q,
                                                           b.probe_ids, b.cand_offsets, b.cand_ids))
    got = gpu(ctx, h, h, p, q, b, flags)
    assert np.array_equal(got, want), (flags, len(got), len(want))
    n = ssj.ssj_verify_batch(ctx, h, h, p, q, b.probe_ids, b.cand_offsets, b.cand_ids,
                             flags=flags | ssj.SSJ_COUNT_ONLY)
    assert n == len(want)
    return want


def test_full_long_sets_exact(ctx):
    """50,000 long sets at t = 3/5 (about 9.2e7 candidates): the sorted (r, s, overlap) list of the
    whole batch equals the oracle's, element by element.  The positional filter rejects every
    candidate of this collection, so the same collection with 20% of its sets replaced by edited
    copies (40 tokens changed) is checked the same way: there several hundred candidates pass,
    with overlaps from about 100 to about 800."""
    c = synth.collection(synth.long_sets())
    h = load(ctx, c, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
    b = feeder_batch(c, 3, 5, threads=16)
    assert b.n_cands > 50_000_000
    _exact_against_threaded_oracle(ctx, c, h, 3, 5, b)
    ssj.ssj_unload_collection(ctx, h)
    spec = synth.long_sets()
    spec.plant_frac, spec.plant_edits = 0.2, 40
    c = synth.collection(spec)
    h = load(ctx, c, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
    b = feeder_batch(c, 3, 5, threads=16)
    want = _exact_against_threaded_oracle(ctx, c, h, 3, 5, b)
    assert len(want) > 500
    # the same candidates as three host batches in one ssj_verify_batches call: large enough that
    # the call runs two launches, the second group's copies overlapping the first group's kernels
    co = b.cand_offsets.astype(np.int64)
    cuts = [0, b.n_probes // 5, b.n_probes // 2, b.n_probes]
    parts = []
    for a, z in zip(cuts[:-1], cuts[1:]):
        parts.append((h, h, 3, 5, b.probe_ids[a:z], (co[a:z + 1] - co[a]).astype(np.uint64),
                      b.cand_ids[co[a]:co[z]], 0))
    res = ssj.ssj_verify_batches(ctx, parts, caps=[len(want) + 16] * 3)
    got = ssj.triples_to_array(np.concatenate(res))
    assert np.array_equal(got, want)
    assert ssj.ssj_device_error(ctx) == 0
    # the same call with the inputs in pinned host memory: the kernels read them over the host
    # link (the default for a call this large), or, with SSJ_HOST_STAGED, they are copied first
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    pinned = [(hh, hs, p, q, pin(pr), pin(po), pin(pc), 0) for hh, hs, p, q, pr, po, pc, _ in parts]
    for fl in (0, ssj.SSJ_HOST_STAGED):
        res = ssj.ssj_verify_batches(ctx, [x[:7] + (fl,) for x in pinned], caps=[len(want) + 16] * 3)
        assert np.array_equal(ssj.triples_to_array(np.concatenate(res)), want), fl
    assert ssj.ssj_device_error(ctx) == 0
    ssj.ssj_unload_collection(ctx, h)


def test_full_serving_collection_and_served_slices(ctx):
    """The 1,000,000-set serving collection: the whole self-join at t in {0.7, 0.8, 0.9} exact
    against the oracle, then request-sized slices (1e3..1e7 pairs) of its candidates submitted
    through the serving path, each equal to the oracle on that slice."""
    c = synth.collection(synth.serving_collection())
    h = load(ctx, c, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
    try:
        batches = {}
        for p, q in [(7, 10), (4, 5), (9, 10)]:
            b = feeder_batch(c, p, q, threads=16)
            batches[(p, q)] = b
            want = ora(c, c, True, p, q, b)
            assert np.array_equal(gpu(ctx, h, h, p, q, b), want), (p, q)
        b = batches[(7, 10)]
        co = b.cand_offsets.astype(np.int64)
        rng = np.random.default_rng(5)
        tickets = []
        sctx = ssj.ssj_create(0, mem_budget_bytes=1 << 30, max_inflight=4)
        hs = ssj.ssj_load_collection(sctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
        try:
            for want_pairs in (1_000, 30_000, 1_000_000, 8_000_000):
                a = int(rng.integers(0, len(b.probe_ids) // 2))
                e = int(np.searchsorted(co, co[a] + want_pairs, side="left"))
                e = max(a + 1, min(e, len(b.probe_ids)))
                sl = synth.Batch(b.probe_ids[a:e], (co[a:e + 1] - co[a]).astype(np.uint64),
                                 b.cand_ids[co[a]:co[e]])
                t = None
                while t is None:
                    t = ssj.ssj_submit(sctx, hs, hs, 7, 10, sl.probe_ids, sl.cand_offsets, sl.cand_ids)
                    if t is None:
                        for tt, ww in tickets:
                            ssj.ssj_poll(sctx, tt, timeout_ms=100)
                tickets.append((t, ora(c, c, True, 7, 10, sl)))
            for t, want in tickets:
                assert ssj.ssj_poll(sctx, t, timeout_ms=-1)
                assert np.array_equal(ssj.triples_to_array(ssj.ssj_results(sctx, t)), want)
        finally:
            ssj.ssj_destroy(sctx)
    finally:
        ssj.ssj_unload_collection(ctx, h)
