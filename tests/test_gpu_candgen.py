"""Self-join with candidate generation on the device (ssj_self_join): the join result
equals the oracle's AllPairs join (and brute force) bit for bit, and with the collection
renumbered by frequency the device generates exactly the oracle's AllPairs candidates."""
import numpy as np
import pytest

import oracle
import synth

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build

pytestmark = pytest.mark.gpu

SIM_FLAGS = {oracle.JACCARD: ssj.SSJ_SIM_JACCARD, oracle.DICE: ssj.SSJ_SIM_DICE,
             oracle.COSINE: ssj.SSJ_SIM_COSINE, oracle.OVERLAP: ssj.SSJ_SIM_OVERLAP}
CASES = [(oracle.JACCARD, (9, 10)), (oracle.JACCARD, (4, 5)), (oracle.JACCARD, (3, 5)), (oracle.DICE, (4, 5)),
         (oracle.COSINE, (7, 10)), (oracle.OVERLAP, (8, 1))]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    h = ssj.ssj_create(0)
    yield h
    ssj.ssj_destroy(h)


def _collections():
    tiny = synth.tiny_self_join(seed=1001, n=800)
    tiny.plant_frac, tiny.plant_edits = 0.15, 2
    short = synth.short_sets(n=20_000)
    short.plant_frac, short.plant_edits = 0.2, 2
    long_ = synth.long_sets(n=800)
    long_.plant_frac, long_.plant_edits = 0.3, 10
    return [synth.collection(x) for x in (tiny, short, long_)]


@pytest.mark.parametrize("sim,pq", CASES)
def test_self_join_matches_oracle_allpairs(ctx, sim, pq):
    for c in _collections():
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
        try:
            want, want_cands = oracle.allpairs_self(c.offsets, c.tokens, *pq, sim=sim)
            want = oracle.sort_triples(want)
            got, n_cands = ssj.ssj_self_join(ctx, h, *pq, SIM_FLAGS[sim])
            assert np.array_equal(ssj.triples_to_array(got), want), (sim, pq, c.n, len(got), len(want))
            assert n_cands == want_cands, (sim, pq, c.n)
            # the positional bound drops candidates, never results
            got_p, n_p = ssj.ssj_self_join(ctx, h, *pq, SIM_FLAGS[sim] | ssj.SSJ_JOIN_POSITIONAL)
            assert np.array_equal(ssj.triples_to_array(got_p), want)
            assert n_p <= n_cands
        finally:
            ssj.ssj_unload_collection(ctx, h)


def test_self_join_raw_tokens_count_only_device_and_sorted(ctx):
    import torch
    # raw (not renumbered) token values, small enough for the device prefix index
    rng = np.random.default_rng(77)
    lists = [sorted(rng.choice(300, size=int(rng.integers(1, 40)), replace=False).tolist()) for _ in range(500)]
    lists += [sorted(set(x) | {299 - i % 7}) for i, x in enumerate(lists[:100])]
    c = synth.from_lists(lists)
    want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, 3, 5))
    assert len(want) > 10
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)  # raw token order
    try:
        got, _ = ssj.ssj_self_join(ctx, h, 3, 5, ssj.SSJ_SORTED)
        arr = np.stack([got["r"], got["s"], got["overlap"]], 1).astype(np.uint32)
        assert np.array_equal(arr, want)  # already in (r, s) order
        cnt, _ = ssj.ssj_self_join(ctx, h, 3, 5, ssj.SSJ_COUNT_ONLY)
        assert cnt == len(want)
        out = torch.zeros(3 * max(len(want), 1), dtype=torch.int32, device="cuda:0")
        cnt2, _ = ssj.ssj_self_join(ctx, h, 3, 5, ssj.SSJ_DEVICE_PTRS, cap=len(want), out=out)
        assert cnt2 == len(want)
        dev = oracle.sort_triples(out[:3 * cnt2].view(-1, 3).cpu().numpy().astype(np.uint32))
        assert np.array_equal(dev, want)
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_self_join(ctx, h, 3, 5, 0, cap=max(len(want) - 1, 1))
        assert ei.value.status == ssj.SSJ_ENOMEM
        for gran in (ssj.SSJ_FORCE_THREAD, ssj.SSJ_FORCE_LANE, ssj.SSJ_FORCE_WARP, ssj.SSJ_FORCE_BLOCK,
                     ssj.SSJ_FORCE_INDEX):
            g, _ = ssj.ssj_self_join(ctx, h, 3, 5, gran)
            assert np.array_equal(ssj.triples_to_array(g), want), gran
    finally:
        ssj.ssj_unload_collection(ctx, h)


def test_self_join_degenerate_collections(ctx):
    for lists in ([], [[1, 2, 3]], [[], [], [5]], [[1, 2], [1, 2], [1, 2]]):
        c = synth.from_lists(lists)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
        try:
            got, _ = ssj.ssj_self_join(ctx, h, 4, 5)
            want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, 4, 5))
            assert np.array_equal(ssj.triples_to_array(got), want), lists
        finally:
            ssj.ssj_unload_collection(ctx, h)


@pytest.mark.parametrize("sim,pq", CASES)
def test_group_join_expanded_on_the_device(ctx, sim, pq):
    """GroupJoin candidates expanded and verified on the device equal the oracle's AllPairs join,
    and the expanded pairs are exactly the AllPairs candidates."""
    specs = []
    for frac, edits in ((0.3, 0), (0.2, 2)):
        spec = synth.tiny_self_join(seed=1001, n=800)
        spec.plant_frac, spec.plant_edits = frac, edits
        specs.append(spec)
    short = synth.short_sets(n=20_000)
    short.plant_frac, short.plant_edits = 0.2, 0
    specs.append(short)
    for spec in specs:
        c = synth.collection(spec)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
        try:
            want, want_cands = oracle.allpairs_self(c.offsets, c.tokens, *pq, sim=sim)
            g = ssj.group_candidates(c.offsets, c.tokens, *pq, sim=sim)
            assert g.n_pairs == want_cands
            got, n_pairs = ssj.ssj_verify_groups(ctx, h, *pq, g, SIM_FLAGS[sim])
            assert n_pairs == want_cands
            assert np.array_equal(ssj.triples_to_array(got), oracle.sort_triples(want)), (sim, pq, c.n)
            cnt, _ = ssj.ssj_verify_groups(ctx, h, *pq, g, SIM_FLAGS[sim] | ssj.SSJ_COUNT_ONLY | ssj.SSJ_FORCE_WARP)
            assert cnt == len(want)
        finally:
            ssj.ssj_unload_collection(ctx, h)
