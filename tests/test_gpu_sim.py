"""GPU parity for the Dice, Cosine and plain-overlap thresholds (Table "Similarity
Functions", Section 2.2.2): bit-exact sorted (r, s, overlap) triples against the
oracle on the same seeded inputs, at every granularity.
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
SIM_FLAGS = {oracle.DICE: ssj.SSJ_SIM_DICE, oracle.COSINE: ssj.SSJ_SIM_COSINE, oracle.OVERLAP: ssj.SSJ_SIM_OVERLAP}
THRESHOLDS = {oracle.DICE: [(9, 10), (4, 5), (3, 5)], oracle.COSINE: [(19, 20), (4, 5), (3, 5)],
              oracle.OVERLAP: [(5, 1), (12, 1), (23, 2)]}


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    h = ssj.ssj_create(0)
    yield h
    ssj.ssj_destroy(h)


def _gpu(ctx, h, p, q, b, flags):
    return ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, p, q, b.probe_ids, b.cand_offsets, b.cand_ids,
                                                     flags=flags))


def _ora(c, p, q, b, sim):
    return oracle.sort_triples(oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, p, q,
                                                   b.probe_ids, b.cand_offsets, b.cand_ids, sim=sim))


@pytest.mark.parametrize("sim", list(SIM_FLAGS))
@pytest.mark.parametrize("gran", GRANULARITIES)
def test_all_pairs_planted(ctx, sim, gran):
    spec = synth.tiny_self_join(seed=1001, n=700)
    spec.plant_frac, spec.plant_edits = 0.15, 2
    c = synth.collection(spec)
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    b = synth.all_pairs_batch(c.n)
    try:
        for p, q in THRESHOLDS[sim]:
            want = _ora(c, p, q, b, sim)
            assert np.array_equal(want, oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim)))
            got = _gpu(ctx, h, p, q, b, SIM_FLAGS[sim] | gran)
            assert np.array_equal(got, want), (sim, gran, p, q, len(got), len(want))
            assert len(want) > 0
    finally:
        ssj.ssj_unload_collection(ctx, h)


@pytest.mark.parametrize("sim", list(SIM_FLAGS))
@pytest.mark.parametrize("gran", GRANULARITIES)
def test_feeder_candidates_short_and_long(ctx, sim, gran):
    """Prefix-filter candidates of each function on scaled short and long collections (sizes
    spanning every bin), against the oracle's AllPairs join of the same function."""
    short = synth.short_sets(n=15_000)
    short.plant_frac, short.plant_edits = 0.2, 2
    long_ = synth.long_sets(n=700)
    long_.plant_frac, long_.plant_edits = 0.3, 10
    for spec in (short, long_):
        c = synth.collection(spec)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
        try:
            for p, q in THRESHOLDS[sim][1:]:
                pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=8, sim=sim)
                b = synth.Batch(pr, co, ci)
                got = _gpu(ctx, h, p, q, b, SIM_FLAGS[sim] | gran)
                want, n_cands = oracle.allpairs_self(c.offsets, c.tokens, p, q, sim)
                assert n_cands == len(ci)
                assert np.array_equal(got, oracle.sort_triples(want)), (sim, gran, p, q, len(got), len(want))
        finally:
            ssj.ssj_unload_collection(ctx, h)


def test_mixed_functions_in_one_launch(ctx):
    """Four instances, one per function, in one batched launch: each equals its single call."""
    import torch
    spec = synth.tiny_self_join(seed=4242, n=500)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    b = synth.all_pairs_batch(c.n)
    dev = torch.device("cuda:0")
    t = (torch.from_numpy(b.probe_ids.astype(np.int32)).to(dev),
         torch.from_numpy(b.cand_offsets.astype(np.int64)).to(dev),
         torch.from_numpy(b.cand_ids.astype(np.int32)).to(dev))
    cases = [(oracle.JACCARD, ssj.SSJ_SIM_JACCARD, 3, 5), (oracle.DICE, ssj.SSJ_SIM_DICE, 3, 5),
             (oracle.COSINE, ssj.SSJ_SIM_COSINE, 3, 5), (oracle.OVERLAP, ssj.SSJ_SIM_OVERLAP, 9, 1)]
    dbs, outs = [], []
    for _, fl, p, q in cases:
        dbs.append(ssj.DeviceBatch(h, h, p, q, *t, b.n_cands, flags=fl, n_probes=b.n_probes))
        outs.append(torch.zeros(3 * b.n_cands, dtype=torch.int32, device=dev))
    counts = torch.zeros(len(cases), dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    m = ssj.ssj_multi_create(ctx, dbs, outs, [b.n_cands] * len(cases), counts)
    try:
        ssj.ssj_multi_launch(ctx, m)
        torch.cuda.synchronize()
        assert ssj.ssj_device_error(ctx) == 0
        n = counts.cpu().numpy()
        for i, (sim, _, p, q) in enumerate(cases):
            got = oracle.sort_triples(outs[i][:3 * int(n[i])].view(-1, 3).cpu().numpy().astype(np.uint32))
            assert np.array_equal(got, _ora(c, p, q, b, sim)), sim
    finally:
        ssj.ssj_multi_destroy(ctx, m)
        ssj.ssj_unload_collection(ctx, h)


def test_threshold_validation(ctx):
    c = synth.collection(synth.tiny_self_join(seed=5, n=50))
    h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
    b = synth.all_pairs_batch(c.n)
    try:
        with pytest.raises(ssj.SsjError):
            _gpu(ctx, h, 6, 5, b, ssj.SSJ_SIM_COSINE)
        with pytest.raises(ssj.SsjError):
            _gpu(ctx, h, 0, 5, b, ssj.SSJ_SIM_DICE)
        # the plain overlap threshold may exceed 1 (p > q)
        got = _gpu(ctx, h, 7, 2, b, ssj.SSJ_SIM_OVERLAP)
        assert np.array_equal(got, _ora(c, 7, 2, b, oracle.OVERLAP))
    finally:
        ssj.ssj_unload_collection(ctx, h)


@pytest.mark.parametrize("gran", GRANULARITIES)
def test_rs_join_from_the_feeder(ctx, gran):
    """An R x S join: the feeder's candidates of R against S (AllPairs and PPJoin) verified on the
    GPU equal the oracle's brute-force R x S join, for each function."""
    r_spec = synth.short_sets(seed=61, n=3000)
    r_spec.vocab = 3000
    s_spec = synth.short_sets(seed=62, n=4000)
    s_spec.vocab = 3000
    cr, cs = synth.collection(r_spec), synth.collection(s_spec)
    # plant near-copies of some sets of R in S
    S = [cs.tokens[cs.offsets[i]:cs.offsets[i + 1]].tolist() for i in range(cs.n)]
    for i in range(0, cr.n, 10):
        S[i] = sorted(set(cr.tokens[cr.offsets[i]:cr.offsets[i + 1]].tolist()) | {10**6 + i})
    cs = synth.from_lists(S)
    hr = ssj.ssj_load_collection(ctx, cr.offsets, cr.tokens)
    hs = ssj.ssj_load_collection(ctx, cs.offsets, cs.tokens)
    try:
        for sim, (p, q) in [(oracle.JACCARD, (4, 5)), (oracle.DICE, (4, 5)), (oracle.COSINE, (3, 5)),
                            (oracle.OVERLAP, (9, 1))]:
            want = oracle.sort_triples(oracle.bruteforce_rs(cr.offsets, cr.tokens, cs.offsets, cs.tokens, p, q,
                                                            sim=sim))
            assert len(want) > 0
            flags = SIM_FLAGS.get(sim, ssj.SSJ_SIM_JACCARD)
            for fl in (0, ssj.SSJ_FEEDER_PPJOIN):
                pr, co, ci = ssj.feeder_all(cr.offsets, cr.tokens, p, q, n_threads=8, sim=sim,
                                            s_offsets=cs.offsets, s_tokens=cs.tokens, flags=fl)
                got = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, hr, hs, p, q, pr, co, ci, flags=flags | gran))
                assert np.array_equal(got, want), (sim, fl, gran, len(got), len(want))
    finally:
        ssj.ssj_unload_collection(ctx, hr)
        ssj.ssj_unload_collection(ctx, hs)
