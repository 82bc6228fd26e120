"""Serving drivers: open-loop replay and the filter/verify co-process."""
import numpy as np
import pytest

import oracle
import synth

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build

pytestmark = pytest.mark.gpu


def test_replay_counts_match_single_batches():
    import torch
    assert torch.cuda.is_available()
    _build.build()
    spec = synth.short_sets(n=20_000)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    ctx = ssj.ssj_create(0, mem_budget_bytes=64 << 20, max_inflight=3)
    try:
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
        reqs, want = [], []
        rng = np.random.default_rng(0)
        for i, (p, q) in enumerate([(3, 5), (7, 10), (4, 5), (9, 10)] * 5):
            pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=4)
            k = int(rng.integers(1, len(pr)))
            a = int(rng.integers(0, len(pr) - k + 1))
            offs = (co[a:a + k + 1] - co[a]).astype(np.uint64)
            cands = ci[int(co[a]):int(co[a + k])]
            reqs.append((h, h, p, q, pr[a:a + k], offs, cands, 0.0005 * i, 0))
            want.append(len(ssj.ssj_verify_batch(ctx, h, h, p, q, pr[a:a + k], offs, cands)))
        lat, st = ssj.ssj_serve_replay(ctx, reqs)
        assert np.all(lat >= 0)
        assert st["results"] == sum(want)
        assert st["pairs"] == sum(len(r[6]) for r in reqs)
    finally:
        ssj.ssj_destroy(ctx)


def test_coprocess_finds_the_join():
    spec = synth.short_sets(n=30_000)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    ctx = ssj.ssj_create(0, mem_budget_bytes=32 << 20, max_inflight=2)
    try:
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
        st = ssj.ssj_serve_coprocess(ctx, h, c.offsets, c.tokens, 3, 5, 4, 10_000)
        _, n_cands = oracle.allpairs_self(c.offsets, c.tokens, 3, 5)
        ap, _ = oracle.allpairs_self(c.offsets, c.tokens, 3, 5)
        assert st["candidates"] == n_cands
        assert st["results"] == len(ap)
        assert st["chunks"] >= n_cands // 10_000
        assert st["join_s"] > 0 and st["filter_only_s"] > 0
    finally:
        ssj.ssj_destroy(ctx)


def test_submit_from_pinned_inputs_then_overwrite():
    """Pinned inputs are copied straight from the caller's arrays; once ssj_submit returns the
    caller may overwrite them (here: with ids that would fail the device checks) without
    changing the result.  Mixed pinned and pageable arrays in one batch take both paths."""
    import torch
    _build.build()
    spec = synth.short_sets(n=20_000)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, 3, 5, n_threads=4)
    want = oracle.sort_triples(oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 3, 5,
                                                   pr, co, ci))

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    ctx = ssj.ssj_create(0, mem_budget_bytes=256 << 20, max_inflight=2)
    try:
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
        for mask in range(8):  # which of probe_ids / cand_offsets / cand_ids are pinned
            arrs = [pinned(a) if mask >> i & 1 else a.copy() for i, a in enumerate((pr, co, ci))]
            t = ssj.ssj_submit(ctx, h, h, 3, 5, *arrs)
            assert t is not None
            for a in arrs:
                a[:] = np.iinfo(a.dtype).max
            assert ssj.ssj_poll(ctx, t, timeout_ms=-1)
            got = ssj.ssj_results(ctx, t)
            np.testing.assert_array_equal(ssj.triples_to_array(got), want)
    finally:
        ssj.ssj_destroy(ctx)


def test_keep_inputs_submissions_match_single_batches():
    """SSJ_KEEP_INPUTS: the call does not wait for the copies of pinned inputs; with the inputs kept
    until the tickets are done, every result equals the synchronous call's."""
    import torch
    _build.build()
    spec = synth.short_sets(n=20_000)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    ctx = ssj.ssj_create(0, mem_budget_bytes=256 << 20, max_inflight=4)
    try:
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
        pinned = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        jobs = []
        for p, q in [(3, 5), (7, 10), (4, 5), (9, 10)]:
            pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=4)
            arrs = (pinned(pr), pinned(co), pinned(ci))
            want = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, p, q, *arrs))
            t = None
            while t is None:
                t = ssj.ssj_submit(ctx, h, h, p, q, *arrs, flags=ssj.SSJ_KEEP_INPUTS)
            jobs.append((t, want, arrs))
        for t, want, _arrs in jobs:
            assert ssj.ssj_poll(ctx, t, timeout_ms=-1)
            np.testing.assert_array_equal(ssj.triples_to_array(ssj.ssj_results(ctx, t)), want)
    finally:
        ssj.ssj_destroy(ctx)
