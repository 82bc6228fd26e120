"""bench.py's algorithmic byte count (A_min and the looser A_pair) on small batches, CPU only."""
import numpy as np

import bench
import oracle
import synth


def _acc(c, batch, p=4, q=5):
    return bench.oracle_accounting([c], [(0, p, q, batch.probe_ids, batch.cand_offsets, batch.cand_ids)])[0]


def test_a_min_formula_and_a_pair_bound():
    c = synth.collection(synth.tiny_self_join(seed=1001, n=200))
    b = synth.all_pairs_batch(c.n)
    a = _acc(c, b)
    tr, cr, cs = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 4, 5, b.probe_ids,
                                     b.cand_offsets, b.cand_ids, consumed=True)
    n_pr, n_ci = len(b.probe_ids), len(b.cand_ids)
    counts = np.diff(b.cand_offsets.astype(np.int64))
    starts = b.cand_offsets[:-1].astype(np.int64)
    # the probe's tokens once per probe: the deepest stop point among its candidates
    max_r = sum(int(cr[s:s + k].max()) for s, k in zip(starts, counts) if k)
    want = 12 * n_pr + 4 * n_ci + 8 * (n_pr + n_ci) + 4 * max_r + 4 * int(cs.sum()) + 12 * len(tr) + 8
    assert a["bytes"] == want
    assert a["hbm_bytes"] == 12 * n_pr + 4 * n_ci + 12 * len(tr) + 8
    assert a["pair_bytes"] - a["bytes"] == 4 * (int(cr.sum()) - max_r) >= 0
    assert a["survivors"] == len(tr) and a["pairs"] == n_ci


def test_a_pair_equals_a_min_with_one_candidate_per_probe():
    c = synth.collection(synth.tiny_self_join(seed=7, n=100))
    probes = np.arange(0, 50, dtype=np.uint32)
    cands = np.arange(50, 100, dtype=np.uint32)
    b = synth.Batch(probes, np.arange(51, dtype=np.uint64), cands)
    a = _acc(c, b, 3, 5)
    assert a["pair_bytes"] == a["bytes"]


def test_stride_sample_takes_whole_probes_at_a_uniform_stride():
    """The CPU baseline's sample: every k-th probe of each batch with all of its candidates (not a
    prefix of the feeder's size-ordered probes), about the asked number of candidates."""
    batches = []
    for seed, probes, per in ((3, 400, 60), (4, 250, 30)):
        b = synth.random_batch(seed, 500, 500, probes, per)
        batches.append((0, 3, 5, b.probe_ids, b.cand_offsets, b.cand_ids))
    total = sum(len(b[5]) for b in batches)
    sample, k = bench.stride_sample(batches, total // 7)
    assert k == -(-total // (total // 7))
    for (_, _, _, pr, co, ci), (_, _, _, spr, sco, sci) in zip(batches, sample):
        pick = np.arange(0, len(pr), k)
        assert np.array_equal(spr, pr[pick])
        co64 = co.astype(np.int64)
        want = np.concatenate([ci[co64[a]:co64[a + 1]] for a in pick])
        assert np.array_equal(sci, want)
        assert int(sco[0]) == 0 and int(sco[-1]) == len(sci) and len(sco) == len(spr) + 1
    whole, k1 = bench.stride_sample(batches, total)
    assert k1 == 1 and whole is batches


def test_both_arms_report_the_same_config():
    """The GPU arm and the reference arm build their `config` with the same function from the same
    workload and candidates, so the two lines can be compared key by key."""
    import types
    args = types.SimpleNamespace(sim="jaccard", ppjoin=False, workload="short_sets")
    cfg = {"workload": "short_sets", "n_sets": 10}
    b = synth.random_batch(1, 50, 50, 20, 5)
    batches = [(0, 3, 5, b.probe_ids, b.cand_offsets, b.cand_ids)]
    c1, c2 = bench.common_config(cfg, batches, args), bench.common_config(dict(cfg), batches, args)
    assert c1 == c2 and c1["pairs_per_step"] == len(b.cand_ids) and c1["instances_per_launch"] == 1
