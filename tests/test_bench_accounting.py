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
