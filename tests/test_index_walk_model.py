"""The walk the index items run, restated on the host and checked against exact set
intersection (CPU only).  The probe r is a bitmap over token values; the candidate s is laid
out in 4-token blocks whose padding repeats its last token.  A step tests the four tokens of s's
current block against the bitmap, then stops at s's last block (subtracting the repeated padding
lanes there) or when the block's last token reaches r's last token (no later token of s can
match), and otherwise rejects once the overlap so far plus the tokens of s left falls below req.  The
claims the kernel relies on: a pair that is not rejected ends with o = |r ∩ s| exactly, a pair
whose overlap reaches req is never rejected, and the walk reads no more blocks of s than
needed to pass r's last token."""
import numpy as np
import pytest


def blocks(tokens):
    t = list(tokens)
    if not t:
        return []
    t += [t[-1]] * ((-len(t)) % 4)
    return [t[k:k + 4] for k in range(0, len(t), 4)]


def index_walk(r, s, req=0, early=False):
    """(overlap counted, rejected, blocks of s read) of the index walk."""
    bitmap = set(r)  # one bit per token value of r
    rmax = r[-1] if len(r) else 0
    o, rems, read = 0, len(s), 0
    if not len(r):
        return 0, False, 0
    for blk in blocks(s):
        read += 1
        bits = [1 if x in bitmap else 0 for x in blk]
        o += sum(bits)
        if rems <= 4 or blk[3] >= rmax:  # s's last block, or no later token of s can match
            if rems < 4:
                o -= (4 - rems) * bits[3]  # the lanes past s's end repeat its last token
            return o, False, read
        rems -= 4
        if early and o + rems < req:
            return o, True, read
    return o, False, read


def _random_sets(rng, n, vocab, lo, hi):
    return [np.unique(rng.integers(0, vocab, size=int(rng.integers(lo, hi + 1)))).tolist() for _ in range(n)]


@pytest.mark.parametrize("vocab", [8, 40, 1000])
def test_overlap_is_exact_on_every_tail_shape(vocab):
    rng = np.random.default_rng(vocab)
    sets = _random_sets(rng, 120, vocab, 0, 14) + [[0], [vocab - 1], list(range(min(vocab, 13)))]
    for r in sets:
        for s in sets:
            o, rej, _ = index_walk(r, s)
            assert not rej
            assert o == len(set(r) & set(s)), (r, s)


def test_bound_never_rejects_a_passing_pair():
    rng = np.random.default_rng(7)
    sets = _random_sets(rng, 150, 60, 1, 30)
    for r in sets:
        for s in sets:
            true_o = len(set(r) & set(s))
            for req in range(0, min(len(r), len(s)) + 1):
                o, rej, _ = index_walk(r, s, req, early=True)
                if true_o >= req:
                    assert not rej and o == true_o, (r, s, req)
                elif not rej:
                    # a pair that runs to its end is still decided correctly by the final test
                    assert o == true_o and o < req


def test_walk_stops_at_r_last_token():
    r = [3, 9, 12]
    s = list(range(0, 40, 1))
    o, rej, read = index_walk(r, s)
    assert (o, rej) == (3, False)
    assert read == 4  # the block holding 12 is the last one read
    assert index_walk([], [1, 2]) == (0, False, 0)
    assert index_walk([5], []) == (0, False, 0)
