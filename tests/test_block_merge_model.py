"""The block merge the thread-per-pair kernels run, restated on the host and checked against
exact set intersection (CPU only).  Sets are laid out in 4-token blocks whose padding repeats
the set's last token; a step counts the matches between the current blocks of r and s (four
membership tests of r's lanes in s's block, minus the repeated lanes of r's last block), then
advances the block with the smaller last lane (both on a tie).  The claims the kernels rely on:
every common token is counted exactly once, so the count equals |r ∩ s|, and the positional
bound o + min(|r| - 4i, |s| - 4j) never rejects a pair whose overlap reaches req."""
import numpy as np
import pytest


def blocks(tokens):
    t = list(tokens)
    if not t:
        return []
    t += [t[-1]] * ((-len(t)) % 4)
    return [t[k:k + 4] for k in range(0, len(t), 4)]


def block_matches(rb, sb, nvr):
    m = [1 if x in sb else 0 for x in rb]
    return sum(m) - (4 - nvr) * m[3]


def block_merge(r, s, req=0, early=False):
    """(overlap counted, rejected) of the block merge with the positional bound."""
    R, S = blocks(r), blocks(s)
    i = j = o = 0
    while i < len(R) and j < len(S):
        remr, rems = len(r) - 4 * i, len(s) - 4 * j
        if early and o + min(remr, rems) < req:
            return o, True
        o += block_matches(R[i], S[j], min(remr, 4))
        ar, as_ = R[i][3] <= S[j][3], S[j][3] <= R[i][3]
        i += ar
        j += as_
    return o, False


def _random_sets(rng, n, vocab, lo, hi):
    return [sorted(rng.choice(vocab, size=int(rng.integers(lo, hi + 1)), replace=False).tolist()) for _ in range(n)]


def test_count_is_the_intersection_for_every_tail_shape():
    rng = np.random.default_rng(3)
    sets = _random_sets(rng, 120, 30, 1, 13) + [[0], [2**32 - 1], [0, 2**32 - 1], [5], [5, 6, 7, 8, 9], [1, 5, 9]]
    for r in sets:
        for s in sets:
            o, rej = block_merge(r, s)
            assert not rej and o == len(set(r) & set(s)), (r, s)


@pytest.mark.parametrize("p,q", [(9, 10), (4, 5), (3, 5), (1, 2)])
def test_positional_bound_never_rejects_a_passing_pair(p, q):
    rng = np.random.default_rng(p * 100 + q)
    base = _random_sets(rng, 60, 200, 2, 40)
    sets = base + [sorted(set(b[:-1]) | {500 + k}) for k, b in enumerate(base)]
    for r in sets:
        for s in sets:
            exact = len(set(r) & set(s))
            req = -(-p * (len(r) + len(s)) // (p + q))
            o, rej = block_merge(r, s, req, early=True)
            if exact >= req:
                assert not rej and o == exact, (r, s)
            else:
                assert rej or o == exact < req
