"""The merge-path split the warp and block kernels run (Section 4.2.3, Intersect Path), restated
on the host and checked against the sequential merge and exact set intersection (CPU only).

A window of the merge of r and s is cut along cross diagonals d = 0, hop, 2 hop, ...; each lane
finds where the merge path crosses its diagonal by a binary search (the largest i with
r[i - 1] <= s[d - i], i.e. the merge takes r first on a tie), then runs up to hop merge steps
from there, counting a match when the step takes r[i] while r[i] == s[j].  The claims the
kernels rely on: the split point is the sequential merge's state after d steps, and the lanes'
counts add up to |r n s|, every common token counted by exactly one lane."""
import math
import random

import pytest

from conftest import golden_path


def split(A, rw, B, sw, d):
    """Lane's start (i, j) on diagonal d: binary search as in the kernels."""
    lo, hi = max(0, d - sw), min(d, rw)
    while lo < hi:
        mid = (lo + hi) // 2
        if A[mid] <= B[d - 1 - mid]:
            lo = mid + 1
        else:
            hi = mid
    return lo, d - lo


def lane_merge(A, rw, B, sw, d, de, steps):
    """Matches counted by the lane whose diagonal is d (at most `steps` steps, none past de)."""
    i, j = split(A, rw, B, sw, d)
    c = 0
    for t in range(steps):
        if d + t >= de:
            break
        if i >= rw:
            take_r = False
        elif j >= sw:
            take_r = True
        else:
            take_r = A[i] <= B[j]
            c += A[i] == B[j]
        if take_r:
            i += 1
        else:
            j += 1
    return c, i, j


def sequential_states(A, B):
    """(i, j) of the plain merge after each step, taking A first on a tie."""
    i = j = 0
    out = [(0, 0)]
    while i < len(A) or j < len(B):
        if j >= len(B) or (i < len(A) and A[i] <= B[j]):
            i += 1
        else:
            j += 1
        out.append((i, j))
    return out


def lanes_count(A, B, lanes):
    n = len(A) + len(B)
    hop = max(1, math.ceil(n / lanes))
    total = 0
    ends = []
    for d in range(0, n, hop):
        c, i, j = lane_merge(A, len(A), B, len(B), d, n, hop)
        total += c
        ends.append((i, j))
    return total, hop, ends


def _golden_rows():
    with open(golden_path("intersect_path_example.txt")) as f:
        return [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]


def test_section_4_2_3_example_diagonals():
    """|r| = |s| = 10 with B = 4 threads: diagonals 5 apart, at 0, 5, 10, 15; each thread's
    start is the sequential merge's state on its diagonal, and the counts add up."""
    for nr, ns, lanes, hop in _golden_rows():
        assert math.ceil((nr + ns) / lanes) == hop
        assert list(range(0, nr + ns, hop)) == [hop * k for k in range(lanes)]
        rng = random.Random(7)
        A = sorted(rng.sample(range(30), nr))
        B = sorted(rng.sample(range(30), ns))
        states = sequential_states(A, B)
        for d in range(0, nr + ns, hop):
            assert split(A, nr, B, ns, d) == states[d]
        total, got_hop, ends = lanes_count(A, B, lanes)
        assert got_hop == hop and total == len(set(A) & set(B))
        # every lane ends where the next one starts
        assert ends[:-1] == [states[d] for d in range(hop, nr + ns, hop)]


@pytest.mark.parametrize("lanes", [1, 2, 3, 4, 32])
def test_lane_counts_add_up_to_the_intersection(lanes):
    rng = random.Random(100 + lanes)
    for _ in range(400):
        na, nb = rng.randint(0, 40), rng.randint(0, 40)
        universe = rng.choice([10, 40, 200])
        A = sorted(rng.sample(range(universe), min(na, universe)))
        B = sorted(rng.sample(range(universe), min(nb, universe)))
        if not A and not B:
            continue
        total, _, _ = lanes_count(A, B, lanes)
        assert total == len(set(A) & set(B)), (A, B, lanes)


def test_split_is_the_sequential_state_on_every_diagonal():
    """Including equal sets, disjoint sets, one set inside the other and an empty side."""
    cases = [(list(range(8)), list(range(8))), ([1, 3, 5, 7], [0, 2, 4, 6]), ([2, 3, 4], list(range(10))),
             ([], [1, 2, 3]), ([1, 2, 3], []), ([5], [5])]
    rng = random.Random(3)
    for _ in range(200):
        cases.append((sorted(rng.sample(range(60), rng.randint(0, 25))),
                      sorted(rng.sample(range(60), rng.randint(0, 25)))))
    for A, B in cases:
        states = sequential_states(A, B)
        for d in range(len(A) + len(B) + 1):
            assert split(A, len(A), B, len(B), d) == states[d], (A, B, d)


def test_window_views_continue_the_merge():
    """The kernels merge in windows: a window holds the next W tokens of each side from the
    current (i0, j0); its W merge steps are split among the lanes by diagonals, and the next
    window starts where the merge path crosses diagonal W.  The counts add up to one whole
    merge's."""
    rng = random.Random(11)
    for _ in range(300):
        A = sorted(rng.sample(range(300), rng.randint(0, 90)))
        B = sorted(rng.sample(range(300), rng.randint(0, 90)))
        W = rng.choice([4, 8, 16, 64])
        i0 = j0 = o = 0
        while i0 < len(A) and j0 < len(B):
            rem = (len(A) - i0) + (len(B) - j0)
            wc = min(W, rem)
            Aw, Bw = A[i0:i0 + wc], B[j0:j0 + wc]
            rw, sw = len(Aw), len(Bw)
            lanes = rng.choice([1, 4, 32])
            hop = max(1, math.ceil(wc / lanes))
            for d in range(0, wc, hop):  # the lanes of the window, each from its own diagonal
                o += lane_merge(Aw, rw, Bw, sw, d, wc, hop)[0]
            i, j = split(Aw, rw, Bw, sw, wc)  # where the window's merge ends
            i0, j0 = i0 + i, j0 + j
        assert o == len(set(A) & set(B))
