"""Pins for the CPU oracle: each checks it against something other than itself.

The sources of truth are the paper's worked examples (tests/golden/), exact
rational arithmetic on the definitions, Python's own set operations, brute
force on tiny inputs, and invariants that any correct join satisfies.
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_path

T_CONFIG = [(19, 20), (9, 10), (17, 20), (4, 5), (3, 4), (7, 10), (13, 20), (3, 5)]


def _rows(name):
    with open(golden_path(name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- threshold

def test_worked_example_jaccard_08_two_10_token_sets_needs_9():
    """Section 2.2.2: two 10-token sets at Jaccard 0.8 need overlap 9."""
    nr, ns, p, q, need = map(int, _rows("jaccard_worked_example.txt")[0].split())
    assert oracle.required_overlap(nr, ns, p, q) == need
    assert oracle.jaccard_pass(need, nr, ns, p, q)
    assert not oracle.jaccard_pass(need - 1, nr, ns, p, q)
    # and on real sets: 9 shared tokens pass, 8 do not
    r = list(range(10))
    s9 = list(range(1, 11))            # shares 1..9
    s8 = list(range(2, 12))            # shares 2..9
    assert oracle.verify_pair(r, s9, p, q)[:2] == (True, 9)
    assert oracle.verify_pair(r, s8, p, q)[0] is False


def _ceil_formula(nr, ns, t: Fraction):
    """Table "Similarity Functions": ceil(t/(1+t) * (|r|+|s|)) in exact rationals."""
    return math.ceil(t / (1 + t) * (nr + ns))


def test_required_overlap_equals_table_formula_small_grid():
    for p, q in T_CONFIG + [(1, 1), (1, 2), (1, 3), (2, 3)]:
        t = Fraction(p, q)
        for nr in range(0, 41):
            for ns in range(0, 41):
                assert oracle.required_overlap(nr, ns, p, q) == _ceil_formula(nr, ns, t), (nr, ns, p, q)


def test_required_overlap_equals_table_formula_large_sizes():
    rng = random.Random(7)
    for _ in range(3000):
        p = rng.randint(1, 2**31 - 1)
        q = rng.randint(p, 2**31 - 1)
        nr = rng.choice([rng.randint(0, 2000), rng.randint(0, 2**31 - 1)])
        ns = rng.choice([rng.randint(0, 2000), rng.randint(0, 2**31 - 1)])
        assert oracle.required_overlap(nr, ns, p, q) == _ceil_formula(nr, ns, Fraction(p, q))


def test_jaccard_pass_is_the_definition():
    """o / |r u s| >= t with |r u s| = |r| + |s| - o, in exact rationals."""
    for p, q in T_CONFIG + [(1, 1), (1, 7)]:
        t = Fraction(p, q)
        for nr in range(0, 25):
            for ns in range(0, 25):
                for o in range(0, min(nr, ns) + 1):
                    union = nr + ns - o
                    want = union > 0 and Fraction(o, union) >= t
                    assert oracle.jaccard_pass(o, nr, ns, p, q) == want, (o, nr, ns, p, q)


def test_threshold_test_agrees_with_required_overlap_up_to_2000():
    """o passes iff o >= ceil-formula, over every size pair up to 2000 at every config t."""
    rng = random.Random(11)
    for p, q in T_CONFIG:
        t = Fraction(p, q)
        for _ in range(2000):
            nr, ns = rng.randint(1, 2000), rng.randint(1, 2000)
            need = _ceil_formula(nr, ns, t)
            lo = max(0, need - 1)
            for o in (lo, need):
                if o <= min(nr, ns):
                    assert oracle.jaccard_pass(o, nr, ns, p, q) == (o >= need)


def test_length_filter_formula():
    """Section 2.2.3: t|r| <= |s| <= |r|/t.  The text's example (t=0.8, |r|=6 -> 4..6) does
    not follow from this formula (it gives 4.8..7.5, i.e. 5..7); the formula is taken."""
    t = Fraction(4, 5)
    ok = [ns for ns in range(0, 20) if oracle.length_ok(6, ns, 4, 5)]
    assert ok == [5, 6, 7]
    for p, q in T_CONFIG:
        t = Fraction(p, q)
        for nr in range(0, 30):
            for ns in range(0, 30):
                want = t * nr <= ns <= (nr / t)
                assert oracle.length_ok(nr, ns, p, q) == want


def test_length_filter_is_exactly_reachability():
    """A pair can pass (with the largest possible overlap min(|r|,|s|)) iff the length filter holds."""
    for p, q in T_CONFIG:
        for nr in range(1, 40):
            for ns in range(1, 40):
                reachable = oracle.jaccard_pass(min(nr, ns), nr, ns, p, q)
                assert reachable == oracle.length_ok(nr, ns, p, q)


# ---------------------------------------------------------------- overlap

def _rand_set(rng, k, V):
    return sorted(rng.sample(range(V), k))


def test_overlap_equals_python_set_intersection():
    rng = random.Random(3)
    for _ in range(3000):
        V = rng.choice([10, 50, 1000, 2**32 - 1])
        a = _rand_set(rng, rng.randint(0, min(V, 60)), min(V, 10**6))
        b = _rand_set(rng, rng.randint(0, min(V, 60)), min(V, 10**6))
        assert oracle.overlap(a, b) == len(set(a) & set(b))
    # extreme token values
    a = [0, 5, 2**32 - 2, 2**32 - 1]
    b = [5, 2**32 - 1]
    assert oracle.overlap(a, b) == 2
    assert oracle.overlap([], b) == 0


# ---------------------------------------------------------------- verification

def test_positional_filter_worked_examples():
    for row in _rows("positional_filter_example.txt"):
        pq, rs, ss, exp = [x.split() for x in row.split("|")]
        p, q = map(int, pq)
        r, s = list(map(int, rs)), list(map(int, ss))
        passes, cr, cs, exact = map(int, exp)
        got = oracle.verify_pair(r, s, p, q, early=True)
        assert (int(got[0]), got[2], got[3]) == (passes, cr, cs)
        assert oracle.verify_pair(r, s, p, q, early=False)[1] == exact
        assert oracle.overlap(r, s) == exact


def test_early_termination_is_sound_and_exact_for_true_pairs():
    rng = random.Random(5)
    for _ in range(5000):
        p, q = rng.choice(T_CONFIG + [(1, 1), (1, 3)])
        V = rng.choice([20, 60, 400])
        k1, k2 = rng.randint(0, min(30, V)), rng.randint(0, min(30, V))
        base = _rand_set(rng, k1, V)
        if rng.random() < 0.5 and k1:
            # near-duplicate so that passing pairs occur often
            s = set(base)
            for _e in range(rng.randint(0, 3)):
                s.discard(rng.choice(base))
                s.add(rng.randrange(V))
            other = sorted(s)
        else:
            other = _rand_set(rng, k2, V)
        truth_o = len(set(base) & set(other))
        union = len(set(base) | set(other))
        truth = union > 0 and Fraction(truth_o, union) >= Fraction(p, q)
        ok_e, o_e, ci, cj = oracle.verify_pair(base, other, p, q, early=True)
        ok_f, o_f, fi, fj = oracle.verify_pair(base, other, p, q, early=False)
        assert ok_e == truth and ok_f == truth
        assert o_f == truth_o
        if ok_e:
            assert o_e == truth_o
        assert ci <= len(base) and cj <= len(other)
        assert ci <= fi and cj <= fj
        # symmetry: verifying (s, r) gives the same decision and overlap
        ok_s, o_s, _, _ = oracle.verify_pair(other, base, p, q, early=False)
        assert ok_s == ok_f and o_s == o_f
        assert o_f <= min(len(base), len(other))


def _py_bruteforce_self(sets, t: Fraction):
    out = []
    for r in range(len(sets)):
        for s in range(r + 1, len(sets)):
            a, b = set(sets[r]), set(sets[s])
            u = len(a | b)
            if u and Fraction(len(a & b), u) >= t:
                out.append((r, s, len(a & b)))
    return out


def _small_collection(seed, n, V, kmax=12, dup_frac=0.3):
    rng = random.Random(seed)
    sets = []
    for i in range(n):
        if sets and rng.random() < dup_frac:
            base = set(rng.choice(sets))
            for _ in range(rng.randint(0, 2)):
                if base and rng.random() < 0.5:
                    base.discard(rng.choice(sorted(base)))
                else:
                    base.add(rng.randrange(V))
            sets.append(sorted(base))
        else:
            sets.append(_rand_set(rng, rng.randint(0, min(kmax, V)), V))
    return sets


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_self_matches_python_definition(seed):
    sets = _small_collection(seed, 70, 40)
    c = synth.from_lists(sets)
    for p, q in [(4, 5), (3, 5), (1, 2), (1, 1), (1, 4)]:
        got = [tuple(map(int, t)) for t in oracle.bruteforce_self(c.offsets, c.tokens, p, q)]
        assert got == _py_bruteforce_self(sets, Fraction(p, q))


def test_bruteforce_rs_matches_python_definition():
    R = _small_collection(1, 30, 30)
    S = _small_collection(2, 40, 30)
    cr, cs = synth.from_lists(R), synth.from_lists(S)
    for p, q in [(4, 5), (1, 2)]:
        t = Fraction(p, q)
        want = []
        for r in range(len(R)):
            for s in range(len(S)):
                a, b = set(R[r]), set(S[s])
                u = len(a | b)
                if u and Fraction(len(a & b), u) >= t:
                    want.append((r, s, len(a & b)))
        got = [tuple(map(int, x)) for x in oracle.bruteforce_rs(cr.offsets, cr.tokens, cs.offsets, cs.tokens, p, q)]
        assert got == want


# ---------------------------------------------------------------- renumbering and AllPairs

def test_renumber_orders_by_ascending_frequency_and_preserves_sets():
    sets = _small_collection(9, 80, 50)
    c = synth.from_lists(sets)
    new, u = oracle.renumber(c.offsets, c.tokens)
    raw_vals, raw_counts = np.unique(c.tokens, return_counts=True)
    assert u == len(raw_vals)
    # expected mapping: sort distinct tokens by (count, id)
    order = sorted(range(len(raw_vals)), key=lambda k: (raw_counts[k], raw_vals[k]))
    mapping = {int(raw_vals[k]): rank for rank, k in enumerate(order)}
    for i in range(c.n):
        want = sorted(mapping[int(x)] for x in c.set(i))
        got = list(map(int, new[c.offsets[i]:c.offsets[i + 1]]))
        assert got == want
    # token 0 is (one of) the least frequent
    _, new_counts = np.unique(new, return_counts=True)
    assert new_counts[0] == raw_counts.min()
    assert list(new_counts) == sorted(new_counts)


@pytest.mark.parametrize("seed", range(8))
def test_allpairs_equals_bruteforce(seed):
    sets = _small_collection(100 + seed, 150, 60, kmax=20)
    c = synth.from_lists(sets)
    for p, q in T_CONFIG + [(1, 2), (1, 1)]:
        bf = oracle.bruteforce_self(c.offsets, c.tokens, p, q)
        ap, ncand = oracle.allpairs_self(c.offsets, c.tokens, p, q)
        assert np.array_equal(oracle.sort_triples(ap), oracle.sort_triples(bf))
        assert ncand <= c.n * (c.n - 1) // 2


def test_allpairs_equals_bruteforce_on_planted_tiny_config():
    spec = synth.tiny_self_join()
    spec.plant_frac, spec.plant_edits = 0.1, 2
    c = synth.collection(spec)
    for p, q in [(4, 5), (3, 5), (9, 10)]:
        bf = oracle.bruteforce_self(c.offsets, c.tokens, p, q)
        ap, _ = oracle.allpairs_self(c.offsets, c.tokens, p, q)
        assert len(bf) > 0
        assert np.array_equal(oracle.sort_triples(ap), oracle.sort_triples(bf))


# ---------------------------------------------------------------- batch verification

def test_candidate_layout_worked_example():
    """Section 3.3.1: r1 has one candidate, r2 none, r3 two; only (r3, s4) is similar."""
    rows = _rows("candidate_layout_example.txt")
    probes = cand_offsets = cand_ids = None
    R, S = {}, {}
    expect = []
    for row in rows:
        head, *rest = row.split()
        if head == "probes":
            probes = list(map(int, rest))
        elif head == "cand_offsets":
            cand_offsets = list(map(int, rest))
        elif head == "cand_ids":
            cand_ids = list(map(int, rest))
        elif head == "R":
            R[int(rest[0].rstrip(":"))] = list(map(int, rest[1:]))
        elif head == "S":
            S[int(rest[0].rstrip(":"))] = list(map(int, rest[1:]))
        elif head == "expect":
            expect.append(tuple(map(int, rest)))
    filler = [1000, 1001]
    Rl = [R.get(i, filler) for i in range(max(R) + 1)]
    Sl = [S.get(i, filler) for i in range(max(S) + 1)]
    cr, cs = synth.from_lists(Rl), synth.from_lists(Sl)
    got = oracle.verify_batch(cr.offsets, cr.tokens, cs.offsets, cs.tokens, False, 4, 5,
                              probes, cand_offsets, cand_ids)
    assert [tuple(map(int, t)) for t in got] == expect
    # the per-probe candidate counts of the text: 1, 0, 2
    assert list(np.diff(cand_offsets)) == [1, 0, 2]


def test_verify_batch_self_join_semantics():
    sets = [[1, 2, 3], [1, 2, 3], [1, 2, 4], [7, 8]]
    c = synth.from_lists(sets)
    # probe 1 lists itself, 0 (a duplicate set) and 2; probe 3 lists 0
    probes = [1, 3]
    offs = [0, 3, 4]
    cands = [1, 0, 2, 0]
    tr = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 1, 2, probes, offs, cands)
    # self pair skipped; (1,0) oriented as (0,1) with overlap 3; (1,2) overlap 2 -> J = 2/4 = 0.5 passes
    assert [tuple(map(int, t)) for t in tr] == [(0, 1, 3), (1, 2, 2)]
    allt = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 1, 2, probes, offs, cands,
                               flags=oracle.EMIT_ALL)
    assert [tuple(map(int, t)) for t in allt] == [(0, 1, 3), (1, 2, 2), (0, 3, 0)]
    with pytest.raises(ValueError):
        oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 1, 2, [9], [0, 0], [])
    with pytest.raises(ValueError):
        oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 0, 2, [1], [0, 1], [0])


def test_verify_batch_agrees_with_bruteforce_over_all_pairs():
    spec = synth.tiny_self_join(n=300)
    spec.plant_frac, spec.plant_edits = 0.15, 3
    c = synth.collection(spec)
    b = synth.all_pairs_batch(c.n)
    for p, q in [(4, 5), (1, 2)]:
        tr, cr, cs = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, p, q,
                                         b.probe_ids, b.cand_offsets, b.cand_ids, consumed=True)
        bf = oracle.bruteforce_self(c.offsets, c.tokens, p, q)
        assert np.array_equal(oracle.sort_triples(tr), oracle.sort_triples(bf))
        sizes = c.sizes().astype(np.int64)
        pr = np.repeat(b.probe_ids, np.diff(b.cand_offsets).astype(np.int64))
        assert np.all(cr <= sizes[pr]) and np.all(cs <= sizes[b.cand_ids])


# ---------------------------------------------------------------- invariants

def test_monotone_in_threshold():
    spec = synth.tiny_self_join(n=400)
    spec.plant_frac, spec.plant_edits = 0.2, 4
    c = synth.collection(spec)
    ts = sorted(T_CONFIG, key=lambda pq: Fraction(*pq))
    prev = None
    for p, q in ts:
        cur = {tuple(map(int, t)) for t in oracle.bruteforce_self(c.offsets, c.tokens, p, q)}
        if prev is not None:
            assert cur <= prev
        prev = cur


def test_renumbering_and_id_permutation_invariance():
    sets = _small_collection(21, 120, 40, kmax=15)
    c = synth.from_lists(sets)
    base = {tuple(map(int, t)) for t in oracle.bruteforce_self(c.offsets, c.tokens, 3, 5)}
    # any bijection on tokens leaves the result unchanged
    new, _ = oracle.renumber(c.offsets, c.tokens)
    ren = {tuple(map(int, t)) for t in oracle.bruteforce_self(c.offsets, new, 3, 5)}
    assert ren == base
    # permuting set ids permutes the result
    rng = random.Random(4)
    perm = list(range(len(sets)))
    rng.shuffle(perm)                      # new id of old set i is perm[i]
    inv = [0] * len(sets)
    for i, pi in enumerate(perm):
        inv[pi] = i
    c2 = synth.from_lists([sets[inv[k]] for k in range(len(sets))])
    got = {tuple(map(int, t)) for t in oracle.bruteforce_self(c2.offsets, c2.tokens, 3, 5)}
    want = {(min(perm[r], perm[s]), max(perm[r], perm[s]), o) for r, s, o in base}
    assert got == want


# ---------------------------------------------------------------- helpers the parity tests lean on

def test_sort_triples_is_the_r_then_s_order_of_python_tuples():
    """sort_triples against Python's own tuple sort, with ids above 2^31 (a signed key would
    misplace them) and triples that share r."""
    rng = np.random.default_rng(11)
    r = rng.integers(0, 2**32, size=400, dtype=np.uint64)
    r[::3] = r[0]  # many triples with the same r
    s = rng.integers(0, 2**32, size=400, dtype=np.uint64)
    o = rng.integers(0, 2000, size=400, dtype=np.uint64)
    t = np.stack([r, s, o], axis=1).astype(np.uint32)
    want = sorted(map(tuple, t.tolist()), key=lambda x: (x[0], x[1]))
    assert oracle.sort_triples(t).tolist() == [list(x) for x in want]
    assert oracle.sort_triples(np.zeros((0, 3), dtype=np.uint32)).shape == (0, 3)


def test_verify_batch_threads_equals_bruteforce_for_any_split():
    """The threaded oracle splits the probes into contiguous ranges: for any number of ranges
    (one, a few, more than there are probes) and a batch with empty candidate lists, its results
    are brute force's on the listed pairs, in the probe order of the single-range call."""
    spec = synth.tiny_self_join(n=240)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    b = synth.all_pairs_batch(c.n)  # probe r is paired with r+1 .. n-1
    # every fifth probe keeps no candidates (empty lists inside the batch)
    co = b.cand_offsets.astype(np.int64)
    counts = np.diff(co)
    keep = np.ones(len(b.cand_ids), dtype=bool)
    dropped = set(range(0, b.n_probes, 5))
    for k in dropped:
        keep[co[k]:co[k + 1]] = False
        counts[k] = 0
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    cands = b.cand_ids[keep]
    args = (c.offsets, c.tokens, c.offsets, c.tokens, True, 3, 5, b.probe_ids, offs, cands)
    whole = np.asarray(oracle.verify_batch(*args)).reshape(-1, 3)
    # brute force over all pairs, less the pairs whose probe (the smaller id) lost its list
    want = [t for t in oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, 3, 5)).tolist()
            if t[0] not in dropped]
    assert len(want) > 20
    assert oracle.sort_triples(whole).tolist() == want
    assert np.all(np.diff(whole[:, 0].astype(np.int64)) >= 0)  # probe order
    for n_threads in (1, 2, 3, 7, b.n_probes + 5):
        got = np.asarray(oracle.verify_batch_threads(*args, n_threads=n_threads)).reshape(-1, 3)
        assert np.array_equal(got, whole), n_threads
    empty = oracle.verify_batch_threads(c.offsets, c.tokens, c.offsets, c.tokens, True, 3, 5, [], [0], [])
    assert empty.shape == (0, 3)
