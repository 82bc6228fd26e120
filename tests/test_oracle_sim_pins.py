"""Pins for the oracle's Dice, Cosine and plain-overlap thresholds (Table
"Similarity Functions" of Section 2.2.2 and the length filter of Section
2.2.3), each against something other than the oracle's own integer forms:
the table's formulas evaluated in 60-digit decimal arithmetic, the
definitions as ratios of Python sets, brute force, and relations between
the functions that hold for every pair of sets.
"""
import random
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_path

getcontext().prec = 60
SIMS = [oracle.JACCARD, oracle.DICE, oracle.COSINE]
T_CONFIG = [(19, 20), (9, 10), (17, 20), (4, 5), (3, 4), (7, 10), (13, 20), (3, 5), (1, 2), (1, 1)]


def _dec_ceil(x: Decimal) -> int:
    return int(x.to_integral_value(rounding="ROUND_CEILING"))


def _table_formula(sim, nr, ns, p, q) -> int:
    """The equivalent-overlap column of Table "Similarity Functions", in 60-digit decimals."""
    t = Decimal(p) / Decimal(q)
    if sim == oracle.JACCARD:
        return _dec_ceil(t / (1 + t) * (nr + ns))
    if sim == oracle.DICE:
        return _dec_ceil(t * (nr + ns) / 2)
    if sim == oracle.COSINE:
        return _dec_ceil(t * (Decimal(nr) * Decimal(ns)).sqrt())
    return _dec_ceil(t)


def _definition(sim, o, nr, ns, p, q) -> bool:
    """The similarity function's value against t, as a ratio (Cosine in 60-digit decimals)."""
    t = Fraction(p, q)
    if sim == oracle.JACCARD:
        return nr + ns - o > 0 and Fraction(o, nr + ns - o) >= t
    if sim == oracle.DICE:
        return nr + ns > 0 and Fraction(2 * o, nr + ns) >= t
    if sim == oracle.COSINE:
        if nr == 0 or ns == 0:
            return False
        return Decimal(o) / (Decimal(nr) * Decimal(ns)).sqrt() >= Decimal(p) / Decimal(q)
    return o >= t


def test_golden_examples_of_the_table():
    """Hand-worked equivalent overlaps (tests/golden/similarity_examples.txt)."""
    names = {"jaccard": oracle.JACCARD, "dice": oracle.DICE, "cosine": oracle.COSINE, "overlap": oracle.OVERLAP}
    with open(golden_path("similarity_examples.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 8
    for name, nr, ns, p, q, need in rows:
        sim, nr, ns, p, q, need = names[name], int(nr), int(ns), int(p), int(q), int(need)
        assert oracle.required_overlap(nr, ns, p, q, sim) == need, (name, nr, ns, p, q)
        assert oracle.sim_pass(need, nr, ns, p, q, sim)
        assert need == 0 or not oracle.sim_pass(need - 1, nr, ns, p, q, sim)


@pytest.mark.parametrize("sim", SIMS)
def test_required_overlap_equals_table_formula(sim):
    for p, q in T_CONFIG:
        for nr in range(0, 33):
            for ns in range(0, 33):
                assert oracle.required_overlap(nr, ns, p, q, sim) == _table_formula(sim, nr, ns, p, q), \
                    (sim, nr, ns, p, q)


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_required_overlap_large_sizes_and_thresholds(sim):
    rng = random.Random(11 + sim)
    for _ in range(1500):
        p = rng.randint(1, 2**31 - 1)
        q = rng.randint(p, 2**31 - 1) if sim != oracle.OVERLAP else rng.randint(1, 2**31 - 1)
        nr, ns = rng.randint(0, 2**32 - 1), rng.randint(0, 2**32 - 1)
        assert oracle.required_overlap(nr, ns, p, q, sim) == _table_formula(sim, nr, ns, p, q), (sim, nr, ns, p, q)


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_pass_is_the_definition_and_the_least_passing_overlap_is_required(sim):
    thresholds = T_CONFIG if sim != oracle.OVERLAP else [(1, 1), (3, 1), (7, 2), (10, 3)]
    for p, q in thresholds:
        for nr in range(0, 21):
            for ns in range(0, 21):
                req = oracle.required_overlap(nr, ns, p, q, sim)
                for o in range(0, min(nr, ns) + 1):
                    want = _definition(sim, o, nr, ns, p, q)
                    assert oracle.sim_pass(o, nr, ns, p, q, sim) == want, (sim, o, nr, ns, p, q)
                    if nr + ns > 0 and (sim != oracle.COSINE or nr * ns > 0):
                        assert want == (o >= req), (sim, o, nr, ns, p, q, req)


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_length_filter_is_exactly_reachability(sim):
    thresholds = T_CONFIG if sim != oracle.OVERLAP else [(1, 1), (3, 1), (7, 2)]
    for p, q in thresholds:
        for nr in range(1, 41):
            for ns in range(1, 41):
                reachable = any(_definition(sim, o, nr, ns, p, q) for o in range(min(nr, ns) + 1))
                assert oracle.length_ok(nr, ns, p, q, sim) == reachable, (sim, nr, ns, p, q)


def _sets(seed, n, kmax, V=40, dup=0.3):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        if out and rng.random() < dup:
            base = set(rng.choice(out))
            if base and rng.random() < 0.5:
                base.discard(rng.choice(sorted(base)))
            else:
                base.add(rng.randrange(V))
            out.append(sorted(base))
        else:
            out.append(sorted(rng.sample(range(V), rng.randint(0, min(kmax, V)))))
    return out


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_bruteforce_matches_python_sets(sim):
    sets = _sets(3 + sim, 60, 25)
    c = synth.from_lists(sets)
    thresholds = [(4, 5), (3, 5), (1, 2)] if sim != oracle.OVERLAP else [(3, 1), (5, 1), (9, 2)]
    for p, q in thresholds:
        want = []
        for r in range(len(sets)):
            for s in range(r + 1, len(sets)):
                o = len(set(sets[r]) & set(sets[s]))
                if _definition(sim, o, len(sets[r]), len(sets[s]), p, q):
                    want.append((r, s, o))
        got = [tuple(map(int, t)) for t in oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim)]
        assert got == want, (sim, p, q)


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_bruteforce_rs_matches_python_sets(sim):
    R, S = _sets(21, 25, 20), _sets(22, 30, 20)
    cr, cs = synth.from_lists(R), synth.from_lists(S)
    p, q = (3, 5) if sim != oracle.OVERLAP else (4, 1)
    want = []
    for r in range(len(R)):
        for s in range(len(S)):
            o = len(set(R[r]) & set(S[s]))
            if _definition(sim, o, len(R[r]), len(S[s]), p, q):
                want.append((r, s, o))
    got = [tuple(map(int, x)) for x in oracle.bruteforce_rs(cr.offsets, cr.tokens, cs.offsets, cs.tokens, p, q, sim)]
    assert got == want


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
@pytest.mark.parametrize("seed", range(3))
def test_allpairs_equals_bruteforce(sim, seed):
    """The prefix and length filters of every function lose no result pair."""
    spec = synth.tiny_self_join(seed=500 + seed, n=400)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    c = synth.collection(spec)
    thresholds = [(9, 10), (4, 5), (3, 5)] if sim != oracle.OVERLAP else [(5, 1), (12, 1), (23, 2)]
    for p, q in thresholds:
        want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim))
        got, n_cands = oracle.allpairs_self(c.offsets, c.tokens, p, q, sim)
        assert np.array_equal(oracle.sort_triples(got), want), (sim, p, q)
        assert n_cands >= len(want)


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_allpairs_equals_bruteforce_dense_sets(sim):
    """Sets over a 24-token vocabulary with sizes 1..24, so that pairs of every size ratio and
    similarity occur, including those just inside each function's length filter and prefix."""
    rng = random.Random(700 + sim)
    sets = [sorted(rng.sample(range(24), rng.randint(1, 24))) for _ in range(300)]
    c = synth.from_lists(sets)
    thresholds = [(9, 10), (7, 10), (1, 2), (3, 10)] if sim != oracle.OVERLAP else [(4, 1), (9, 1), (31, 2)]
    for p, q in thresholds:
        want = oracle.sort_triples(oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim))
        got, _ = oracle.allpairs_self(c.offsets, c.tokens, p, q, sim)
        assert np.array_equal(oracle.sort_triples(got), want), (sim, p, q, len(got), len(want))
        assert len(want) > 0


@pytest.mark.parametrize("sim", SIMS + [oracle.OVERLAP])
def test_early_termination_decides_as_the_definition(sim):
    rng = random.Random(40 + sim)
    thresholds = T_CONFIG if sim != oracle.OVERLAP else [(2, 1), (6, 1), (13, 2)]
    for _ in range(3000):
        V = rng.randint(5, 60)
        r = sorted(rng.sample(range(V), rng.randint(0, min(V, 30))))
        s = sorted(rng.sample(range(V), rng.randint(0, min(V, 30))))
        p, q = rng.choice(thresholds)
        o = len(set(r) & set(s))
        ok, got_o, ci, cj = oracle.verify_pair(r, s, p, q, True, sim)
        assert ok == _definition(sim, o, len(r), len(s), p, q), (sim, r, s, p, q)
        if ok:
            assert got_o == o
        assert ci <= len(r) and cj <= len(s)
        assert oracle.verify_pair(r, s, p, q, False, sim)[1] == o


def test_function_order_jaccard_dice_cosine():
    """Dice = 2J/(1+J) >= J and Cosine >= Dice (the geometric mean is at most the arithmetic
    mean), so at one threshold the result sets nest: Jaccard within Dice within Cosine."""
    sets = _sets(77, 80, 20, V=30, dup=0.4)
    c = synth.from_lists(sets)
    for p, q in [(4, 5), (3, 5), (1, 2)]:
        res = [set(map(tuple, oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim).tolist())) for sim in SIMS]
        assert res[0] <= res[1] <= res[2]
        assert len(res[2]) > len(res[0])


@pytest.mark.parametrize("sim", SIMS)
def test_monotone_in_threshold(sim):
    sets = _sets(90 + sim, 70, 20, V=30, dup=0.4)
    c = synth.from_lists(sets)
    prev = None
    for p, q in sorted(T_CONFIG, key=lambda pq: Fraction(*pq)):
        cur = set(map(tuple, oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim).tolist()))
        if prev is not None:
            assert cur <= prev
        prev = cur


def test_verify_batch_sim_agrees_with_bruteforce_over_all_pairs():
    c = synth.collection(synth.tiny_self_join(seed=808, n=150))
    b = synth.all_pairs_batch(c.n)
    for sim in SIMS + [oracle.OVERLAP]:
        p, q = (3, 5) if sim != oracle.OVERLAP else (6, 1)
        got = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, p, q,
                                  b.probe_ids, b.cand_offsets, b.cand_ids, sim=sim)
        want = oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim)
        assert np.array_equal(oracle.sort_triples(got), oracle.sort_triples(want)), sim


def test_invalid_thresholds_rejected():
    c = synth.collection(synth.tiny_self_join(seed=9, n=20))
    for sim, p, q in [(oracle.DICE, 0, 5), (oracle.COSINE, 6, 5), (oracle.DICE, 3, 0), (oracle.OVERLAP, 0, 1)]:
        with pytest.raises(ValueError):
            oracle.bruteforce_self(c.offsets, c.tokens, p, q, sim)
    # the plain overlap threshold may exceed 1
    oracle.bruteforce_self(c.offsets, c.tokens, 7, 2, oracle.OVERLAP)
