"""CPU-only checks of the C ABI library and the host-side feeder.

No compute call reaches the GPU here: the library is loaded, its exported
symbols are compared with the declarations in include/*.h, and the CPU
candidate feeder (host code) is checked for completeness against the oracle.
"""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import synth
from conftest import ROOT

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    return ssj.lib()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(ssj_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.mark.parametrize("name", ["libssj.so", "libssj_checked.so"])
def test_every_declared_function_is_exported_and_bound(name):
    """The product library and its checked build export every function include/*.h declares."""
    declared = _declared_functions()
    assert "ssj_verify_batch" in declared and "ssj_submit" in declared
    path = os.path.join(os.path.dirname(ssj.LIB_PATH), name)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True)
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    missing = declared - exported
    assert not missing, f"declared but not exported: {missing}"
    assert declared == set(ssj.SIGNATURES), (declared ^ set(ssj.SIGNATURES))


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1812_09141_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", text), f"{f} mentions the oracle"


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ssj.SsjError):
        ssj.ssj_create(0)


# ---------------------------------------------------------------- feeder (host code)

def _planted(n=600, frac=0.15, edits=2, seed=1001):
    spec = synth.tiny_self_join(seed=seed, n=n)
    spec.plant_frac, spec.plant_edits = frac, edits
    return synth.collection(spec)


@pytest.mark.parametrize("pq", [(19, 20), (4, 5), (7, 10), (3, 5), (1, 2), (1, 1)])
def test_feeder_candidates_cover_every_result(pq):
    c = _planted()
    pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, *pq, n_threads=3, chunk=997)
    assert co[0] == 0 and np.all(np.diff(co.astype(np.int64)) >= 0) and co[-1] == len(ci)
    # every pair at most once, never (r, r)
    pairs = set()
    for k in range(len(pr)):
        for s in ci[co[k]:co[k + 1]]:
            key = (min(pr[k], s), max(pr[k], s))
            assert pr[k] != s and key not in pairs
            pairs.add(key)
    bf = oracle.bruteforce_self(c.offsets, c.tokens, *pq)
    assert {(int(r), int(s)) for r, s, _ in bf} <= pairs
    tr = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, *pq, pr, co, ci)
    assert np.array_equal(oracle.sort_triples(tr), oracle.sort_triples(bf))


@pytest.mark.parametrize("sim,pq", [(oracle.DICE, (4, 5)), (oracle.DICE, (3, 5)), (oracle.COSINE, (9, 10)),
                                    (oracle.COSINE, (3, 5)), (oracle.OVERLAP, (6, 1)), (oracle.OVERLAP, (23, 2))])
def test_feeder_other_similarity_functions(sim, pq):
    """The feeder's prefix and length filters for Dice, Cosine and the plain overlap threshold
    produce exactly the oracle AllPairs candidates, which cover every brute-force result."""
    rng = np.random.default_rng(5 + sim)
    lists = [sorted(rng.choice(40, size=int(rng.integers(1, 30)), replace=False).tolist()) for _ in range(400)]
    for c in (_planted(), synth.from_lists(lists)):
        pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, *pq, n_threads=3, chunk=1013, sim=sim)
        pairs = {(min(int(r), int(s)), max(int(r), int(s)))
                 for r, k0, k1 in zip(pr, co[:-1], co[1:]) for s in ci[k0:k1]}
        assert len(pairs) == len(ci)
        bf = oracle.bruteforce_self(c.offsets, c.tokens, *pq, sim=sim)
        assert {(int(r), int(s)) for r, s, _ in bf} <= pairs
        _, n_cands = oracle.allpairs_self(c.offsets, c.tokens, *pq, sim=sim)
        assert n_cands == len(ci)
        tr = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, *pq, pr, co, ci, sim=sim)
        assert np.array_equal(oracle.sort_triples(tr), oracle.sort_triples(bf))


def _pairs(pr, co, ci, self_join=True):
    out = set()
    for r, k0, k1 in zip(pr, co[:-1], co[1:]):
        for s in ci[k0:k1]:
            out.add((min(int(r), int(s)), max(int(r), int(s))) if self_join else (int(r), int(s)))
    return out


@pytest.mark.parametrize("sim,pq", [(oracle.JACCARD, (4, 5)), (oracle.JACCARD, (3, 5)), (oracle.DICE, (7, 10)),
                                    (oracle.COSINE, (4, 5)), (oracle.OVERLAP, (5, 1))])
def test_feeder_rs_join_covers_every_result(sim, pq):
    """R x S: every brute-force result pair of R against S is a candidate, once."""
    rng = np.random.default_rng(31 + sim)
    R = [sorted(rng.choice(60, size=int(rng.integers(1, 30)), replace=False).tolist()) for _ in range(300)]
    S = [sorted(rng.choice(60, size=int(rng.integers(1, 30)), replace=False).tolist()) for _ in range(250)]
    S += [sorted(set(R[i]) | {59}) for i in range(0, 300, 7)]  # near-copies of some sets of R
    cr, cs = synth.from_lists(R), synth.from_lists(S)
    for ppjoin in (0, ssj.SSJ_FEEDER_PPJOIN):
        pr, co, ci = ssj.feeder_all(cr.offsets, cr.tokens, *pq, n_threads=3, chunk=501, sim=sim,
                                    s_offsets=cs.offsets, s_tokens=cs.tokens, flags=ppjoin)
        pairs = _pairs(pr, co, ci, self_join=False)
        assert len(pairs) == len(ci)
        bf = oracle.bruteforce_rs(cr.offsets, cr.tokens, cs.offsets, cs.tokens, *pq, sim=sim)
        assert len(bf) > 0
        assert {(int(r), int(s)) for r, s, _ in bf} <= pairs
        tr = oracle.verify_batch(cr.offsets, cr.tokens, cs.offsets, cs.tokens, False, *pq, pr, co, ci, sim=sim)
        assert np.array_equal(oracle.sort_triples(tr), oracle.sort_triples(bf))


@pytest.mark.parametrize("sim,pq", [(oracle.JACCARD, (4, 5)), (oracle.JACCARD, (3, 5)), (oracle.DICE, (4, 5)),
                                    (oracle.COSINE, (7, 10)), (oracle.OVERLAP, (8, 1))])
def test_feeder_ppjoin_prunes_without_losing_results(sim, pq):
    """PPJoin's positional filter: candidates are a subset of AllPairs' and still cover every
    result (self-join)."""
    pruned = 0
    for c in (_planted(n=700), synth.from_lists(
            [sorted(np.random.default_rng(9).choice(40, size=k, replace=False).tolist())
             for k in np.random.default_rng(10).integers(1, 30, size=400)])):
        allp = ssj.feeder_all(c.offsets, c.tokens, *pq, n_threads=2, sim=sim)
        ppj = ssj.feeder_all(c.offsets, c.tokens, *pq, n_threads=2, sim=sim, flags=ssj.SSJ_FEEDER_PPJOIN)
        a, b = _pairs(*allp), _pairs(*ppj)
        assert b <= a and len(b) == len(ppj[2])
        bf = oracle.bruteforce_self(c.offsets, c.tokens, *pq, sim=sim)
        assert {(int(r), int(s)) for r, s, _ in bf} <= b
        pruned += len(a) - len(b)
    # with a plain overlap threshold k every prefix position leaves k tokens on both sides, so
    # the positional bound never falls below k; the normalized functions do prune
    assert pruned == 0 if sim == oracle.OVERLAP else pruned > 0


@pytest.mark.parametrize("sim,pq", [(oracle.JACCARD, (4, 5)), (oracle.JACCARD, (3, 5)), (oracle.DICE, (4, 5)),
                                    (oracle.COSINE, (7, 10)), (oracle.OVERLAP, (8, 1))])
def test_group_candidates_expand_to_allpairs_candidates(sim, pq):
    """GroupJoin: expanding the group candidates (probe group x candidate group members, and the
    pairs inside groups with a non-empty prefix) gives exactly the AllPairs candidates."""
    for frac, edits in ((0.3, 0), (0.15, 2)):
        spec = synth.tiny_self_join(seed=1001, n=700)
        spec.plant_frac, spec.plant_edits = frac, edits
        c = synth.collection(spec)
        g = ssj.group_candidates(c.offsets, c.tokens, *pq, sim=sim)
        go, mem = g.group_offsets.astype(np.int64), g.members
        sizes = np.diff(c.offsets.astype(np.int64))
        assert sorted(mem.tolist()) == list(range(c.n))
        pairs = set()
        for k, pgi in enumerate(g.probe_groups):
            for cgi in g.cand_groups[g.cand_offsets[k]:g.cand_offsets[k + 1]]:
                assert cgi < pgi  # earlier groups only
                for a in mem[go[pgi]:go[pgi + 1]]:
                    for b in mem[go[cgi]:go[cgi + 1]]:
                        pairs.add((min(int(a), int(b)), max(int(a), int(b))))
        for gi in range(len(go) - 1):
            A = mem[go[gi]:go[gi + 1]]
            size = int(sizes[A[0]])
            assert all(int(sizes[x]) == size for x in A)
            nonempty = size > 0 and (sim != oracle.OVERLAP or -(-pq[0] // pq[1]) <= size)
            if nonempty:
                pairs |= {(min(int(A[i]), int(A[j])), max(int(A[i]), int(A[j])))
                          for i in range(len(A)) for j in range(i + 1, len(A))}
        assert len(pairs) == g.n_pairs
        pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, *pq, n_threads=2, sim=sim)
        assert pairs == _pairs(pr, co, ci)
        assert oracle.allpairs_self(c.offsets, c.tokens, *pq, sim=sim)[1] == g.n_pairs


def test_feeder_threads_and_chunking_do_not_change_candidates():
    c = _planted(n=800)
    ref = ssj.feeder_all(c.offsets, c.tokens, 3, 5, n_threads=1, chunk=1 << 20)
    for threads, chunk in [(4, 1), (2, 13), (8, 4096)]:
        got = ssj.feeder_all(c.offsets, c.tokens, 3, 5, n_threads=threads, chunk=chunk)
        # chunking may split a probe's list; compare the flat (probe, cand) sequence
        def flat(b):
            pr, co, ci = b
            return np.repeat(pr, np.diff(co.astype(np.int64))), ci
        assert all(np.array_equal(x, y) for x, y in zip(flat(ref), flat(got)))


def test_feeder_rejects_bad_input():
    c = synth.from_lists([[1, 2], [3, 3]])
    with pytest.raises(ssj.SsjError):
        ssj.ssj_feeder_create(c.offsets, c.tokens, 1, 2)
    c = synth.from_lists([[1, 2], [3]])
    with pytest.raises(ssj.SsjError):
        ssj.ssj_feeder_create(c.offsets, c.tokens, 0, 2)
    with pytest.raises(ssj.SsjError):
        ssj.ssj_feeder_create(c.offsets, c.tokens, 3, 2)


def test_feeder_handles_empty_sets_and_empty_collection():
    c = synth.from_lists([[], [1, 2], [], [1, 2]])
    pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, 1, 2)
    assert sorted((min(a, b), max(a, b)) for a, b in zip(np.repeat(pr, np.diff(co.astype(np.int64))), ci)) == [(1, 3)]
    c = synth.from_lists([])
    pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, 1, 2)
    assert len(pr) == 0 and len(ci) == 0
