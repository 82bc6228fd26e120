"""CPU oracle for the verification phase of exact set similarity joins.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg and reference arm of ``bench.py`` may import this package.  The library
(``paper_1812_09141_gb300``) never imports, links or calls it; the two share
no code.

The arithmetic lives in ``oracle.c`` (plain C, single-threaded, exact
integers).  This module only marshals numpy arrays through ctypes and
returns results as (r, s, overlap) uint32 triples.

Functions and the passages they follow:

* ``required_overlap`` / ``jaccard_pass`` / ``sim_pass`` - Table "Similarity
  Functions" (Section 2.2.2): Jaccard, Dice, Cosine (and the plain overlap
  threshold) with t = p/q in exact integer form (``sim`` selects the
  function; Jaccard by default).
* ``length_ok`` - the length filter of Section 2.2.3, per function.
* ``overlap`` - intersection count by a sorted-list merge (Section 4.2.2).
* ``verify_pair`` - the verification loop of Section 3.1 with the
  positional stopping rule of Section 2.2.3.
* ``bruteforce_self`` / ``bruteforce_rs`` - the problem definition of
  Section 3 over all pairs.
* ``verify_batch`` - verification of a grouped candidate list (Section
  3.3.1 layout).  ``verify_batch_threads`` runs the same C routine over
  contiguous probe ranges on several host threads (candidate pairs are
  independent, Section 3) and concatenates the results: a faster driver
  for full-size parity tests, with no arithmetic of its own.
* ``renumber`` - token renumbering by ascending frequency (Section 2.2.1).
* ``allpairs_self`` - algorithm ALL (Sections 2.2.3, 2.2.4, 3.1).
* ``sort_triples`` - the canonical (r, s) order in which result lists are
  compared (the paper leaves output order open, Section 3.3.1).

Every function is pinned by a test in ``tests/test_oracle_pins.py`` against
something other than itself (the paper's worked example, exact rationals,
Python set operations, brute force, invariants).
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

EARLY = 1
EMIT_ALL = 2

# similarity functions (Table "Similarity Functions"), threshold t = p/q
JACCARD, DICE, COSINE, OVERLAP = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c with plain gcc into _oracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32, u64, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            u32p, u64p = ctypes.POINTER(u32), ctypes.POINTER(u64)
            lib.oracle_required_overlap.restype = u64
            lib.oracle_required_overlap.argtypes = [u64, u64, u64, u64]
            lib.oracle_jaccard_pass.restype = ctypes.c_int
            lib.oracle_jaccard_pass.argtypes = [u64, u64, u64, u64, u64]
            lib.oracle_length_ok.restype = ctypes.c_int
            lib.oracle_length_ok.argtypes = [u64, u64, u64, u64]
            lib.oracle_overlap.restype = u32
            lib.oracle_overlap.argtypes = [u32p, u32, u32p, u32]
            lib.oracle_verify_pair.restype = ctypes.c_int
            lib.oracle_verify_pair.argtypes = [u32p, u32, u32p, u32, u64, u64, ctypes.c_int, u32p, u32p, u32p]
            lib.oracle_bruteforce_self.restype = i64
            lib.oracle_bruteforce_self.argtypes = [u64p, u32p, u32, u64, u64, u32p, u64]
            lib.oracle_bruteforce_rs.restype = i64
            lib.oracle_bruteforce_rs.argtypes = [u64p, u32p, u32, u64p, u32p, u32, u64, u64, u32p, u64]
            lib.oracle_verify_batch.restype = i64
            lib.oracle_verify_batch.argtypes = [u64p, u32p, u32, u64p, u32p, u32, ctypes.c_int, u64, u64,
                                                u32, u32p, u64p, u32p, ctypes.c_int, u32p, u64, u32p, u32p]
            lib.oracle_renumber.restype = i64
            lib.oracle_renumber.argtypes = [u64p, u32p, u32, u32p]
            lib.oracle_allpairs_self.restype = i64
            lib.oracle_allpairs_self.argtypes = [u64p, u32p, u32, u64, u64, u32p, u64, u64p]
            c_int = ctypes.c_int
            lib.oracle_sim_pass.restype = c_int
            lib.oracle_sim_pass.argtypes = [c_int, u64, u64, u64, u64, u64]
            lib.oracle_required_overlap_sim.restype = u64
            lib.oracle_required_overlap_sim.argtypes = [c_int, u64, u64, u64, u64]
            lib.oracle_length_ok_sim.restype = c_int
            lib.oracle_length_ok_sim.argtypes = [c_int, u64, u64, u64, u64]
            lib.oracle_verify_pair_sim.restype = c_int
            lib.oracle_verify_pair_sim.argtypes = [c_int, u32p, u32, u32p, u32, u64, u64, c_int, u32p, u32p, u32p]
            lib.oracle_bruteforce_self_sim.restype = i64
            lib.oracle_bruteforce_self_sim.argtypes = [c_int, u64p, u32p, u32, u64, u64, u32p, u64]
            lib.oracle_bruteforce_rs_sim.restype = i64
            lib.oracle_bruteforce_rs_sim.argtypes = [c_int, u64p, u32p, u32, u64p, u32p, u32, u64, u64, u32p, u64]
            lib.oracle_verify_batch_sim.restype = i64
            lib.oracle_verify_batch_sim.argtypes = [c_int, u64p, u32p, u32, u64p, u32p, u32, c_int, u64, u64,
                                                    u32, u32p, u64p, u32p, c_int, u32p, u64, u32p, u32p]
            lib.oracle_allpairs_self_sim.restype = i64
            lib.oracle_allpairs_self_sim.argtypes = [c_int, u64p, u32p, u32, u64, u64, u32p, u64, u64p]
            _lib = lib
    return _lib


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint32)
    return a


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint64)
    return a


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _triples(fn, cap_hint=1024):
    """Call fn(out, cap) twice if needed so every triple fits; return (k,3) uint32."""
    cap = max(int(cap_hint), 1)
    while True:
        out = np.empty(3 * cap, dtype=np.uint32)
        k = fn(out, cap)
        if k < 0:
            raise ValueError(f"oracle error {k}")
        if k <= cap:
            return out[:3 * k].reshape(k, 3)
        cap = k


def required_overlap(nr: int, ns: int, p: int, q: int, sim: int = JACCARD) -> int:
    if sim == JACCARD:
        return int(_load().oracle_required_overlap(nr, ns, p, q))
    return int(_load().oracle_required_overlap_sim(sim, nr, ns, p, q))


def jaccard_pass(o: int, nr: int, ns: int, p: int, q: int) -> bool:
    return bool(_load().oracle_jaccard_pass(o, nr, ns, p, q))


def sim_pass(o: int, nr: int, ns: int, p: int, q: int, sim: int = JACCARD) -> bool:
    return bool(_load().oracle_sim_pass(sim, o, nr, ns, p, q))


def length_ok(nr: int, ns: int, p: int, q: int, sim: int = JACCARD) -> bool:
    if sim == JACCARD:
        return bool(_load().oracle_length_ok(nr, ns, p, q))
    return bool(_load().oracle_length_ok_sim(sim, nr, ns, p, q))


def overlap(a, b) -> int:
    """|a n b| for ascending duplicate-free a, b (empty arrays allowed)."""
    la, lb = len(a), len(b)
    a, b = _u32(a), _u32(b)
    return int(_load().oracle_overlap(_p32(a), la, _p32(b), lb))


def verify_pair(r, s, p: int, q: int, early: bool = True, sim: int = JACCARD):
    """Returns (passes, overlap, consumed_r, consumed_s)."""
    lr, ls = len(r), len(s)
    r, s = _u32(r), _u32(s)
    o, ci, cj = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    lib = _load()
    refs = (ctypes.byref(o), ctypes.byref(ci), ctypes.byref(cj))
    if sim == JACCARD:
        ok = lib.oracle_verify_pair(_p32(r), lr, _p32(s), ls, p, q, int(early), *refs)
    else:
        ok = lib.oracle_verify_pair_sim(sim, _p32(r), lr, _p32(s), ls, p, q, int(early), *refs)
    return bool(ok), o.value, ci.value, cj.value


def bruteforce_self(offsets, tokens, p: int, q: int, sim: int = JACCARD) -> np.ndarray:
    offs, toks = _u64(offsets), _u32(tokens)
    n = len(offsets) - 1
    lib = _load()
    if sim == JACCARD:
        return _triples(lambda out, cap: lib.oracle_bruteforce_self(_p64(offs), _p32(toks), n, p, q, _p32(out), cap))
    return _triples(lambda out, cap: lib.oracle_bruteforce_self_sim(sim, _p64(offs), _p32(toks), n, p, q,
                                                                    _p32(out), cap))


def bruteforce_rs(r_offsets, r_tokens, s_offsets, s_tokens, p: int, q: int, sim: int = JACCARD) -> np.ndarray:
    ro, rt, so, st = _u64(r_offsets), _u32(r_tokens), _u64(s_offsets), _u32(s_tokens)
    nr, ns = len(r_offsets) - 1, len(s_offsets) - 1
    lib = _load()
    if sim == JACCARD:
        return _triples(lambda out, cap: lib.oracle_bruteforce_rs(_p64(ro), _p32(rt), nr, _p64(so), _p32(st), ns,
                                                                  p, q, _p32(out), cap))
    return _triples(lambda out, cap: lib.oracle_bruteforce_rs_sim(sim, _p64(ro), _p32(rt), nr, _p64(so), _p32(st),
                                                                  ns, p, q, _p32(out), cap))


def verify_batch(r_offsets, r_tokens, s_offsets, s_tokens, self_join: bool, p: int, q: int,
                 probe_ids, cand_offsets, cand_ids, flags: int = EARLY, consumed: bool = False,
                 sim: int = JACCARD):
    """Verify a grouped candidate batch.  Returns triples, or (triples, consumed_r, consumed_s)."""
    ro, rt, so, st = _u64(r_offsets), _u32(r_tokens), _u64(s_offsets), _u32(s_tokens)
    nr, ns = len(r_offsets) - 1, len(s_offsets) - 1
    pr, co, ci = _u32(probe_ids), _u64(cand_offsets), _u32(cand_ids)
    n_probes = len(probe_ids)
    n_cands = int(cand_offsets[-1]) if len(cand_offsets) else 0
    cr = np.zeros(max(n_cands, 1), dtype=np.uint32) if consumed else None
    cs = np.zeros(max(n_cands, 1), dtype=np.uint32) if consumed else None
    lib = _load()

    def call(out, cap):
        args = (_p64(ro), _p32(rt), nr, _p64(so), _p32(st), ns, int(self_join), p, q,
                n_probes, _p32(pr), _p64(co), _p32(ci), flags, _p32(out), cap,
                _p32(cr) if consumed else None, _p32(cs) if consumed else None)
        if sim == JACCARD:
            return lib.oracle_verify_batch(*args)
        return lib.oracle_verify_batch_sim(sim, *args)
    tr = _triples(call, cap_hint=max(n_cands, 1))
    if consumed:
        return tr, cr[:n_cands], cs[:n_cands]
    return tr


def verify_batch_threads(r_offsets, r_tokens, s_offsets, s_tokens, self_join: bool, p: int, q: int,
                         probe_ids, cand_offsets, cand_ids, flags: int = EARLY, sim: int = JACCARD,
                         n_threads: int | None = None) -> np.ndarray:
    """verify_batch over contiguous probe ranges of about equal candidate counts, one range per
    host thread (the C routine releases the GIL), results concatenated in probe order."""
    n_threads = n_threads or os.cpu_count() or 1
    co = np.asarray(cand_offsets, dtype=np.int64)
    pr = np.asarray(probe_ids)
    ci = np.asarray(cand_ids)
    if len(pr) == 0:
        return np.zeros((0, 3), dtype=np.uint32)
    bounds = np.searchsorted(co, np.linspace(0, co[-1], n_threads + 1), side="left")
    bounds[0], bounds[-1] = 0, len(pr)
    bounds = np.maximum.accumulate(np.minimum(bounds, len(pr)))
    jobs = [(a, b) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]

    def run(job):
        a, b = job
        return verify_batch(r_offsets, r_tokens, s_offsets, s_tokens, self_join, p, q, pr[a:b],
                            (co[a:b + 1] - co[a]).astype(np.uint64), ci[co[a]:co[b]], flags=flags, sim=sim)

    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        parts = list(ex.map(run, jobs))
    parts = [np.asarray(x, dtype=np.uint32).reshape(-1, 3) for x in parts]
    return np.concatenate(parts) if parts else np.zeros((0, 3), dtype=np.uint32)


def renumber(offsets, tokens):
    """Returns (new_tokens, n_distinct): tokens renumbered by ascending frequency, sets re-sorted."""
    offs, toks = _u64(offsets), _u32(tokens)
    n = len(offsets) - 1
    out = np.empty_like(toks)
    u = _load().oracle_renumber(_p64(offs), _p32(toks), n, _p32(out))
    if u < 0:
        raise MemoryError("oracle_renumber")
    return out[:len(tokens)], int(u)


def allpairs_self(offsets, tokens, p: int, q: int, sim: int = JACCARD):
    """AllPairs self-join.  Returns (triples, n_candidates)."""
    offs, toks = _u64(offsets), _u32(tokens)
    n = len(offsets) - 1
    nc = ctypes.c_uint64()
    lib = _load()
    if sim == JACCARD:
        fn = lambda out, cap: lib.oracle_allpairs_self(_p64(offs), _p32(toks), n, p, q, _p32(out), cap,
                                                       ctypes.byref(nc))
    else:
        fn = lambda out, cap: lib.oracle_allpairs_self_sim(sim, _p64(offs), _p32(toks), n, p, q, _p32(out), cap,
                                                           ctypes.byref(nc))
    tr = _triples(fn, cap_hint=1 << 16)
    return tr, int(nc.value)


def sort_triples(t: np.ndarray) -> np.ndarray:
    """Triples sorted by (r, s) - the canonical order for comparisons."""
    t = np.asarray(t, dtype=np.uint32).reshape(-1, 3)
    if len(t) == 0:
        return t
    key = (t[:, 0].astype(np.uint64) << np.uint64(32)) | t[:, 1].astype(np.uint64)
    return t[np.argsort(key, kind="stable")]
