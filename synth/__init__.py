"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds input generation only: set sizes, Zipf token draws,
planted near-duplicates and candidate id lists.  None of the join's
arithmetic lives here (no overlap, threshold, filter or renumbering), so it
can feed both the CPU oracle and the CUDA library without coupling them.

The workload shapes follow the paper's setting (Section 5: self-joins with
Jaccard over collections whose set sizes are skewed and whose tokens are
Zipf-like); the real datasets are not available, so these stand in for them.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_gen.so")
_lock = threading.Lock()
_lib = None

SIZE_UNIFORM = 0
SIZE_LOGNORMAL = 1


def build(force: bool = False) -> str:
    """Compile gen.c into _gen.so next to it (plain gcc, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.synth_sizes.restype = ctypes.c_uint64
            lib.synth_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, u32p]
            lib.synth_tokens.restype = ctypes.c_int
            lib.synth_tokens.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p, ctypes.c_double,
                                         ctypes.c_uint32, u64p, u32p]
            lib.synth_plant.restype = ctypes.c_uint32
            lib.synth_plant.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u64p, u32p, ctypes.c_double,
                                        ctypes.c_uint32]
            lib.synth_random_batch.restype = ctypes.c_uint64
            lib.synth_random_batch.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_uint32, u32p, u64p, u32p]
            lib.synth_loguniform.restype = ctypes.c_double
            lib.synth_loguniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                             ctypes.c_double]
            lib.synth_uniform.restype = ctypes.c_double
            lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_double]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


@dataclass
class CollectionSpec:
    """One synthetic collection: n sets, a size law, and a Zipf token law."""
    n: int
    size_kind: int            # SIZE_UNIFORM or SIZE_LOGNORMAL
    a: float                  # uniform: unused; lognormal: arithmetic mean
    b: float                  # uniform: unused; lognormal: sigma
    lo: int
    hi: int
    zipf_s: float
    vocab: int
    seed: int
    plant_frac: float = 0.0   # fraction of sets overwritten by edited copies
    plant_edits: int = 0


@dataclass
class Collection:
    offsets: np.ndarray       # uint64, n+1
    tokens: np.ndarray        # uint32, sorted-unique within each set
    spec: CollectionSpec | None = None

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.uint32)

    def set(self, i: int) -> np.ndarray:
        return self.tokens[self.offsets[i]:self.offsets[i + 1]]


def collection(spec: CollectionSpec) -> Collection:
    lib = _load()
    sizes = np.empty(spec.n, dtype=np.uint32)
    total = lib.synth_sizes(spec.seed, spec.n, spec.size_kind, spec.a, spec.b, spec.lo, spec.hi,
                            _p(sizes, ctypes.c_uint32))
    offsets = np.empty(spec.n + 1, dtype=np.uint64)
    tokens = np.empty(max(int(total), 1), dtype=np.uint32)
    rc = lib.synth_tokens(spec.seed, spec.n, _p(sizes, ctypes.c_uint32), spec.zipf_s, spec.vocab,
                          _p(offsets, ctypes.c_uint64), _p(tokens, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("synth_tokens failed (a set size exceeds the vocabulary?)")
    tokens = tokens[:int(total)]
    if spec.plant_frac > 0:
        lib.synth_plant(spec.seed, spec.n, _p(offsets, ctypes.c_uint64), _p(tokens, ctypes.c_uint32),
                        spec.plant_frac, spec.plant_edits)
    return Collection(offsets, tokens, spec)


def from_lists(sets) -> Collection:
    """A collection from Python lists (each sorted ascending, unique)."""
    sizes = [len(s) for s in sets]
    offsets = np.zeros(len(sets) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(sizes, dtype=np.uint64)
    tokens = np.array([t for s in sets for t in s], dtype=np.uint32)
    return Collection(offsets, tokens)


@dataclass
class Batch:
    """Grouped candidate list: probe_ids[k] is checked against
    cand_ids[cand_offsets[k]:cand_offsets[k+1]] (the probe / offset /
    candidate-id layout of the paper's Section 3.3.1, Fig. candidatesoutputlayout)."""
    probe_ids: np.ndarray     # uint32
    cand_offsets: np.ndarray  # uint64, n_probes+1
    cand_ids: np.ndarray      # uint32

    @property
    def n_probes(self) -> int:
        return len(self.probe_ids)

    @property
    def n_cands(self) -> int:
        return int(self.cand_offsets[-1]) if len(self.cand_offsets) else 0


def all_pairs_batch(n: int) -> Batch:
    """Every pair r < s of an n-set self-join, grouped by r (brute-force candidates)."""
    probe_ids = np.arange(n, dtype=np.uint32)
    counts = (n - 1 - np.arange(n, dtype=np.int64))
    offsets = np.zeros(n + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(counts)
    total = int(offsets[-1])
    # candidates of r are r+1 .. n-1
    starts = np.repeat(np.arange(n, dtype=np.int64) + 1, counts)
    within = np.arange(total, dtype=np.int64) - np.repeat(offsets[:-1].astype(np.int64), counts)
    cand_ids = (starts + within).astype(np.uint32)
    return Batch(probe_ids, offsets, cand_ids)


def random_batch(seed: int, n_r: int, n_s: int, n_probes: int, max_per_probe: int) -> Batch:
    """Uniform random probes and candidates (ids may repeat, may equal the probe)."""
    lib = _load()
    probe_ids = np.empty(n_probes, dtype=np.uint32)
    offs = np.empty(n_probes + 1, dtype=np.uint64)
    total = lib.synth_random_batch(seed, n_r, n_s, n_probes, max_per_probe, _p(probe_ids, ctypes.c_uint32),
                                   _p(offs, ctypes.c_uint64), None)
    cands = np.empty(max(int(total), 1), dtype=np.uint32)
    lib.synth_random_batch(seed, n_r, n_s, n_probes, max_per_probe, _p(probe_ids, ctypes.c_uint32),
                           _p(offs, ctypes.c_uint64), _p(cands, ctypes.c_uint32))
    return Batch(probe_ids, offs, cands[:int(total)])


# --------------------------------------------------------------------------
# The five workloads.  Thresholds are exact rationals p/q.
# --------------------------------------------------------------------------

T_VALUES = {0.95: (19, 20), 0.9: (9, 10), 0.85: (17, 20), 0.8: (4, 5), 0.75: (3, 4),
            0.7: (7, 10), 0.65: (13, 20), 0.6: (3, 5)}


def tiny_self_join(seed: int = 1001, n: int = 1000) -> CollectionSpec:
    """1,000 sets, sizes uniform 5..50, Zipf(1.0) over 10,000 tokens (t = 4/5, all pairs)."""
    return CollectionSpec(n, SIZE_UNIFORM, 0, 0, 5, 50, 1.0, 10_000, seed)


def short_sets(seed: int = 1002, n: int = 200_000) -> CollectionSpec:
    """200,000 sets, lognormal(mean 20, sigma 0.6) sizes clipped 2..200, Zipf(1.0) over 1e6 tokens."""
    return CollectionSpec(n, SIZE_LOGNORMAL, 20.0, 0.6, 2, 200, 1.0, 1_000_000, seed)


def long_sets(seed: int = 1003, n: int = 50_000) -> CollectionSpec:
    """50,000 sets, lognormal(mean 300, sigma 0.6) sizes clipped 50..2000, Zipf(0.8) over 1e5 tokens."""
    return CollectionSpec(n, SIZE_LOGNORMAL, 300.0, 0.6, 50, 2000, 0.8, 100_000, seed)


def serving_collection(seed: int = 1005, n: int = 1_000_000) -> CollectionSpec:
    """1,000,000 sets, lognormal(mean 12, sigma 0.6) clipped 2..200, Zipf(1.0) over 2e6 tokens."""
    return CollectionSpec(n, SIZE_LOGNORMAL, 12.0, 0.6, 2, 200, 1.0, 2_000_000, seed)


@dataclass
class InstanceSpec:
    coll: CollectionSpec
    p: int
    q: int


def uneven_instances(count: int = 256, seed: int = 1004, n_lo: int = 500, n_hi: int = 50_000,
                     mean_lo: float = 5.0, mean_hi: float = 500.0, vocab: int = 100_000) -> list[InstanceSpec]:
    """Independent self-join instances with uneven shapes: n log-uniform [n_lo, n_hi], mean set
    size log-uniform [mean_lo, mean_hi] (sigma 0.6, clipped to [2, min(4*mean, 2000)]), Zipf s
    uniform [0.6, 1.2], t uniform over {0.6, 0.65, ..., 0.95}."""
    lib = _load()
    ts = sorted(T_VALUES.values(), key=lambda pq: Fraction(*pq))
    out = []
    for i in range(count):
        n = int(round(lib.synth_loguniform(seed, 4 * i + 0, n_lo, n_hi)))
        mean = lib.synth_loguniform(seed, 4 * i + 1, mean_lo, mean_hi)
        s = lib.synth_uniform(seed, 4 * i + 2, 0.6, 1.2)
        ti = min(int(lib.synth_uniform(seed, 4 * i + 3, 0, len(ts))), len(ts) - 1)
        hi = int(min(4 * mean, 2000))
        hi = max(hi, 2)
        spec = CollectionSpec(n, SIZE_LOGNORMAL, mean, 0.6, 2, hi, s, vocab, seed * 1000 + i)
        out.append(InstanceSpec(spec, *ts[ti]))
    return out
