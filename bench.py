#!/usr/bin/env python3
"""Benchmark: candidate pairs verified per second on one GB300.

Workload (default "uneven_instances"): 256 independent prefix-filter
self-joins verified in one batched launch (one plan and one persistent
verify kernel over every instance): collection sizes log-uniform 500..50,000
sets, mean set size log-uniform 5..500 (lognormal, sigma 0.6), Zipf s in
[0.6, 1.2] over 1e5 tokens, t uniform over {0.6, ..., 0.95}.  The CPU feeder
produces the candidate batches once (untimed); the granularity is chosen by
the library's autotuner beforehand.  Synthetic, seeded data.  Other
workloads: tiny (all 499,500 pairs of 1,000 sets), short_sets (200k short
sets, four thresholds), long_sets, serving_collection, rs_short, serving
(continuous batching only), candgen.

value   pairs/s with inputs resident in HBM; L2 is flushed (512 MiB write)
        before every timed step; CUDA events on the launching stream; max
        over ranks.  With N ranks every batch is split into N contiguous
        probe ranges, one per rank (strong scaling; no data exchange).
e2e     the same metric through the public synchronous call with pinned
        host buffers: the inputs' transfer (copies, or in calls of 2^25+
        candidates the kernels' own reads of the pinned inputs over the host
        link), kernels and the result readback in the timed region.
served  (default workload, one rank) continuous batching on the resident
        1,000,000-set collection: p50/p99 submit-to-result latency of 1,000
        Poisson-arriving requests at 0.5x and 0.9x of the closed-loop peak,
        device-memory budget M_c = 4 GiB.
roofline  algorithmic bytes of the verify kernel (candidate stream, set
        descriptors, the tokens the positional filter lets the merge read,
        results) over its own event-timed duration, against the measured HBM
        copy bandwidth; l2_aware_roofline adds the L2 read rate measured by
        the library's probe; a_pair the looser count with the probe's
        tokens read once per pair.
warm_l2 / plain_per_batch  the same launch without the flush, and one
        plan + verify call per instance instead of one batched launch.
cpu_baseline / --impl reference  the CPU oracle as it stands, on host cores.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidate pairs verified/sec and GB/s vs HBM peak; p50/p99 batch latency"
SIM = 0                   # similarity function of every instance (0 Jaccard, 1 Dice, 2 Cosine, 3 overlap)
SIM_NAMES = {"jaccard": 0, "dice": 1, "cosine": 2, "overlap": 3}
OVERLAP_THRESHOLDS = [(6, 1), (8, 1), (10, 1), (12, 1)]
REF_STEP_PAIRS = 3_000_000  # candidates per step of the reference (CPU oracle) arm
INSTANCES = 0               # uneven_instances: 0 = all 256 (--instances, for profiling runs only)
UNIT = "pairs/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20


# --------------------------------------------------------------------------- workloads

def workload(name: str):
    """Returns (config dict, [collections], [(collection index, p, q), ...])."""
    import synth
    if name == "uneven_instances":
        specs = synth.uneven_instances()
        if INSTANCES:
            specs = specs[:INSTANCES]  # profiling runs: the first instances only
        colls = [synth.collection(ins.coll) for ins in specs]
        inst = [(i, ins.p, ins.q) for i, ins in enumerate(specs)]
        cfg = {"workload": name if not INSTANCES else f"{name}[:{INSTANCES}]",
               "description": f"{len(specs)} independent self-joins in one launch: n log-uniform "
               "[500, 50000], mean set size log-uniform [5, 500] (sigma 0.6, clip [2, min(4 mean, 2000)]), "
               "Zipf s uniform [0.6, 1.2] over 1e5 tokens, t uniform over {0.6, ..., 0.95}",
               "instances": len(inst), "n_sets": int(sum(c.n for c in colls)),
               "n_tokens": int(sum(len(c.tokens) for c in colls)), "seed": 1004}
        return cfg, colls, inst
    if name == "tiny":
        c = synth.collection(synth.tiny_self_join())
        cfg = {"workload": name, "description": "brute-force self-join: all 499,500 pairs of 1,000 sets "
               "(sizes uniform 5..50, Zipf(1.0) over 1e4 tokens), t = 4/5", "n_sets": c.n,
               "n_tokens": int(len(c.tokens)), "seed": 1001, "thresholds": ["4/5"], "candidates": "all pairs"}
        return cfg, [c], [(0, 4, 5)]
    if name == "rs_short":
        # one seeded collection with planted near-duplicates, split into R (first 100k sets) and
        # S (the other 150k), so that S holds edited copies of sets of R
        spec = synth.short_sets(seed=1006, n=250_000)
        spec.plant_frac, spec.plant_edits = 0.3, 2
        c = synth.collection(spec)
        cut = int(c.offsets[100_000])
        cr = types.SimpleNamespace(n=100_000, offsets=c.offsets[:100_001].copy(), tokens=c.tokens[:cut].copy())
        cs = types.SimpleNamespace(n=150_000, offsets=(c.offsets[100_000:] - c.offsets[100_000]).astype(np.uint64),
                                   tokens=c.tokens[cut:].copy())
        ts = [(4, 5), (7, 10), (3, 5), (1, 2)] if SIM != 3 else OVERLAP_THRESHOLDS
        cfg = {"workload": name, "description": "R x S join: one seeded collection of 250k short sets "
               "(lognormal(20, 0.6) clip [2,200], Zipf(1.0) over 1e6, seed 1006, 30% planted near-duplicates "
               "with 2 edits) split into R = the first 100k and S = the other 150k; feeder candidates of R "
               "against S",
               "n_sets": cr.n + cs.n, "n_tokens": int(len(cr.tokens) + len(cs.tokens)),
               "thresholds": [f"{p}/{q}" for p, q in ts]}
        return cfg, [cr, cs], [((0, 1), p, q) for p, q in ts]
    if name == "short_sets":
        spec = synth.short_sets()
        ts = [(9, 10), (4, 5), (7, 10), (3, 5)]
        label = "prefix-filter self-join, 200k short sets, t in {0.9,0.8,0.7,0.6}"
    elif name == "long_sets":
        spec = synth.long_sets()
        ts = [(3, 5)]
        label = "prefix-filter self-join, 50k long sets, t=0.6"
    elif name == "serving_collection":
        spec = synth.serving_collection()
        ts = [(7, 10), (4, 5), (9, 10)]
        label = "prefix-filter self-join, 1M sets mean 12, t in {0.7,0.8,0.9}"
    else:
        raise SystemExit(f"unknown workload {name}")
    if SIM == 3:
        ts = OVERLAP_THRESHOLDS
    c = synth.collection(spec)
    cfg = {"workload": name, "description": label, "n_sets": c.n, "n_tokens": int(len(c.tokens)),
           "size_law": f"{'lognormal' if spec.size_kind else 'uniform'}({spec.a},{spec.b}) clip [{spec.lo},{spec.hi}]",
           "zipf_s": spec.zipf_s, "vocab": spec.vocab, "seed": spec.seed,
           "thresholds": [f"{p}/{q}" for p, q in ts]}
    return cfg, [c], [(0, p, q) for p, q in ts]


def coll_pair(colls, k):
    """(R collection, S collection, self-join?) of an instance's collection index k, which is an
    int for a self-join or a pair (r, s) for an R x S join."""
    if isinstance(k, tuple):
        return colls[k[0]], colls[k[1]], False
    return colls[k], colls[k], True


def make_batches(colls, inst, all_pairs: bool = False, ppjoin: bool = False):
    """CPU feeder (AllPairs prefix filter) candidates for every instance, or every pair r < s
    (brute force) when all_pairs: (ci, p, q, probes, offsets, cands)."""
    import paper_1812_09141_gb300 as ssj
    threads = max(1, min(16, os.cpu_count() or 1))
    import synth
    out = []
    for ci, p, q in inst:
        cR, cS, selfj = coll_pair(colls, ci)
        if all_pairs:
            b = synth.all_pairs_batch(cR.n)
            pr, co, cands = b.probe_ids, b.cand_offsets, b.cand_ids
        else:
            pr, co, cands = ssj.feeder_all(cR.offsets, cR.tokens, p, q, n_threads=threads, sim=SIM,
                                           s_offsets=None if selfj else cS.offsets,
                                           s_tokens=None if selfj else cS.tokens,
                                           flags=ssj.SSJ_FEEDER_PPJOIN if ppjoin else 0)
        out.append((ci, p, q, pr, co, cands))
    return out


# --------------------------------------------------------------------------- CPU oracle leg

def oracle_accounting(colls, batches):
    """Algorithmic bytes of each batch from the oracle's sequential stop points:
    12 B per probe (id + offset), 4 B per candidate id, 8 B per touched set
    descriptor (probe and candidate), 4 B per token the merge must read (the
    probe's tokens once per probe, the candidate's up to the stop point), 12 B
    per result triple and 8 B for the count.  Batches are accounted on several
    host threads (the C oracle releases the GIL)."""
    import oracle

    def one(b):
        k, p, q, pr, co, ci = b
        cR, cS, selfj = coll_pair(colls, k)
        tr, cr, cs = oracle.verify_batch(cR.offsets, cR.tokens, cS.offsets, cS.tokens, selfj, p, q, pr, co, ci,
                                         consumed=True, sim=SIM)
        counts = np.diff(co.astype(np.int64))
        pr_max = np.zeros(len(pr), dtype=np.int64)
        if len(ci):
            nz = counts > 0
            starts = co[:-1].astype(np.int64)[nz]
            pr_max[nz] = np.maximum.reduceat(cr.astype(np.int64), starts)
        a = (12 * len(pr) + 4 * len(ci) + 8 * (len(pr) + len(ci)) + 4 * int(pr_max.sum())
             + 4 * int(cs.astype(np.int64).sum()) + 12 * len(tr) + 8)
        # the part that comes from HBM even with the collection resident in L2:
        # the candidate stream and the output
        a_hbm = 12 * len(pr) + 4 * len(ci) + 12 * len(tr) + 8
        # the looser per-pair figure: both sides' consumed tokens for every pair
        a_pair = (12 * len(pr) + 4 * len(ci) + 8 * (len(pr) + len(ci)) + 4 * int(cr.astype(np.int64).sum())
                  + 4 * int(cs.astype(np.int64).sum()) + 12 * len(tr) + 8)
        return {"bytes": int(a), "hbm_bytes": int(a_hbm), "pair_bytes": int(a_pair), "survivors": int(len(tr)),
                "pairs": int(len(ci))}

    with cf.ThreadPoolExecutor(max(1, min(len(batches), os.cpu_count() or 1))) as ex:
        return list(ex.map(one, batches))


def stride_sample(batches, target_pairs: int):
    """Every k-th probe of each batch with all of its candidates, k chosen so that the sample
    holds about target_pairs candidates (k = 1: the whole batches).  A uniform stride over probes
    is not biased by the feeder's size order.  Returns (sample batches, k)."""
    pairs_step = sum(len(b[5]) for b in batches)
    stride = max(1, int(math.ceil(pairs_step / max(target_pairs, 1))))
    if stride == 1:
        return batches, 1
    sample = []
    for k, p, q, pr, co, ci in batches:
        co64 = co.astype(np.int64)
        pick = np.arange(0, len(pr), stride)
        counts = co64[pick + 1] - co64[pick]
        offs = np.zeros(len(pick) + 1, dtype=np.uint64)
        offs[1:] = np.cumsum(counts)
        cands = (np.concatenate([ci[co64[a]:co64[a + 1]] for a in pick]) if len(pick)
                 else np.zeros(0, dtype=np.uint32))
        sample.append((k, p, q, pr[pick], offs, cands.astype(np.uint32)))
    return sample, stride


def cpu_baseline(colls, batches, min_seconds=10.0, max_seconds=30.0, pass_pairs=4_000_000):
    """The oracle (single-threaded C) timed on the host over a fixed sample of the workload's
    batches (stride_sample, about pass_pairs candidates), repeated for at least min_seconds."""
    import oracle
    pairs_step = sum(len(b[5]) for b in batches)
    sample, stride = stride_sample(batches, pass_pairs)
    pairs, total_t, reps = 0, 0.0, 0
    while total_t < min_seconds and reps < 1000:
        for k, p, q, pr, co, ci in sample:
            cR, cS, selfj = coll_pair(colls, k)
            t0 = time.perf_counter()
            oracle.verify_batch(cR.offsets, cR.tokens, cS.offsets, cS.tokens, selfj, p, q, pr, co, ci, sim=SIM)
            total_t += time.perf_counter() - t0
            pairs += len(ci)
            if total_t > max_seconds:
                break
        reps += 1
        if total_t > max_seconds:
            break
    what = (f"{pairs / max(pairs_step, 1):.2f} steps of {pairs_step}" if stride == 1 else
            f"every {stride}-th probe of each of the {len(batches)} batches with all its candidates, "
            f"{reps} pass(es)")
    return {"value": pairs / total_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{pairs} candidate pairs of the workload ({what}), {total_t:.1f} s of single-threaded CPU work"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def cpu_baseline_threads(colls, batches, min_seconds=5.0):
    """The same oracle calls over all host cores: each batch split into contiguous probe ranges
    of about equal candidate counts, one range per thread (the C oracle releases the GIL)."""
    import oracle
    n_thr = os.cpu_count() or 1
    jobs = []
    for k, p, q, pr, co, ci in batches:
        co = co.astype(np.int64)
        bounds = np.searchsorted(co, np.linspace(0, co[-1], n_thr + 1), side="left")
        bounds[0], bounds[-1] = 0, len(pr)
        for a, b in zip(bounds[:-1], bounds[1:]):
            if b > a:
                jobs.append((k, p, q, pr[a:b], (co[a:b + 1] - co[a]).astype(np.uint64), ci[co[a]:co[b]]))
    pairs_step = sum(len(b[5]) for b in batches)

    def run(job):
        k, p, q, pr, co, ci = job
        cR, cS, selfj = coll_pair(colls, k)
        oracle.verify_batch(cR.offsets, cR.tokens, cS.offsets, cS.tokens, selfj, p, q, pr, co, ci, sim=SIM)

    steps, t = 0, 0.0
    with cf.ThreadPoolExecutor(n_thr) as ex:
        while t < min_seconds and steps < 1000:
            t0 = time.perf_counter()
            list(ex.map(run, jobs))
            t += time.perf_counter() - t0
            steps += 1
    return {"value": pairs_step * steps / t, "unit": UNIT, "cores": n_thr, "kind": "oracle",
            "sample": f"{steps} full steps ({pairs_step} pairs each) split into probe ranges over {n_thr} threads"}


# --------------------------------------------------------------------------- measurement helpers

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(workload_name: str):
    """DRAM bytes per verify launch from the committed ncu summary, if it was taken on the
    current kernel source (the summary records the sha256 of verify.cu)."""
    path = os.path.join(ROOT, "profiles", f"verify_kernel_{workload_name}.md")
    src = os.path.join(ROOT, "paper_1812_09141_gb300", "csrc", "verify.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        m_sha = re.search(r"verify\.cu sha256:\s*([0-9a-f]{64})", text)
        m_tr = re.search(r"dram bytes per verify launch:\s*([0-9.eE+]+)", text)
        if m_sha and m_tr and m_sha.group(1) == sha:
            return float(m_tr.group(1))
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the GPU works."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.perf_counter(), ln.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- ranks

def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value over the ranks of the job (every rank gets it), then a barrier.
    Each rank verifies its own contiguous probe range of every batch against its own copy of the
    collections (the path has no exchange step), so the job's time is its slowest rank's."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_value(pairs_all_ranks: int, steps: int, total_s: float) -> float:
    """Pairs/s of the whole job: the ranks share every step's pairs (each verifies its own probe
    ranges), so the job verifies pairs_all_ranks per step in the slowest rank's time."""
    return pairs_all_ranks * steps / total_s


def rank_share(batches, rank: int, world: int):
    """This rank's part of every batch: a contiguous range of probes holding about 1/world of the
    batch's candidates (the probe ranges of the ranks tile the batch, so every candidate is
    verified by exactly one rank).  Offsets are rebased to the range."""
    if world == 1:
        return batches
    out = []
    for k, p, q, pr, co, ci in batches:
        co64 = co.astype(np.int64)
        cut = np.searchsorted(co64, np.linspace(0, co64[-1], world + 1), side="left")
        cut[0], cut[-1] = 0, len(pr)
        cut = np.maximum.accumulate(np.minimum(cut, len(pr)))
        a, b = int(cut[rank]), int(cut[rank + 1])
        out.append((k, p, q, pr[a:b], (co64[a:b + 1] - co64[a]).astype(np.uint64), ci[co64[a]:co64[b]]))
    return out


def input_bytes_of(colls, batches):
    """Bytes of a step's inputs as they sit on the device: token arrays and set offsets of the
    collections, probe ids, candidate offsets and candidate ids of the batches."""
    return (sum(4 * len(c.tokens) + 8 * c.n for c in colls)
            + sum(4 * len(b[3]) + 8 * len(b[4]) + 4 * len(b[5]) for b in batches))


def common_config(cfg, colls, batches, args):
    """The config both arms report (same keys and values): the workload, its candidates, and how
    the GPU arm keeps timed steps from reusing L2 (inputs larger than L2, and a flush between
    steps)."""
    nbytes = input_bytes_of(colls, batches)
    l2 = (f"inputs {nbytes / 1e6:.0f} MB, " + ("larger than" if nbytes > 129e6 else "within")
          + " the 129 MB L2; " + (f"the GPU arm writes {args.l2_flush_mb} MiB before every timed step"
                                  if args.l2_flush_mb else "no flush between steps (profiling run)"))
    return dict(cfg, pairs_per_step=int(sum(len(b[5]) for b in batches)), instances_per_launch=len(batches),
                similarity=args.sim,
                candidates=("AllPairs prefix filter" + (" + PPJoin" if args.ppjoin else ""))
                if args.workload != "tiny" else "all pairs",
                l2_between_steps=l2)


# --------------------------------------------------------------------------- GPU arm

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_1812_09141_gb300 as ssj
    from paper_1812_09141_gb300 import _build

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg, colls, inst = workload(args.workload)
    all_batches = make_batches(colls, inst, all_pairs=args.workload == "tiny", ppjoin=args.ppjoin)
    batches = rank_share(all_batches, rank, world)
    pairs_step = sum(len(b[5]) for b in batches)
    pairs_all = sum(len(b[5]) for b in all_batches)
    sim_flags = SIM << 8

    stream = torch.cuda.Stream(device=dev)
    ctx = ssj.ssj_create(local_rank, flags=ssj.SSJ_CTX_PROFILE, stream=stream.cuda_stream)
    # renumbering by frequency is for self-joins; an R x S join keeps the raw token order
    rs_join = any(isinstance(k, tuple) for k, _, _ in inst)
    load_flags = ssj.SSJ_VALIDATE | (0 if rs_join else ssj.SSJ_RENUMBER_BY_FREQ) | (ssj.SSJ_PIN_L2 if args.pin_l2 else 0)
    handles = [ssj.ssj_load_collection(ctx, c.offsets, c.tokens, load_flags) for c in colls]

    def hpair(k):
        return (handles[k[0]], handles[k[1]]) if isinstance(k, tuple) else (handles[k], handles[k])

    dbs, outs, caps, keep = [], [], [], []
    for ci, p, q, pr, co, cands in batches:
        t_pr = torch.from_numpy(pr.astype(np.int32)).to(dev)
        t_co = torch.from_numpy(co.astype(np.int64)).to(dev)
        t_ci = torch.from_numpy(cands.astype(np.int32)).to(dev)
        keep.append((t_pr, t_co, t_ci))
        hR, hS = hpair(ci)
        dbs.append(ssj.DeviceBatch(hR, hS, p, q, t_pr, t_co, t_ci, len(cands), flags=sim_flags, n_probes=len(pr)))
        cap = max(min(len(cands), args.out_cap), 1)
        outs.append(torch.empty(cap * 3, dtype=torch.int32, device=dev))
        caps.append(cap)
    counts = torch.zeros(len(batches), dtype=torch.int64, device=dev)
    flush = torch.empty(max(args.l2_flush_mb << 18, 1), dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    if args.granularity:
        # a fixed setting (profiling runs: no tuning launches before the timed ones)
        t, l, w, b, d, ix = parse_granularity(args.granularity)
        ssj.ssj_set_granularity(ctx, t, l, w, b)
        ssj.ssj_set_short_pairs(ctx, d)
        ssj.ssj_set_index_items(ctx, ix)
        multi = ssj.ssj_multi_create(ctx, dbs, outs, caps, counts)
        tune = {"thread_max_key": t, "lane_max_key": l, "warp_max_key": w, "block_threads": b,
                "drain_min_live": d, "index_min_cands": ix, "chosen_by": "--granularity"}
    else:
        multi = ssj.ssj_multi_create(ctx, dbs, outs, caps, counts)
        # granularity and block size chosen by the library's autotuner on this launch (untimed)
        tune = ssj.ssj_multi_autotune(ctx, multi, stream.cuda_stream, reps=5)
        tune["chosen_by"] = "ssj_multi_autotune (median of 5 launches per setting)"
        ssj.ssj_set_granularity(ctx, tune["thread_max_key"], tune["lane_max_key"],
                                min(tune["warp_max_key"], 1 << 30), tune["block_threads"])
        ssj.ssj_set_short_pairs(ctx, tune["drain_min_live"])
        ssj.ssj_set_index_items(ctx, tune["index_min_cands"])

    clocks = ClockSampler(local_rank)
    clocks.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1)
            ssj.ssj_multi_launch(ctx, multi, stream.cuda_stream)
        stream.synchronize()
        if ssj.ssj_device_error(ctx):
            raise RuntimeError("device-side batch check fired")
        ssj.ssj_profile_read(ctx)  # drop warm-up launches
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ssj.ssj_multi_launch(ctx, multi, stream.cuda_stream)
            e1.record(stream)
            evs.append((e0, e1))
        stream.synchronize()
        torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    launches, plan_ms, verify_ms = ssj.ssj_profile_read(ctx)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    result_counts = [int(x) for x in counts.cpu().tolist()]

    # the same launch replayed from a CUDA graph (captured by the library)
    graph_ms = []
    with torch.cuda.stream(stream):
        ssj.ssj_multi_graph_launch(ctx, multi, stream.cuda_stream)  # capture + first replay
        for _ in range(min(args.steps, 20)):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ssj.ssj_multi_graph_launch(ctx, multi, stream.cuda_stream)
            e1.record(stream)
            graph_ms.append((e0, e1))
        stream.synchronize()
    graph_ms = [a.elapsed_time(b) for a, b in graph_ms]
    if [int(x) for x in counts.cpu().tolist()] != result_counts:
        raise RuntimeError("graph replay returned different counts")

    # warm L2: the same batched launch with nothing evicted in between
    warm = []
    with torch.cuda.stream(stream):
        for _ in range(min(args.steps, 20)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ssj.ssj_multi_launch(ctx, multi, stream.cuda_stream)
            e1.record(stream)
            warm.append((e0, e1))
        stream.synchronize()
    warm_ms = [a.elapsed_time(b) for a, b in warm]

    # the plain per-batch path: one stream-ordered call (plan + verify) per instance
    ssj.ssj_reserve(ctx, max(len(b[3]) for b in batches), max(len(b[5]) for b in batches))
    pcounts = torch.zeros(len(batches), dtype=torch.int64, device=dev)
    lib = ssj.lib()
    calls = [(ctypes.byref(db.batch), o.data_ptr(), cap, pcounts.data_ptr() + 8 * i)
             for i, (db, o, cap) in enumerate(zip(dbs, outs, caps))]
    plain = []
    with torch.cuda.stream(stream):
        for _ in range(min(args.steps, 20)):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for bp, op, cap, cp in calls:
                st = lib.ssj_verify_batch_async(ctx, bp, op, cap, cp, stream.cuda_stream)
                if st != ssj.SSJ_OK:
                    raise RuntimeError(ssj.ssj_last_error(ctx))
            e1.record(stream)
            plain.append((e0, e1))
        stream.synchronize()
    plain_ms = [a.elapsed_time(b) for a, b in plain]
    if [int(x) for x in pcounts.cpu().tolist()] != result_counts:
        raise RuntimeError("per-batch calls returned different counts")
    ssj.ssj_profile_read(ctx)  # drop their profile records

    # read-bandwidth probes: L2-resident buffer and a buffer far above L2
    l2_gbs = ssj.ssj_read_bandwidth(ctx, 32 << 20, 200)
    hbm_read_gbs = ssj.ssj_read_bandwidth(ctx, 4 << 30, 5)

    # ---------------- end to end through the public synchronous call, host buffers
    pinned = []
    for ci, p, q, pr, co, cands in batches:
        tp = torch.from_numpy(pr.astype(np.uint32).view(np.int32)).pin_memory()
        tc = torch.from_numpy(co.astype(np.uint64).view(np.int64)).pin_memory()
        ti = torch.from_numpy(cands.astype(np.uint32).view(np.int32)).pin_memory()
        pinned.append((hpair(ci), p, q, tp.numpy().view(np.uint32), tc.numpy().view(np.uint64),
                       ti.numpy().view(np.uint32), (tp, tc, ti)))
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps, 20))
    e2e_t = e2e_single_t = e2e_staged_t = 0.0
    h2d = sum(4 * len(b[3]) + 8 * (len(b[3]) + 1) + 4 * len(b[5]) for b in pinned)
    d2h = 0
    step_batches = [(hr, hs, p, q, pr, co, ci, sim_flags) for (hr, hs), p, q, pr, co, ci, _keep in pinned]
    with torch.cuda.stream(stream):
        for it in range(e2e_steps + 1 if e2e_steps else 0):
            # one call for every instance of the step (one batched launch)
            flush.fill_(1)
            stream.synchronize()
            t0 = time.perf_counter()
            res = ssj.ssj_verify_batches(ctx, step_batches)
            dt = time.perf_counter() - t0
            res_total = sum(len(r) for r in res)
            # the same call with every pinned input copied to the device before the kernels run
            flush.fill_(1)
            stream.synchronize()
            t0 = time.perf_counter()
            res_s = ssj.ssj_verify_batches(ctx, [x[:7] + (x[7] | ssj.SSJ_HOST_STAGED,) for x in step_batches])
            dt_staged = time.perf_counter() - t0
            if sum(len(r) for r in res_s) != res_total:
                raise RuntimeError("staged-copy call returned different counts")
            # one synchronous call per instance
            flush.fill_(1)
            stream.synchronize()
            t0 = time.perf_counter()
            for (hr, hs), p, q, pr, co, ci, _keep in pinned:
                ssj.ssj_verify_batch(ctx, hr, hs, p, q, pr, co, ci, flags=sim_flags)
            dt_single = time.perf_counter() - t0
            if it > 0:  # the first pass sizes the staging buffers
                e2e_t += dt
                e2e_single_t += dt_single
                e2e_staged_t += dt_staged
                d2h = 12 * res_total + 8 * len(pinned) + 4
    clocks.stop()
    ssj.ssj_profile_read(ctx)
    ssj.ssj_multi_destroy(ctx, multi)
    ssj.ssj_destroy(ctx)

    # end-to-end times: the slowest rank's
    e2e_t = max_over_ranks(e2e_t, world, dev)
    e2e_single_t = max_over_ranks(e2e_single_t, world, dev)
    e2e_staged_t = max_over_ranks(e2e_staged_t, world, dev)
    result = {"total_ms": total_ms, "step_ms": step_ms, "verify_ms": verify_ms, "plan_ms": plan_ms,
              "launches": launches, "counts": result_counts, "pairs_step": pairs_step, "pairs_all": pairs_all,
              "graph_ms": graph_ms, "cfg": common_config(cfg, colls, all_batches, args),
              "e2e_value": pairs_all * e2e_steps / e2e_t if e2e_t > 0 else None, "h2d": h2d, "d2h": d2h,
              "e2e_single_value": pairs_all * e2e_steps / e2e_single_t if e2e_single_t > 0 else None,
              "e2e_staged_value": pairs_all * e2e_steps / e2e_staged_t if e2e_staged_t > 0 else None,
              "clocks": clocks.summary(), "tune": tune, "warm_ms": warm_ms, "plain_ms": plain_ms,
              "l2_gbs": l2_gbs, "hbm_read_gbs": hbm_read_gbs}
    return result, colls, batches


def measure_serving(requests: int, budgets=(4, 1), coprocess: bool = True, seed: int = 2024):
    """Continuous batching on a resident 1M-set collection: closed-loop peak, then open-loop
    Poisson arrivals at 0.5x and 0.9x of that peak, for each device-memory budget M_c (GiB); and,
    if coprocess, the filter/verify co-process (Section 3.2) with chunks handed over as the CPU
    filter makes them."""
    import torch
    import synth
    import paper_1812_09141_gb300 as ssj

    c = synth.collection(synth.serving_collection())
    ts = [(7, 10), (4, 5), (9, 10)]
    threads = max(1, min(16, os.cpu_count() or 1))
    pools = []

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()

    # request inputs sit in pinned host memory, as a server's receive buffers would
    for p, q in ts:
        pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=threads)
        pools.append((p, q, pinned(pr), co.astype(np.int64), pinned(ci)))
    rng = np.random.default_rng(seed)
    n_req = requests

    def make_requests(arrivals, h):
        picks = []
        for i in range(n_req):
            p, q, pr, co, ci = pools[int(rng.integers(0, len(pools)))]
            want = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e7)))))
            want = min(want, int(co[-1]))
            a = int(rng.integers(0, len(pr)))
            # probes a .. b-1 with about `want` candidates (wrapping is avoided by moving a back)
            target = co[a] + want
            b = int(np.searchsorted(co, target, side="left"))
            if b > len(pr):
                b = len(pr)
                a = int(np.searchsorted(co, co[-1] - want, side="right")) - 1
                a = max(a, 0)
            b = max(b, a + 1)
            picks.append((p, q, pr, co, ci, a, b))
        arena = pinned(np.zeros(sum(b - a + 1 for *_, a, b in picks), dtype=np.uint64))
        reqs, sizes, at = [], [], 0
        for i, (p, q, pr, co, ci, a, b) in enumerate(picks):
            offs = arena[at:at + b - a + 1]
            at += b - a + 1
            offs[:] = co[a:b + 1] - co[a]
            cands = ci[int(co[a]):int(co[b])]
            # request buffers stay untouched until the replay has collected every result
            reqs.append((h, h, p, q, pr[a:b], offs, cands, float(arrivals[i]), ssj.SSJ_KEEP_INPUTS))
            sizes.append(len(cands))
        return reqs, np.array(sizes)

    out = {"workload": "serving", "collection": "1M sets, lognormal(12, 0.6) clip [2,200], Zipf(1.0) over 2e6",
           "requests": n_req, "request_sizes": "log-uniform [1e3, 1e7] pairs, slices of the CPU filter's "
           "candidates at t in {0.7, 0.8, 0.9}, in pinned host memory kept until collected (SSJ_KEEP_INPUTS)",
           "latency": "host clock from ssj_submit to the completion that ssj_poll reports", "runs": []}
    for budget_gb in budgets:
        ctx = ssj.ssj_create(0, mem_budget_bytes=budget_gb << 30, max_inflight=8)
        try:
            h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_VALIDATE | ssj.SSJ_RENUMBER_BY_FREQ)
            # warm-up and closed-loop peak
            reqs, sizes = make_requests(np.zeros(n_req), h)
            ssj.ssj_serve_replay(ctx, reqs[:50])
            lat, st = ssj.ssj_serve_replay(ctx, reqs)
            peak = st["pairs"] / st["wall_s"]
            run = {"budget_gib": budget_gb, "closed_loop": {"pairs_per_s": peak, "p50_ms": 1e3 * np.percentile(lat, 50),
                                                             "p99_ms": 1e3 * np.percentile(lat, 99),
                                                             "max_inflight": st["max_inflight"]}}
            mean_size = float(sizes.mean())
            for load in (0.5, 0.9):
                rate = load * peak / mean_size          # requests per second
                arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
                reqs, sizes2 = make_requests(arrivals, h)
                lat, st = ssj.ssj_serve_replay(ctx, reqs)
                run[f"open_loop_{load}"] = {"offered_pairs_per_s": load * peak,
                                            "achieved_pairs_per_s": st["pairs"] / st["wall_s"],
                                            "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                                            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                            "p50_ms_small": 1e3 * float(np.percentile(lat[sizes2 < 1e5], 50)),
                                            "p99_ms_large": 1e3 * float(np.percentile(lat[sizes2 >= 1e6], 99)),
                                            "max_inflight": st["max_inflight"], "eagain": st["eagain"]}
            if coprocess and budget_gb == 4:
                cp = ssj.ssj_serve_coprocess(ctx, h, c.offsets, c.tokens, 7, 10, threads, 1 << 20)
                run["coprocess_t0.7"] = dict(cp, chunk_cands=1 << 20, filter_threads=threads)
            out["runs"].append(run)
        finally:
            ssj.ssj_destroy(ctx)
    return out


def run_serving(args):
    import torch
    from paper_1812_09141_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    print(json.dumps(measure_serving(args.requests)), flush=True)


def run_candgen(args):
    """Self-join with candidate generation on the device (ssj_self_join) against the CPU feeder
    (16 threads) followed by the same GPU verification, and GroupJoin (CPU group candidates
    expanded and verified on the device), on the short-set and long-set collections; wall
    clock; results and candidate counts must agree."""
    import torch
    import synth
    import paper_1812_09141_gb300 as ssj
    from paper_1812_09141_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    threads = max(1, min(16, os.cpu_count() or 1))
    ctx = ssj.ssj_create(0)
    out = {"workload": "candgen", "runs": []}
    try:
        for name, spec, ts in (("short_sets", synth.short_sets(), [(9, 10), (4, 5), (7, 10), (3, 5)]),
                               ("long_sets", synth.long_sets(), [(9, 10), (4, 5)])):
            c = synth.collection(spec)
            h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens, ssj.SSJ_RENUMBER_BY_FREQ)
            for p, q in ts:
                row = {"collection": name, "t": f"{p}/{q}"}
                for label, fl in (("device", 0), ("device_positional", ssj.SSJ_JOIN_POSITIONAL)):
                    ssj.ssj_self_join(ctx, h, p, q, fl | ssj.SSJ_COUNT_ONLY)  # warm-up
                    times = []
                    for _ in range(3):
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        cnt, nc = ssj.ssj_self_join(ctx, h, p, q, fl | ssj.SSJ_COUNT_ONLY)
                        times.append(time.perf_counter() - t0)
                    row[label] = {"s": float(np.median(times)), "candidates": nc, "results": cnt,
                                  "candidates_per_s": nc / float(np.median(times))}
                t0 = time.perf_counter()
                pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, p, q, n_threads=threads)
                t_feed = time.perf_counter() - t0
                t0 = time.perf_counter()
                cnt_cpu = ssj.ssj_verify_batch(ctx, h, h, p, q, pr, co, ci, flags=ssj.SSJ_COUNT_ONLY)
                t_ver = time.perf_counter() - t0
                row["cpu_feeder_then_gpu"] = {"feeder_s": t_feed, "verify_s": t_ver, "candidates": len(ci),
                                              "results": cnt_cpu, "feeder_threads": threads}
                if cnt_cpu != row["device"]["results"] or len(ci) != row["device"]["candidates"]:
                    row["mismatch"] = True
                # GroupJoin: CPU grouping and group candidates, expansion + verification on the device
                t0 = time.perf_counter()
                g = ssj.group_candidates(c.offsets, c.tokens, p, q)
                t_grp = time.perf_counter() - t0
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                cnt_g, n_pairs = ssj.ssj_verify_groups(ctx, h, p, q, g, ssj.SSJ_COUNT_ONLY)
                t_gv = time.perf_counter() - t0
                row["groupjoin"] = {"groups": int(len(g.group_offsets) - 1), "probe_groups": int(len(g.probe_groups)),
                                    "candidate_group_entries": int(len(g.cand_groups)), "expanded_pairs": n_pairs,
                                    "results": cnt_g, "cpu_grouping_s": t_grp, "device_expand_verify_s": t_gv}
                if cnt_g != cnt_cpu or n_pairs != len(ci):
                    row["mismatch"] = True
                out["runs"].append(row)
            ssj.ssj_unload_collection(ctx, h)
    finally:
        ssj.ssj_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The CPU oracle as it stands (single-threaded C) on this workload's candidates.  Each step
    verifies a fixed bounded sample: every k-th probe of each batch (with all of its candidates),
    k chosen so that the sample holds about REF_STEP_PAIRS candidates, or the whole step when it
    is smaller; a uniform stride over probes, so the sample is not biased by the feeder's size
    order."""
    import oracle
    cfg, colls, inst = workload(args.workload)
    batches = make_batches(colls, inst, all_pairs=args.workload == "tiny", ppjoin=args.ppjoin)
    pairs_step = sum(len(b[5]) for b in batches)
    sample, stride = stride_sample(batches, REF_STEP_PAIRS)
    sample_pairs = sum(len(x[5]) for x in sample)

    def one_step():
        for k, p, q, pr, co, ci in sample:
            cR, cS, selfj = coll_pair(colls, k)
            oracle.verify_batch(cR.offsets, cR.tokens, cS.offsets, cS.tokens, selfj, p, q, pr, co, ci, sim=SIM)
    for _ in range(args.warmup):  # untimed warm-up steps, as in the GPU arm
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    v = sample_pairs * args.steps / dt
    whole = stride == 1
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.gpus > 1 else "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", "config": common_config(cfg, colls, batches, args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": (f"{args.steps} full steps of the workload ({pairs_step} pairs each)"
                                        if whole else
                                        f"{args.steps} steps of a fixed sample of {sample_pairs} of the "
                                        f"{pairs_step} candidate pairs of a step: every {stride}-th probe of "
                                        f"each of the {len(batches)} batches with all its candidates")
                                       + f", after {args.warmup} untimed warm-up steps, one host thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


WORKLOADS = ("uneven_instances", "tiny", "short_sets", "long_sets", "serving_collection", "rs_short", "serving",
             "candgen")


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="uneven_instances", choices=WORKLOADS)
    ap.add_argument("--no-serving", action="store_true", help="skip the served-latency leg of the default workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l2-flush-mb", type=int, default=L2_FLUSH_BYTES >> 20,
                    help="bytes written between timed steps to evict L2 (0 disables; only for profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--out-cap", type=int, default=1 << 26, help="most result triples kept per instance")
    ap.add_argument("--requests", type=int, default=1000, help="requests of the serving workload")
    ap.add_argument("--sim", default="jaccard", choices=sorted(SIM_NAMES),
                    help="similarity function of every instance (overlap uses thresholds 6, 8, 10, 12)")
    ap.add_argument("--ppjoin", action="store_true", help="PPJoin positional filter in the CPU feeder")
    ap.add_argument("--granularity", default="", help="thread,lane,warp,block_threads[,drain_min_live[,index_min_cands]]: "
                    "fixed setting instead of the autotuner's (profiling runs)")
    ap.add_argument("--pin-l2", action="store_true",
                    help="load the collections with SSJ_PIN_L2 (persisting-L2 window over the token array)")
    ap.add_argument("--instances", type=int, default=0,
                    help="uneven_instances: verify only the first N instances (profiling runs on a smaller case)")
    return ap


def parse_granularity(text: str):
    """--granularity: thread, lane and warp bin keys and block_threads, then optionally
    drain_min_live and index_min_cands (0 when absent)."""
    g = [int(x) for x in text.split(",")]
    if not 4 <= len(g) <= 6 or min(g) < 0:
        raise ValueError(f"--granularity wants 4 to 6 non-negative integers, got {text!r}")
    return tuple(g[:4]) + (g[4] if len(g) > 4 else 0, g[5] if len(g) > 5 else 0)


def main():
    args = build_parser().parse_args()
    if args.granularity:
        try:
            parse_granularity(args.granularity)
        except ValueError as e:
            raise SystemExit(str(e))
    global SIM, INSTANCES
    SIM = SIM_NAMES[args.sim]
    INSTANCES = args.instances
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "serving" and args.impl == "ours":
        if rank == 0:
            run_serving(args)
        return
    if args.workload == "candgen" and args.impl == "ours":
        if rank == 0:
            run_candgen(args)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res, colls, batches = run_ours(args, rank, world, local_rank)
    served = None
    if world == 1 and args.workload == "uneven_instances" and not args.no_serving:
        # the served path on the resident 1M-set collection, in the same line
        served = measure_serving(args.requests, budgets=(4,), coprocess=False)
    if rank != 0:
        return
    pairs_step = res["pairs_step"]
    total_s = res["total_ms"] / 1e3
    input_bytes = input_bytes_of(colls, batches)
    value = whole_job_value(res["pairs_all"], args.steps, total_s)
    peak, peak_kind = measured_hbm_peak()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": res["cfg"],
            "l2_between_steps": (f"flushed before every timed step ({args.l2_flush_mb} MiB write)"
                                 if args.l2_flush_mb else "not flushed (profiling run)"),
            "parallelism": (f"{world} ranks, each a contiguous probe range of every batch" if world > 1
                            else "single GPU"),
            "device_input_bytes": int(input_bytes), "inputs_fit_l2": bool(input_bytes < 129e6),
            "l2_pinned": bool(args.pin_l2)}
    sm = sorted(res["step_ms"])
    line["latency_ms"] = {"p50": float(np.percentile(sm, 50)), "p99": float(np.percentile(sm, 99)),
                          "per": "one batched launch (every instance of the step), device time"}
    gm = res["graph_ms"]
    line["graph_replay_ms_per_step"] = float(np.median(gm)) if gm else None
    line["gpu_launches"] = 2 * res["launches"]
    line["granularity"] = res["tune"]
    if served is not None:
        run = served["runs"][0]
        line["served"] = {
            "workload": "continuous batching on the resident 1,000,000-set collection (lognormal mean 12, "
                        "Zipf 1.0 over 2e6 tokens), t in {0.7, 0.8, 0.9}",
            "requests": served["requests"], "request_sizes": served["request_sizes"],
            "latency": served["latency"], "mem_budget_gib": run["budget_gib"],
            "closed_loop_pairs_per_s": run["closed_loop"]["pairs_per_s"],
            "p50_ms_at_0.5x": run["open_loop_0.5"]["p50_ms"], "p99_ms_at_0.5x": run["open_loop_0.5"]["p99_ms"],
            "p50_ms_at_0.9x": run["open_loop_0.9"]["p50_ms"], "p99_ms_at_0.9x": run["open_loop_0.9"]["p99_ms"],
            "runs": served["runs"]}
    wm = sorted(res["warm_ms"])
    line["warm_l2"] = {"pairs_per_s": pairs_step / (np.median(wm) / 1e3), "p50_ms": float(np.percentile(wm, 50)),
                       "p99_ms": float(np.percentile(wm, 99)), "runs": len(wm)}
    pm = sorted(res["plain_ms"])
    line["plain_per_batch"] = {"pairs_per_s": pairs_step / (np.median(pm) / 1e3), "p50_ms": float(np.percentile(pm, 50)),
                               "p99_ms": float(np.percentile(pm, 99)), "runs": len(pm),
                               "call": "ssj_verify_batch_async per instance (plan + verify each), L2 flushed"}
    line["kernel_ms_per_step"] = {"verify": res["verify_ms"] / args.steps, "plan": res["plan_ms"] / args.steps}
    line["survivors_per_step"] = sum(res["counts"])
    line["e2e"] = {"value": res["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                   "d2h_bytes_per_step": res["d2h"],
                   "call": "ssj_verify_batches: every instance of the step in one call (host pointers, pinned); "
                           "a call of 2^25+ candidates has the kernels read the pinned inputs over the host link "
                           "(NVLink-C2C) inside the timed region, a smaller one copies them first",
                   "per_instance_calls": {"value": res["e2e_single_value"], "unit": UNIT,
                                          "call": "ssj_verify_batch per instance"},
                   "staged_copies": {"value": res["e2e_staged_value"], "unit": UNIT,
                                     "call": "ssj_verify_batches with SSJ_HOST_STAGED: every input copied to the "
                                             "device first (two launches, the second group's copies overlapping "
                                             "the first group's kernels)"}}
    line["clocks"] = res["clocks"]

    if world == 1 and not args.no_cpu_baseline:
        acc = oracle_accounting(colls, batches)
        bytes_step = sum(a["bytes"] for a in acc)
        if [a["survivors"] for a in acc] != res["counts"]:
            line["count_mismatch"] = {"oracle": [a["survivors"] for a in acc], "gpu": res["counts"]}
        verify_s_step = res["verify_ms"] / 1e3 / args.steps
        achieved = bytes_step / verify_s_step / 1e9
        traffic = recorded_traffic(args.workload)
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": traffic,
                            "kernel": "verify_kernel", "peak_source": f"{peak_kind} copy bandwidth",
                            "algorithmic_bytes_per_launch": bytes_step}
        line["gbs_vs_hbm_peak"] = {"achieved_gbs": achieved, "frac": achieved / peak}
        pair_step = sum(a["pair_bytes"] for a in acc)
        line["a_pair"] = {"bytes_per_launch": pair_step, "achieved_gbs": pair_step / verify_s_step / 1e9,
                          "frac": pair_step / verify_s_step / 1e9 / peak,
                          "note": "both sides' consumed tokens counted for every pair (the probe's tokens once "
                                  "per pair, not once per probe)"}
        hbm_step = sum(a["hbm_bytes"] for a in acc)
        l2 = res["l2_gbs"]
        bound_s = max(hbm_step / (peak * 1e9), bytes_step / (l2 * 1e9))
        warm_verify_s = np.median(res["warm_ms"]) / 1e3
        line["l2_aware_roofline"] = {
            "l2_read_gbs": l2, "hbm_read_gbs_probe": res["hbm_read_gbs"], "hbm_peak_gbs": peak,
            "A_min": bytes_step, "A_hbm": hbm_step,
            "frac_cold": bound_s / verify_s_step, "frac_warm_step": bound_s / warm_verify_s,
            "formula": "max(A_hbm/BW_hbm, A_min/BW_l2) / t; t = verify kernel time (cold: L2 flushed before "
                       "the step) or whole warm step; BW_l2 from ssj_read_bandwidth over a 32 MiB buffer"}
        line["cpu_baseline"] = cpu_baseline(colls, batches)
        line["cpu_baseline"]["cpu_model"] = cpu_model()
        line["cpu_baseline_all_cores"] = cpu_baseline_threads(colls, batches)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
