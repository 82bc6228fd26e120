"""Python binding of libssj: GPU verification for exact set similarity joins.

Thin ctypes layer over the C ABI in ``include/ssj.h`` and
``include/ssj_feeder.h``: the functions below carry the C names and only
marshal arguments (numpy arrays for host memory, torch CUDA tensors or raw
integers for device memory).  Every step of the verification runs in the
library's CUDA kernels; there is no Python or CPU fallback, and importing
this package fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SSJ_LIBRARY=checked loads the checked build (every kernel index tested, an
# out-of-bounds one reported as device error bit 4 instead of faulting).
LIB_PATH = os.path.join(_HERE, "libssj_checked.so" if os.environ.get("SSJ_LIBRARY") == "checked" else "libssj.so")

# status codes
SSJ_OK, SSJ_EINVAL, SSJ_ENOMEM, SSJ_EAGAIN, SSJ_ETIMEDOUT, SSJ_EBUSY, SSJ_ENOTFOUND, SSJ_EDEVICE = range(8)
STATUS_NAMES = ["SSJ_OK", "SSJ_EINVAL", "SSJ_ENOMEM", "SSJ_EAGAIN", "SSJ_ETIMEDOUT", "SSJ_EBUSY",
                "SSJ_ENOTFOUND", "SSJ_EDEVICE"]

# load flags
SSJ_RENUMBER_BY_FREQ = 0x1
SSJ_VALIDATE = 0x2
SSJ_PIN_L2 = 0x4
# batch flags
SSJ_COUNT_ONLY = 0x1
SSJ_SORTED = 0x2
SSJ_DEVICE_PTRS = 0x4
SSJ_EMIT_ALL = 0x8
SSJ_FORCE_THREAD = 0x10
SSJ_FORCE_WARP = 0x20
SSJ_FORCE_BLOCK = 0x40
SSJ_FORCE_LANE = 0x80
SSJ_FORCE_INDEX = 0x2000
SSJ_HOST_STAGED = 0x4000
SSJ_SIM_JACCARD = 0x000
SSJ_SIM_DICE = 0x100
SSJ_SIM_COSINE = 0x200
SSJ_SIM_OVERLAP = 0x300
SSJ_SIM_MASK = 0x300
SSJ_FEEDER_PPJOIN = 0x1
SSJ_JOIN_POSITIONAL = 0x400
SSJ_KEEP_INPUTS = 0x800
SSJ_HOST_DIRECT = 0x1000
SSJ_WIDE_REGISTERS = 0x10000
SSJ_BULK_STAGING = 0x20000
# context flags
SSJ_CTX_PROFILE = 0x1

TRIPLE_DTYPE = np.dtype([("r", np.uint32), ("s", np.uint32), ("overlap", np.uint32)])


class SsjError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class ssj_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint32), ("stream", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class ssj_batch(ctypes.Structure):
    _fields_ = [("R", ctypes.c_uint32), ("S", ctypes.c_uint32), ("p", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("n_probes", ctypes.c_uint32), ("probe_ids", ctypes.c_void_p), ("cand_offsets", ctypes.c_void_p),
                ("cand_ids", ctypes.c_void_p), ("n_cands", ctypes.c_uint64), ("flags", ctypes.c_uint32)]


class ssj_request(ctypes.Structure):
    _fields_ = [("batch", ssj_batch), ("arrival_s", ctypes.c_double)]


class ssj_tune_result(ctypes.Structure):
    _fields_ = [("thread_max_key", ctypes.c_uint32), ("lane_max_key", ctypes.c_uint32), ("warp_max_key", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("drain_min_live", ctypes.c_uint32),
                ("settings_tried", ctypes.c_uint32),
                ("best_ms", ctypes.c_float), ("initial_ms", ctypes.c_float),
                ("index_min_cands", ctypes.c_uint32)]


class ssj_feeder_opts(ctypes.Structure):
    _fields_ = [("sim", ctypes.c_uint32), ("p", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("n_threads", ctypes.c_uint32)]


class ssj_group_batch(ctypes.Structure):
    _fields_ = [("coll", ctypes.c_uint32), ("p", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("n_groups", ctypes.c_uint32), ("group_offsets", ctypes.c_void_p),
                ("members", ctypes.c_void_p), ("n_probe_groups", ctypes.c_uint32),
                ("probe_groups", ctypes.c_void_p), ("cand_offsets", ctypes.c_void_p),
                ("cand_groups", ctypes.c_void_p)]


class ssj_serve_stats(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("pairs", ctypes.c_uint64), ("results", ctypes.c_uint64),
                ("eagain", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32)]


class ssj_coprocess_stats(ctypes.Structure):
    _fields_ = [("filter_only_s", ctypes.c_double), ("join_s", ctypes.c_double), ("gpu_busy_s", ctypes.c_double),
                ("candidates", ctypes.c_uint64), ("results", ctypes.c_uint64), ("chunks", ctypes.c_uint32)]


class ssj_triple(ctypes.Structure):
    _fields_ = [("r", ctypes.c_uint32), ("s", ctypes.c_uint32), ("overlap", ctypes.c_uint32)]


# every exported symbol with (restype, argtypes); the tests check this list against include/*.h
_VP, _U32, _U64, _INT = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_P = ctypes.POINTER
SIGNATURES = {
    "ssj_create": (_INT, [_P(ssj_config), _P(_VP)]),
    "ssj_destroy": (None, [_VP]),
    "ssj_last_error": (ctypes.c_char_p, [_VP]),
    "ssj_load_collection": (_INT, [_VP, _VP, _VP, _U32, _U32, _P(_U32)]),
    "ssj_unload_collection": (_INT, [_VP, _U32]),
    "ssj_collection_info": (_INT, [_VP, _U32, _P(_U32), _P(_U64)]),
    "ssj_verify_batch": (_INT, [_VP, _P(ssj_batch), _VP, _U64, _P(_U64)]),
    "ssj_verify_batch_async": (_INT, [_VP, _P(ssj_batch), _VP, _U64, _VP, _VP]),
    "ssj_verify_batch_noalloc": (_INT, [_VP, _P(ssj_batch), _VP, _U64, _VP, _VP]),
    "ssj_reserve": (_INT, [_VP, _U32, _U64]),
    "ssj_multi_create": (_INT, [_VP, _P(ssj_batch), _U32, _P(_VP), _P(_U64), _VP, _P(_VP)]),
    "ssj_multi_launch": (_INT, [_VP, _VP, _VP]),
    "ssj_multi_graph_launch": (_INT, [_VP, _VP, _VP]),
    "ssj_multi_destroy": (None, [_VP, _VP]),
    "ssj_self_join": (_INT, [_VP, _U32, _U32, _U32, _U32, _VP, _U64, _P(_U64), _P(_U64)]),
    "ssj_verify_batches": (_INT, [_VP, _P(ssj_batch), _U32, _P(_VP), _P(_U64), _P(_U64)]),
    "ssj_multi_autotune": (_INT, [_VP, _VP, _VP, _U32, _P(ssj_tune_result)]),
    "ssj_read_bandwidth": (_INT, [_VP, _U64, _U32, _P(ctypes.c_double)]),
    "ssj_device_error": (_INT, [_VP, _P(_U32)]),
    "ssj_submit": (_INT, [_VP, _P(ssj_batch), _P(_U64)]),
    "ssj_poll": (_INT, [_VP, _U64, _INT, _P(_INT)]),
    "ssj_results": (_INT, [_VP, _U64, _VP, _U64, _P(_U64)]),
    "ssj_set_granularity": (_INT, [_VP, _U32, _U32, _U32, _U32]),
    "ssj_set_short_pairs": (_INT, [_VP, _U32]),
    "ssj_set_index_items": (_INT, [_VP, _U32]),
    "ssj_profile_read": (_INT, [_VP, _P(_U32), _P(ctypes.c_double), _P(ctypes.c_double)]),
    "ssj_serve_replay": (_INT, [_VP, _P(ssj_request), _U32, _P(ctypes.c_double), _P(ssj_serve_stats)]),
    "ssj_serve_coprocess": (_INT, [_VP, _U32, _VP, _VP, _U32, _U32, _U32, _U32, _U64, _P(ssj_coprocess_stats)]),
    "ssj_feeder_create": (_INT, [_VP, _VP, _U32, _U32, _U32, _U32, _P(_VP)]),
    "ssj_feeder_create_sim": (_INT, [_VP, _VP, _U32, _U32, _U32, _U32, _U32, _P(_VP)]),
    "ssj_feeder_create_ex": (_INT, [_VP, _VP, _U32, _VP, _VP, _U32, _P(ssj_feeder_opts), _P(_VP)]),
    "ssj_groups_create": (_INT, [_VP, _VP, _U32, _P(ssj_feeder_opts), _P(_VP)]),
    "ssj_groups_info": (_INT, [_VP, _P(_U32), _P(_U32), _P(_U64), _P(_U64)]),
    "ssj_groups_copy": (_INT, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ssj_groups_destroy": (None, [_VP]),
    "ssj_verify_groups": (_INT, [_VP, _P(ssj_group_batch), _VP, _U64, _P(_U64), _P(_U64)]),
    "ssj_feeder_next": (_INT, [_VP, _U32, _U64, _VP, _VP, _VP, _P(_U32), _P(_U64), _P(_INT)]),
    "ssj_feeder_progress": (_INT, [_VP, _P(_U64), _P(_U32), _P(_U32)]),
    "ssj_feeder_destroy": (None, [_VP]),
}

_lib = None


def lib():
    """The loaded libssj.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              f"or python paper_1812_09141_gb300/_build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# pointer marshalling
# --------------------------------------------------------------------------

def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, (a.ctypes.data if a.size else None)


def _devptr(x) -> int | None:
    """Device address of a torch CUDA tensor, or an integer address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor for a device pointer")
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _check(ctx, status: int):
    if status != SSJ_OK:
        msg = lib().ssj_last_error(ctx).decode() if ctx else ""
        raise SsjError(status, msg)


# --------------------------------------------------------------------------
# C functions with their C names (argument marshalling only)
# --------------------------------------------------------------------------

def ssj_create(device: int = 0, mem_budget_bytes: int = 0, max_inflight: int = 0, stream: int | None = None,
               flags: int = 0) -> int:
    cfg = ssj_config(device, mem_budget_bytes, max_inflight, stream, flags)
    out = ctypes.c_void_p()
    _check(None, lib().ssj_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def ssj_destroy(ctx: int) -> None:
    lib().ssj_destroy(ctx)


def ssj_last_error(ctx: int) -> str:
    return lib().ssj_last_error(ctx).decode()


def ssj_load_collection(ctx: int, offsets, tokens, flags: int = 0) -> int:
    offs, po = _host(offsets, np.uint64)
    toks, pt = _host(tokens, np.uint32)
    out = ctypes.c_uint32()
    _check(ctx, lib().ssj_load_collection(ctx, po, pt, len(offs) - 1, flags, ctypes.byref(out)))
    return out.value


def ssj_unload_collection(ctx: int, coll: int) -> None:
    _check(ctx, lib().ssj_unload_collection(ctx, coll))


def ssj_collection_info(ctx: int, coll: int) -> tuple[int, int]:
    n, t = ctypes.c_uint32(), ctypes.c_uint64()
    _check(ctx, lib().ssj_collection_info(ctx, coll, ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


@dataclass
class _HostBatch:
    batch: ssj_batch
    keep: tuple


def _make_batch(R, S, p, q, probe_ids, cand_offsets, cand_ids, flags, n_cands=None, n_probes=None) -> _HostBatch:
    if flags & SSJ_DEVICE_PTRS:
        if n_probes is None:
            if not hasattr(probe_ids, "numel"):
                raise ValueError("n_probes is required with raw device pointers")
            n_probes = int(probe_ids.numel())
        if n_cands is None:
            raise ValueError("n_cands is required with device pointers")
        b = ssj_batch(R, S, p, q, n_probes, _devptr(probe_ids), _devptr(cand_offsets), _devptr(cand_ids),
                      int(n_cands), flags)
        return _HostBatch(b, (probe_ids, cand_offsets, cand_ids))
    pr, pp = _host(probe_ids, np.uint32)
    co, pc = _host(cand_offsets, np.uint64)
    ci, pi = _host(cand_ids, np.uint32)
    b = ssj_batch(R, S, p, q, len(pr), pp, pc, pi, 0 if n_cands is None else int(n_cands), flags)
    return _HostBatch(b, (pr, co, ci))


def ssj_verify_batch(ctx: int, R: int, S: int, p: int, q: int, probe_ids, cand_offsets, cand_ids,
                     flags: int = 0, out=None, cap: int | None = None, n_cands: int | None = None,
                     n_probes: int | None = None):
    """Synchronous verification.  Host mode returns a structured array of triples (or the
    count with SSJ_COUNT_ONLY).  With SSJ_DEVICE_PTRS, `out` is a device tensor/pointer of
    `cap` triples and the count is returned."""
    hb = _make_batch(R, S, p, q, probe_ids, cand_offsets, cand_ids, flags, n_cands, n_probes)
    n_out = ctypes.c_uint64()
    if flags & SSJ_DEVICE_PTRS:
        _check(ctx, lib().ssj_verify_batch(ctx, ctypes.byref(hb.batch), _devptr(out), int(cap or 0),
                                           ctypes.byref(n_out)))
        return n_out.value
    if flags & SSJ_COUNT_ONLY:
        _check(ctx, lib().ssj_verify_batch(ctx, ctypes.byref(hb.batch), None, 0, ctypes.byref(n_out)))
        return n_out.value
    if cap is None:
        cap = int(hb.batch.n_cands) if hb.batch.n_cands else int(hb.keep[1][-1]) if len(hb.keep[1]) else 0
    res = np.empty(max(cap, 1), dtype=TRIPLE_DTYPE)
    st = lib().ssj_verify_batch(ctx, ctypes.byref(hb.batch), res.ctypes.data, cap, ctypes.byref(n_out))
    _check(ctx, st)
    return res[:n_out.value]


def ssj_self_join(ctx: int, coll: int, p: int, q: int, flags: int = 0, cap: int | None = None, out=None):
    """Self-join with device candidate generation.  Host mode: returns (structured triples,
    n_candidates), or (count, n_candidates) with SSJ_COUNT_ONLY.  With SSJ_DEVICE_PTRS, `out` is a
    device tensor/address of `cap` triples and (count, n_candidates) is returned."""
    n_out, n_c = ctypes.c_uint64(), ctypes.c_uint64()
    if flags & SSJ_COUNT_ONLY:
        _check(ctx, lib().ssj_self_join(ctx, coll, p, q, flags, None, 0, ctypes.byref(n_out), ctypes.byref(n_c)))
        return n_out.value, n_c.value
    if flags & SSJ_DEVICE_PTRS:
        _check(ctx, lib().ssj_self_join(ctx, coll, p, q, flags, _devptr(out), int(cap), ctypes.byref(n_out),
                                        ctypes.byref(n_c)))
        return n_out.value, n_c.value
    if cap is None:
        # ask for the count first (a COUNT_ONLY pass), then fetch
        cnt, _ = ssj_self_join(ctx, coll, p, q, flags | SSJ_COUNT_ONLY)
        cap = max(cnt, 1)
    res = np.empty(max(int(cap), 1), dtype=TRIPLE_DTYPE)
    _check(ctx, lib().ssj_self_join(ctx, coll, p, q, flags, res.ctypes.data, int(cap), ctypes.byref(n_out),
                                    ctypes.byref(n_c)))
    return res[:n_out.value], n_c.value


def ssj_verify_batches(ctx: int, batches: list, caps: list | None = None):
    """Several host batches in one call (one batched launch; a call of 2^25+ candidates over two or
    more batches runs two, the second group's inputs moving while the first group's kernels run,
    and its pinned inputs are read by the kernels directly).  batches: list of (R, S, p, q, probe_ids,
    cand_offsets, cand_ids, flags).  Returns a list with, per batch, its structured triples (or
    its count with SSJ_COUNT_ONLY)."""
    n = len(batches)
    hbs = [_make_batch(R, S, p, q, pr, co, ci, fl) for R, S, p, q, pr, co, ci, fl in batches]
    arr = (ssj_batch * max(n, 1))(*[h.batch for h in hbs])
    if caps is None:
        caps = [max(int(h.keep[1][-1]) if len(h.keep[1]) else 0, 1) for h in hbs]
    res = [np.empty(max(int(c), 1), dtype=TRIPLE_DTYPE) for c in caps]
    outp = (ctypes.c_void_p * max(n, 1))(*[r.ctypes.data for r in res])
    capa = (ctypes.c_uint64 * max(n, 1))(*[int(c) for c in caps])
    nout = (ctypes.c_uint64 * max(n, 1))()
    _check(ctx, lib().ssj_verify_batches(ctx, arr, n, outp, capa, nout))
    return [int(nout[i]) if batches[i][7] & SSJ_COUNT_ONLY else res[i][:nout[i]] for i in range(n)]


def ssj_verify_batch_async(ctx: int, R: int, S: int, p: int, q: int, probe_ids, cand_offsets, cand_ids, n_cands: int,
                           d_out, cap: int, d_count, stream: int | None = None, flags: int = 0,
                           n_probes: int | None = None) -> None:
    """Enqueue verification of device-resident inputs on `stream` (device pointers only)."""
    hb = _make_batch(R, S, p, q, probe_ids, cand_offsets, cand_ids, flags | SSJ_DEVICE_PTRS, n_cands, n_probes)
    _check(ctx, lib().ssj_verify_batch_async(ctx, ctypes.byref(hb.batch), _devptr(d_out), int(cap),
                                             _devptr(d_count), stream))


def ssj_verify_batch_noalloc(ctx: int, R: int, S: int, p: int, q: int, probe_ids, cand_offsets, cand_ids,
                             n_cands: int, d_out, cap: int, d_count, stream: int | None = None, flags: int = 0,
                             n_probes: int | None = None) -> None:
    """Like ssj_verify_batch_async, but the library allocates nothing: for callers that cannot let a
    library allocate device memory mid-call (own arena / caching allocator, or latency-critical paths
    where cudaMalloc would synchronise the device).  Uses the library's fixed 32 MiB scratch block;
    calls that overlap on the GPU share it and race."""
    hb = _make_batch(R, S, p, q, probe_ids, cand_offsets, cand_ids, flags | SSJ_DEVICE_PTRS, n_cands, n_probes)
    _check(ctx, lib().ssj_verify_batch_noalloc(ctx, ctypes.byref(hb.batch), _devptr(d_out), int(cap),
                                               _devptr(d_count), stream))


class DeviceBatch:
    """A batch whose arrays live on the device (torch CUDA tensors or raw addresses)."""

    def __init__(self, R: int, S: int, p: int, q: int, probe_ids, cand_offsets, cand_ids, n_cands: int,
                 flags: int = 0, n_probes: int | None = None):
        self._hb = _make_batch(R, S, p, q, probe_ids, cand_offsets, cand_ids, flags | SSJ_DEVICE_PTRS, n_cands,
                               n_probes)

    @property
    def batch(self) -> ssj_batch:
        return self._hb.batch


def ssj_multi_create(ctx: int, batches: list, outs: list, caps: list, d_counts) -> int:
    """Prepare one launch over several device batches (DeviceBatch objects).  outs[i]: device
    tensor (or address) for batch i's triples, caps[i] its capacity, d_counts: device int64
    tensor of len(batches)."""
    n = len(batches)
    arr = (ssj_batch * max(n, 1))(*[b.batch for b in batches])
    outp = (ctypes.c_void_p * max(n, 1))(*[_devptr(o) for o in outs])
    capa = (ctypes.c_uint64 * max(n, 1))(*[int(c) for c in caps])
    m = ctypes.c_void_p()
    _check(ctx, lib().ssj_multi_create(ctx, arr, n, outp, capa, _devptr(d_counts), ctypes.byref(m)))
    return m.value


def ssj_multi_launch(ctx: int, m: int, stream: int | None = None) -> None:
    _check(ctx, lib().ssj_multi_launch(ctx, m, stream))


def ssj_multi_graph_launch(ctx: int, m: int, stream: int | None = None) -> None:
    _check(ctx, lib().ssj_multi_graph_launch(ctx, m, stream))


def ssj_multi_destroy(ctx: int, m: int) -> None:
    lib().ssj_multi_destroy(ctx, m)


def ssj_multi_autotune(ctx: int, m: int, stream: int | None = None, reps: int = 5) -> dict:
    """Tune the granularity of a prepared launch; returns the chosen setting and timings."""
    r = ssj_tune_result()
    _check(ctx, lib().ssj_multi_autotune(ctx, m, stream, reps, ctypes.byref(r)))
    return {"thread_max_key": r.thread_max_key, "lane_max_key": r.lane_max_key, "warp_max_key": r.warp_max_key,
            "block_threads": r.block_threads, "drain_min_live": r.drain_min_live,
            "index_min_cands": r.index_min_cands, "settings_tried": r.settings_tried,
            "best_ms": r.best_ms, "initial_ms": r.initial_ms}


def ssj_read_bandwidth(ctx: int, nbytes: int, passes: int = 20) -> float:
    """Device read bandwidth (GB/s) over a buffer of nbytes (see ssj.h)."""
    g = ctypes.c_double()
    _check(ctx, lib().ssj_read_bandwidth(ctx, nbytes, passes, ctypes.byref(g)))
    return g.value


def ssj_reserve(ctx: int, n_probes: int, n_cands: int) -> None:
    _check(ctx, lib().ssj_reserve(ctx, n_probes, n_cands))


def ssj_device_error(ctx: int) -> int:
    code = ctypes.c_uint32()
    _check(ctx, lib().ssj_device_error(ctx, ctypes.byref(code)))
    return code.value


def ssj_submit(ctx: int, R: int, S: int, p: int, q: int, probe_ids, cand_offsets, cand_ids, flags: int = 0,
               n_cands: int | None = None, n_probes: int | None = None) -> int | None:
    """Admit a batch; returns its ticket, or None when the call answered SSJ_EAGAIN."""
    hb = _make_batch(R, S, p, q, probe_ids, cand_offsets, cand_ids, flags, n_cands, n_probes)
    t = ctypes.c_uint64()
    st = lib().ssj_submit(ctx, ctypes.byref(hb.batch), ctypes.byref(t))
    if st == SSJ_EAGAIN:
        return None
    _check(ctx, st)
    return t.value


def ssj_poll(ctx: int, ticket: int, timeout_ms: int = 0) -> bool:
    done = ctypes.c_int()
    st = lib().ssj_poll(ctx, ticket, timeout_ms, ctypes.byref(done))
    if st == SSJ_ETIMEDOUT:
        return False
    _check(ctx, st)
    return bool(done.value)


def ssj_results(ctx: int, ticket: int, count_only: bool = False):
    """Collect a finished ticket: structured triples (or the count if count_only)."""
    n = ctypes.c_uint64()
    _check(ctx, lib().ssj_results(ctx, ticket, None, 0, ctypes.byref(n)))
    if count_only:
        dummy = np.empty(1, dtype=TRIPLE_DTYPE)
        _check(ctx, lib().ssj_results(ctx, ticket, dummy.ctypes.data, 0, ctypes.byref(n)))
        return n.value
    res = np.empty(max(n.value, 1), dtype=TRIPLE_DTYPE)
    _check(ctx, lib().ssj_results(ctx, ticket, res.ctypes.data, n.value, ctypes.byref(n)))
    return res[:n.value]


def ssj_set_granularity(ctx: int, thread_max_key: int = 0, lane_max_key: int = 0, warp_max_key: int = 0,
                        block_threads: int = 0) -> None:
    _check(ctx, lib().ssj_set_granularity(ctx, thread_max_key, lane_max_key, warp_max_key, block_threads))


def ssj_set_index_items(ctx: int, min_cands: int) -> None:
    """Probes with at least min_cands candidates become index items (0: none)."""
    _check(ctx, lib().ssj_set_index_items(ctx, min_cands))


def ssj_set_short_pairs(ctx: int, drain_min_live: int = 0) -> None:
    """Short-pair refill threshold of later launches: 1..24, or 0 (the default, 16)."""
    _check(ctx, lib().ssj_set_short_pairs(ctx, drain_min_live))


def ssj_profile_read(ctx: int) -> tuple[int, float, float]:
    """(launches, plan kernel ms, verify kernel ms) since the last read (SSJ_CTX_PROFILE contexts)."""
    n, a, b = ctypes.c_uint32(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().ssj_profile_read(ctx, ctypes.byref(n), ctypes.byref(a), ctypes.byref(b)))
    return n.value, a.value, b.value


# serving drivers -------------------------------------------------------------

def ssj_serve_replay(ctx: int, requests: list) -> tuple[np.ndarray, dict]:
    """Open-loop replay.  requests: list of (R, S, p, q, probe_ids, cand_offsets, cand_ids,
    arrival_s, flags) with host arrays.  Returns (latency_s per request, stats dict)."""
    n = len(requests)
    arr = (ssj_request * max(n, 1))()
    keep = []
    for i, (R, S, p, q, pr, co, ci, t, fl) in enumerate(requests):
        hb = _make_batch(R, S, p, q, pr, co, ci, fl)
        keep.append(hb)
        arr[i].batch = hb.batch
        arr[i].arrival_s = float(t)
    lat = np.zeros(max(n, 1), dtype=np.float64)
    st = ssj_serve_stats()
    _check(ctx, lib().ssj_serve_replay(ctx, arr, n, lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(st)))
    return lat[:n], {"wall_s": st.wall_s, "pairs": st.pairs, "results": st.results, "eagain": st.eagain,
                     "max_inflight": st.max_inflight}


def ssj_serve_coprocess(ctx: int, coll: int, offsets, tokens, p: int, q: int, n_threads: int,
                        chunk_cands: int) -> dict:
    offs, po = _host(offsets, np.uint64)
    toks, pt = _host(tokens, np.uint32)
    st = ssj_coprocess_stats()
    _check(ctx, lib().ssj_serve_coprocess(ctx, coll, po, pt, len(offs) - 1, p, q, n_threads, chunk_cands,
                                          ctypes.byref(st)))
    return {"filter_only_s": st.filter_only_s, "join_s": st.join_s, "gpu_busy_s": st.gpu_busy_s,
            "candidates": st.candidates, "results": st.results, "chunks": st.chunks}


# feeder --------------------------------------------------------------------

def ssj_feeder_create(offsets, tokens, p: int, q: int, n_threads: int = 1) -> int:
    offs, po = _host(offsets, np.uint64)
    toks, pt = _host(tokens, np.uint32)
    out = ctypes.c_void_p()
    _check(None, lib().ssj_feeder_create(po, pt, len(offs) - 1, p, q, n_threads, ctypes.byref(out)))
    return out.value


def ssj_feeder_create_sim(offsets, tokens, sim: int, p: int, q: int, n_threads: int = 1) -> int:
    """sim: 0 Jaccard, 1 Dice, 2 Cosine, 3 plain overlap (SSJ_SIM_* >> 8)."""
    offs, po = _host(offsets, np.uint64)
    toks, pt = _host(tokens, np.uint32)
    out = ctypes.c_void_p()
    _check(None, lib().ssj_feeder_create_sim(po, pt, len(offs) - 1, sim, p, q, n_threads, ctypes.byref(out)))
    return out.value


def ssj_feeder_next(f: int, max_probes: int, max_cands: int):
    """Next chunk as (probe_ids, cand_offsets, cand_ids, done)."""
    pr = np.empty(max_probes, dtype=np.uint32)
    co = np.empty(max_probes + 1, dtype=np.uint64)
    ci = np.empty(max(max_cands, 1), dtype=np.uint32)
    npb, nc, done = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_int()
    _check(None, lib().ssj_feeder_next(f, max_probes, max_cands, pr.ctypes.data, co.ctypes.data, ci.ctypes.data,
                                       ctypes.byref(npb), ctypes.byref(nc), ctypes.byref(done)))
    k = npb.value
    return pr[:k], co[:k + 1], ci[:nc.value], bool(done.value)


def ssj_feeder_progress(f: int) -> tuple[int, int, int]:
    nc, probed, n = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(None, lib().ssj_feeder_progress(f, ctypes.byref(nc), ctypes.byref(probed), ctypes.byref(n)))
    return nc.value, probed.value, n.value


def ssj_feeder_destroy(f: int) -> None:
    lib().ssj_feeder_destroy(f)


def ssj_feeder_create_ex(r_offsets, r_tokens, s_offsets=None, s_tokens=None, sim: int = 0, p: int = 1,
                         q: int = 1, flags: int = 0, n_threads: int = 1) -> int:
    """Self-join of R (s_offsets None) or R x S join feeder; flags: SSJ_FEEDER_PPJOIN."""
    ro, rpo = _host(r_offsets, np.uint64)
    rt, rpt = _host(r_tokens, np.uint32)
    n_s, spo, spt = 0, None, None
    if s_offsets is not None:
        so, spo = _host(s_offsets, np.uint64)
        st, spt = _host(s_tokens, np.uint32)
        n_s = len(so) - 1
    o = ssj_feeder_opts(sim, p, q, flags, n_threads)
    out = ctypes.c_void_p()
    _check(None, lib().ssj_feeder_create_ex(rpo, rpt, len(ro) - 1, spo, spt, n_s, ctypes.byref(o),
                                            ctypes.byref(out)))
    return out.value


def feeder_all(offsets, tokens, p: int, q: int, n_threads: int = 1, chunk: int = 1 << 22, sim: int = 0,
               s_offsets=None, s_tokens=None, flags: int = 0):
    """Run the feeder to completion; returns one concatenated batch (probe_ids, offsets, cands).
    sim selects the similarity function (SSJ_SIM_* >> 8; Jaccard by default); s_offsets /
    s_tokens make it an R x S join of (offsets, tokens) against them; flags: SSJ_FEEDER_PPJOIN."""
    if s_offsets is None and flags == 0:
        f = (ssj_feeder_create(offsets, tokens, p, q, n_threads) if sim == 0 else
             ssj_feeder_create_sim(offsets, tokens, sim, p, q, n_threads))
    else:
        f = ssj_feeder_create_ex(offsets, tokens, s_offsets, s_tokens, sim, p, q, flags, n_threads)
    try:
        probes, offs, cands = [], [np.zeros(1, dtype=np.uint64)], []
        base = 0
        n_sets = len(offsets) - 1
        while True:
            pr, co, ci, done = ssj_feeder_next(f, max(n_sets, 1), chunk)
            probes.append(pr)
            offs.append(co[1:] + base)
            cands.append(ci)
            base += len(ci)
            if done:
                break
        return (np.concatenate(probes).astype(np.uint32), np.concatenate(offs).astype(np.uint64),
                np.concatenate(cands).astype(np.uint32))
    finally:
        ssj_feeder_destroy(f)


def triples_to_array(t) -> np.ndarray:
    """Structured triples -> (k, 3) uint32, sorted by (r, s)."""
    a = np.stack([t["r"], t["s"], t["overlap"]], axis=1).astype(np.uint32) if len(t) else np.zeros((0, 3), np.uint32)
    if len(a):
        a = a[np.lexsort((a[:, 1], a[:, 0]))]
    return a


# GroupJoin -----------------------------------------------------------------

class Groups:
    """GroupJoin candidates: group_offsets, members, probe_groups, cand_offsets, cand_groups (numpy),
    and n_pairs, the member pairs they stand for."""

    def __init__(self, group_offsets, members, probe_groups, cand_offsets, cand_groups, n_pairs):
        self.group_offsets, self.members = group_offsets, members
        self.probe_groups, self.cand_offsets, self.cand_groups = probe_groups, cand_offsets, cand_groups
        self.n_pairs = n_pairs


def group_candidates(offsets, tokens, p: int, q: int, sim: int = 0) -> Groups:
    """Run ssj_groups_create and copy the groups out."""
    offs, po = _host(offsets, np.uint64)
    toks, pt = _host(tokens, np.uint32)
    o = ssj_feeder_opts(sim, p, q, 0, 1)
    h = ctypes.c_void_p()
    _check(None, lib().ssj_groups_create(po, pt, len(offs) - 1, ctypes.byref(o), ctypes.byref(h)))
    try:
        ng, npg = ctypes.c_uint32(), ctypes.c_uint32()
        ncg, npairs = ctypes.c_uint64(), ctypes.c_uint64()
        _check(None, lib().ssj_groups_info(h, ctypes.byref(ng), ctypes.byref(npg), ctypes.byref(ncg),
                                           ctypes.byref(npairs)))
        go = np.zeros(ng.value + 1, dtype=np.uint64)
        mem = np.zeros(max(len(offs) - 1, 1), dtype=np.uint32)
        pg = np.zeros(max(npg.value, 1), dtype=np.uint32)
        co = np.zeros(npg.value + 1, dtype=np.uint64)
        cg = np.zeros(max(ncg.value, 1), dtype=np.uint32)
        _check(None, lib().ssj_groups_copy(h, go.ctypes.data, mem.ctypes.data, pg.ctypes.data, co.ctypes.data,
                                           cg.ctypes.data))
        return Groups(go, mem[:len(offs) - 1], pg[:npg.value], co, cg[:ncg.value], npairs.value)
    finally:
        lib().ssj_groups_destroy(h)


def ssj_verify_groups(ctx: int, coll: int, p: int, q: int, g: Groups, flags: int = 0, cap: int | None = None):
    """Expand and verify GroupJoin candidates on the device.  Returns (structured triples, n_pairs),
    or (count, n_pairs) with SSJ_COUNT_ONLY."""
    keep = [np.ascontiguousarray(a, dtype=t) for a, t in ((g.group_offsets, np.uint64), (g.members, np.uint32),
                                                            (g.probe_groups, np.uint32), (g.cand_offsets, np.uint64),
                                                            (g.cand_groups, np.uint32))]
    ptr = [a.ctypes.data if a.size else None for a in keep]
    gb = ssj_group_batch(coll, p, q, flags, len(keep[0]) - 1, ptr[0], ptr[1], len(keep[2]), ptr[2], ptr[3], ptr[4])
    n_out, n_pairs = ctypes.c_uint64(), ctypes.c_uint64()
    if flags & SSJ_COUNT_ONLY:
        _check(ctx, lib().ssj_verify_groups(ctx, ctypes.byref(gb), None, 0, ctypes.byref(n_out), ctypes.byref(n_pairs)))
        return n_out.value, n_pairs.value
    cap = g.n_pairs if cap is None else cap
    res = np.empty(max(int(cap), 1), dtype=TRIPLE_DTYPE)
    _check(ctx, lib().ssj_verify_groups(ctx, ctypes.byref(gb), res.ctypes.data, int(cap), ctypes.byref(n_out),
                                        ctypes.byref(n_pairs)))
    return res[:n_out.value], n_pairs.value

