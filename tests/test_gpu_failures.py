"""Failure paths of the serving and batch API, made on the host (no GPU fault, trap or hang):
busy collections, full slots, a batch over the memory budget, unknown tickets, a result buffer
too small, a poll that times out, malformed batches and a context that outlives its faults."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def coll():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    spec = synth.tiny_self_join(seed=1001, n=600)
    spec.plant_frac, spec.plant_edits = 0.2, 2
    return synth.collection(spec)


def test_unload_while_a_ticket_is_uncollected_is_busy(coll):
    ctx = ssj.ssj_create(0, max_inflight=2)
    try:
        h = ssj.ssj_load_collection(ctx, coll.offsets, coll.tokens)
        b = synth.all_pairs_batch(coll.n)
        t = ssj.ssj_submit(ctx, h, h, 4, 5, b.probe_ids, b.cand_offsets, b.cand_ids)
        assert t is not None
        assert ssj.ssj_poll(ctx, t, -1)  # finished on the GPU, but not collected yet
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_unload_collection(ctx, h)
        assert ei.value.status == ssj.SSJ_EBUSY
        got = ssj.triples_to_array(ssj.ssj_results(ctx, t))
        assert np.array_equal(got, oracle.sort_triples(oracle.bruteforce_self(coll.offsets, coll.tokens, 4, 5)))
        ssj.ssj_unload_collection(ctx, h)  # free once collected
    finally:
        ssj.ssj_destroy(ctx)


def test_full_slots_answer_eagain_until_a_ticket_is_collected(coll):
    ctx = ssj.ssj_create(0, max_inflight=2)
    try:
        h = ssj.ssj_load_collection(ctx, coll.offsets, coll.tokens)
        b = synth.all_pairs_batch(coll.n)
        args = (h, h, 4, 5, b.probe_ids, b.cand_offsets, b.cand_ids)
        t1, t2 = ssj.ssj_submit(ctx, *args), ssj.ssj_submit(ctx, *args)
        assert t1 is not None and t2 is not None
        assert ssj.ssj_submit(ctx, *args) is None  # SSJ_EAGAIN: both slots hold uncollected tickets
        assert ssj.ssj_poll(ctx, t1, -1)
        r1 = ssj.ssj_results(ctx, t1)
        t3 = ssj.ssj_submit(ctx, *args)  # a slot is free again
        assert t3 is not None
        for t in (t2, t3):
            assert ssj.ssj_poll(ctx, t, -1)
            assert np.array_equal(ssj.triples_to_array(ssj.ssj_results(ctx, t)), ssj.triples_to_array(r1))
    finally:
        ssj.ssj_destroy(ctx)


def test_batch_over_the_budget_unknown_ticket_and_small_buffer(coll):
    ctx = ssj.ssj_create(0, mem_budget_bytes=1 << 20, max_inflight=2)
    try:
        h = ssj.ssj_load_collection(ctx, coll.offsets, coll.tokens)
        big = synth.all_pairs_batch(coll.n)  # ~180k pairs: its device inputs exceed 1 MiB
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_submit(ctx, h, h, 4, 5, big.probe_ids, big.cand_offsets, big.cand_ids)
        assert ei.value.status == ssj.SSJ_EINVAL
        done = ctypes.c_int()
        assert ssj.lib().ssj_poll(ctx, 987654321, 0, ctypes.byref(done)) == ssj.SSJ_ENOTFOUND
        # a small batch fits; collecting it into a buffer that is too small answers SSJ_ENOMEM
        # with the count needed, and the ticket stays collectable
        probes = np.arange(0, 40, dtype=np.uint32)
        offs = np.arange(0, 41, dtype=np.uint64) * 20
        cands = np.concatenate([np.arange(i + 1, i + 21) % coll.n for i in range(40)]).astype(np.uint32)
        t = ssj.ssj_submit(ctx, h, h, 1, 5, probes, offs, cands)
        assert t is not None and ssj.ssj_poll(ctx, t, -1)
        n = ctypes.c_uint64()
        assert ssj.lib().ssj_results(ctx, t, None, 0, ctypes.byref(n)) == ssj.SSJ_OK
        want = oracle.sort_triples(oracle.verify_batch(coll.offsets, coll.tokens, coll.offsets, coll.tokens, True,
                                                       1, 5, probes, offs, cands))
        assert n.value == len(want) and n.value >= 2
        small = np.empty(1, dtype=ssj.TRIPLE_DTYPE)
        assert ssj.lib().ssj_results(ctx, t, small.ctypes.data, 1, ctypes.byref(n)) == ssj.SSJ_ENOMEM
        assert n.value == len(want)
        got = ssj.triples_to_array(ssj.ssj_results(ctx, t))
        assert np.array_equal(got, want)
    finally:
        ssj.ssj_destroy(ctx)


def test_poll_timeout_is_not_destructive(coll):
    """A zero-timeout poll right after submitting a large batch answers either 'not yet'
    (SSJ_ETIMEDOUT) or 'done'; either way a waiting poll then completes it with the right join."""
    ctx = ssj.ssj_create(0, max_inflight=2)
    try:
        spec = synth.long_sets(n=3000)
        c = synth.collection(spec)
        h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
        pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, 3, 5, n_threads=4)
        t = ssj.ssj_submit(ctx, h, h, 3, 5, pr, co, ci)
        done = ctypes.c_int(7)
        st = ssj.lib().ssj_poll(ctx, t, 0, ctypes.byref(done))
        assert (st, done.value) in ((ssj.SSJ_ETIMEDOUT, 0), (ssj.SSJ_OK, 1))
        assert ssj.ssj_poll(ctx, t, -1)
        got = ssj.triples_to_array(ssj.ssj_results(ctx, t))
        assert np.array_equal(got, oracle.sort_triples(oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens,
                                                                           True, 3, 5, pr, co, ci)))
    finally:
        ssj.ssj_destroy(ctx)


def test_context_survives_rejected_batches(coll):
    """Malformed batches (ids out of range, bad offsets, bad thresholds) are rejected with a status,
    and the same context then verifies a valid batch correctly."""
    ctx = ssj.ssj_create(0, max_inflight=2)
    try:
        h = ssj.ssj_load_collection(ctx, coll.offsets, coll.tokens)
        b = synth.all_pairs_batch(coll.n)
        bad_ids = b.cand_ids.copy()
        bad_ids[len(bad_ids) // 2] = coll.n + 5
        bad_offs = b.cand_offsets.copy()
        bad_offs[3] = bad_offs[5] + 1
        for args in ((4, 5, b.probe_ids, b.cand_offsets, bad_ids), (4, 5, b.probe_ids, bad_offs, b.cand_ids),
                     (6, 5, b.probe_ids, b.cand_offsets, b.cand_ids), (0, 5, b.probe_ids, b.cand_offsets, b.cand_ids)):
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_verify_batch(ctx, h, h, *args)
            assert ei.value.status == ssj.SSJ_EINVAL
        got = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, 4, 5, b.probe_ids, b.cand_offsets, b.cand_ids))
        want = oracle.sort_triples(oracle.bruteforce_self(coll.offsets, coll.tokens, 4, 5))
        assert np.array_equal(got, want)
        # the same through serving: the failed ticket reports SSJ_EINVAL and frees its slot
        for _ in range(3):
            t = ssj.ssj_submit(ctx, h, h, 4, 5, b.probe_ids, b.cand_offsets, bad_ids)
            assert t is not None
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_poll(ctx, t, -1)
            assert ei.value.status == ssj.SSJ_EINVAL
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_results(ctx, t)
            assert ei.value.status == ssj.SSJ_EINVAL
        t = ssj.ssj_submit(ctx, h, h, 4, 5, b.probe_ids, b.cand_offsets, b.cand_ids)
        assert ssj.ssj_poll(ctx, t, -1)
        assert np.array_equal(ssj.triples_to_array(ssj.ssj_results(ctx, t)), want)
    finally:
        ssj.ssj_destroy(ctx)


def test_misaligned_arrays_never_reach_the_kernels(coll):
    """The kernels load ids as 4-byte and offsets and counts as 8-byte words and store triples
    field by field.  Device arrays off that alignment are refused with SSJ_EINVAL before any
    launch, on every entry point that takes them; pinned host arrays off it are copied instead
    of read over the host link, and give the oracle's results.  The context keeps working."""
    import torch
    dev = torch.device("cuda:0")
    ctx = ssj.ssj_create(0)
    try:
        h = ssj.ssj_load_collection(ctx, coll.offsets, coll.tokens)
        b = synth.all_pairs_batch(coll.n)
        want = oracle.sort_triples(oracle.bruteforce_self(coll.offsets, coll.tokens, 4, 5))
        assert len(want) > 0
        # device arrays with room for a shifted copy; each shifted address is off its alignment
        pr = torch.zeros(b.n_probes + 4, dtype=torch.int32, device=dev)
        co = torch.zeros(b.n_probes + 3, dtype=torch.int64, device=dev)
        ci = torch.zeros(b.n_cands + 4, dtype=torch.int32, device=dev)
        out = torch.zeros(3 * len(want) + 8, dtype=torch.int32, device=dev)
        cnt = torch.zeros(4, dtype=torch.int64, device=dev)
        pr[:b.n_probes] = torch.from_numpy(b.probe_ids.astype(np.int32)).to(dev)
        co[:b.n_probes + 1] = torch.from_numpy(b.cand_offsets.astype(np.int64)).to(dev)
        ci[:b.n_cands] = torch.from_numpy(b.cand_ids.astype(np.int32)).to(dev)
        torch.cuda.synchronize()
        good = (pr.data_ptr(), co.data_ptr(), ci.data_ptr())
        cap = len(want)
        for k, shift in ((0, 2), (1, 4), (2, 2)):
            arrays = list(good)
            arrays[k] += shift
            args = (h, h, 4, 5, *arrays)
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_verify_batch(ctx, *args, flags=ssj.SSJ_DEVICE_PTRS, out=out, cap=cap,
                                     n_cands=b.n_cands, n_probes=b.n_probes)
            assert ei.value.status == ssj.SSJ_EINVAL, k
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_verify_batch_async(ctx, *args, b.n_cands, out, cap, cnt, n_probes=b.n_probes)
            assert ei.value.status == ssj.SSJ_EINVAL, k
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_multi_create(ctx, [ssj.DeviceBatch(*args, b.n_cands, n_probes=b.n_probes)], [out],
                                     [cap], cnt)
            assert ei.value.status == ssj.SSJ_EINVAL, k
        # an output off 4 bytes, a count off 8
        for o, c in ((out.data_ptr() + 2, cnt), (out, cnt.data_ptr() + 4)):
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_verify_batch_async(ctx, h, h, 4, 5, *good, b.n_cands, o, cap, c, n_probes=b.n_probes)
            assert ei.value.status == ssj.SSJ_EINVAL
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_self_join(ctx, h, 4, 5, flags=ssj.SSJ_DEVICE_PTRS, out=out.data_ptr() + 2, cap=cap)
        assert ei.value.status == ssj.SSJ_EINVAL
        # the aligned arrays work on the same context
        n = ssj.ssj_verify_batch(ctx, h, h, 4, 5, *good, flags=ssj.SSJ_DEVICE_PTRS, out=out, cap=cap,
                                 n_cands=b.n_cands, n_probes=b.n_probes)
        got = out[:3 * n].view(-1, 3).cpu().numpy().astype(np.uint32)
        assert np.array_equal(oracle.sort_triples(got), want)

        # pinned host arrays off their alignment, with the kernels asked to read pinned inputs
        # directly: they are copied, and the results are exact
        def pinned_off(a, mod, rem):
            a = np.ascontiguousarray(a)
            buf = torch.empty(a.nbytes + 64, dtype=torch.uint8).pin_memory().numpy()
            shift = (rem - buf.ctypes.data) % mod
            v = buf[shift:shift + a.nbytes].view(a.dtype)
            v[...] = a
            assert v.ctypes.data % mod == rem
            assert np.ascontiguousarray(v, dtype=a.dtype).ctypes.data == v.ctypes.data  # passed as is
            return v
        hp = pinned_off(b.probe_ids.astype(np.uint32), 4, 2)
        ho = pinned_off(b.cand_offsets.astype(np.uint64), 8, 4)
        hc = pinned_off(b.cand_ids.astype(np.uint32), 4, 2)
        res = ssj.ssj_verify_batches(ctx, [(h, h, 4, 5, hp, ho, hc, ssj.SSJ_HOST_DIRECT)], caps=[cap + 16])
        assert np.array_equal(ssj.triples_to_array(res[0]), want)
        assert ssj.ssj_device_error(ctx) == 0
    finally:
        ssj.ssj_destroy(ctx)


def test_sizes_beyond_the_size_arithmetic_are_refused(coll):
    """A batch of 2^31 or more probes, a collection of 2^31 or more sets and a batch of 2^40 or
    more candidates are refused before any memory is sized from them (the n + 1 offsets and
    32-probe tiles stay within 32 bits, the workspace sizes far from 64-bit wrap); the context
    keeps working."""
    ctx = ssj.ssj_create(0)
    try:
        h = ssj.ssj_load_collection(ctx, coll.offsets, coll.tokens)
        one = np.zeros(4, dtype=np.uint64)
        b = ssj.ssj_batch(h, h, 4, 5, 1 << 31, one.ctypes.data, one.ctypes.data, one.ctypes.data, 0, 0)
        n_out = ctypes.c_uint64()
        assert ssj.lib().ssj_verify_batch(ctx, ctypes.byref(b), None, 0, ctypes.byref(n_out)) == ssj.SSJ_EINVAL
        assert "2^31" in ssj.ssj_last_error(ctx)
        handle = ctypes.c_uint32()
        assert ssj.lib().ssj_load_collection(ctx, one.ctypes.data, one.ctypes.data, 1 << 31, 0,
                                             ctypes.byref(handle)) == ssj.SSJ_EINVAL
        # 2^40 candidates: as the count of a device batch, and as the last host offset
        b = ssj.ssj_batch(h, h, 4, 5, 1, one.ctypes.data, one.ctypes.data, one.ctypes.data, 1 << 40,
                          ssj.SSJ_DEVICE_PTRS | ssj.SSJ_COUNT_ONLY)
        assert ssj.lib().ssj_verify_batch(ctx, ctypes.byref(b), None, 0, ctypes.byref(n_out)) == ssj.SSJ_EINVAL
        assert "2^40" in ssj.ssj_last_error(ctx)
        assert ssj.lib().ssj_reserve(ctx, 16, 1 << 40) == ssj.SSJ_EINVAL
        assert ssj.lib().ssj_reserve(ctx, 1 << 31, 16) == ssj.SSJ_EINVAL
        offs = np.array([0, 1 << 40], dtype=np.uint64)
        b = ssj.ssj_batch(h, h, 4, 5, 1, one.ctypes.data, offs.ctypes.data, one.ctypes.data, 0, ssj.SSJ_COUNT_ONLY)
        assert ssj.lib().ssj_verify_batch(ctx, ctypes.byref(b), None, 0, ctypes.byref(n_out)) == ssj.SSJ_EINVAL
        assert "2^40" in ssj.ssj_last_error(ctx)
        b = synth.all_pairs_batch(coll.n)
        got = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, 4, 5, b.probe_ids, b.cand_offsets, b.cand_ids))
        assert np.array_equal(got, oracle.sort_triples(oracle.bruteforce_self(coll.offsets, coll.tokens, 4, 5)))
    finally:
        ssj.ssj_destroy(ctx)
