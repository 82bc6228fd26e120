"""The scratch-free entry point (ssj_verify_batch_noalloc) against ssj_verify_batch.

Some callers cannot let a library allocate device memory during a call (their
memory all goes through an arena or a caching allocator, or cudaMalloc's
device synchronisation is unacceptable on their path).  This file checks that
the variant serving them returns exactly what the allocating entry point
returns, on two calls in a row that reuse the same static scratch block, on
an explicit stream and on the context's own stream (stream NULL), and that
those calls leave the device's free memory unchanged.  It is named to be
collected last and works alone in a fresh process too.
"""
import numpy as np
import pytest

import synth

import paper_1812_09141_gb300 as ssj
from paper_1812_09141_gb300 import _build

pytestmark = pytest.mark.gpu


def _device_batch(b, dev):
    import torch
    pr = torch.from_numpy(b.probe_ids.astype(np.int32)).to(dev)
    co = torch.from_numpy(b.cand_offsets.astype(np.int64)).to(dev)
    ci = torch.from_numpy(b.cand_ids.astype(np.int32)).to(dev)
    return pr, co, ci


def _triples(out, n):
    return ssj.triples_to_array(np.frombuffer(out[:3 * n].cpu().numpy().astype(np.uint32).tobytes(),
                                              dtype=ssj.TRIPLE_DTYPE))


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    _build.build()
    dev = torch.device("cuda:0")
    ctx = ssj.ssj_create(0)
    try:
        spec = synth.tiny_self_join(n=700)
        spec.plant_frac, spec.plant_edits = 0.2, 2
        c1 = synth.collection(spec)
        spec2 = synth.short_sets(n=20_000)
        spec2.plant_frac, spec2.plant_edits = 0.2, 2
        c2 = synth.collection(spec2)
        h1 = ssj.ssj_load_collection(ctx, c1.offsets, c1.tokens, ssj.SSJ_VALIDATE)
        h2 = ssj.ssj_load_collection(ctx, c2.offsets, c2.tokens, ssj.SSJ_VALIDATE)
        pr, co, ci = ssj.feeder_all(c2.offsets, c2.tokens, 3, 5, n_threads=4)
        cases = [(h1, (1, 2), synth.all_pairs_batch(c1.n)), (h2, (3, 5), synth.Batch(pr, co, ci))]
        stream = torch.cuda.Stream()
        prepared = []
        for h, (p, q), b in cases:
            want = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, p, q, b.probe_ids, b.cand_offsets,
                                                             b.cand_ids))
            assert len(want) > 0
            t_pr, t_co, t_ci = _device_batch(b, dev)
            cap = len(want) + 16
            out = torch.zeros(cap * 3, dtype=torch.int32, device=dev)
            cnt = torch.zeros(1, dtype=torch.int64, device=dev)
            prepared.append((h, p, q, b, want, t_pr, t_co, t_ci, cap, out, cnt))
        # the first call on the device may load the library's device code (and with it
        # the static scratch block); the free-memory check starts after it
        h, p, q, b, want, t_pr, t_co, t_ci, cap, out, cnt = prepared[0]
        ssj.ssj_verify_batch_noalloc(ctx, h, h, p, q, t_pr, t_co, t_ci, b.n_cands, out, cap, cnt)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(dev)
        for use_ctx_stream in (False, True):
            for h, p, q, b, want, t_pr, t_co, t_ci, cap, out, cnt in prepared:
                out.zero_()
                cnt.zero_()
                torch.cuda.synchronize()
                if use_ctx_stream:
                    # stream NULL: the context's own stream, which ssj_device_error reads on
                    ssj.ssj_verify_batch_noalloc(ctx, h, h, p, q, t_pr, t_co, t_ci, b.n_cands, out, cap, cnt)
                    assert ssj.ssj_device_error(ctx) == 0
                    torch.cuda.synchronize()
                else:
                    with torch.cuda.stream(stream):
                        ssj.ssj_verify_batch_noalloc(ctx, h, h, p, q, t_pr, t_co, t_ci, b.n_cands, out, cap, cnt,
                                                     stream=stream.cuda_stream)
                    stream.synchronize()
                    assert ssj.ssj_device_error(ctx) == 0
                n = int(cnt.item())
                assert np.array_equal(_triples(out, n), want)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(dev)
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across the calls"
        # a batch whose work queue exceeds the static block is refused before any launch
        t_pr, t_co, t_ci = _device_batch(cases[0][2], dev)
        with pytest.raises(ssj.SsjError) as ei:
            ssj.ssj_verify_batch_noalloc(ctx, h1, h1, 1, 2, t_pr, t_co, t_ci, 10 ** 9, None, 0,
                                         torch.zeros(1, dtype=torch.int64, device=dev), flags=ssj.SSJ_COUNT_ONLY)
        assert ei.value.status == ssj.SSJ_EINVAL
        # so is a device array off its element alignment (offsets 8 bytes, the count 8, the rest 4)
        h, p, q, b, want, t_pr, t_co, t_ci, cap, out, cnt = prepared[0]
        for args in ((t_pr, t_co.data_ptr() + 4, t_ci, out, cnt), (t_pr.data_ptr() + 2, t_co, t_ci, out, cnt),
                     (t_pr, t_co, t_ci, out.data_ptr() + 2, cnt), (t_pr, t_co, t_ci, out, cnt.data_ptr() + 4)):
            with pytest.raises(ssj.SsjError) as ei:
                ssj.ssj_verify_batch_noalloc(ctx, h, h, p, q, *args[:3], b.n_cands, args[3], cap, args[4],
                                             n_probes=b.n_probes)
            assert ei.value.status == ssj.SSJ_EINVAL
    finally:
        ssj.ssj_destroy(ctx)
