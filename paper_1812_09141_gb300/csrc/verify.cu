// Verification kernels for sm_103a.
//
// What is computed (Section 3.1 and Table "Similarity Functions"): for every
// listed candidate pair (r, s), the overlap o = |r n s| of the two sorted
// token sets by merging, stopping early once o + min(|r|-i, |s|-j) falls
// below the required overlap (positional filter, Section 2.2.3), and the
// pair is kept iff o*(p+q) >= p*(|r|+|s|) (Jaccard t = p/q).
//
// How the work is laid out (the paper's Alternatives A-C of Section 3.3.2,
// re-designed for one GB300):
//   * plan_kernel, one thread per probe: validates the grouped candidate
//     list, records for every 32-candidate chunk which probe owns its first
//     candidate, and emits block work items for probes whose sets are long.
//   * verify_kernel, persistent (one wave of CTAs over the 152 SMs):
//       phase 1 - block items: one CTA per pair, Intersect Path across the
//                 whole CTA (Alternative C, Section 4.2.2-4.2.3);
//       phase 2 - a flat pass over the candidate stream in 32-candidate
//                 chunks: each lane resolves its probe with a shuffle
//                 search, short pairs are merged one per thread
//                 (Alternative A/B), medium pairs by the whole warp with a
//                 32-lane merge path.
//   The cooperative merges run in windows of G*D merge steps; the
//   positional bound is tested between windows, and a pair that is not
//   rejected runs to the end of the merge so its overlap is exact.
//   Survivors are compacted into (r, s, o) triples with warp-aggregated
//   atomics on one global cursor (output select, Section 3.3.2), or only
//   counted (output count).
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "ssj_internal.h"

namespace ssj {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kWarpD = 8;                          // merge steps per lane per window (warp)
constexpr uint32_t kWarpWin = 32 * kWarpD;         // merge steps per window (warp)
constexpr uint32_t kWarpBuf = kWarpWin + 16;       // tokens staged per side (warp)
constexpr int kBlockD = 8;                         // merge steps per thread per window (block)
constexpr uint32_t kBlockRCap = 4096;              // r kept whole in shared memory up to this

__device__ __forceinline__ uint32_t sel4(const uint4& v, uint32_t k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// ceil(p*(nr+ns)/(p+q)): Jaccard's equivalent overlap with t = p/q.
// nr, ns < 2^31 and p, q < 2^31 keep every product below 2^63.
__device__ __forceinline__ uint32_t required_overlap(uint32_t nr, uint32_t ns, uint32_t p, uint32_t q) {
    const uint64_t num = (uint64_t)p * (uint64_t)(nr + ns);
    const uint64_t den = (uint64_t)p + (uint64_t)q;
    return (uint32_t)((num + den - 1) / den);
}

__device__ __forceinline__ void emit_triple(const VerifyArgs& a, unsigned long long idx, uint32_t r, uint32_t s,
                                            uint32_t o) {
    if (idx < a.cap) {
        uint32_t x = r, y = s;
        if (a.self_join && y < x) { x = s; y = r; }
        ssj_triple* t = a.out + idx;
        t->r = x;
        t->s = y;
        t->overlap = o;
    }
}

// -------------------------------------------------------------------------
// Sequential merge of one pair by one thread (Alternatives A/B).  Both sets
// are read from global memory 16 bytes at a time (sets start 16-byte
// aligned; the padding keeps the last 16-byte read inside the array).
// Returns the overlap; *rejected is set when the positional bound fired.
// -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t thread_merge(const uint4* __restrict__ r4, uint32_t nr,
                                                 const uint4* __restrict__ s4, uint32_t ns, uint32_t req,
                                                 bool early, bool* rejected) {
    uint32_t i = 0, j = 0, o = 0;
    *rejected = false;
    if (nr == 0 || ns == 0) return 0;
    uint4 rv = __ldg(r4), sv = __ldg(s4);
    while (i < nr && j < ns) {
        if (early) {
            const uint32_t left = min(nr - i, ns - j);
            if (o + left < req) { *rejected = true; break; }
        }
        const uint32_t x = sel4(rv, i & 3u), y = sel4(sv, j & 3u);
        const bool ta = x <= y, tb = x >= y;
        o += (ta && tb) ? 1u : 0u;
        if (ta) {
            ++i;
            if ((i & 3u) == 0 && i < nr) rv = __ldg(r4 + (i >> 2));
        }
        if (tb) {
            ++j;
            if ((j & 3u) == 0 && j < ns) sv = __ldg(s4 + (j >> 2));
        }
    }
    return o;
}

// Copy the 16-byte chunks covering tokens [x0, x0+n) of a set into dst
// (16-byte aligned): dst[k] holds token (x0 & ~3) + k.
template <int G>
__device__ __forceinline__ void stage(const uint4* __restrict__ set4, uint32_t x0, uint32_t n, uint32_t* dst,
                                      int lane) {
    const uint32_t c_lo = x0 >> 2, c_hi = (x0 + n + 3) >> 2;
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint32_t c = c_lo + lane; c < c_hi; c += G) d4[c - c_lo] = __ldg(set4 + c);
}

// One lane's share of a window: binary search of its cross diagonal
// (merge path with "take r when r[i] <= s[j]"), then up to D merge steps.
// A match is counted by the step that takes r[i] while r[i] == s[j], so
// every match is counted exactly once across lanes (Section 4.2.3 with the
// tie rule fixed).  A, B: window-local views; rw, sw: their valid lengths.
template <int D>
__device__ __forceinline__ void lane_merge(const uint32_t* A, uint32_t rw, const uint32_t* B, uint32_t sw,
                                           uint32_t d, uint32_t de, uint32_t* c_out, uint32_t* i_out,
                                           uint32_t* j_out) {
    uint32_t lo = d > sw ? d - sw : 0u;
    uint32_t hi = min(d, rw);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    uint32_t i = lo, j = d - lo, c = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
        if (d + (uint32_t)t < de) {
            bool ta;
            if (i >= rw) {
                ta = false;
            } else if (j >= sw) {
                ta = true;
            } else {
                const uint32_t x = A[i], y = B[j];
                ta = x <= y;
                c += (x == y) ? 1u : 0u;
            }
            i += ta ? 1u : 0u;
            j += ta ? 0u : 1u;
        }
    }
    *c_out = c;
    *i_out = i;
    *j_out = j;
}

// -------------------------------------------------------------------------
// Warp-cooperative merge of one pair (all 32 lanes, uniform arguments).
// abuf, bbuf: this warp's staging buffers (kWarpBuf tokens each).
// -------------------------------------------------------------------------
__device__ uint32_t warp_merge(const uint4* __restrict__ r4, uint32_t nr, const uint4* __restrict__ s4, uint32_t ns,
                               uint32_t req, bool early, uint32_t* abuf, uint32_t* bbuf, int lane, bool* rejected) {
    uint32_t i0 = 0, j0 = 0, o = 0;
    *rejected = false;
    for (;;) {
        const uint32_t left = min(nr - i0, ns - j0);
        if (early && o + left < req) { *rejected = true; break; }
        if (left == 0) break;
        const uint32_t rem = (nr - i0) + (ns - j0);
        const uint32_t Wc = min(kWarpWin, rem);
        const uint32_t rw = min(nr - i0, Wc), sw = min(ns - j0, Wc);
        stage<32>(r4, i0, rw, abuf, lane);
        stage<32>(s4, j0, sw, bbuf, lane);
        __syncwarp();
        const uint32_t* A = abuf + (i0 & 3u);
        const uint32_t* B = bbuf + (j0 & 3u);
        const uint32_t d = min((uint32_t)lane * kWarpD, Wc), de = min(d + kWarpD, Wc);
        uint32_t c = 0, ie = 0, je = 0;
        if (d < de) lane_merge<kWarpD>(A, rw, B, sw, d, de, &c, &ie, &je);
        const uint32_t total = __reduce_add_sync(kFull, c);
        const int last = (int)((Wc - 1) / kWarpD);
        ie = __shfl_sync(kFull, ie, last);
        je = __shfl_sync(kFull, je, last);
        __syncwarp();
        i0 += ie;
        j0 += je;
        o += total;
    }
    return o;
}

// -------------------------------------------------------------------------
// Block-cooperative merge of one pair (Alternative C).  r is staged whole in
// rbuf when it fits (r_staged), else per window in wbuf_r.
// -------------------------------------------------------------------------
template <int BT>
struct BlockSmem {
    uint32_t red[BT / 32];
    uint32_t end_i, end_j;
    uint32_t item;
};

template <int BT>
__device__ uint32_t block_merge(const uint4* __restrict__ r4, uint32_t nr, const uint4* __restrict__ s4,
                                uint32_t ns, uint32_t req, bool early, const uint32_t* rbuf, bool r_staged,
                                uint32_t* wbuf_r, uint32_t* wbuf_s, BlockSmem<BT>* sm, bool* rejected) {
    constexpr uint32_t W = BT * kBlockD;
    const int tid = threadIdx.x;
    uint32_t i0 = 0, j0 = 0, o = 0;
    bool rej = false;
    for (;;) {
        const uint32_t left = min(nr - i0, ns - j0);
        if (early && o + left < req) { rej = true; break; }
        if (left == 0) break;
        const uint32_t rem = (nr - i0) + (ns - j0);
        const uint32_t Wc = min(W, rem);
        const uint32_t rw = min(nr - i0, Wc), sw = min(ns - j0, Wc);
        const uint32_t* A;
        if (r_staged) {
            A = rbuf + i0;
        } else {
            stage<BT>(r4, i0, rw, wbuf_r, tid);
            A = wbuf_r + (i0 & 3u);
        }
        stage<BT>(s4, j0, sw, wbuf_s, tid);
        __syncthreads();
        const uint32_t* B = wbuf_s + (j0 & 3u);
        const uint32_t d = min((uint32_t)tid * kBlockD, Wc), de = min(d + kBlockD, Wc);
        uint32_t c = 0, ie = 0, je = 0;
        if (d < de) lane_merge<kBlockD>(A, rw, B, sw, d, de, &c, &ie, &je);
        c = __reduce_add_sync(kFull, c);
        if ((tid & 31) == 0) sm->red[tid >> 5] = c;
        if (d < de && de == Wc) { sm->end_i = ie; sm->end_j = je; }
        __syncthreads();
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) total += sm->red[w];
        i0 += sm->end_i;
        j0 += sm->end_j;
        o += total;
        __syncthreads();  // everyone has read red/end_* and the window buffers
    }
    *rejected = rej;
    return o;
}

}  // namespace

// -------------------------------------------------------------------------
// Plan: one thread per probe.
// -------------------------------------------------------------------------
__global__ void plan_kernel(VerifyArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_probes; k += stride) {
        const uint64_t c0 = a.cand_offsets[k], c1 = a.cand_offsets[k + 1];
        if ((k == 0 && c0 != 0) || (k + 1 == a.n_probes && c1 != a.n_cands) || c1 < c0 || c1 > a.n_cands) {
            atomicOr(&a.ctr->err, ERR_OFFSETS);
            continue;
        }
        if (c1 == c0) continue;
        // chunks whose first candidate belongs to this probe
        for (uint64_t m = (c0 + kChunk - 1) / kChunk; m * kChunk < c1; ++m) a.hint[m] = k;
        const uint32_t r = a.probe_ids[k];
        if (r >= a.R.n_sets) continue;  // reported by the verify pass
        const uint32_t nr = a.R.desc[r].y;
        bool block;
        if (a.flags & VF_FORCE_BLOCK) block = true;
        else if (a.flags & (VF_FORCE_THREAD | VF_FORCE_WARP)) block = false;
        else block = 2ull * nr > (uint64_t)a.warp_max_key;
        if (!block) continue;
        const uint64_t n = c1 - c0;
        const uint32_t items = (uint32_t)((n + kBlockItemCands - 1) / kBlockItemCands);
        const uint32_t base = atomicAdd(&a.ctr->block_items, items);
        for (uint32_t it = 0; it < items; ++it) {
            if (base + it >= a.item_cap) { atomicOr(&a.ctr->err, ERR_OFFSETS); break; }
            const uint64_t s0 = c0 + (uint64_t)it * kBlockItemCands;
            BlockItem bi;
            bi.r = r;
            bi.n = (uint32_t)min((uint64_t)kBlockItemCands, c1 - s0);
            bi.c0 = s0;
            a.items[base + it] = bi;
        }
    }
}

// -------------------------------------------------------------------------
// Persistent verification kernel.
// -------------------------------------------------------------------------
template <int BT>
__global__ void __launch_bounds__(BT) verify_kernel(VerifyArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ BlockSmem<BT> bsm;
    constexpr uint32_t kBlockWin = BT * kBlockD;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const bool count_only = (a.flags & VF_COUNT_ONLY) != 0;
    const bool emit_all = (a.flags & VF_EMIT_ALL) != 0;
    const bool early = !emit_all;
    unsigned long long local_count = 0;  // count-only mode

    if (a.ctr->err & ERR_OFFSETS) return;  // hints are not trustworthy

    // ---------------- phase 1: block-per-pair items ----------------------
    {
        uint32_t* rbuf = smem;                                // kBlockRCap + 16
        uint32_t* wr = smem + kBlockRCap + 16;                // kBlockWin + 16
        uint32_t* ws = wr + kBlockWin + 16;                   // kBlockWin + 16
        const uint32_t n_items = a.ctr->block_items;
        for (;;) {
            if (tid == 0) bsm.item = atomicAdd(&a.ctr->block_cursor, 1u);
            __syncthreads();
            const uint32_t it = bsm.item;
            __syncthreads();
            if (it >= n_items || it >= a.item_cap) break;
            const BlockItem bi = a.items[it];
            const uint2 dr = a.R.desc[bi.r];
            const uint32_t nr = dr.y;
            const uint4* r4 = a.R.toks4 + dr.x;
            const bool r_staged = nr + 4 <= kBlockRCap;
            if (r_staged) {
                stage<BT>(r4, 0, nr, rbuf, tid);
                __syncthreads();
            }
            for (uint32_t m = 0; m < bi.n; ++m) {
                const uint64_t c = bi.c0 + m;
                const uint32_t s = a.cand_ids[c];
                if (s >= a.S.n_sets) {
                    if (tid == 0) atomicOr(&a.ctr->err, ERR_CAND_ID);
                    continue;
                }
                if (a.self_join && s == bi.r) continue;
                const uint2 ds = a.S.desc[s];
                const uint32_t ns = ds.y;
                const uint32_t req = required_overlap(nr, ns, a.p, a.q);
                if (!emit_all && (nr + ns == 0 || req > min(nr, ns))) continue;  // length filter
                bool rej;
                const uint32_t o = block_merge<BT>(r4, nr, a.S.toks4 + ds.x, ns, req, early, rbuf, r_staged, wr, ws,
                                                   &bsm, &rej);
                const bool pass = emit_all || (!rej && nr + ns > 0 && o >= req);
                if (pass && tid == 0) {
                    if (count_only) {
                        ++local_count;
                    } else {
                        const unsigned long long idx = atomicAdd(a.count, 1ull);
                        emit_triple(a, idx, bi.r, s, o);
                    }
                }
            }
            __syncthreads();  // rbuf reuse
        }
    }

    // ---------------- phase 2: flat chunks of 32 candidates -------------
    {
        uint32_t* abuf = smem + warp * (2 * kWarpBuf);
        uint32_t* bbuf = abuf + kWarpBuf;
        const uint64_t n_chunks = (a.n_cands + kChunk - 1) / kChunk;
        // warp-local survivor buffer for cooperative pairs: lane k holds the k-th
        uint32_t buf_r = 0, buf_s = 0, buf_o = 0, nbuf = 0;
        const bool force_thread = (a.flags & VF_FORCE_THREAD) != 0;
        const bool force_warp = (a.flags & VF_FORCE_WARP) != 0;
        const bool force_block = (a.flags & VF_FORCE_BLOCK) != 0;
        for (;;) {
            uint32_t m32 = 0;
            if (lane == 0) m32 = atomicAdd(&a.ctr->chunk_cursor, 1u);
            const uint64_t m = __shfl_sync(kFull, m32, 0);
            if (m >= n_chunks || force_block) break;
            const uint64_t base = m * kChunk;
            const uint64_t c = base + lane;
            const bool valid = c < a.n_cands;

            // resolve the probe of each lane: k = hint + #{offsets <= c}
            // (every shuffle below is executed by all 32 lanes)
            uint32_t kk = min(a.hint[m], a.n_probes - 1);
            uint32_t k = kk;
            bool resolved = !valid;
            for (uint32_t guard = 0;; ++guard) {
                const uint32_t idx = kk + 1 + lane;
                const uint64_t b = idx <= a.n_probes ? a.cand_offsets[idx] : ~0ull;
                uint32_t pos = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint64_t bm = __shfl_sync(kFull, b, pos + step - 1);
                    if (bm <= c) pos += step;
                }
                const uint64_t b_last = __shfl_sync(kFull, b, 31);
                if (pos == 31 && b_last <= c) pos = 32;
                if (!resolved && pos < 32) { k = kk + pos; resolved = true; }
                if (__all_sync(kFull, resolved)) break;
                // offsets are validated by plan_kernel, so the owner is found within
                // n_probes/32 windows; the guard only turns a broken invariant into an error
                if (guard > (a.n_probes >> 5) + 1 || kk + 32 >= a.n_probes) {
                    if (lane == 0) atomicOr(&a.ctr->err, ERR_OFFSETS);
                    if (!resolved) { k = a.n_probes; resolved = true; }
                    break;
                }
                kk += 32;
            }

            // per-lane pair
            uint32_t r = 0, s = 0, nr = 0, ns = 0, req = 0;
            uint2 dr = make_uint2(0, 0), ds = make_uint2(0, 0);
            bool live = false;
            if (valid && k < a.n_probes) {
                r = a.probe_ids[k];
                s = __ldcs(a.cand_ids + c);
                if (r >= a.R.n_sets) {
                    atomicOr(&a.ctr->err, ERR_PROBE_ID);
                } else if (s >= a.S.n_sets) {
                    atomicOr(&a.ctr->err, ERR_CAND_ID);
                } else if (!(a.self_join && r == s)) {
                    dr = a.R.desc[r];
                    nr = dr.y;
                    const bool block_probe =
                        force_block || (!force_thread && !force_warp && 2ull * nr > (uint64_t)a.warp_max_key);
                    if (!block_probe) {
                        ds = a.S.desc[s];
                        ns = ds.y;
                        req = required_overlap(nr, ns, a.p, a.q);
                        live = emit_all || (nr + ns > 0 && req <= min(nr, ns));  // length filter
                    }
                }
            }
            const bool thread_pair =
                live && !force_warp && (force_thread || (uint64_t)nr + ns <= (uint64_t)a.thread_max_key);
            const bool warp_pair = live && !thread_pair;

            // one pair per thread
            bool pass = false;
            uint32_t o = 0;
            if (thread_pair) {
                bool rej;
                o = thread_merge(a.R.toks4 + dr.x, nr, a.S.toks4 + ds.x, ns, req, early, &rej);
                pass = emit_all || (!rej && o >= req);
            }
            const uint32_t pmask = __ballot_sync(kFull, pass);
            if (pmask) {
                if (count_only) {
                    local_count += (lane == 0) ? __popc(pmask) : 0;
                } else {
                    unsigned long long b0 = 0;
                    if (lane == 0) b0 = atomicAdd(a.count, (unsigned long long)__popc(pmask));
                    b0 = __shfl_sync(kFull, b0, 0);
                    if (pass) emit_triple(a, b0 + __popc(pmask & ((1u << lane) - 1u)), r, s, o);
                }
            }

            // one pair per warp, for the lanes that hold medium pairs
            uint32_t wmask = __ballot_sync(kFull, warp_pair);
            while (wmask) {
                const int src = __ffs(wmask) - 1;
                wmask &= wmask - 1;
                const uint32_t pr = __shfl_sync(kFull, r, src);
                const uint32_t ps = __shfl_sync(kFull, s, src);
                const uint32_t pnr = __shfl_sync(kFull, nr, src);
                const uint32_t pns = __shfl_sync(kFull, ns, src);
                const uint32_t preq = __shfl_sync(kFull, req, src);
                const uint32_t rx = __shfl_sync(kFull, dr.x, src);
                const uint32_t sx = __shfl_sync(kFull, ds.x, src);
                bool rej;
                const uint32_t po =
                    warp_merge(a.R.toks4 + rx, pnr, a.S.toks4 + sx, pns, preq, early, abuf, bbuf, lane, &rej);
                const bool ppass = emit_all || (!rej && po >= preq);
                if (ppass) {
                    if (count_only) {
                        local_count += (lane == 0) ? 1u : 0u;
                    } else {
                        if (lane == (int)nbuf) { buf_r = pr; buf_s = ps; buf_o = po; }
                        ++nbuf;
                        if (nbuf == 32) {
                            unsigned long long b0 = 0;
                            if (lane == 0) b0 = atomicAdd(a.count, 32ull);
                            b0 = __shfl_sync(kFull, b0, 0);
                            emit_triple(a, b0 + lane, buf_r, buf_s, buf_o);
                            nbuf = 0;
                        }
                    }
                }
            }
        }
        if (nbuf) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(a.count, (unsigned long long)nbuf);
            b0 = __shfl_sync(kFull, b0, 0);
            if ((uint32_t)lane < nbuf) emit_triple(a, b0 + lane, buf_r, buf_s, buf_o);
        }
    }

    if (count_only) {
        // lanes hold partial counts; one atomic per warp
        unsigned long long v = local_count;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(kFull, v, off);
        if (lane == 0 && v) atomicAdd(a.count, v);
    }
}

// -------------------------------------------------------------------------
// Host side of the launch.
// -------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static uint32_t block_item_cap(uint32_t n_probes, uint64_t n_cands) {
    const uint64_t cap = (uint64_t)n_probes + (n_cands + kBlockItemCands - 1) / kBlockItemCands;
    return (uint32_t)(cap > 0xFFFFFFF0ull ? 0xFFFFFFF0ull : cap);
}

size_t workspace_bytes(uint32_t n_probes, uint64_t n_cands) {
    const uint64_t n_chunks = (n_cands + kChunk - 1) / kChunk;
    return align256(sizeof(Counters)) + align256(sizeof(uint32_t) * (n_chunks + 1)) +
           align256(sizeof(BlockItem) * ((size_t)block_item_cap(n_probes, n_cands) + 1));
}

void bind_workspace(VerifyArgs& a, void* ws, uint32_t n_probes, uint64_t n_cands) {
    char* p = static_cast<char*>(ws);
    const uint64_t n_chunks = (n_cands + kChunk - 1) / kChunk;
    a.ctr = reinterpret_cast<Counters*>(p);
    p += align256(sizeof(Counters));
    a.hint = reinterpret_cast<uint32_t*>(p);
    p += align256(sizeof(uint32_t) * (n_chunks + 1));
    a.items = reinterpret_cast<BlockItem*>(p);
    a.item_cap = block_item_cap(n_probes, n_cands);
}

template <int BT>
static size_t verify_smem_bytes() {
    constexpr uint32_t kBlockWin = BT * kBlockD;
    const size_t block_phase = sizeof(uint32_t) * (kBlockRCap + 16 + 2 * (kBlockWin + 16));
    const size_t warp_phase = sizeof(uint32_t) * (BT / 32) * 2 * kWarpBuf;
    return block_phase > warp_phase ? block_phase : warp_phase;
}

// CTAs per SM of the persistent kernel, per device (the attribute and the
// occupancy query run once per device and block size).
template <int BT>
static cudaError_t resident_ctas(int* per_sm) {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDev && cache[dev].load() > 0) {
        *per_sm = cache[dev].load();
        return cudaSuccess;
    }
    const size_t smem = verify_smem_bytes<BT>();
    e = cudaFuncSetAttribute(verify_kernel<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, verify_kernel<BT>, BT, smem);
    if (e != cudaSuccess) return e;
    if (n < 1) n = 1;
    if (dev >= 0 && dev < kMaxDev) cache[dev].store(n);
    *per_sm = n;
    return cudaSuccess;
}

template <int BT>
static cudaError_t launch_bt(const VerifyArgs& a, cudaStream_t st, int num_sms) {
    int per_sm = 0;
    cudaError_t e = resident_ctas<BT>(&per_sm);
    if (e != cudaSuccess) return e;
    verify_kernel<BT><<<num_sms * per_sm, BT, verify_smem_bytes<BT>(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_verify(const VerifyArgs& a, cudaStream_t st, int num_sms, uint32_t block_threads,
                          cudaEvent_t* ev) {
    cudaError_t e = cudaMemsetAsync(a.ctr, 0, sizeof(Counters), st);
    if (e != cudaSuccess) return e;
    if (a.count) {
        e = cudaMemsetAsync(a.count, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[0], st);
    if (a.n_probes == 0 || a.n_cands == 0) {
        if (ev) {
            cudaEventRecord(ev[1], st);
            cudaEventRecord(ev[2], st);
        }
        return cudaSuccess;
    }
    {
        const int threads = 256;
        uint64_t blocks = (a.n_probes + threads - 1) / threads;
        const uint64_t max_blocks = (uint64_t)num_sms * 16;
        if (blocks > max_blocks) blocks = max_blocks;
        plan_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], st);
    switch (block_threads) {
        case 128: e = launch_bt<128>(a, st, num_sms); break;
        case 512: e = launch_bt<512>(a, st, num_sms); break;
        default: e = launch_bt<256>(a, st, num_sms); break;
    }
    if (ev) cudaEventRecord(ev[2], st);
    return e;
}

}  // namespace ssj
