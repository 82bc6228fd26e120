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
//     list and bins each probe by |r|+|s| (estimated as 2|r|; the length
//     filter keeps |s| within [t|r|, |r|/t]).  Short probes append their
//     pairs to a compacted (probe, candidate) list; longer probes become
//     warp or block work items.  Space is reserved with one atomic per warp.
//   * verify_kernel, persistent (one wave of CTAs over the SMs):
//       phase 1 - block items: one CTA per pair, Intersect Path across the
//                 whole CTA (Alternative C, Sections 4.2.2-4.2.3), r kept in
//                 shared memory for the item's candidates; and index items:
//                 the CTA holds r as a bitmap over the token values (one bit
//                 per value, in shared memory) and every thread walks one
//                 candidate s at a time through the merge, s side by s side:
//                 each token of s is tested against r by one bit lookup, so
//                 r's tokens are read once per item instead of once per
//                 pair (Alternative B with the probe in shared memory,
//                 Section 3.3.2; the s-side positional bound of Section
//                 2.2.3 after every 16-byte block);
//       phase 2 - warp items: one warp per pair, 32-lane merge path, r kept
//                 in the warp's shared memory for the item's candidates;
//       phase 3 - short pairs, one pair per thread (Alternatives A/B), 32
//                 consecutive pairs of the compacted list per warp step.
//                 The merge compares 16-byte blocks (4 tokens of r against
//                 4 of s, 16 compares; the block with the smaller last token
//                 advances).  Pass 1: every lane loads the first three blocks
//                 of both sets and runs exactly three block steps, unrolled
//                 and predicated, which decides most pairs (the positional
//                 bound rejects them early).  Pass 2: undecided pairs are
//                 parked with their merge state in a per-warp shared buffer
//                 and finished 32 at a time by a loop.
//     Heavy work goes first so that short pairs fill the tail.  The first
//     unit of each phase is assigned statically (CTA / warp index), later
//     ones through one atomic per unit, so small batches need no atomics.
//   The cooperative merges run in windows of G*D merge steps; the
//   positional bound is tested between windows, and a pair that is not
//   rejected runs to the end of the merge so its overlap is exact.
//   Survivors are compacted into (r, s, o) triples with warp-aggregated
//   atomics on one global cursor (output select, Section 3.3.2), or only
//   counted (output count).
#include <atomic>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "arith.h"
#include "ssj_internal.h"

namespace ssj {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kWarpD = 8;                          // merge steps per lane per window (warp)
constexpr uint32_t kWarpWin = 32 * kWarpD;         // merge steps per window (warp)
constexpr uint32_t kWarpRCap = 1024;               // r kept whole in a warp's shared memory up to this
constexpr uint32_t kWarpABuf = kWarpRCap + 16;     // r buffer (whole r, or one window of it)
constexpr uint32_t kWarpBBuf = kWarpWin + 16;      // s window buffer
constexpr int kBlockD = 8;                         // merge steps per thread per window (block)
constexpr uint32_t kBlockRCap = 4096;              // r kept whole in shared memory up to this
constexpr uint32_t kFlatGrab = 4;                  // 32-pair chunks taken per dynamic grab in phase 3
constexpr uint32_t kCont = 64;                     // parked pairs per warp in phase 3
constexpr int kPlanThreads = 256;                  // plan kernel block size

// Checked build (SSJ_CHECKED): the functions that are not inlined take the
// token arrays' remaining extents and the error word as extra arguments;
// the product build passes nothing and the checks compile away.
#ifdef SSJ_CHECKED
#define CHK_PARAMS , uint64_t chk_rlim, uint64_t chk_slim, uint32_t* chk_err
#define CHK_ARGS(rl, sl, e) , (rl), (sl), (e)
#define CHK_ERR_PARAM , uint32_t* chk_err
#define CHK_ERR_ARG(e) , (e)
#define CHK_RLIM chk_rlim
#define CHK_SLIM chk_slim
#define CHK_ERR chk_err
#else
#define CHK_PARAMS
#define CHK_ARGS(rl, sl, e)
#define CHK_ERR_PARAM
#define CHK_ERR_ARG(e)
#define CHK_RLIM (~0ull)
#define CHK_SLIM (~0ull)
#define CHK_ERR (static_cast<uint32_t*>(nullptr))
#endif

// Checked build: false, and ERR_BOUNDS set, when idx is not below n.
__device__ __forceinline__ bool in_bounds(uint64_t idx, uint64_t n, uint32_t* err) {
    if (kChecked && idx >= n) {
        atomicOr(err, ERR_BOUNDS);
        return false;
    }
    return true;
}

// Block idx of a token array with lim blocks from base on (the checked
// build reads zeros past the end).
__device__ __forceinline__ uint4 ld_block(const uint4* base, uint64_t idx, uint64_t lim, uint32_t* err) {
    if (!in_bounds(idx, lim, err)) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg(base + idx);
}

// ---------------------------------------------------------------------------
// One-dimensional bulk copies global -> shared memory (cp.async.bulk on the
// copy engine, completion counted in bytes on an mbarrier), used to stage
// the probe set and candidate sets of block and warp items.  Addresses and
// sizes are multiples of 16 bytes (sets start on 16-byte chunks).  Waits are
// bounded: one thread polls the barrier for at most about a second of SM
// clocks and reports a timeout (ERR_GUARD) instead of spinning forever.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The calling thread arrives on bar expecting `bytes` more bytes, then asks
// the copy engine for `bytes` bytes from src to dst (previous generic-proxy
// accesses of dst are ordered before the copy by the proxy fence).
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Poll bar until the phase with the given parity has completed; false (and
// ERR_GUARD) if that takes more than about a second.
constexpr long long kBulkWaitCycles = 2000000000ll;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kBulkWaitCycles) {
            atomicOr(err, ERR_GUARD);
            return false;
        }
        __nanosleep(20);
    }
}

// Chunks [c_lo, c_hi) of a token array (16 bytes each) into dst by one bulk
// copy on bar; the checked build tests both ends against the array's and
// the buffer's extents and skips the copy (arriving without bytes) when one
// is out of range.
__device__ __forceinline__ void bulk_stage(uint32_t* dst, const uint4* set4, uint32_t c_lo, uint32_t c_hi, uint64_t lim,
                                           uint32_t dst_blocks, uint64_t* bar, uint32_t* err) {
    const uint32_t n = c_hi - c_lo;
    if (n == 0 || !in_bounds(c_hi - 1, lim, err) || !in_bounds(n - 1, dst_blocks, err)) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
        return;
    }
    bulk_copy(dst, set4 + c_lo, 16u * n, bar);
}

// A parked pair with its merge state.
struct ContEntry {
    uint4 m0;  // probe slot (its r id is rid[slot]), s id, current 16-byte block of r, of s (token array indices)
    uint4 m1;  // tokens of r and of s from the current blocks on, required overlap, overlap so far
    uint4 m2;  // instance, unused, unused, unused
};
constexpr uint32_t kDrainMinLive = 16;             // default: pass 2 re-parks a warp's pairs below this many live lanes
constexpr uint32_t kTableBytes = kCont * sizeof(ContEntry);

// Phases 2 and 3 run per warp and the warps of a CTA change phase at
// different times, so each warp owns one fixed slice of shared memory that
// both phases use (phase 1 uses the whole CTA's memory and ends with a
// CTA barrier before any warp moves on).
constexpr uint32_t kWarpPhase2Bytes = (kWarpABuf + kWarpBBuf) * 4;
constexpr uint32_t kWarpSliceBytes =
    ((kWarpPhase2Bytes > kTableBytes ? kWarpPhase2Bytes : kTableBytes) + 15u) & ~15u;

// 1 if x equals one of the four tokens of s (distinct within a block).
__device__ __forceinline__ uint32_t match4(uint32_t x, const uint4& s) {
    return (x == s.x) | (x == s.y) | (x == s.z) | (x == s.w);
}

// Merge state of one pair compared block by block.
struct BlockState {
    uint32_t qi, qj, o;  // current block of r and of s, overlap so far
    bool fin, rej;
};

// Matches between the valid tokens of an r block and an s block whose
// padding repeats the set's last token (the collection layout): a repeated
// s token changes no membership test, and the r lanes past nvr valid ones
// all repeat the last valid token, whose match is subtracted again.
__device__ __forceinline__ uint32_t block_matches(const uint4& rc, const uint4& sc, uint32_t nvr) {
    const uint32_t mw = match4(rc.w, sc);
    return match4(rc.x, sc) + match4(rc.y, sc) + match4(rc.z, sc) + mw - (4u - nvr) * mw;
}

// One block step: count the matches between block qi of r (rc) and block qj
// of s (sc), then advance the block whose last valid token is smaller (both
// on a tie).  Every matching pair of tokens sits in a pair of blocks that is
// current together exactly once, so the count is exact.  Before the step the
// positional bound o + min(|r| - 4qi, |s| - 4qj) < req rejects the pair; the
// bound counts whole current blocks, so it only over-estimates the reachable
// overlap and never rejects a passing pair.  A block's last lane holds its
// last valid token (the padding repeats it).  The step is predicated code:
// the lanes of a warp are at different points of different pairs, so a lane
// whose pair is decided computes and discards instead of branching away.
__device__ __forceinline__ void block_step(const uint4& rc, const uint4& sc, uint32_t nr, uint32_t ns, uint32_t req,
                                           bool early, BlockState& st, bool& adv_r, bool& adv_s) {
    const uint32_t remr = nr - 4 * st.qi, rems = ns - 4 * st.qj;
    const bool bad = !st.fin && early && st.o + min(remr, rems) < req;
    const bool go = !st.fin && !bad;
    st.rej = st.rej || bad;
    const uint32_t c = block_matches(rc, sc, min(remr, 4u));
    st.o += go ? c : 0u;
    adv_r = go && rc.w <= sc.w;
    adv_s = go && sc.w <= rc.w;
    st.qi += adv_r ? 1u : 0u;
    st.qj += adv_s ? 1u : 0u;
    st.fin = st.fin || bad || 4 * st.qi >= nr || 4 * st.qj >= ns;
}

// Equivalent overlap of the instance's similarity function with t = p/q
// (Table "Similarity Functions"; exact, see arith.h): Jaccard and Dice
// divide p(|r|+|s|) by den = p+q or 2q with the precomputed reciprocal,
// Cosine takes the exact ceil(t sqrt(|r||s|)) (den = q), the plain overlap
// threshold is den itself.
__device__ __forceinline__ uint32_t required_overlap(uint32_t sim, uint32_t p, uint32_t den, uint64_t magic,
                                                     uint32_t nr, uint32_t ns) {
    if (sim == SIM_COSINE) return required_overlap_cosine(p, den, nr, ns);
    if (sim == SIM_OVERLAP) return den;
    return required_overlap_magic(nr, ns, p, den, magic);
}

// Write result idx of an instance (if it fits its capacity), as (min, max)
// ids for a self-join.
__device__ __forceinline__ void emit_triple(ssj_triple* out, uint64_t cap, bool self_join, unsigned long long idx,
                                            uint32_t r, uint32_t s, uint32_t o) {
    if (idx < cap) {
        uint32_t x = r, y = s;
        if (self_join && y < x) { x = s; y = r; }
        ssj_triple* t = out + idx;
        t->r = x;
        t->s = y;
        t->overlap = o;
    }
}

// Copy the 16-byte chunks covering tokens [x0, x0+n) of a set into dst
// (16-byte aligned): dst[k] holds token (x0 & ~3) + k.
// (lim: blocks of the token array from set4 on; dst_blocks: room at dst;
// both checked in the checked build only.)
template <int G>
__device__ __forceinline__ void stage(const uint4* __restrict__ set4, uint32_t x0, uint32_t n, uint32_t* dst,
                                      int lane, uint64_t lim, uint32_t dst_blocks, uint32_t* err) {
    const uint32_t c_lo = x0 >> 2, c_hi = (x0 + n + 3) >> 2;
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint32_t c = c_lo + lane; c < c_hi; c += G)
        if (in_bounds(c - c_lo, dst_blocks, err)) d4[c - c_lo] = ld_block(set4, c, lim, err);
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
// If r_staged, abuf holds all of r (abuf[k] = r[k]); otherwise abuf is a
// window buffer.  bbuf is the s window buffer, filled per window by the
// lanes' 16-byte loads or, with wbar (bulk staging), by one bulk copy on the
// warp's barrier (phase parity *wph); a copy that does not complete sets
// *failed and ends the merge.
// -------------------------------------------------------------------------
__device__ uint32_t warp_merge(const uint4* __restrict__ r4, uint32_t nr, const uint4* __restrict__ s4, uint32_t ns,
                               uint32_t req, bool early, bool r_staged, uint32_t* abuf, uint32_t* bbuf, int lane,
                               uint64_t* wbar, uint32_t* wph, uint64_t slim, uint32_t* err, bool* failed,
                               bool* rejected CHK_PARAMS) {
    uint32_t i0 = 0, j0 = 0, o = 0;
    *rejected = false;
    *failed = false;
    for (;;) {
        const uint32_t left = min(nr - i0, ns - j0);
        if (early && o + left < req) { *rejected = true; break; }
        if (left == 0) break;
        const uint32_t rem = (nr - i0) + (ns - j0);
        const uint32_t Wc = min(kWarpWin, rem);
        const uint32_t rw = min(nr - i0, Wc), sw = min(ns - j0, Wc);
        const uint32_t* A;
        if (r_staged) {
            A = abuf + i0;
        } else {
            stage<32>(r4, i0, rw, abuf, lane, CHK_RLIM, kWarpABuf / 4, CHK_ERR);
            A = abuf + (i0 & 3u);
        }
        if (wbar) {  // bulk staging: the window of s by one bulk copy, lane 0 waits
            uint32_t ok = 1;
            if (lane == 0) {
                bulk_stage(bbuf, s4, j0 >> 2, (j0 + sw + 3) >> 2, slim, kWarpBBuf / 4, wbar, err);
                ok = mbar_wait(wbar, *wph, err) ? 1u : 0u;
            }
            *wph ^= 1u;
            if (!__shfl_sync(kFull, ok, 0)) {
                *failed = true;
                break;
            }
        } else {
            stage<32>(s4, j0, sw, bbuf, lane, CHK_SLIM, kWarpBBuf / 4, CHK_ERR);
        }
        __syncwarp();
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
// rbuf when it fits (r_staged), else per window in wbuf_r; s is staged whole
// in wbuf_s by the caller (s_staged: bulk staging) or per window.
// -------------------------------------------------------------------------
template <int BT>
struct BlockSmem {
    uint64_t bar[3];  // bulk staging: r, and the two candidate buffers
    uint32_t red[BT / 32];
    uint32_t end_i, end_j;
    uint32_t item;
    uint32_t next;       // index items: next candidate of the item
    uint32_t staged[2];  // bulk staging: candidate buffer b holds the whole set s of its candidate
    uint32_t ok;         // bulk staging: the last wait completed
};

template <int BT>
__device__ uint32_t block_merge(const uint4* __restrict__ r4, uint32_t nr, const uint4* __restrict__ s4,
                                uint32_t ns, uint32_t req, bool early, const uint32_t* rbuf, bool r_staged,
                                uint32_t* wbuf_r, uint32_t* wbuf_s, bool s_staged, BlockSmem<BT>* sm,
                                bool* rejected CHK_PARAMS) {
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
            stage<BT>(r4, i0, rw, wbuf_r, tid, CHK_RLIM, (W + 16) / 4, CHK_ERR);
            A = wbuf_r + (i0 & 3u);
        }
        const uint32_t* B;
        if (s_staged) {  // all of s is in wbuf_s already (bulk copy)
            B = wbuf_s + j0;
        } else {
            stage<BT>(s4, j0, sw, wbuf_s, tid, CHK_SLIM, (W + 16) / 4, CHK_ERR);
            B = wbuf_s + (j0 & 3u);
        }
        __syncthreads();
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

// Block step of pass 2 on a (block cursor, tokens remaining) state; the same
// step as block_step: positional bound, 16 compares between the current
// blocks, then the block with the smaller last valid token advances (both on
// a tie), predicated like block_step.  rn / sn hold the next block of each
// side, loaded one step ahead.
__device__ __forceinline__ void lean_step(uint4& rc, uint4& rn, uint4& sc, uint4& sn, const uint4* rb,
                                          const uint4* sb, uint32_t& rcur, uint32_t& scur, uint32_t& remr,
                                          uint32_t& rems, uint32_t& o, uint32_t req, bool early, bool& fin,
                                          bool& rej, uint64_t rlim, uint64_t slim, uint32_t* err) {
    const bool bad = !fin && early && o + min(remr, rems) < req;
    const bool go = !fin && !bad;
    rej = rej || bad;
    const uint32_t c = block_matches(rc, sc, min(remr, 4u));
    o += go ? c : 0u;
    const bool ar = go && rc.w <= sc.w, as = go && sc.w <= rc.w;
    rc.x = ar ? rn.x : rc.x;
    rc.y = ar ? rn.y : rc.y;
    rc.z = ar ? rn.z : rc.z;
    rc.w = ar ? rn.w : rc.w;
    sc.x = as ? sn.x : sc.x;
    sc.y = as ? sn.y : sc.y;
    sc.z = as ? sn.z : sc.z;
    sc.w = as ? sn.w : sc.w;
    rcur += ar ? 1u : 0u;
    scur += as ? 1u : 0u;
    remr = ar ? (remr > 4 ? remr - 4 : 0u) : remr;
    rems = as ? (rems > 4 ? rems - 4 : 0u) : rems;
    if (ar && remr > 4) rn = ld_block(rb, rcur + 1, rlim, err);
    if (as && rems > 4) sn = ld_block(sb, scur + 1, slim, err);
    fin = fin || bad || remr == 0 || rems == 0;
}

// Pass 2 of the short-pair phase: the parked pairs [n_cont - m, n_cont) are
// taken one per lane (lanes may belong to different instances) and merged
// while at least min_live lanes are still undecided; decided pairs are
// emitted, undecided ones parked again, compacted, so that lanes are refilled
// from later pairs instead of idling behind the longest merge of the warp.
// min_live = 1 finishes every pair.  A parked pair carries its probe slot;
// the r id is read from it only for a survivor.  Returns the new number of
// parked pairs.
__device__ __noinline__ uint32_t drain_parked(ContEntry* cont, uint32_t n_cont, uint32_t m, uint32_t min_live,
                                              const Instance* table, const uint32_t* rid_of_slot,
                                              int lane CHK_ERR_PARAM) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint4 zero4 = make_uint4(0, 0, 0, 0);
    const uint32_t base = n_cont - m;
    const bool have = (uint32_t)lane < m && in_bounds(base + lane, kCont, CHK_ERR);
    uint32_t slot = 0, sid = 0, rcur = 0, scur = 0, remr = 0, rems = 0, req = 0, o = 0, inst = 0;
    const uint4* rb = nullptr;
    const uint4* sb = nullptr;
    uint64_t rlim = 0, slim = 0;
    bool early = true, fin = true, rej = false;
    uint4 rc = zero4, rn = zero4, sc = zero4, sn = zero4;
    if (have) {
        const ContEntry* ce = cont + base + lane;
        const uint4 m0 = ce->m0, m1 = ce->m1, m2 = ce->m2;
        slot = m0.x;
        sid = m0.y;
        rcur = m0.z;
        scur = m0.w;
        remr = m1.x;
        rems = m1.y;
        req = m1.z;
        o = m1.w;
        inst = m2.x;
        const Instance& I = table[inst];
        rb = I.r_toks4;
        sb = I.s_toks4;
        rlim = I.r_n_chunks;
        slim = I.s_n_chunks;
        early = !(I.flags & VF_EMIT_ALL);
        fin = remr == 0 || rems == 0;
        rc = ld_block(rb, rcur, rlim, CHK_ERR);
        if (remr > 4) rn = ld_block(rb, rcur + 1, rlim, CHK_ERR);
        sc = ld_block(sb, scur, slim, CHK_ERR);
        if (rems > 4) sn = ld_block(sb, scur + 1, slim, CHK_ERR);
    }
    __syncwarp();  // every entry is read before any is written again
    while ((uint32_t)__popc(__ballot_sync(kFull, !fin)) >= min_live) {  // two steps per check
        if (!fin) lean_step(rc, rn, sc, sn, rb, sb, rcur, scur, remr, rems, o, req, early, fin, rej, rlim, slim, CHK_ERR);
        if (!fin) lean_step(rc, rn, sc, sn, rb, sb, rcur, scur, remr, rems, o, req, early, fin, rej, rlim, slim, CHK_ERR);
    }
    // survivors: one atomic per instance among the warp's lanes (lanes may hold different instances)
    const bool pass = have && fin && (!early || (!rej && o >= req));
    const uint32_t pmask = __ballot_sync(kFull, pass);
    if (pmask) {
        const uint32_t grp = __match_any_sync(kFull, inst) & pmask;  // passing lanes of my instance
        if (pass) {
            const Instance& I = table[inst];
            const int leader = __ffs(grp) - 1;
            unsigned long long b0 = 0;
            if (lane == leader) b0 = atomicAdd(I.count, (unsigned long long)__popc(grp));
            b0 = __shfl_sync(grp, b0, leader);
            if (!(I.flags & VF_COUNT_ONLY))
                emit_triple(I.out, I.cap, (I.flags & VF_SELF_JOIN) != 0, b0 + __popc(grp & lt_mask),
                            rid_of_slot[slot], sid, o);
        }
    }
    const bool again = have && !fin;
    const uint32_t amask = __ballot_sync(kFull, again);
    if (again) {
        ContEntry* ce = cont + base + __popc(amask & lt_mask);
        ce->m0 = make_uint4(slot, sid, rcur, scur);
        ce->m1 = make_uint4(remr, rems, req, o);
        ce->m2 = make_uint4(inst, 0u, 0u, 0u);
    }
    __syncwarp();
    return base + __popc(amask);
}

// Warp-local survivor buffer for pairs decided by the whole warp (one work
// item, so one instance): lane k holds the k-th buffered triple; flushed
// with one atomic per 32 and at the end of every item.
struct WarpOut {
    uint32_t r = 0, s = 0, o = 0, n = 0;

    __device__ void push(const Instance& I, int lane, uint32_t pr, uint32_t ps, uint32_t po) {
        if (lane == (int)n) { r = pr; s = ps; o = po; }
        if (++n == 32) flush(I, lane);
    }
    __device__ void flush(const Instance& I, int lane) {
        if (n == 0) return;
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(I.count, (unsigned long long)n);
        b0 = __shfl_sync(kFull, b0, 0);
        if ((uint32_t)lane < n) emit_triple(I.out, I.cap, (I.flags & VF_SELF_JOIN) != 0, b0 + lane, r, s, o);
        n = 0;
    }
};

// One lane item (Alternative B): the item's probe r is staged whole in the
// warp's shared memory (rsm, 16-byte blocks), each lane verifies one of the
// item's candidates at a time with the block merge, reading r's blocks from
// shared memory and s's from global memory one block ahead; a lane that
// finishes takes the item's next candidate.  Survivors are emitted with one
// atomic per warp step.
__device__ __noinline__ void lane_item(const Instance& I, const WorkItem& wi, uint32_t nr, const uint4* rsm, int lane,
                          uint32_t* err) {
    const uint32_t flags = I.flags;
    const bool emit_all = (flags & VF_EMIT_ALL) != 0, early = !emit_all;
    const bool self_join = (flags & VF_SELF_JOIN) != 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t rq = (nr + 3) >> 2;
    const uint4 zero4 = make_uint4(0, 0, 0, 0);
    uint32_t cursor = 0;  // next candidate of the item (warp-uniform)
    bool active = false;
    uint32_t s_id = 0, ns = 0, req = 0, sq = 0;
    const uint4* s4 = nullptr;
    uint64_t slim = 0;
    BlockState st;
    st.qi = st.qj = st.o = 0;
    st.fin = true;
    st.rej = false;
    uint4 rc = zero4, sc = zero4, sn = zero4;
    for (;;) {
        const uint32_t idle = __ballot_sync(kFull, !active);
        if (idle && cursor < wi.n) {
            const uint32_t my = cursor + __popc(idle & lt_mask);
            if (!active && my < wi.n) {
                const uint32_t s = in_bounds(wi.c0 + my, I.n_cands, err) ? I.cand_ids[wi.c0 + my] : ~0u;
                if (s >= I.s_n_sets) {
                    atomicOr(err, ERR_CAND_ID);
                } else if (!(self_join && s == wi.r)) {
                    const uint2 ds = I.s_desc[s];
                    const uint32_t q = required_overlap(I.sim, I.p, I.den, I.magic, nr, ds.y);
                    if (emit_all || (nr + ds.y > 0 && q <= min(nr, ds.y))) {  // length filter
                        active = true;
                        s_id = s;
                        ns = ds.y;
                        req = q;
                        sq = (ns + 3) >> 2;
                        s4 = I.s_toks4 + ds.x;
                        slim = I.s_n_chunks - ds.x;
                        st.qi = st.qj = st.o = 0;
                        st.rej = false;
                        st.fin = nr == 0 || ns == 0;
                        rc = rq ? rsm[0] : zero4;
                        sc = sq ? ld_block(s4, 0, slim, err) : zero4;
                        sn = sq > 1 ? ld_block(s4, 1, slim, err) : zero4;
                    }
                }
            }
            cursor += __popc(idle);
        }
        if (!__any_sync(kFull, active)) {
            if (cursor >= wi.n) break;
            continue;
        }
        if (active && !st.fin) {
            bool ar, as;
            block_step(rc, sc, nr, ns, req, early, st, ar, as);
            if (ar && st.qi < rq && in_bounds(st.qi, kWarpABuf / 4, err)) rc = rsm[st.qi];
            if (as) {
                sc = sn;
                if (st.qj + 1 < sq) sn = ld_block(s4, st.qj + 1, slim, err);
            }
        }
        const bool done = active && st.fin;
        const bool pass = done && (emit_all || (!st.rej && st.o >= req));
        const uint32_t pmask = __ballot_sync(kFull, pass);
        if (pmask) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(I.count, (unsigned long long)__popc(pmask));
            if (!(flags & VF_COUNT_ONLY)) {
                b0 = __shfl_sync(kFull, b0, 0);
                if (pass) emit_triple(I.out, I.cap, self_join, b0 + __popc(pmask & lt_mask), wi.r, s_id, st.o);
            }
        }
        if (done) active = false;
    }
}

// Set (or, with clear, zero the words of) the bits of r's tokens; r's
// padding repeats its last token, so whole blocks are used.
template <int BT>
__device__ __forceinline__ void bm_mark(uint32_t* bm, const uint4* r4, uint32_t nr, uint64_t rlim, uint32_t n_words,
                                        bool clear, int tid, uint32_t* err) {
    for (uint32_t c = tid; c < ((nr + 3) >> 2); c += BT) {
        const uint4 b = ld_block(r4, c, rlim, err);
        const uint32_t v[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = v[k] >> 5;
            if (!in_bounds(w, n_words, err)) continue;
            if (clear) bm[w] = 0u;
            else atomicOr(bm + w, 1u << (v[k] & 31u));
        }
    }
}

// Asynchronous 16-byte copy global -> shared memory (cp.async, cached in L2
// only) and its per-thread groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One index item: candidates [c0, c0 + n) of probe r, verified by every
// thread of the CTA, one candidate per thread at a time.  r is held as a
// bitmap over the token values (bm, all zero on entry and on return).  A
// candidate s is merged against r from the s side: block by block (16
// bytes, 4 tokens), each token tested by one bit lookup, so the state after
// a block is the merge's state after s's token j: o matches, |s| - j tokens
// of s left.  The merge stops when o + (|s| - j) falls below the required
// overlap (the positional bound of Section 2.2.3 with the s side's
// remainder; never stricter than the merge's bound, so no passing pair is
// lost) or when s's block reaches r's last token (no later token of s can
// match); a pair that is not rejected runs to that point, so its overlap is
// exactly |r n s|.
//
// The walk is software-pipelined so that no thread waits on a load it has
// just issued, and its common path is short.  Each warp prepares its
// candidates 32 at a time: their ids are loaded, one round later their
// descriptors, one round later again the required overlap and the length
// filter decide which enter the warp's queue (shared memory), and the next
// batch's ids are loaded in that same step.  A round is
// kIndexSteps walk steps followed by one maintenance step (preparation,
// survivors out, idle lanes refilled from the queue).  In a walk step a lane
// asks for one more block of s (cp.async into its own ring of kIndexRing
// blocks in shared memory, at most kIndexRing blocks ahead of its walk) and
// merges a block it asked for in an earlier step.
constexpr uint32_t kIndexRing = 4;   // blocks of s per thread in the ring
constexpr uint32_t kIndexQueue = 64; // prepared candidates per warp
constexpr int kIndexSteps = 4;       // walk steps per round

// Bit of token value x in the probe bitmap, as one shift-and-mask of the
// word (the funnel shift takes the shift amount modulo 32).
__device__ __forceinline__ uint32_t bm_test(const uint32_t* bm, uint32_t x, uint32_t n_words, uint32_t* err) {
    const uint32_t w = x >> 5;
    if (!in_bounds(w, n_words, err)) return 0u;
    const uint32_t word = bm[w];
    return __funnelshift_r(word, word, x) & 1u;
}

template <int BT>
__device__ __noinline__ void index_item(const Instance& I, const WorkItem& wi, uint32_t nr, const uint4* r4,
                                        uint64_t rlim, uint32_t* bm, uint32_t n_words, uint4* rings,
                                        uint4* queues, BlockSmem<BT>* sm, uint32_t* err) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t flags = I.flags;
    const bool emit_all = (flags & VF_EMIT_ALL) != 0, early = !emit_all;
    const bool self_join = (flags & VF_SELF_JOIN) != 0;
    uint4* ring = rings + (size_t)tid * kIndexRing;
    uint4* queue = queues + (size_t)warp * kIndexQueue;
    // candidate preparation (warp-uniform stage: 0 takes 32 candidates, 1 loads descriptors,
    // 2 filters and queues); queue cursors are free-running.  Warp w's first batch is
    // candidates [32w, 32w + 32): its ids and descriptors are loaded while r's bits are set,
    // so the walk starts one round after the item does; later batches are taken from the
    // item's cursor, which starts after the first batches.
    uint32_t pstage = 0, qhead = 0, qtail = 0;
    bool pdone = 32u * (BT / 32) >= wi.n;  // warp-uniform: no candidates left to take
    const uint32_t my0 = 32u * (uint32_t)warp + (uint32_t)lane;
    bool p_ok = my0 < wi.n && in_bounds(wi.c0 + my0, I.n_cands, err);
    uint32_t p_id = p_ok ? I.cand_ids[wi.c0 + my0] : 0u;
    uint2 p_desc = make_uint2(0u, 0u);
    if (tid == 0) sm->next = 32u * (BT / 32);
    bm_mark<BT>(bm, r4, nr, rlim, n_words, false, tid, err);
    // r's last token (the padding repeats it in the last block's last lane)
    const uint32_t rmax = nr ? ld_block(r4, (nr - 1) >> 2, rlim, err).w : 0u;
    if (32u * (uint32_t)warp < wi.n) {  // warp-uniform: the first batch's descriptors
        if (p_ok && p_id >= I.s_n_sets) {
            atomicOr(err, ERR_CAND_ID);
            p_ok = false;
        }
        if (p_ok && self_join && p_id == wi.r) p_ok = false;
        if (p_ok) p_desc = I.s_desc[p_id];
        pstage = 2;
    }
    __syncthreads();

    // the lane's pair: next block to merge (jb) and to ask for (jr), ring slot of its block 0
    // (rb); a finished pair keeps s_id / o until the maintenance step sends it out
    bool active = false, out = false;
    uint32_t s_id = 0, rems = 0, req = 0, o = 0, jb = 0, jr = 0, rb = 0;
    const uint4* s4 = nullptr;
    uint64_t slim = 0;
    for (;;) {
        // ---- walk steps
#pragma unroll
        for (int step = 0; step < kIndexSteps; ++step) {
            const uint32_t avail = jr;      // blocks asked for in earlier steps
            const uint32_t ahead = jr - jb;  // asked for, not yet merged (rems counts tokens from block jb)
            if (active && ahead < kIndexRing && 4 * ahead < rems) {
                if (in_bounds(jr, slim, err)) cp_async16(ring + ((rb + jr) & (kIndexRing - 1)), s4 + jr);
                ++jr;
            }
            cp_async_commit();
            cp_async_wait<1>();  // every block asked for before this step is in
            if (active && jb < avail) {
                const uint4 sc = ring[(rb + jb) & (kIndexRing - 1)];
                const uint32_t bw = bm_test(bm, sc.w, n_words, err);
                o += bm_test(bm, sc.x, n_words, err) + bm_test(bm, sc.y, n_words, err) +
                     bm_test(bm, sc.z, n_words, err) + bw;
                ++jb;
                if (rems <= 4 || sc.w >= rmax) {  // s's last block, or no later token of s can match
                    if (rems < 4) o -= (4u - rems) * bw;  // the lanes past s's end repeat its last token
                    rems = 0;
                    active = false;
                    out = emit_all || o >= req;
                } else {
                    rems -= 4;
                    if (early && o + rems < req) {
                        active = false;
                        out = emit_all;
                    }
                }
            }
        }
        // ---- maintenance: survivors out
        const uint32_t pmask = __ballot_sync(kFull, out);
        if (pmask) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(I.count, (unsigned long long)__popc(pmask));
            if (!(flags & VF_COUNT_ONLY)) {
                b0 = __shfl_sync(kFull, b0, 0);
                if (out) emit_triple(I.out, I.cap, self_join, b0 + __popc(pmask & lt_mask), wi.r, s_id, o);
            }
            out = false;
        }
        // ---- preparation (a batch queued here makes room for the next one to be taken in the
        // same step, so a batch is taken every second round)
        if (pstage == 1) {
            if (p_ok && p_id >= I.s_n_sets) {
                atomicOr(err, ERR_CAND_ID);
                p_ok = false;
            }
            if (p_ok && self_join && p_id == wi.r) p_ok = false;
            if (p_ok) p_desc = I.s_desc[p_id];
            pstage = 2;
        } else {
            if (pstage == 2) {
                uint32_t q = 0;
                if (p_ok) {
                    q = required_overlap(I.sim, I.p, I.den, I.magic, nr, p_desc.y);
                    p_ok = emit_all || (nr + p_desc.y > 0 && q <= min(nr, p_desc.y));  // length filter
                }
                const uint32_t m = __ballot_sync(kFull, p_ok);
                if (p_ok) queue[(qtail + __popc(m & lt_mask)) % kIndexQueue] = make_uint4(p_id, p_desc.x, p_desc.y, q);
                qtail += __popc(m);
                pstage = 0;
                __syncwarp();
            }
            if (pstage == 0) {
                if (!pdone && qtail - qhead + 32 <= kIndexQueue) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(&sm->next, 32u);
                    base = __shfl_sync(kFull, base, 0);
                    if (base + 32 >= wi.n) pdone = true;
                    const uint32_t my = base + (uint32_t)lane;
                    p_ok = my < wi.n && in_bounds(wi.c0 + my, I.n_cands, err);
                    if (p_ok) p_id = I.cand_ids[wi.c0 + my];
                    if (base < wi.n) pstage = 1;
                }
            }
        }
        // ---- idle lanes take queued candidates
        const uint32_t idle = __ballot_sync(kFull, !active);
        if (idle && qtail != qhead) {
            const uint32_t k = min((uint32_t)__popc(idle), qtail - qhead);
            const uint32_t rank = __popc(idle & lt_mask);
            if (!active && rank < k) {
                const uint4 e = queue[(qhead + rank) % kIndexQueue];
                rb = (rb + jr) & (kIndexRing - 1);  // continue the lane's ring after its last request
                s_id = e.x;
                rems = e.z;
                req = e.w;
                o = 0;
                jb = 0;
                jr = 0;
                s4 = I.s_toks4 + e.y;
                slim = I.s_n_chunks - e.y;
                if (rems == 0 || nr == 0) {
                    out = emit_all;  // an empty side: overlap 0
                } else {
                    active = true;
                }
            }
            qhead += k;
            __syncwarp();
        }
        if (pdone && pstage == 0 && qhead == qtail && !__any_sync(kFull, active || out)) break;
    }
    cp_async_wait<0>();  // the ring's last copies (asked for past a pair's end) are in
    __syncthreads();     // every thread is done with the bitmap
    bm_mark<BT>(bm, r4, nr, rlim, n_words, true, tid, err);
    __syncthreads();
}

// Granularity of a probe with |r| = nr and n candidates: 0 thread per pair,
// 1 warp per pair, 2 block per pair, 3 lane per pair with r in the warp's
// shared memory (Alternative B; needs r to fit and enough candidates to
// occupy the lanes), 4 index items (probes with many candidates, when the
// launch's token values fit the probe bitmap).
__device__ __forceinline__ uint32_t probe_bin(const VerifyArgs& a, uint32_t flags, uint32_t nr, uint64_t n) {
    const bool lane_ok = nr + 4 <= kWarpRCap;
    if (flags & VF_FORCE_INDEX) return a.index_words ? 4u : (lane_ok ? 3u : 1u);
    if (flags & VF_FORCE_BLOCK) return 2;
    if (flags & VF_FORCE_WARP) return 1;
    if (flags & VF_FORCE_THREAD) return 0;
    if (flags & VF_FORCE_LANE) return lane_ok ? 3u : 1u;
    if (a.index_words && a.index_min_cands && n >= a.index_min_cands) return 4;
    const uint64_t key = 2ull * nr;  // |r|+|s| at |s| = |r|
    if (key <= a.thread_max_key) return 0;
    if (key <= a.lane_max_key && lane_ok && n >= kLaneMinCands) return 3;
    return key <= a.warp_max_key ? 1u : 2u;
}

// Instance fields read by the plan kernel (from the kernel parameters for a
// one-batch launch, else from the device table).
struct PlanInst {
    const uint32_t* probe_ids;
    const uint64_t* cand_offsets;
    const uint32_t* cand_ids;
    const uint2* r_desc;
    uint64_t n_cands;
    uint32_t r_n_sets, n_probes, tile_base, flags;
};

__device__ __forceinline__ PlanInst plan_inst(const VerifyArgs& a, uint32_t i) {
    PlanInst q;
    if (a.table) {
        const Instance* I = a.table + i;
        q.probe_ids = I->probe_ids;
        q.cand_offsets = I->cand_offsets;
        q.cand_ids = I->cand_ids;
        q.r_desc = I->r_desc;
        q.n_cands = I->n_cands;
        q.r_n_sets = I->r_n_sets;
        q.n_probes = I->n_probes;
        q.tile_base = I->tile_base;
        q.flags = I->flags;
    } else {
        q.probe_ids = a.single.probe_ids;
        q.cand_offsets = a.single.cand_offsets;
        q.cand_ids = a.single.cand_ids;
        q.r_desc = a.single.r_desc;
        q.n_cands = a.single.n_cands;
        q.r_n_sets = a.single.r_n_sets;
        q.n_probes = a.single.n_probes;
        q.tile_base = a.single.tile_base;
        q.flags = a.single.flags;
    }
    return q;
}

}  // namespace

// -------------------------------------------------------------------------
// Plan.  The probes of every instance are cut into tiles of 32; warp w takes
// tiles w, w + n_warps, ...  Lane l of tile t of an instance with T tiles
// takes probe t + l*T, so a warp's 32 probes are spread over the instance and
// warps get similar amounts of copying even when probes come in size order.
// Each probe is validated and binned; short probes append their pairs to
// the compacted list (a warp's range is padded to whole 32-slot chunks, so
// a chunk never mixes instances), longer probes become work items.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(VerifyArgs a) {
    constexpr int kPlanWarps = kPlanThreads / 32;
    // per-warp list sizes and the CTA's list bases, double-buffered by round
    // parity so that a warp one round ahead never overwrites what others read
    __shared__ unsigned long long s_tot[2][3][kPlanWarps];
    __shared__ unsigned long long s_base[2][3];
    // each warp's tile, for the copy of the short pairs by the whole CTA
    __shared__ unsigned long long s_incl[2][kPlanWarps][32];  // inclusive prefix of the lanes' short pairs
    __shared__ unsigned long long s_c0[2][kPlanWarps][32];    // the lanes' first candidates
    __shared__ uint32_t s_slot[2][kPlanWarps][32];            // the lanes' probe slots
    __shared__ unsigned long long s_pre[2][kPlanWarps + 1];   // exclusive prefix of the tiles' padded ranges
    __shared__ const uint32_t* s_cand[2][kPlanWarps];         // the tiles' candidate arrays
    __shared__ unsigned long long s_ncand[2][kPlanWarps];     // their lengths (checked build)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (blockIdx.x == 0) {
        if (!a.table && threadIdx.x == 0) a.table_out[0] = a.single;
        for (uint32_t i = threadIdx.x; i < a.n_inst; i += blockDim.x)
            *(a.table ? a.table[i].count : a.single.count) = 0ull;
    }
    // Rounds are uniform over the CTA: warp w of the CTA takes tile g0 + w.
    // The three lists (short pairs, warp/lane items, block items) are
    // reserved with one atomic per CTA and round, not per warp.
    // With few tiles a CTA takes fewer than one per warp, so that more CTAs
    // share the copying.
    const uint32_t per_round =
        a.n_tiles >= gridDim.x * (uint32_t)kPlanWarps ? kPlanWarps : max(1u, (a.n_tiles + gridDim.x - 1) / gridDim.x);
    uint32_t par = 0;
    for (uint32_t g0 = blockIdx.x * per_round; g0 < a.n_tiles; g0 += gridDim.x * per_round, par ^= 1u) {
        const uint32_t g = g0 + (uint32_t)warp;
        const bool tile_ok = (uint32_t)warp < per_round && g < a.n_tiles;
        // instance owning tile g: the last one whose tile_base <= g
        uint32_t inst = 0;
        if (a.table) {
            uint32_t lo = 0, hi = a.n_inst - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (a.table[mid].tile_base <= g) lo = mid; else hi = mid - 1;
            }
            inst = lo;
        }
        const PlanInst I = plan_inst(a, inst);
        const uint32_t T = (I.n_probes + 31) >> 5;
        const uint32_t t = g - I.tile_base;
        const uint32_t k = t + (uint32_t)lane * T;           // local probe index
        const uint32_t slot = I.tile_base * 32u + (uint32_t)lane * T + t;  // probe slot, unique per launch
        uint64_t c0 = 0, n = 0;
        uint32_t r = 0, bin = 0;
        uint2 rdesc = make_uint2(0, 0);
        if (tile_ok && k < I.n_probes) {
            c0 = I.cand_offsets[k];
            const uint64_t c1 = I.cand_offsets[k + 1];
            if ((k == 0 && c0 != 0) || (k + 1 == I.n_probes && c1 != I.n_cands) || c1 < c0 || c1 > I.n_cands) {
                atomicOr(&a.ctr->err, ERR_OFFSETS);
            } else {
                r = I.probe_ids[k];
                if (r >= I.r_n_sets) {
                    if (c1 > c0) atomicOr(&a.ctr->err, ERR_PROBE_ID);
                } else {
                    rdesc = I.r_desc[r];
                    if (in_bounds(slot, 32ull * a.n_tiles + 1, &a.ctr->err)) {
                        a.rdesc[slot] = rdesc;
                        a.rid[slot] = r;
                    }
                    n = c1 - c0;
                    bin = probe_bin(a, I.flags, rdesc.y, n);
                }
            }
        }
        // short probes: the warp's pairs form one contiguous, chunk-aligned range
        // of the list; it is copied flat and coalesced, each slot finding its probe
        // by a search over the lanes' prefix sums
        const unsigned long long tn = (bin == 0) ? n : 0;
        unsigned long long tincl = tn;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, tincl, off);
            if (lane >= off) tincl += y;
        }
        const unsigned long long ttotal = __shfl_sync(kFull, tincl, 31);
        const unsigned long long tpadded = (ttotal + 31) & ~31ull;
        // work item counts (lane items share the warp item list, marked by mode 1)
        const uint32_t wc = bin == 3 ? a.lane_item_cands : a.warp_item_cands;
        const uint32_t bc = bin == 4 ? a.index_item_cands : a.block_item_cands;
        const unsigned long long wn = (bin == 1 || bin == 3) ? (n + wc - 1) / wc : 0;
        const unsigned long long bn = (bin == 2 || bin == 4) ? (n + bc - 1) / bc : 0;
        unsigned long long wincl = wn, bincl = bn;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long yw = __shfl_up_sync(kFull, wincl, off);
            const unsigned long long yb = __shfl_up_sync(kFull, bincl, off);
            if (lane >= off) { wincl += yw; bincl += yb; }
        }
        if (lane == 31) {
            s_tot[par][0][warp] = tpadded;
            s_tot[par][1][warp] = wincl;
            s_tot[par][2][warp] = bincl;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            unsigned long long sum = 0;
#pragma unroll
            for (int w = 0; w < kPlanWarps; ++w) sum += s_tot[par][threadIdx.x][w];
            unsigned long long* ctr = threadIdx.x == 0 ? &a.ctr->thread_pairs
                                                       : (threadIdx.x == 1 ? &a.ctr->warp_items : &a.ctr->block_items);
            s_base[par][threadIdx.x] = sum ? atomicAdd(ctr, sum) : 0ull;
        }
        __syncthreads();
        unsigned long long tbase0 = s_base[par][0], wbase = s_base[par][1], bbase = s_base[par][2];
        for (int w = 0; w < warp; ++w) {
            tbase0 += s_tot[par][0][w];
            wbase += s_tot[par][1][w];
            bbase += s_tot[par][2][w];
        }
        wbase += wincl - wn;  // this lane's first item
        bbase += bincl - bn;
        // short pairs: the CTA's tiles have one contiguous, chunk-aligned range of
        // the list (warp order); all its threads copy it flat and coalesced, each
        // slot finding its tile by the prefix of the tiles' ranges and its probe
        // by a search over that tile's lane prefix sums
        s_incl[par][warp][lane] = tincl;
        s_c0[par][warp][lane] = c0;
        s_slot[par][warp][lane] = slot;
        if (lane == 0) s_cand[par][warp] = I.cand_ids;
        if (kChecked && lane == 0) s_ncand[par][warp] = I.n_cands;
        if (threadIdx.x == 0) {
            unsigned long long acc = 0;
            for (int w = 0; w < kPlanWarps; ++w) {
                s_pre[par][w] = acc;
                acc += s_tot[par][0][w];
            }
            s_pre[par][kPlanWarps] = acc;
        }
        if (tpadded && tbase0 + tpadded > a.pair_cap) {  // cannot happen with a sized workspace
            if (lane == 0) atomicOr(&a.ctr->err, ERR_GUARD);
        } else {
            for (unsigned long long c = lane; c < tpadded / 32; c += 32) a.chunk_inst[tbase0 / 32 + c] = inst;
        }
        __syncthreads();
        {
            const unsigned long long cta_base = s_base[par][0], cta_total = s_pre[par][kPlanWarps];
            if (cta_base + cta_total <= a.pair_cap) {
                // each thread writes 4 consecutive slots (cta_total is a multiple of
                // 32, so all 4 exist): it locates the first by binary search and
                // follows the tile and probe boundaries for the other three
                for (unsigned long long f0 = 4ull * threadIdx.x; f0 < cta_total; f0 += 4ull * kPlanThreads) {
                    int w = 0;
#pragma unroll
                    for (int step = kPlanWarps / 2; step >= 1; step >>= 1)
                        if (s_pre[par][w + step] <= f0) w += step;
                    uint32_t pos = 0, out[8];
                    bool located = false;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const unsigned long long f = f0 + e;
                        while (f >= s_pre[par][w + 1]) {  // into the next tile with slots
                            ++w;
                            located = false;
                        }
                        const unsigned long long fl = f - s_pre[par][w];
                        out[2 * e] = kNoProbe;
                        out[2 * e + 1] = 0u;
                        if (fl < s_incl[par][w][31]) {
                            if (!located) {
                                pos = 0;
#pragma unroll
                                for (int step = 16; step >= 1; step >>= 1)
                                    if (s_incl[par][w][pos + step - 1] <= fl) pos += step;
                                located = true;
                            } else {
                                while (s_incl[par][w][pos] <= fl) ++pos;  // past probes that end before fl
                            }
                            const unsigned long long ex = pos ? s_incl[par][w][pos - 1] : 0ull;
                            const unsigned long long ci = s_c0[par][w][pos] + (fl - ex);
                            out[2 * e] = s_slot[par][w][pos];
                            out[2 * e + 1] =
                                in_bounds(ci, kChecked ? s_ncand[par][w] : 0ull, &a.ctr->err) ? s_cand[par][w][ci] : 0u;
                        }
                    }
                    uint4* dst = reinterpret_cast<uint4*>(a.pairs + cta_base + f0);
                    dst[0] = make_uint4(out[0], out[1], out[2], out[3]);
                    dst[1] = make_uint4(out[4], out[5], out[6], out[7]);
                }
            }
        }
        // longer probes: work items of up to warp_item_cands / lane_item_cands /
        // block_item_cands candidates
        for (unsigned long long it = 0; it < wn; ++it) {
            if (wbase + it >= a.warp_item_cap) { atomicOr(&a.ctr->err, ERR_GUARD); break; }
            const uint64_t s0 = c0 + it * wc;
            WorkItem wi;
            wi.r = r;
            wi.n = (uint32_t)min((uint64_t)wc, c0 + n - s0);
            wi.c0 = s0;
            wi.inst = inst;
            wi.pad = bin == 3 ? 1u : 0u;
            a.warp_items[wbase + it] = wi;
        }
        for (unsigned long long it = 0; it < bn; ++it) {
            if (bbase + it >= a.block_item_cap) { atomicOr(&a.ctr->err, ERR_GUARD); break; }
            const uint64_t s0 = c0 + it * bc;
            WorkItem bi;
            bi.r = r;
            bi.n = (uint32_t)min((uint64_t)bc, c0 + n - s0);
            bi.c0 = s0;
            bi.inst = inst;
            bi.pad = bin == 4 ? 1u : 0u;
            a.block_items[bbase + it] = bi;
        }
    }
}

// -------------------------------------------------------------------------
// Persistent verification kernel.  Instance fields come from the device table
// (table_out), loaded once per work item or per 32-pair chunk.
// -------------------------------------------------------------------------
// MINB: CTAs per SM the registers are budgeted for (1024 / BT: 64 registers
// per thread; fewer CTAs leave more registers per thread).
template <int BT, int MINB>
__global__ void __launch_bounds__(BT, MINB) verify_kernel(VerifyArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ BlockSmem<BT> bsm;
    __shared__ uint64_t s_wbar[BT / 32];  // bulk staging: one barrier per warp for phase 2
    constexpr uint32_t kBlockWin = BT * kBlockD;
    constexpr int kWarps = BT / 32;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uint32_t n_warps_total = gridDim.x * kWarps;
    const uint32_t gwarp = blockIdx.x * kWarps + warp;
    const Instance* table = a.table_out;

    if (a.ctr->err & (ERR_OFFSETS | ERR_GUARD)) return;  // the plan is not trustworthy

    // Static first-round assignment: phase 1 takes CTAs [0, n_bs); phase 2 starts
    // on the warps after those, phase 3 on the warps after phase 2's, so a small
    // batch spreads over idle warps at once.  Later rounds are dynamic.
    const unsigned long long n_block = min(a.ctr->block_items, (unsigned long long)a.block_item_cap);
    const unsigned long long n_warp = min(a.ctr->warp_items, (unsigned long long)a.warp_item_cap);
    const uint32_t n_bs = (uint32_t)min(n_block, (unsigned long long)gridDim.x);
    const uint32_t free2 = n_bs * kWarps;
    const uint32_t slots2 = n_warps_total - free2;
    const uint32_t free3 = free2 + (uint32_t)min(n_warp, (unsigned long long)slots2);
    const uint32_t slots3 = n_warps_total - free3;

    // ---------------- phase 1: block-per-pair items ----------------------
    if (n_block) {
        uint32_t* rbuf = smem;                                // kBlockRCap + 16
        uint32_t* wr = smem + kBlockRCap + 16;                // kBlockWin + 16
        uint32_t* ws = wr + kBlockWin + 16;                   // kBlockWin + 16
        uint32_t* bm = smem;                                  // index items' probe bitmap (a.index_words)
        bool bm_zero = false;                                 // CTA-uniform: bm holds zeros only
        uint32_t r_phase = 0;                                 // bulk staging: parity of bar[0]'s next phase
        uint32_t ph[2] = {0u, 0u};                            // the same for the candidate buffers' barriers
        if (a.bulk_stage) {
            if (tid == 0)
                for (int k = 0; k < 3; ++k) mbar_init(&bsm.bar[k], 1);
            __syncthreads();
        }
        for (uint32_t round = 0;; ++round) {
            if (tid == 0) bsm.item = round == 0 ? blockIdx.x : gridDim.x + atomicAdd(&a.ctr->block_cursor, 1u);
            __syncthreads();
            const uint32_t it = bsm.item;
            __syncthreads();
            if (it >= n_block) break;
            const WorkItem bi = a.block_items[it];
            if (!in_bounds(bi.inst, a.n_inst, &a.ctr->err)) continue;  // (uniform over the CTA)
            const Instance& I = table[bi.inst];
            const uint32_t flags = I.flags;
            const bool emit_all = (flags & VF_EMIT_ALL) != 0, early = !emit_all;
            const bool self_join = (flags & VF_SELF_JOIN) != 0;
            if (!in_bounds(bi.r, I.r_n_sets, &a.ctr->err)) continue;
            const uint2 dr = I.r_desc[bi.r];
            const uint32_t nr = dr.y;
            const uint4* r4 = I.r_toks4 + dr.x;
            if (bi.pad == 1) {  // index item (uniform over the CTA)
                if (!bm_zero) {  // the bitmap shares its memory with the block-merge buffers
                    uint4* b4 = reinterpret_cast<uint4*>(bm);
                    for (uint32_t k = tid; k < a.index_words / 4; k += BT) b4[k] = make_uint4(0u, 0u, 0u, 0u);
                    __syncthreads();
                    bm_zero = true;
                }
                uint4* rings = reinterpret_cast<uint4*>(bm + a.index_words);
                index_item<BT>(I, bi, nr, r4, I.r_n_chunks - dr.x, bm, a.index_words, rings, rings + BT * kIndexRing,
                               &bsm, &a.ctr->err);
                continue;
            }
            bm_zero = false;
            const bool r_staged = nr + 4 <= kBlockRCap;
            const uint64_t rlim = I.r_n_chunks - dr.x;
            // bulk staging (a.bulk_stage): r by one bulk copy; each candidate's whole s by one bulk
            // copy into buffer m & 1 (wr / ws), issued while the previous candidate merges
            const bool bulk = a.bulk_stage && r_staged;
            uint32_t* sbuf[2] = {wr, ws};
            // thread 0: stage candidate m's s if it will be merged and fits a buffer
            auto prefetch = [&](uint32_t m) -> uint32_t {
                if (m >= bi.n || !in_bounds(bi.c0 + m, I.n_cands, &a.ctr->err)) return 0u;
                const uint32_t sx = I.cand_ids[bi.c0 + m];
                if (sx >= I.s_n_sets || (self_join && sx == bi.r)) return 0u;
                const uint2 dx = I.s_desc[sx];
                const uint32_t rq = required_overlap(I.sim, I.p, I.den, I.magic, nr, dx.y);
                if (!emit_all && (nr + dx.y == 0 || rq > min(nr, dx.y))) return 0u;
                if (dx.y == 0 || dx.y + 4 > kBlockWin + 16) return 0u;
                bulk_stage(sbuf[m & 1], I.s_toks4 + dx.x, 0u, (dx.y + 3) >> 2, I.s_n_chunks - dx.x,
                           (kBlockWin + 16) / 4, &bsm.bar[1 + (m & 1)], &a.ctr->err);
                return 1u;
            };
            if (bulk) {
                if (tid == 0) {
                    bulk_stage(rbuf, r4, 0u, (nr + 3) >> 2, rlim, (kBlockRCap + 16) / 4, &bsm.bar[0], &a.ctr->err);
                    bsm.staged[0] = prefetch(0);
                    bsm.staged[1] = 0u;
                    bsm.ok = mbar_wait(&bsm.bar[0], r_phase, &a.ctr->err) ? 1u : 0u;
                    if (!bsm.ok && bsm.staged[0]) mbar_wait(&bsm.bar[1], ph[0], &a.ctr->err);  // own copy in flight
                }
                r_phase ^= 1u;
                __syncthreads();
                if (!bsm.ok) return;  // (uniform) a copy did not complete: reported, the CTA stops
            } else if (r_staged) {
                stage<BT>(r4, 0, nr, rbuf, tid, rlim, (kBlockRCap + 16) / 4, &a.ctr->err);
                __syncthreads();
            }
            for (uint32_t m = 0; m < bi.n; ++m) {
                bool s_whole = false;
                if (bulk) {
                    // candidate m - 1 is merged (its buffer is free again); stage m + 1 into it
                    s_whole = bsm.staged[m & 1] != 0;
                    __syncthreads();
                    if (tid == 0) {
                        bsm.staged[(m + 1) & 1] = prefetch(m + 1);
                        if (s_whole) {
                            bsm.ok = mbar_wait(&bsm.bar[1 + (m & 1)], ph[m & 1], &a.ctr->err) ? 1u : 0u;
                            bsm.staged[m & 1] = 0u;  // consumed
                            if (!bsm.ok && bsm.staged[(m + 1) & 1])  // own copy in flight
                                mbar_wait(&bsm.bar[1 + ((m + 1) & 1)], ph[(m + 1) & 1], &a.ctr->err);
                        }
                    }
                    if (s_whole) ph[m & 1] ^= 1u;
                    __syncthreads();
                    if (s_whole && !bsm.ok) return;  // (uniform) reported, the CTA stops
                }
                if (!in_bounds(bi.c0 + m, I.n_cands, &a.ctr->err)) break;
                const uint32_t s = I.cand_ids[bi.c0 + m];
                if (s >= I.s_n_sets) {
                    if (tid == 0) atomicOr(&a.ctr->err, ERR_CAND_ID);
                    continue;
                }
                if (self_join && s == bi.r) continue;
                const uint2 ds = I.s_desc[s];
                const uint32_t ns = ds.y;
                const uint32_t req = required_overlap(I.sim, I.p, I.den, I.magic, nr, ns);
                if (!emit_all && (nr + ns == 0 || req > min(nr, ns))) continue;  // length filter
                bool rej;
                const uint32_t o = block_merge<BT>(r4, nr, I.s_toks4 + ds.x, ns, req, early, rbuf, r_staged, wr,
                                                   bulk ? sbuf[m & 1] : ws, s_whole, &bsm, &rej
                                                   CHK_ARGS(I.r_n_chunks - dr.x, I.s_n_chunks - ds.x, &a.ctr->err));
                const bool pass = emit_all || (!rej && o >= req);
                if (pass && tid == 0) {
                    const unsigned long long idx = atomicAdd(I.count, 1ull);
                    if (!(flags & VF_COUNT_ONLY)) emit_triple(I.out, I.cap, self_join, idx, bi.r, s, o);
                }
            }
            __syncthreads();  // rbuf reuse
            if (bulk) {
                // a copy issued for a candidate the loop did not reach (it stopped at a bad index
                // of the checked build): wait for it so the barrier phases stay in step
                const uint32_t left0 = bsm.staged[0], left1 = bsm.staged[1];
                if (tid == 0) {
                    if (left0) mbar_wait(&bsm.bar[1], ph[0], &a.ctr->err);
                    if (left1) mbar_wait(&bsm.bar[2], ph[1], &a.ctr->err);
                }
                if (left0) ph[0] ^= 1u;
                if (left1) ph[1] ^= 1u;
                __syncthreads();
            }
        }
    }

    // ---------------- phase 2: warp-per-pair items -----------------------
    if (n_warp) {
        WarpOut wout;
        uint32_t* abuf = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(smem) + warp * kWarpSliceBytes);
        uint32_t* bbuf = abuf + kWarpABuf;
        // bulk staging: the warp's own barrier (phase parity wph, warp-uniform)
        uint64_t* wbar = a.bulk_stage ? &s_wbar[warp] : nullptr;
        uint32_t wph = 0;
        if (wbar) {
            if (lane == 0) mbar_init(wbar, 1);
            __syncwarp();
        }
        for (uint32_t round = 0;; ++round) {
            uint32_t it = 0;
            if (lane == 0) {
                if (round == 0 && gwarp >= free2) it = gwarp - free2;
                else it = slots2 + atomicAdd(&a.ctr->warp_cursor, 1u);
            }
            it = __shfl_sync(kFull, it, 0);
            if (it >= n_warp) break;
            const WorkItem wi = a.warp_items[it];
            if (!in_bounds(wi.inst, a.n_inst, &a.ctr->err)) continue;  // (uniform over the warp)
            const Instance& I = table[wi.inst];
            const uint32_t flags = I.flags;
            const bool emit_all = (flags & VF_EMIT_ALL) != 0, early = !emit_all;
            const bool self_join = (flags & VF_SELF_JOIN) != 0;
            if (!in_bounds(wi.r, I.r_n_sets, &a.ctr->err)) continue;
            const uint2 dr = I.r_desc[wi.r];
            const uint32_t nr = dr.y;
            const uint4* r4 = I.r_toks4 + dr.x;
            const bool r_staged = nr + 4 <= kWarpRCap;
            if (r_staged && wbar) {  // r by one bulk copy, lane 0 waits
                uint32_t ok = 1;
                if (lane == 0) {
                    bulk_stage(abuf, r4, 0u, (nr + 3) >> 2, I.r_n_chunks - dr.x, kWarpABuf / 4, wbar, &a.ctr->err);
                    ok = mbar_wait(wbar, wph, &a.ctr->err) ? 1u : 0u;
                }
                wph ^= 1u;
                if (!__shfl_sync(kFull, ok, 0)) return;  // reported; the warp stops
                __syncwarp();
            } else if (r_staged) {
                stage<32>(r4, 0, nr, abuf, lane, I.r_n_chunks - dr.x, kWarpABuf / 4, &a.ctr->err);
                __syncwarp();
            }
            if (wi.pad == 1 && r_staged) {
                lane_item(I, wi, nr, reinterpret_cast<const uint4*>(abuf), lane, &a.ctr->err);
                __syncwarp();  // abuf reuse
                continue;
            }
            for (uint32_t m = 0; m < wi.n; ++m) {
                if (!in_bounds(wi.c0 + m, I.n_cands, &a.ctr->err)) break;
                const uint32_t s = I.cand_ids[wi.c0 + m];
                if (s >= I.s_n_sets) {
                    if (lane == 0) atomicOr(&a.ctr->err, ERR_CAND_ID);
                    continue;
                }
                if (self_join && s == wi.r) continue;
                const uint2 ds = I.s_desc[s];
                const uint32_t ns = ds.y;
                const uint32_t req = required_overlap(I.sim, I.p, I.den, I.magic, nr, ns);
                if (!emit_all && (nr + ns == 0 || req > min(nr, ns))) continue;  // length filter
                bool rej, failed;
                const uint32_t o =
                    warp_merge(r4, nr, I.s_toks4 + ds.x, ns, req, early, r_staged, abuf, bbuf, lane, wbar, &wph,
                               I.s_n_chunks - ds.x, &a.ctr->err, &failed,
                               &rej CHK_ARGS(I.r_n_chunks - dr.x, I.s_n_chunks - ds.x, &a.ctr->err));
                if (failed) return;  // (warp-uniform) reported; the warp stops
                const bool pass = emit_all || (!rej && o >= req);
                if (pass) {
                    if (flags & VF_COUNT_ONLY) {
                        if (lane == 0) atomicAdd(I.count, 1ull);
                    } else {
                        wout.push(I, lane, wi.r, s, o);
                    }
                }
            }
            wout.flush(I, lane);
            __syncwarp();  // abuf reuse
        }
    }

    // ---------------- phase 3: short pairs, one per thread ----------------
    {
        ContEntry* cont = reinterpret_cast<ContEntry*>(reinterpret_cast<char*>(smem) + warp * kWarpSliceBytes);
        uint32_t n_cont = 0;  // warp-uniform
        const unsigned long long n_pairs = min(a.ctr->thread_pairs, (unsigned long long)a.pair_cap);
        const unsigned long long n_units = (n_pairs + 32 * kFlatGrab - 1) / (32 * kFlatGrab);
        const unsigned lt_mask = (1u << lane) - 1u;
        const uint4 zero4 = make_uint4(0, 0, 0, 0);

        // Pass 2 (drain_parked): the last m parked pairs, one per lane, merged
        // while at least min_live lanes still work; the rest are parked again.
        auto drain = [&](uint32_t m, uint32_t live) {
            n_cont = drain_parked(cont, n_cont, m, live, table, a.rid, lane CHK_ERR_ARG(&a.ctr->err));
        };
        const uint32_t min_live = a.drain_min_live ? min(max(a.drain_min_live, 1u), 24u) : kDrainMinLive;

        for (uint32_t round = 0;; ++round) {
            uint32_t u = 0;
            if (lane == 0) {
                if (round == 0 && gwarp >= free3) u = gwarp - free3;
                else u = slots3 + atomicAdd(&a.ctr->chunk_cursor, 1u);
            }
            u = __shfl_sync(kFull, u, 0);
            if (u >= n_units) break;
            for (uint32_t sub = 0; sub < kFlatGrab; ++sub) {
                const unsigned long long first = ((unsigned long long)u * kFlatGrab + sub) * 32;
                if (first >= n_pairs) break;  // warp-uniform
                // the chunk's instance (uniform)
                if (!in_bounds(first / 32, a.pair_cap / 32 + 1, &a.ctr->err)) break;
                const uint32_t inst = a.chunk_inst[first / 32];
                if (!in_bounds(inst, a.n_inst, &a.ctr->err)) continue;
                const Instance& I = table[inst];
                const uint32_t flags = I.flags;
                const bool emit_all = (flags & VF_EMIT_ALL) != 0, early = !emit_all;
                const bool self_join = (flags & VF_SELF_JOIN) != 0;
                const uint32_t s_n_sets = I.s_n_sets, p = I.p, den = I.den, sim = I.sim;
                const uint64_t magic = I.magic;
                const uint4* r_toks4 = I.r_toks4;
                const uint4* s_toks4 = I.s_toks4;
                // ---- pass 1
                bool live = false;
                uint32_t pr_k = 0, ps_id = 0, nr = 0, ns = 0, req = 0;
                uint2 dr = make_uint2(0, 0), ds = make_uint2(0, 0);
                {
                    PairRef pr;
                    pr.k = kNoProbe;
                    pr.s = 0;
                    if (in_bounds(first + lane, a.pair_cap, &a.ctr->err)) pr = a.pairs[first + lane];
                    if (pr.k != kNoProbe && !in_bounds(pr.k, 32ull * a.n_tiles + 1, &a.ctr->err)) pr.k = kNoProbe;
                    if (pr.k != kNoProbe) {
                        ps_id = pr.s;
                        if (ps_id >= s_n_sets) {
                            atomicOr(&a.ctr->err, ERR_CAND_ID);
                        } else {
                            pr_k = pr.k;
                            dr = a.rdesc[pr_k];
                            ds = I.s_desc[ps_id];
                            nr = dr.y;
                            ns = ds.y;
                            // (r, r) of a self-join: non-empty sets have disjoint blocks, so
                            // equal descriptors name the same set; empty ones need the id
                            const bool same = self_join && dr.x == ds.x && nr == ns && (nr > 0 || a.rid[pr_k] == ps_id);
                            if (!same) {
                                req = required_overlap(sim, p, den, magic, nr, ns);
                                live = emit_all || (nr + ns > 0 && req <= min(nr, ns));  // length filter
                            }
                        }
                    }
                }
                uint4 r0 = zero4, r1 = zero4, r2 = zero4, s0 = zero4, s1 = zero4, s2 = zero4;
                if (live) {
                    const uint4* r4 = r_toks4 + dr.x;
                    const uint4* s4 = s_toks4 + ds.x;
                    const uint64_t rlim = I.r_n_chunks - dr.x, slim = I.s_n_chunks - ds.x;
                    if (nr > 0) r0 = ld_block(r4, 0, rlim, &a.ctr->err);
                    if (nr > 4) r1 = ld_block(r4, 1, rlim, &a.ctr->err);
                    if (nr > 8) r2 = ld_block(r4, 2, rlim, &a.ctr->err);
                    if (ns > 0) s0 = ld_block(s4, 0, slim, &a.ctr->err);
                    if (ns > 4) s1 = ld_block(s4, 1, slim, &a.ctr->err);
                    if (ns > 8) s2 = ld_block(s4, 2, slim, &a.ctr->err);
                }
                BlockState st;
                st.qi = st.qj = st.o = 0;
                st.rej = false;
                st.fin = !live || nr == 0 || ns == 0;
#pragma unroll
                for (int step = 0; step < 3; ++step) {
                    bool ar, as;
                    block_step(r0, s0, nr, ns, req, early, st, ar, as);
                    if (ar) { r0 = r1; r1 = r2; }
                    if (as) { s0 = s1; s1 = s2; }
                }
                // decided pairs
                const bool pass = live && st.fin && (emit_all || (!st.rej && st.o >= req));
                const uint32_t pmask = __ballot_sync(kFull, pass);
                if (pmask) {
                    unsigned long long b0 = 0;
                    if (lane == 0) b0 = atomicAdd(I.count, (unsigned long long)__popc(pmask));
                    if (!(flags & VF_COUNT_ONLY)) {
                        b0 = __shfl_sync(kFull, b0, 0);
                        if (pass)
                            emit_triple(I.out, I.cap, self_join, b0 + __popc(pmask & lt_mask), a.rid[pr_k], ps_id,
                                        st.o);
                    }
                }
                // undecided pairs: park them with their merge state
                const bool park = live && !st.fin;
                const uint32_t kmask = __ballot_sync(kFull, park);
                if (kmask) {
                    while (n_cont + 32 > kCont) drain(32, min_live);  // room for a full warp of parked pairs
                    if (park && in_bounds(n_cont + __popc(kmask & lt_mask), kCont, &a.ctr->err)) {
                        ContEntry* ce = cont + n_cont + __popc(kmask & lt_mask);
                        ce->m0 = make_uint4(pr_k, ps_id, dr.x + st.qi, ds.x + st.qj);
                        ce->m1 = make_uint4(nr - 4 * st.qi, ns - 4 * st.qj, req, st.o);
                        ce->m2 = make_uint4(inst, 0u, 0u, 0u);
                    }
                    n_cont += __popc(kmask);
                    __syncwarp();
                    if (n_cont >= 32) drain(32, min_live);
                }
            }
        }
        // the tail: keep refilling lanes while more than a warp is parked, then finish
        while (n_cont) drain(min(n_cont, 32u), n_cont > 32 ? min_live : 1u);
    }
}

// -------------------------------------------------------------------------
// Host side of the launch.
// -------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static uint64_t item_cap(uint64_t n_probes, uint64_t n_cands, uint32_t per_item) {
    const uint64_t cap = n_probes + (n_cands + per_item - 1) / per_item;
    return cap > 0xFFFFFFF0ull ? 0xFFFFFFF0ull : cap;
}

// Candidates per warp / block work item: small batches get one candidate
// per item so that every warp holds at most one pair of the critical path;
// large batches get up to kWarpItemCands / kBlockItemCands to bound the
// number of dynamic-scheduling atomics.  (Estimates: 32 resident warps and
// 4 resident CTAs per SM.)
static void item_sizes(uint64_t n_cands, int num_sms, uint32_t* per_warp_item, uint32_t* per_block_item,
                       uint32_t* per_lane_item, uint32_t* per_index_item) {
    const uint64_t warps = 32ull * (uint64_t)num_sms, ctas = 4ull * (uint64_t)num_sms;
    uint64_t w = n_cands / (64 * warps), b = n_cands / (64 * ctas), l = n_cands / (8 * warps);
    *per_warp_item = (uint32_t)(w < 1 ? 1 : (w > kWarpItemCands ? kWarpItemCands : w));
    *per_block_item = (uint32_t)(b < 1 ? 1 : (b > kBlockItemCands ? kBlockItemCands : b));
    l = l < 32 ? 32 : (l > kLaneItemCands ? kLaneItemCands : l);
    *per_lane_item = (uint32_t)(l & ~31ull);
    // index items: a few per CTA of the wave, at least one block's worth of candidates (never
    // fewer than a block item, so the block list's capacity covers them)
    uint64_t x = n_cands / (4 * ctas);
    x = x < 512 ? 512 : (x > kIndexItemCands ? kIndexItemCands : x);
    *per_index_item = (uint32_t)(x < *per_block_item ? *per_block_item : x);
}

static uint64_t pair_cap(const LaunchShape& sh) { return sh.total_cands + 32ull * sh.n_tiles + 32; }

LaunchShape single_shape(uint32_t n_probes, uint64_t n_cands) {
    LaunchShape sh;
    sh.n_inst = 1;
    sh.n_tiles = (n_probes + 31) / 32;
    sh.total_probes = n_probes;
    sh.total_cands = n_cands;
    return sh;
}

size_t workspace_bytes(const LaunchShape& sh, int num_sms) {
    uint32_t wc, bc, lc, ic;
    item_sizes(sh.total_cands, num_sms, &wc, &bc, &lc, &ic);
    const uint64_t slots = 32ull * sh.n_tiles + 1, pc = pair_cap(sh);
    return align256(sizeof(Counters)) + align256(sizeof(Instance) * ((size_t)sh.n_inst + 1)) +
           align256(sizeof(uint2) * slots) + align256(sizeof(uint32_t) * slots) +
           align256(sizeof(uint32_t) * (pc / 32 + 1)) + align256(sizeof(PairRef) * pc) +
           align256(sizeof(WorkItem) * ((size_t)item_cap(sh.total_probes, sh.total_cands, wc) + 1)) +
           align256(sizeof(WorkItem) * ((size_t)item_cap(sh.total_probes, sh.total_cands, bc) + 1));
}

size_t workspace_bytes(uint32_t n_probes, uint64_t n_cands, int num_sms) {
    return workspace_bytes(single_shape(n_probes, n_cands), num_sms);
}

void bind_workspace(VerifyArgs& a, void* ws, const LaunchShape& sh, int num_sms) {
    char* p = static_cast<char*>(ws);
    item_sizes(sh.total_cands, num_sms, &a.warp_item_cands, &a.block_item_cands, &a.lane_item_cands,
               &a.index_item_cands);
    const uint64_t slots = 32ull * sh.n_tiles + 1;
    a.n_inst = sh.n_inst;
    a.n_tiles = sh.n_tiles;
    a.total_probes = sh.total_probes;
    a.total_cands = sh.total_cands;
    a.ctr = reinterpret_cast<Counters*>(p);
    p += align256(sizeof(Counters));
    a.table_out = reinterpret_cast<Instance*>(p);
    p += align256(sizeof(Instance) * ((size_t)sh.n_inst + 1));
    a.rdesc = reinterpret_cast<uint2*>(p);
    p += align256(sizeof(uint2) * slots);
    a.rid = reinterpret_cast<uint32_t*>(p);
    p += align256(sizeof(uint32_t) * slots);
    a.pair_cap = pair_cap(sh);
    a.chunk_inst = reinterpret_cast<uint32_t*>(p);
    p += align256(sizeof(uint32_t) * (a.pair_cap / 32 + 1));
    a.pairs = reinterpret_cast<PairRef*>(p);
    p += align256(sizeof(PairRef) * a.pair_cap);
    a.warp_items = reinterpret_cast<WorkItem*>(p);
    a.warp_item_cap = (uint32_t)item_cap(sh.total_probes, sh.total_cands, a.warp_item_cands);
    p += align256(sizeof(WorkItem) * ((size_t)a.warp_item_cap + 1));
    a.block_items = reinterpret_cast<WorkItem*>(p);
    a.block_item_cap = (uint32_t)item_cap(sh.total_probes, sh.total_cands, a.block_item_cands);
}

void bind_workspace(VerifyArgs& a, void* ws, uint32_t n_probes, uint64_t n_cands, int num_sms) {
    bind_workspace(a, ws, single_shape(n_probes, n_cands), num_sms);
}

// Dynamic shared memory of the verify kernel: the largest of the block
// phase's buffers, the per-warp slices of phases 2 and 3, and the index
// items' probe bitmap (index_words words; it overlaps the others).
template <int BT>
static size_t verify_smem_bytes(uint32_t index_words) {
    constexpr uint32_t kBlockWin = BT * kBlockD;
    const size_t block_phase = sizeof(uint32_t) * (kBlockRCap + 16 + 2 * (kBlockWin + 16));
    const size_t warp_phases = (size_t)(BT / 32) * kWarpSliceBytes;
    // index items: the bitmap, then each thread's block ring, then each warp's candidate queue
    const size_t bitmap = index_words ? sizeof(uint32_t) * (size_t)index_words +
                                            sizeof(uint4) * ((size_t)BT * kIndexRing + (size_t)(BT / 32) * kIndexQueue)
                                      : 0;
    size_t m = block_phase > warp_phases ? block_phase : warp_phases;
    return bitmap > m ? bitmap : m;
}

// CTAs per SM of the persistent kernel for a dynamic shared-memory size, per
// device: the size attribute is raised once per device and variant to the
// largest size any launch uses, the occupancy query runs once per size
// (sizes come in 4 KiB steps above the fixed part).
template <int BT, int MINB>
static cudaError_t resident_ctas(size_t smem, int* per_sm) {
    constexpr int kMaxDev = 64;
    constexpr int kSteps = 64;
    static std::atomic<int> attr_set[kMaxDev];
    static std::atomic<int> cache[kMaxDev][kSteps];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t base = verify_smem_bytes<BT>(0);
    const size_t step = smem > base ? (smem - base + 4095) / 4096 : 0;
    const bool cacheable = dev >= 0 && dev < kMaxDev && step < (size_t)kSteps;
    if (cacheable && cache[dev][step].load() > 0) {
        *per_sm = cache[dev][step].load();
        return cudaSuccess;
    }
    if (!(dev >= 0 && dev < kMaxDev && attr_set[dev].load())) {
        const size_t most = verify_smem_bytes<BT>(kIndexMaxWords);
        e = cudaFuncSetAttribute(verify_kernel<BT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kMaxDev) attr_set[dev].store(1);
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, verify_kernel<BT, MINB>, BT, smem);
    if (e != cudaSuccess) return e;
    if (n < 1) n = 1;
    if (cacheable) cache[dev][step].store(n);
    *per_sm = n;
    return cudaSuccess;
}

template <int BT, int MINB>
static cudaError_t launch_bt(const VerifyArgs& a, cudaStream_t st, int num_sms) {
    int per_sm = 0;
    const size_t smem = verify_smem_bytes<BT>(a.index_words);
    cudaError_t e = resident_ctas<BT, MINB>(smem, &per_sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(num_sms * per_sm));
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (a.l2_base && a.l2_bytes) {
        // the collection's tokens persist in the L2 set-aside during this launch
        memset(attr, 0, sizeof(attr));
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(a.l2_base);
        attr[0].val.accessPolicyWindow.num_bytes = a.l2_bytes;
        attr[0].val.accessPolicyWindow.hitRatio = a.l2_hit_ratio;
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    e = cudaLaunchKernelEx(&cfg, verify_kernel<BT, MINB>, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// block_threads: 128, 256 or 512, optionally | kWideRegisters (the variant
// budgeted for fewer CTAs per SM, with more registers per thread: 7 of 8
// CTAs of 128 threads, 3 of 4 of 256, 1 of 2 of 512) and | kBulkStaging (a
// launch argument, not a variant).
template <class F>
static cudaError_t dispatch_variant(uint32_t block_threads, F&& f) {
    const bool wide = (block_threads & kWideRegisters) != 0;
    switch (block_threads & ~(kWideRegisters | kBulkStaging)) {
        case 128: return wide ? f.template operator()<128, 7>() : f.template operator()<128, 8>();
        case 512: return wide ? f.template operator()<512, 1>() : f.template operator()<512, 2>();
        default: return wide ? f.template operator()<256, 3>() : f.template operator()<256, 4>();
    }
}

struct PrepareVariant {
    uint32_t index_words;
    template <int BT, int MINB>
    cudaError_t operator()() const {
        int per_sm = 0;
        return resident_ctas<BT, MINB>(verify_smem_bytes<BT>(index_words), &per_sm);
    }
};

struct LaunchVariant {
    const VerifyArgs& a;
    cudaStream_t st;
    int num_sms;
    template <int BT, int MINB>
    cudaError_t operator()() const {
        return launch_bt<BT, MINB>(a, st, num_sms);
    }
};

cudaError_t prepare_verify(uint32_t block_threads, uint32_t index_words) {
    return dispatch_variant(block_threads, PrepareVariant{index_words});
}

cudaError_t launch_verify(const VerifyArgs& a, cudaStream_t st, int num_sms, uint32_t block_threads,
                          cudaEvent_t* ev) {
    cudaError_t e = cudaMemsetAsync(a.ctr, 0, sizeof(Counters), st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], st);
    if (a.n_inst == 0) {
        if (ev) {
            cudaEventRecord(ev[1], st);
            cudaEventRecord(ev[2], st);
        }
        return cudaSuccess;
    }
    // the plan kernel also runs for empty batches: it clears the instances' counts
    {
        // at most one wave of CTAs; a CTA takes up to kPlanThreads / 32 tiles per round
        static int plan_ctas_per_sm = 0;  // resident CTAs per SM (same value from every thread)
        if (plan_ctas_per_sm == 0) {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, plan_kernel, kPlanThreads, 0) != cudaSuccess || n < 1)
                n = 4;
            plan_ctas_per_sm = n;
        }
        // one tile per CTA while tiles are fewer than a wave of CTAs (a tile's candidates are copied
        // by the whole CTA, so few tiles still fill the GPU), else a wave with several tiles each
        const int threads = kPlanThreads;
        uint64_t blocks = a.n_tiles;
        const uint64_t max_blocks = (uint64_t)num_sms * (uint64_t)plan_ctas_per_sm;
        if (blocks > max_blocks) blocks = max_blocks;
        if (blocks < 1) blocks = 1;
        plan_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], st);
    VerifyArgs va = a;
    va.bulk_stage = (block_threads & kBulkStaging) ? 1u : 0u;
    e = dispatch_variant(block_threads, LaunchVariant{va, st, num_sms});
    if (ev) cudaEventRecord(ev[2], st);
    return e;
}

}  // namespace ssj
