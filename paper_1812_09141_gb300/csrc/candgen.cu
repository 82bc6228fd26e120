// Candidate generation on the device for a self-join: the prefix filter and
// inverted-index probing of algorithm ALL (Sections 2.2.3, 2.2.4, 3.1),
// which the paper leaves on the CPU and names as future work (Section 6).
// The candidates come out in the grouped (probe ids, offsets, candidate ids)
// layout of a device batch, so verification follows without a host round trip.
//
// Steps, on one stream:
//   1. order the sets by size (counting sort; ties in any order: the set of
//      unordered candidate pairs does not depend on it);
//   2. index every set's prefix: per token, the entries (position in that
//      order, position of the token in the set, set size, set id), by a
//      count / scan / scatter over the prefix tokens;
//   3. count, per probe, the index entries that can yield a candidate (an
//      earlier set in the order, passing the length filter), to size a hash
//      table and the output;
//   4. one warp per probe walks its prefix tokens' entries, keeps those of
//      earlier sets that pass the length filter (and optionally the
//      positional bound of the matching token, PPJoin-style), deduplicates
//      (probe, candidate) with a hash set of 64-bit keys, and appends the new
//      candidates to the output through a per-warp buffer; one atomic on a
//      packed (groups, candidates) counter reserves a group and its range, so
//      the group offsets are contiguous in group order.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "arith.h"
#include "ssj_internal.h"

namespace ssj {
namespace {

constexpr int kGenWarps = 8;             // warps per CTA of the probing kernel
constexpr uint32_t kGenBuf = 256;        // candidates buffered per warp before a flush
constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr uint64_t kEmpty = ~0ull;

struct Params {
    const uint4* toks4;
    const uint2* desc;
    uint32_t n;
    uint32_t sim, p, q;     // sim: SIM_*; t = p/q
    uint32_t positional;    // apply the positional bound at the matching token
};

__device__ __forceinline__ const uint32_t* set_tokens(const Params& P, uint2 d) {
    return reinterpret_cast<const uint32_t*>(P.toks4 + d.x);
}

// Least overlap a set of size len shares with any partner that can reach t
// (Jaccard t|x|, Dice t|x|/(2-t), Cosine t^2|x|, plain overlap t, rounded
// up); also the smallest partner size the length filter admits.
__device__ __forceinline__ uint64_t min_overlap(const Params& P, uint32_t len) {
    const uint64_t p = P.p, q = P.q;
    switch (P.sim) {
        case SIM_DICE: return ((uint64_t)len * p + (2 * q - p) - 1) / (2 * q - p);
        case SIM_COSINE: {  // p^2 len needs 128 bits
            const unsigned __int128 d = (unsigned __int128)q * q;
            return (uint64_t)(((unsigned __int128)p * p * len + d - 1) / d);
        }
        case SIM_OVERLAP: return (p + q - 1) / q;
        default: return ((uint64_t)len * p + q - 1) / q;
    }
}

// Prefix of len - min_overlap + 1 tokens (none if no partner can reach t).
__device__ __forceinline__ uint32_t prefix_len(const Params& P, uint32_t len) {
    if (len == 0) return 0;
    const uint64_t need = min_overlap(P, len);
    if (need > len) return 0;
    const uint64_t pl = (uint64_t)len + 1 - need;
    return pl > len ? len : (uint32_t)pl;
}

// Equivalent overlap of a pair (for the positional bound).
__device__ __forceinline__ uint32_t pair_required(const Params& P, uint32_t nr, uint32_t ns) {
    switch (P.sim) {
        case SIM_DICE: return required_overlap_magic(nr, ns, P.p, 2 * P.q, div_magic(2ull * P.q));
        case SIM_COSINE: return required_overlap_cosine(P.p, P.q, nr, ns);
        case SIM_OVERLAP: return (uint32_t)(((uint64_t)P.p + P.q - 1) / P.q);
        default: return required_overlap_magic(nr, ns, P.p, P.p + P.q, div_magic((uint64_t)P.p + P.q));
    }
}

__global__ void size_hist_kernel(Params P, uint64_t* hist) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(hist + P.desc[i].y), 1ull);
}

__global__ void place_kernel(Params P, uint64_t* cursor, uint32_t* order, uint32_t* rank) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const uint32_t pos =
            (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + P.desc[i].y), 1ull);
        order[pos] = i;
        rank[i] = pos;
    }
}

// one warp per set: count its prefix tokens per token
__global__ void token_count_kernel(Params P, uint64_t* tcnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < P.n; i += warps) {
        const uint2 d = P.desc[i];
        const uint32_t* t = set_tokens(P, d);
        const uint32_t pl = prefix_len(P, d.y);
        for (uint32_t a = lane; a < pl; a += 32) atomicAdd(reinterpret_cast<unsigned long long*>(tcnt + t[a]), 1ull);
    }
}

// one warp per set: its prefix entries into the token lists
__global__ void postings_kernel(Params P, const uint32_t* rank, uint64_t* tcur, uint4* post) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < P.n; i += warps) {
        const uint2 d = P.desc[i];
        const uint32_t* t = set_tokens(P, d);
        const uint32_t pl = prefix_len(P, d.y);
        const uint32_t pos = rank[i];
        for (uint32_t a = lane; a < pl; a += 32) {
            const uint64_t slot = atomicAdd(reinterpret_cast<unsigned long long*>(tcur + t[a]), 1ull);
            post[slot] = make_uint4(pos, a, d.y, i);
        }
    }
}

// Does index entry e (a set at position e.x, token position e.y, size e.z)
// matched at probe token position a yield a candidate of the probe at
// position rpos with size L?
__device__ __forceinline__ bool entry_ok(const Params& P, uint4 e, uint32_t rpos, uint32_t L, uint64_t min_size,
                                         uint32_t a) {
    if (e.x >= rpos || e.z < min_size) return false;  // earlier sets only; length filter
    if (P.positional) {
        // at most min(a, j) matches before this one, one here, min(|r|-a-1, |s|-j-1) after
        const uint32_t ub = min(a, e.y) + 1 + min(L - a - 1, e.z - e.y - 1);
        if (ub < pair_required(P, L, e.z)) return false;
    }
    return true;
}

// one warp per probe position: entries that pass entry_ok, summed per warp
__global__ void precount_kernel(Params P, const uint32_t* order, const uint64_t* toff, const uint4* post,
                                unsigned long long* total) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long mine = 0;
    for (uint32_t rpos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; rpos < P.n; rpos += warps) {
        const uint32_t r = order[rpos];
        const uint2 d = P.desc[r];
        const uint32_t* t = set_tokens(P, d);
        const uint32_t L = d.y, pl = prefix_len(P, L);
        const uint64_t min_size = min_overlap(P, L);
        for (uint32_t a = 0; a < pl; ++a) {
            const uint32_t tok = t[a];
            for (uint64_t e = toff[tok] + lane; e < toff[tok + 1]; e += 32)
                mine += entry_ok(P, post[e], rpos, L, min_size, a) ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(kAll, mine, o);
    if (lane == 0 && mine) atomicAdd(total, mine);
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Insert key; true if it was not there.  The table has a power-of-two size
// at least twice the number of keys ever inserted, so a free slot is always
// found within the table.  Should the probe loop ever run through the whole
// table (a sizing bug), the key cannot be stored: ERR_GUARD is set, so the
// call fails with SSJ_EDEVICE instead of losing the candidate silently.
__device__ __forceinline__ bool hash_insert(unsigned long long* table, uint64_t mask, uint64_t key, uint32_t* err) {
    uint64_t h = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(table + h, (unsigned long long)kEmpty, (unsigned long long)key);
        if (prev == kEmpty) return true;
        if (prev == key) return false;
        h = (h + 1) & mask;
    }
    atomicOr(err, ERR_GUARD);
    return false;
}

struct GenOut {
    uint32_t* probe_ids;           // per group: probe set id
    uint64_t* cand_offsets;        // per group: first candidate (the final entry is written last)
    uint32_t* cand_ids;
    unsigned long long* packed;    // groups << 40 | candidates
    uint64_t group_cap, cand_cap;
    uint32_t* err;
};

__global__ void __launch_bounds__(kGenWarps * 32) generate_kernel(Params P, const uint32_t* order,
                                                                  const uint64_t* toff, const uint4* post,
                                                                  unsigned long long* table, uint64_t mask,
                                                                  GenOut O) {
    __shared__ uint32_t buf[kGenWarps][kGenBuf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t* b = buf[warp];
    for (uint32_t rpos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; rpos < P.n; rpos += warps) {
        const uint32_t r = order[rpos];
        const uint2 d = P.desc[r];
        const uint32_t* t = set_tokens(P, d);
        const uint32_t L = d.y, pl = prefix_len(P, L);
        const uint64_t min_size = min_overlap(P, L);
        uint32_t nb = 0;  // buffered candidates (warp-uniform)
        auto flush = [&]() {
            unsigned long long old = 0;
            if (lane == 0) old = atomicAdd(O.packed, (1ull << 40) | (unsigned long long)nb);
            old = __shfl_sync(kAll, old, 0);
            const uint64_t g = old >> 40, start = old & ((1ull << 40) - 1);
            if (g >= O.group_cap || start + nb > O.cand_cap) {  // cannot happen with sized outputs
                if (lane == 0) atomicOr(O.err, ERR_GUARD);
            } else {
                if (lane == 0) {
                    O.probe_ids[g] = r;
                    O.cand_offsets[g] = start;
                }
                for (uint32_t k = lane; k < nb; k += 32) O.cand_ids[start + k] = b[k];
            }
            __syncwarp();
            nb = 0;
        };
        for (uint32_t a = 0; a < pl; ++a) {
            const uint32_t tok = t[a];
            const uint64_t e0 = toff[tok], e1 = toff[tok + 1];
            for (uint64_t base = e0; base < e1; base += 32) {
                const uint64_t e = base + lane;
                bool fresh = false;
                uint32_t sid = 0;
                if (e < e1) {
                    const uint4 en = post[e];
                    if (entry_ok(P, en, rpos, L, min_size, a)) {
                        fresh = hash_insert(table, mask, ((uint64_t)rpos << 32) | en.x, O.err);
                        sid = en.w;
                    }
                }
                const unsigned fm = __ballot_sync(kAll, fresh);
                if (fresh) b[nb + __popc(fm & lt)] = sid;
                nb += __popc(fm);
                __syncwarp();
                if (nb > kGenBuf - 32) flush();
            }
        }
        if (nb) flush();
    }
}

// ---------------------------------------------------------------------------
// GroupJoin expansion: entry k < n_probe_groups is a probe group with its
// candidate groups (every member of the probe group against every member of
// those groups); entry n_probe_groups + g is group g itself (each member
// against the later members, when the group's prefix is not empty).
// ---------------------------------------------------------------------------

struct GroupArgs {
    const uint64_t* group_offsets;
    const uint32_t* members;
    const uint32_t* probe_groups;
    const uint64_t* cand_offsets;
    const uint32_t* cand_groups;
    uint32_t n_groups, n_probe_groups;
};

// one warp per entry: probes, pairs and (inter entries) candidates per probe
__global__ void group_count_kernel(Params P, GroupArgs G, uint64_t* n_probes, uint64_t* n_pairs, uint64_t* per_probe) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n_entries = G.n_probe_groups + G.n_groups;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_entries; k += warps) {
        uint64_t probes = 0, pairs = 0, sum = 0;
        if (k < G.n_probe_groups) {
            const uint32_t g = G.probe_groups[k];
            const uint64_t m = G.group_offsets[g + 1] - G.group_offsets[g];
            for (uint64_t c = G.cand_offsets[k] + lane; c < G.cand_offsets[k + 1]; c += 32) {
                const uint32_t h = G.cand_groups[c];
                sum += G.group_offsets[h + 1] - G.group_offsets[h];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o);
            probes = sum ? m : 0;
            pairs = m * sum;
        } else {
            const uint32_t g = k - G.n_probe_groups;
            const uint64_t b = G.group_offsets[g], m = G.group_offsets[g + 1] - b;
            if (m >= 2 && prefix_len(P, P.desc[G.members[b]].y) > 0) {
                probes = m - 1;
                pairs = m * (m - 1) / 2;
            }
        }
        if (lane == 0) {
            n_probes[k] = probes;
            n_pairs[k] = pairs;
            per_probe[k] = sum;
        }
    }
}

// one warp per entry: write the expanded probes, offsets and candidates
__global__ void group_write_kernel(GroupArgs G, const uint64_t* probe_off, const uint64_t* pair_off,
                                   const uint64_t* per_probe, uint32_t* probe_ids, uint64_t* cand_offsets,
                                   uint32_t* cand_ids) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n_entries = G.n_probe_groups + G.n_groups;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_entries; k += warps) {
        const uint64_t p0 = probe_off[k], np = probe_off[k + 1] - p0, c0 = pair_off[k];
        if (np == 0) continue;
        if (k < G.n_probe_groups) {
            const uint32_t g = G.probe_groups[k];
            const uint64_t b = G.group_offsets[g], S = per_probe[k];
            for (uint64_t i = 0; i < np; ++i) {
                if (lane == 0) {
                    probe_ids[p0 + i] = G.members[b + i];
                    cand_offsets[p0 + i] = c0 + i * S;
                }
                uint64_t w = c0 + i * S;  // the candidate groups' members, in order
                for (uint64_t c = G.cand_offsets[k]; c < G.cand_offsets[k + 1]; ++c) {
                    const uint32_t h = G.cand_groups[c];
                    const uint64_t hb = G.group_offsets[h], hm = G.group_offsets[h + 1] - hb;
                    for (uint64_t j = lane; j < hm; j += 32) cand_ids[w + j] = G.members[hb + j];
                    w += hm;
                }
            }
        } else {
            const uint32_t g = k - G.n_probe_groups;
            const uint64_t b = G.group_offsets[g], m = G.group_offsets[g + 1] - b;
            for (uint64_t i = 0; i < np; ++i) {
                const uint64_t w = c0 + i * (2 * m - i - 1) / 2;  // pairs of the members before i
                if (lane == 0) {
                    probe_ids[p0 + i] = G.members[b + i];
                    cand_offsets[p0 + i] = w;
                }
                for (uint64_t j = i + 1 + lane; j < m; j += 32) cand_ids[w + (j - i - 1)] = G.members[b + j];
            }
        }
    }
}

unsigned grid_for(uint64_t work, unsigned per_block, int num_sms, unsigned per_sm) {
    const uint64_t want = (work + per_block - 1) / per_block;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms * per_sm));
}

}  // namespace

cudaError_t candgen_run(const CandgenInput& in, cudaStream_t st, int num_sms, CandgenIndex* ix, uint64_t* host_word) {
    Params P;
    P.toks4 = in.toks4;
    P.desc = in.desc;
    P.n = in.n;
    P.sim = in.sim;
    P.p = in.p;
    P.q = in.q;
    P.positional = in.positional;
    cudaError_t e;
    const unsigned tb = 256;
    if (in.stage == 0) {
        // order by size, then count prefix tokens
        e = cudaMemsetAsync(ix->size_hist, 0, 8ull * (in.max_len + 2), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ix->tcnt, 0, 8ull * (in.vocab + 1), st);
        if (e != cudaSuccess) return e;
        if (in.n) {
            size_hist_kernel<<<grid_for(in.n, tb, num_sms, 8), tb, 0, st>>>(P, ix->size_hist);
            e = exclusive_scan_u64(ix->size_hist, in.max_len + 2, ix->scan_scratch, ix->total, st);
            if (e != cudaSuccess) return e;
            place_kernel<<<grid_for(in.n, tb, num_sms, 8), tb, 0, st>>>(P, ix->size_hist, ix->order, ix->rank);
            token_count_kernel<<<grid_for(32ull * in.n, tb, num_sms, 8), tb, 0, st>>>(P, ix->tcnt);
        }
        e = cudaMemcpyAsync(ix->toff, ix->tcnt, 8ull * (in.vocab + 1), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = exclusive_scan_u64(ix->toff, in.vocab + 1, ix->scan_scratch, ix->total, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_word, ix->total, 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(st);  // *host_word: index entries
    }
    if (in.stage == 1) {
        // fill the token lists, then count the entries that can yield candidates
        e = cudaMemcpyAsync(ix->tcnt, ix->toff, 8ull * (in.vocab + 1), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ix->total, 0, 8, st);
        if (e != cudaSuccess) return e;
        if (in.n) {
            postings_kernel<<<grid_for(32ull * in.n, tb, num_sms, 8), tb, 0, st>>>(P, ix->rank, ix->tcnt, ix->post);
            precount_kernel<<<grid_for(32ull * in.n, tb, num_sms, 8), tb, 0, st>>>(
                P, ix->order, ix->toff, ix->post, reinterpret_cast<unsigned long long*>(ix->total));
        }
        e = cudaMemcpyAsync(host_word, ix->total, 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(st);  // *host_word: entries passing the filters
    }
    // stage 2: probe, deduplicate and emit
    e = cudaMemsetAsync(in.table, 0xFF, 8ull * (in.table_mask + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(in.out.packed, 0, 8, st);
    if (e != cudaSuccess) return e;
    if (in.n) {
        GenOut O;
        O.probe_ids = in.out.probe_ids;
        O.cand_offsets = in.out.cand_offsets;
        O.cand_ids = in.out.cand_ids;
        O.packed = in.out.packed;
        O.group_cap = in.out.group_cap;
        O.cand_cap = in.out.cand_cap;
        O.err = in.out.err;
        generate_kernel<<<grid_for(32ull * in.n, kGenWarps * 32, num_sms, 4), kGenWarps * 32, 0, st>>>(
            P, ix->order, ix->toff, ix->post, in.table, in.table_mask, O);
    }
    e = cudaMemcpyAsync(host_word, in.out.packed, 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);  // *host_word: groups << 40 | candidates
}

cudaError_t expand_groups(const GroupExpand& x, cudaStream_t st, int num_sms, uint64_t* host_words) {
    Params P;
    memset(&P, 0, sizeof(P));
    P.toks4 = x.toks4;
    P.desc = x.desc;
    P.sim = x.sim;
    P.p = x.p;
    P.q = x.q;
    GroupArgs G;
    G.group_offsets = x.group_offsets;
    G.members = x.members;
    G.probe_groups = x.probe_groups;
    G.cand_offsets = x.cand_offsets;
    G.cand_groups = x.cand_groups;
    G.n_groups = x.n_groups;
    G.n_probe_groups = x.n_probe_groups;
    const uint64_t n_entries = (uint64_t)x.n_groups + x.n_probe_groups;
    const unsigned tb = 256;
    cudaError_t e;
    if (x.stage == 0) {
        e = cudaMemsetAsync(x.probe_off + n_entries, 0, 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(x.pair_off + n_entries, 0, 8, st);
        if (e != cudaSuccess) return e;
        if (n_entries)
            group_count_kernel<<<grid_for(32 * n_entries, tb, num_sms, 8), tb, 0, st>>>(P, G, x.probe_off, x.pair_off,
                                                                                         x.per_probe);
        e = exclusive_scan_u64(x.probe_off, n_entries + 1, x.scan_scratch, x.total, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_words, x.total, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = exclusive_scan_u64(x.pair_off, n_entries + 1, x.scan_scratch, x.total, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_words + 1, x.total, 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(st);  // host_words: expanded probes, expanded pairs
    }
    if (n_entries)
        group_write_kernel<<<grid_for(32 * n_entries, tb, num_sms, 8), tb, 0, st>>>(G, x.probe_off, x.pair_off,
                                                                                     x.per_probe, x.probe_ids,
                                                                                     x.cand_offsets_out, x.cand_ids);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // closing offset: the total number of pairs
    return cudaMemcpyAsync(x.cand_offsets_out + host_words[0], x.pair_off + n_entries, 8, cudaMemcpyDeviceToDevice, st);
}

}  // namespace ssj
