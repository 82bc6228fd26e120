// Internal declarations shared by the host API (api.cu) and the kernels
// (verify.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ssj.h"

namespace ssj {

// Device layout of one collection (Section 3.3.1, Fig. datasetslayout):
// tokens linearised with every set starting on a 16-byte boundary so that
// sets are read with 128-bit loads; desc[i] = (first 16-byte chunk, length).
struct DevColl {
    const uint4* toks4;
    const uint2* desc;
    uint32_t n_sets;
};

// Work item for warp- or block-per-pair verification: n candidates of probe
// set r starting at candidate index c0.
struct WorkItem {
    uint32_t r;
    uint32_t n;
    uint64_t c0;
};

// One short pair of the compacted list: probe index k (into probe_ids) and
// candidate set id s.
struct PairRef {
    uint32_t k;
    uint32_t s;
};

// Per-call counters, cleared by one memset before the plan kernel.
struct Counters {
    unsigned long long thread_pairs;  // entries of the compacted short-pair list
    unsigned long long warp_items;    // warp work items written by the plan kernel
    unsigned long long block_items;   // block work items written by the plan kernel
    uint32_t block_cursor;            // dynamic cursors of the verify kernel
    uint32_t warp_cursor;
    uint32_t chunk_cursor;
    uint32_t err;                     // device-side check bits (see ssj_device_error)
};

enum : uint32_t {
    ERR_PROBE_ID = 1u,
    ERR_CAND_ID = 2u,
    ERR_OFFSETS = 4u,
    ERR_GUARD = 8u,   // an internal loop bound was reached (a bug, reported instead of hanging)
};

enum : uint32_t {
    VF_COUNT_ONLY = 1u,
    VF_EMIT_ALL = 2u,
    VF_FORCE_THREAD = 4u,
    VF_FORCE_WARP = 8u,
    VF_FORCE_BLOCK = 16u,
};


constexpr uint32_t kWarpItemCands = 8;   // most candidates per warp work item
constexpr uint32_t kBlockItemCands = 16; // most candidates per block work item
constexpr uint32_t kThreadKeyCap = 1024; // largest 2|r| verified one pair per thread

struct VerifyArgs {
    DevColl R, S;
    uint32_t p, q;
    uint32_t den;                 // p + q
    uint64_t magic;               // div_magic(p + q), for the required overlap
    uint32_t self_join;
    uint32_t flags;               // VF_*
    uint32_t n_probes;
    const uint32_t* probe_ids;
    const uint64_t* cand_offsets;
    const uint32_t* cand_ids;
    uint64_t n_cands;
    ssj_triple* out;
    uint64_t cap;
    unsigned long long* count;    // result pairs (may exceed cap)
    Counters* ctr;
    uint2* rdesc;                 // per probe: descriptor of its set r (plan output)
    PairRef* pairs;               // compacted short pairs (plan output)
    WorkItem* warp_items;
    WorkItem* block_items;
    uint32_t warp_item_cap, block_item_cap;
    uint32_t warp_item_cands, block_item_cands;  // candidates per work item
    uint32_t thread_max_key;      // 2|r| <= this: one thread per pair
    uint32_t warp_max_key;        // 2|r| <= this: one warp per pair; above: one block
};

// Scratch a call needs, in bytes, for n_probes / n_cands on a device with
// num_sms SMs.
size_t workspace_bytes(uint32_t n_probes, uint64_t n_cands, int num_sms);

// Carve the workspace and fill the scratch pointers of a.
void bind_workspace(VerifyArgs& a, void* ws, uint32_t n_probes, uint64_t n_cands, int num_sms);

// Enqueue the whole verification (counter clear, plan, verify) on st.
// ev (optional, 3 events): recorded before the plan kernel, between plan and
// verify, and after the verify kernel, on st.
cudaError_t launch_verify(const VerifyArgs& a, cudaStream_t st, int num_sms, uint32_t block_threads,
                          cudaEvent_t* ev = nullptr);

}  // namespace ssj
