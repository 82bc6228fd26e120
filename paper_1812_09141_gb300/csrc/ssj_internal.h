// Internal declarations shared by the host API (api.cu, noalloc.cu) and the
// kernels (verify.cu).  Not part of the public ABI.
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

enum : uint32_t {
    VF_COUNT_ONLY = 1u,
    VF_EMIT_ALL = 2u,
    VF_FORCE_THREAD = 4u,
    VF_FORCE_WARP = 8u,
    VF_FORCE_BLOCK = 16u,
    VF_SELF_JOIN = 32u,
    VF_FORCE_LANE = 64u,
    VF_FORCE_INDEX = 128u,
};

// One join instance of a launch: its collections, grouped candidate list,
// threshold and output.  A launch verifies any number of instances; the
// table of them lives in device memory (the workspace).
struct Instance {
    const uint4* r_toks4;
    const uint2* r_desc;
    const uint4* s_toks4;
    const uint2* s_desc;
    const uint32_t* probe_ids;
    const uint64_t* cand_offsets;
    const uint32_t* cand_ids;
    ssj_triple* out;
    unsigned long long* count;  // result pairs of this instance (may exceed cap)
    uint64_t magic;             // div_magic(den) for Jaccard and Dice
    uint64_t n_cands;
    uint64_t cap;
    uint64_t r_n_chunks, s_n_chunks;  // 16-byte blocks of the token arrays (bounds of the checked build)
    uint32_t r_n_sets, s_n_sets;
    uint32_t p, den;            // t = p / q; den: see SIM_*
    uint32_t n_probes;
    uint32_t tile_base;         // first plan tile (32 probes) of this instance
    uint32_t flags;             // VF_*
    uint32_t sim;               // SIM_*
};

// Similarity function of an instance, and what den / magic hold for it.
enum : uint32_t {
    SIM_JACCARD = 0,  // den = p + q, magic = div_magic(den)
    SIM_DICE = 1,     // den = 2q, magic = div_magic(den)
    SIM_COSINE = 2,   // den = q
    SIM_OVERLAP = 3,  // den = ceil(p / q), the required overlap itself
};

// Work item for warp-, lane- or block-per-pair verification: n candidates of
// probe set r starting at candidate index c0, in instance inst.  In the warp
// list, mode 0 is one warp per pair, mode 1 one lane per pair (r in shared
// memory).  In the block list, mode 0 is one thread block per pair, mode 1
// an index item: the whole block holds r as a bitmap over the token values
// and every thread verifies one candidate at a time against it.
struct WorkItem {
    uint32_t r;
    uint32_t n;
    uint64_t c0;
    uint32_t inst;
    uint32_t pad;  // mode
};

// One short pair of the compacted list: probe slot k (index into the
// launch's per-probe arrays) and candidate set id s.  k == kNoProbe marks a
// padding slot.
struct PairRef {
    uint32_t k;
    uint32_t s;
};
constexpr uint32_t kNoProbe = 0xFFFFFFFFu;

// Per-call counters, cleared by one memset before the plan kernel.
struct Counters {
    unsigned long long thread_pairs;  // slots of the compacted short-pair list (multiple of 32)
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
    ERR_BOUNDS = 16u, // checked build (SSJ_CHECKED): an index was out of bounds; the access was skipped
};

// The checked build (-DSSJ_CHECKED, libssj_checked.so) tests every index of
// the plan and verify kernels against its array's extent before the access;
// an index out of bounds sets ERR_BOUNDS and the access is skipped (a load
// reads zeros), so a bug shows as an error status, never as a fault.
#ifdef SSJ_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

constexpr uint32_t kWarpItemCands = 8;   // most candidates per warp work item
constexpr uint32_t kBlockItemCands = 16; // most candidates per block work item
constexpr uint32_t kLaneItemCands = 128; // most candidates per lane work item
constexpr uint32_t kLaneMinCands = 16;   // fewest candidates of a probe sent to the lane bin
constexpr uint32_t kIndexMaxWords = 24576;  // largest probe bitmap (32-bit words, 96 KiB): token values below 786,432
constexpr uint32_t kIndexItemCands = 8192;  // most candidates per index item

// Kernel arguments of one launch (passed by value).
struct VerifyArgs {
    Instance single;              // the instance of a one-batch launch (table == nullptr)
    const Instance* table;        // device table of n_inst instances, or nullptr
    Instance* table_out;          // where the plan kernel stores `single` for the verify kernel
    uint32_t n_inst;
    uint32_t n_tiles;             // plan tiles over all instances
    uint32_t total_probes;        // probe slots over all instances (instance-major)
    uint64_t total_cands;
    Counters* ctr;
    uint2* rdesc;                 // per probe slot: descriptor of its set r
    uint32_t* rid;                // per probe slot: id of its set r
    uint32_t* chunk_inst;         // per 32-slot chunk of the pair list: its instance
    PairRef* pairs;               // compacted short pairs
    WorkItem* warp_items;
    WorkItem* block_items;
    uint64_t pair_cap;
    uint32_t warp_item_cap, block_item_cap;
    uint32_t warp_item_cands, block_item_cands;  // candidates per work item
    uint32_t lane_item_cands;
    uint32_t thread_max_key;      // 2|r| <= this: one thread per pair
    uint32_t lane_max_key;        // 2|r| <= this (and r fits, >= kLaneMinCands candidates): one lane per pair
    uint32_t warp_max_key;        // 2|r| <= this: one warp per pair; above: one block
    uint32_t drain_min_live;      // short-pair pass 2 re-parks below this many live lanes (0: default 16)
    uint32_t index_words;         // probe bitmap words (every token value of the launch's collections below
                                  // 32 * index_words); 0: no index items
    uint32_t index_min_cands;     // probes with at least this many candidates become index items (0: none)
    uint32_t index_item_cands;    // candidates per index item
    uint32_t bulk_stage;          // block and warp items stage sets by bulk copies (cp.async.bulk)
    // host side only: an L2 access-policy window (persisting) for the verify kernel's launch, or none
    const void* l2_base;
    uint64_t l2_bytes;
    float l2_hit_ratio;
};

// Bitmap words for index items over collections whose token values are all
// below vocab_bound (0 when that exceeds kIndexMaxWords); a multiple of 4.
inline uint32_t index_words_for(uint64_t vocab_bound) {
    const uint64_t w = ((vocab_bound + 31) / 32 + 3) & ~3ull;
    return (w == 0 || w > kIndexMaxWords) ? 0u : (uint32_t)w;
}

// Sizes of one launch, from which the workspace is carved.
struct LaunchShape {
    uint32_t n_inst;
    uint32_t n_tiles;
    uint32_t total_probes;
    uint64_t total_cands;
};

// Scratch a launch of this shape needs, in bytes, on a device with num_sms SMs.
size_t workspace_bytes(const LaunchShape& sh, int num_sms);
// Shape of a one-batch launch.
LaunchShape single_shape(uint32_t n_probes, uint64_t n_cands);
size_t workspace_bytes(uint32_t n_probes, uint64_t n_cands, int num_sms);

// Carve the workspace and fill the scratch pointers of a.
void bind_workspace(VerifyArgs& a, void* ws, const LaunchShape& sh, int num_sms);
void bind_workspace(VerifyArgs& a, void* ws, uint32_t n_probes, uint64_t n_cands, int num_sms);

// block_threads flag selecting the verify kernel variant compiled for three
// quarters of the CTAs per SM (more registers per thread, fewer spills).
constexpr uint32_t kWideRegisters = SSJ_WIDE_REGISTERS;
// block_threads flag: block and warp items stage the sets by bulk copies.
constexpr uint32_t kBulkStaging = SSJ_BULK_STAGING;

// Set the verify kernel's launch attributes for this device (done by the
// first launch anyway; call before capturing a launch into a graph).
cudaError_t prepare_verify(uint32_t block_threads, uint32_t index_words = 0);

// Enqueue the whole verification (counter clear, plan, verify) on st.
// ev (optional, 3 events): recorded before the plan kernel, between plan and
// verify, and after the verify kernel, on st.
cudaError_t launch_verify(const VerifyArgs& a, cudaStream_t st, int num_sms, uint32_t block_threads,
                          cudaEvent_t* ev = nullptr);

// Exclusive prefix sum of n 64-bit values in place on st; *total (device)
// receives the sum.  scratch holds scan_scratch_words(n) values.
size_t scan_scratch_words(uint64_t n);
cudaError_t exclusive_scan_u64(uint64_t* data, uint64_t n, uint64_t* scratch, uint64_t* total, cudaStream_t st);

// Device candidate generation of a self-join (candgen.cu).  Scratch of the
// prefix index, sized by the caller: size_hist max_len + 2 words, order and
// rank n each, tcnt and toff vocab + 1 words each, scan_scratch
// scan_scratch_words(max(max_len + 2, vocab + 1)), total 1 word, post one
// uint4 per index entry (known after stage 0).
struct CandgenIndex {
    uint64_t* size_hist;
    uint32_t* order;
    uint32_t* rank;
    uint64_t* tcnt;
    uint64_t* toff;
    uint64_t* scan_scratch;
    uint64_t* total;
    uint4* post;
};

struct CandgenOutput {
    uint32_t* probe_ids;          // group -> probe set id
    uint64_t* cand_offsets;       // group -> first candidate
    uint32_t* cand_ids;
    unsigned long long* packed;   // groups << 40 | candidates
    uint64_t group_cap, cand_cap;
    uint32_t* err;                // ERR_GUARD if a capacity was exceeded
};

struct CandgenInput {
    const uint4* toks4;
    const uint2* desc;
    uint32_t n, max_len, vocab;   // vocab: largest token + 1
    uint32_t sim, p, q;           // SIM_*, t = p/q
    uint32_t positional;          // positional bound at the matching prefix token
    int stage;                    // 0: order + token counts; 1: lists + filtered count; 2: probe and emit
    unsigned long long* table;    // stage 2: hash set of (probe position, candidate position)
    uint64_t table_mask;          // its size - 1 (a power of two minus one)
    CandgenOutput out;
};

// Run one stage on st and wait for it; *host_word (pinned) receives stage
// 0: index entries, stage 1: entries passing the filters (an upper bound of
// the candidates), stage 2: the packed group / candidate counter.
cudaError_t candgen_run(const CandgenInput& in, cudaStream_t st, int num_sms, CandgenIndex* ix,
                        uint64_t* host_word);

// GroupJoin expansion on the device (candgen.cu).  Entries: the probe
// groups, then every group (pairs inside it).  probe_off / pair_off /
// per_probe hold n_entries + 1 words; scan_scratch
// scan_scratch_words(n_entries + 1); total one word.
struct GroupExpand {
    const uint4* toks4;
    const uint2* desc;
    uint32_t sim, p, q;
    const uint64_t* group_offsets;
    const uint32_t* members;
    const uint32_t* probe_groups;
    const uint64_t* cand_offsets;
    const uint32_t* cand_groups;
    uint32_t n_groups, n_probe_groups;
    uint64_t* probe_off;
    uint64_t* pair_off;
    uint64_t* per_probe;
    uint64_t* scan_scratch;
    uint64_t* total;
    int stage;                 // 0: count and scan; 1: write
    uint32_t* probe_ids;       // stage 1 outputs: the expanded grouped batch
    uint64_t* cand_offsets_out;
    uint32_t* cand_ids;
};

// Stage 0 waits and leaves (expanded probes, expanded pairs) in
// host_words[0..1] (pinned); stage 1 enqueues the writes (host_words[0]
// must still hold the probe count).
cudaError_t expand_groups(const GroupExpand& x, cudaStream_t st, int num_sms, uint64_t* host_words);

// One launch of the read-bandwidth probe: `passes` sweeps over bytes (a
// multiple of 16) at buf, on st; sink is a device word the kernel may write.
cudaError_t read_probe(const void* buf, uint64_t bytes, uint32_t passes, uint32_t* sink, int num_sms,
                       cudaStream_t st);

}  // namespace ssj
