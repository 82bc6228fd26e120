/*
 * ssj.h - C ABI of the GB300 verification library for exact set similarity
 * joins (Bellas & Gounaris, "Speeding-up the Verification Phase of Set
 * Similarity Joins in the GPGPU paradigm").
 *
 * Problem (Section 3, Definition): given collections R and S of token sets
 * and a threshold t, find every (r, s) in R x S with Jaccard(r, s) >= t.
 * A CPU filter (Section 2.2.3-2.2.4) emits candidate pairs; this library
 * performs the verification phase (Section 3.3) on the GPU: for each
 * candidate it intersects the two sorted token arrays by merging, stops as
 * soon as the threshold can no longer be reached (positional filter,
 * Section 2.2.3), and keeps the pair iff o*(p+q) >= p*(|r|+|s|), the exact
 * integer form of the Jaccard equivalent overlap of Table "Similarity
 * Functions" with t = p/q.
 *
 * Conventions for every call:
 *   - Every call returns an ssj_status and never aborts the process.
 *   - Unless a flag says otherwise, pointers are HOST pointers and are only
 *     read during the call.
 *   - Set ids are 0-based indices into the collection as loaded.
 *   - Tokens are uint32; each set must be strictly increasing.
 *   - The library owns every device buffer it allocates (collections,
 *     batch slots, work queues); the caller owns everything it passes in.
 *   - A context is bound to one CUDA device and is not thread-safe except
 *     where a function says so (ssj_submit / ssj_poll / ssj_results may be
 *     called from different threads).
 */
#ifndef SSJ_H
#define SSJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssj_ctx ssj_ctx;   /* opaque, owned by the library */
typedef uint32_t ssj_coll;        /* handle of a loaded collection */

/* One result pair: set ids and their exact overlap |r n s|.  For a self-join
 * r < s (the smaller id first); for R != S, r is in R and s is in S. */
typedef struct {
    uint32_t r, s, overlap;
} ssj_triple;

typedef enum {
    SSJ_OK = 0,
    SSJ_EINVAL = 1,    /* malformed argument or batch (ids, offsets, threshold, order) */
    SSJ_ENOMEM = 2,    /* device/host allocation failed, or a caller buffer is too small */
    SSJ_EAGAIN = 3,    /* no free slot or memory budget right now: retry later */
    SSJ_ETIMEDOUT = 4, /* ssj_poll: the batch did not finish within the timeout */
    SSJ_EBUSY = 5,     /* the object is in use by an in-flight batch */
    SSJ_ENOTFOUND = 6, /* unknown collection handle or ticket */
    SSJ_EDEVICE = 7    /* a CUDA call failed or a device-side check fired */
} ssj_status;

/* ------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------ */

typedef struct {
    int device;                 /* CUDA device ordinal */
    uint64_t mem_budget_bytes;  /* M_c of Table "Notation": device bytes that in-flight
                                   candidate batches (inputs, work queue, outputs) may
                                   occupy at once; 0 selects 4 GiB, the paper's default
                                   (Section 5.2) */
    uint32_t max_inflight;      /* batch slots for ssj_submit; 0 selects 4 */
    void* stream;               /* cudaStream_t used by the synchronous calls; NULL
                                   makes the library create its own */
    uint32_t flags;             /* SSJ_CTX_PROFILE or 0 */
} ssj_config;

#define SSJ_CTX_PROFILE 0x1u    /* record CUDA events around the kernels of every synchronous
                                   or stream-ordered verification (see ssj_profile_read) */

/* Create a context on config->device.  *out receives the handle.
 * Errors: SSJ_EINVAL (NULL arguments, unknown flags, bad device),
 * SSJ_EDEVICE (CUDA initialisation failed). */
ssj_status ssj_create(const ssj_config* config, ssj_ctx** out);

/* Wait for in-flight batches, free every device buffer and the context.
 * NULL is accepted and ignored. */
void ssj_destroy(ssj_ctx* ctx);

/* Text of the last error raised on this context (never NULL, "" when
 * there was none).  The string stays valid until the next failing call on
 * the context. */
const char* ssj_last_error(ssj_ctx* ctx);

/* ------------------------------------------------------------------------
 * Collections (Section 3.3.1, Fig. datasetslayout: all tokens linearised in
 * one array plus an offsets array delimiting the sets, copied to the device
 * once).
 * ------------------------------------------------------------------------ */

#define SSJ_RENUMBER_BY_FREQ 0x1u  /* replace tokens by their rank in ascending global
                                      frequency, ties by token value (Section 2.2.1), and
                                      re-sort each set; results are unchanged, only the
                                      device layout is.  Self-joins only: a batch whose R
                                      and S differ rejects renumbered collections. */
#define SSJ_VALIDATE 0x2u          /* check that every set is strictly increasing */
#define SSJ_PIN_L2 0x4u            /* keep the token array L2-resident (Section 3.3.1: the
                                      collection is copied once and read by every batch):
                                      the context's persisting-L2 set-aside is raised to
                                      the array's size (up to the device's maximum; a limit
                                      of this context only, restored when the last pinned
                                      collection is unloaded) and every verification launch
                                      that reads the collection carries a persisting
                                      access-policy window over it (for a launch over
                                      several collections: the first pinned one) */

/* Load a collection of n_sets sets.  offsets (n_sets+1 entries, host) are
 * nondecreasing with offsets[0] = 0; set i is tokens[offsets[i] ..
 * offsets[i+1]) (host).  n_sets is below 2^31 and each set must hold
 * fewer than 2^31 tokens.
 * The data are copied; the caller may free them on return.
 * Device layout: tokens padded so that every set starts on a 16-byte
 * boundary (the padding repeats the set's last token), plus one 8-byte (start, length)
 * descriptor per set.  Empty sets are allowed and never match.
 * Errors: SSJ_EINVAL (NULL pointers, decreasing offsets, unsorted set with
 * SSJ_VALIDATE, unknown flag, n_sets of 2^31 or more), SSJ_ENOMEM, SSJ_EDEVICE. */
ssj_status ssj_load_collection(ssj_ctx* ctx, const uint64_t* offsets, const uint32_t* tokens,
                               uint32_t n_sets, uint32_t flags, ssj_coll* out);

/* Free a collection.  SSJ_EBUSY if a submitted batch that uses it has not
 * been collected with ssj_results; SSJ_ENOTFOUND for an unknown handle. */
ssj_status ssj_unload_collection(ssj_ctx* ctx, ssj_coll coll);

/* Number of sets and of (unpadded) tokens of a loaded collection. */
ssj_status ssj_collection_info(ssj_ctx* ctx, ssj_coll coll, uint32_t* n_sets, uint64_t* n_tokens);

/* ------------------------------------------------------------------------
 * Candidate batches (Section 3.3.1, Fig. candidatesoutputlayout: the ids of
 * candidate sets C, delimited per probe set by offsets C_O).
 * ------------------------------------------------------------------------ */

#define SSJ_COUNT_ONLY 0x1u     /* only count result pairs (aggregation on top of the join,
                                   Section 3.2, "output count") */
#define SSJ_SORTED 0x2u         /* return triples sorted by (r, s) */
#define SSJ_DEVICE_PTRS 0x4u    /* probe_ids, cand_offsets, cand_ids and the output array are
                                   DEVICE pointers (same device as the context), each aligned to
                                   its element size (4 bytes for ids and triples, 8 for
                                   cand_offsets and counts; SSJ_EINVAL otherwise) */
#define SSJ_EMIT_ALL 0x8u       /* diagnostic: emit every listed pair (except self pairs of a
                                   self-join) with its exact overlap, no threshold test and no
                                   early termination */
#define SSJ_FORCE_THREAD 0x10u  /* verify every pair with one thread (Alternative A/B style) */
#define SSJ_FORCE_WARP 0x20u    /* verify every pair with one warp (merge path over 32 lanes) */
#define SSJ_FORCE_BLOCK 0x40u   /* verify every pair with one thread block (Alternative C) */
#define SSJ_FORCE_LANE 0x80u    /* verify every pair with one lane, the probe set held in the
                                   warp's shared memory (Alternative B); probes longer than
                                   1,020 tokens go to the warp path */
#define SSJ_FORCE_INDEX 0x2000u /* verify every pair with one thread against the probe set held
                                   as a bitmap over the token values in the thread block's
                                   shared memory (index items, see ssj_set_index_items); where
                                   the collections' token values reach 786,432 or more, the
                                   lane path instead */

/* Similarity function (Table "Similarity Functions", Section 2.2.2), in the
 * flags' bits 8-9; t = p/q.  Each pair is kept iff its overlap o reaches the
 * function's equivalent overlap, tested exactly in integers:
 *   Jaccard  o / (|r|+|s|-o) >= t   <=>  o (p+q) >= p (|r|+|s|)    (default)
 *   Dice     2o / (|r|+|s|) >= t    <=>  2 q o >= p (|r|+|s|)
 *   Cosine   o / sqrt(|r||s|) >= t  <=>  (q o)^2 >= p^2 |r| |s|
 *   Overlap  o >= t                 <=>  q o >= p   (p may exceed q)
 * The positional early termination uses the same equivalent overlap. */
#define SSJ_SIM_JACCARD 0x000u
#define SSJ_SIM_DICE 0x100u
#define SSJ_SIM_COSINE 0x200u
#define SSJ_SIM_OVERLAP 0x300u
#define SSJ_SIM_MASK 0x300u
#define SSJ_KEEP_INPUTS 0x800u      /* ssj_submit: the caller keeps pinned host inputs unchanged
                                       until the ticket is done, so the call does not wait for
                                       their host-to-device copies (ignored for pageable inputs) */
#define SSJ_HOST_DIRECT 0x1000u     /* ssj_verify_batches: host arrays in pinned memory that the
                                       device can address are read by the kernels directly over
                                       the host link (NVLink-C2C on Grace systems) instead of
                                       being copied first; other arrays (pageable, or off
                                       their element alignment) are copied.  Calls of
                                       2^25 or more candidates do this by default */
#define SSJ_HOST_STAGED 0x4000u     /* ssj_verify_batches: copy this batch's pinned inputs to the
                                       device before the kernels run, even in a large call */
#define SSJ_JOIN_POSITIONAL 0x400u  /* ssj_self_join: drop a candidate at a matching prefix token
                                       when min(i, j) + 1 + min(|r|-i-1, |s|-j-1) (i, j: the token's
                                       positions) is below the pair's equivalent overlap */

typedef struct {
    ssj_coll R, S;                /* R == S: self-join */
    uint32_t p, q;                /* threshold t = p/q, 0 < p <= q < 2^31 (SSJ_SIM_OVERLAP:
                                     0 < p, q < 2^31); Jaccard unless flags select another function */
    uint32_t n_probes;            /* below 2^31 (SSJ_EINVAL otherwise) */
    const uint32_t* probe_ids;    /* n_probes ids into R */
    const uint64_t* cand_offsets; /* n_probes+1 nondecreasing offsets, cand_offsets[0] = 0 */
    const uint32_t* cand_ids;     /* cand_offsets[n_probes] ids into S; probe k is paired with
                                     cand_ids[cand_offsets[k] .. cand_offsets[k+1]) */
    uint64_t n_cands;             /* cand_offsets[n_probes], below 2^40 (also summed over the
                                     batches of one call or prepared launch).  Required with
                                     SSJ_DEVICE_PTRS (the host does not read device offsets; the
                                     device checks it); with host pointers 0 means "take it from
                                     cand_offsets" */
    uint32_t flags;               /* SSJ_COUNT_ONLY | SSJ_SORTED | SSJ_DEVICE_PTRS | ... | SSJ_SIM_* */
} ssj_batch;

/*
 * Verify one batch synchronously.
 * Semantics: every listed pair is verified; a self-join skips pairs whose
 * two ids are equal and reports (min id, max id).  Pairs are not
 * deduplicated: each listed pair yields at most one triple.  Without
 * SSJ_SORTED the triple order is unspecified.
 * out / cap: room for cap triples (host memory, or device memory with
 * SSJ_DEVICE_PTRS); may be NULL with cap = 0 to query the count.
 * *n_out receives the number of result pairs.  If it exceeds cap, only the
 * first cap are written (which ones is unspecified unless SSJ_SORTED) and
 * SSJ_ENOMEM is returned.  With SSJ_COUNT_ONLY nothing is written to out.
 * Errors: SSJ_EINVAL (bad threshold, id out of range, decreasing offsets,
 * renumbered collections in an R != S batch), SSJ_ENOTFOUND, SSJ_ENOMEM,
 * SSJ_EDEVICE.
 */
ssj_status ssj_verify_batch(ssj_ctx* ctx, const ssj_batch* batch, ssj_triple* out, uint64_t cap,
                            uint64_t* n_out);

/*
 * Verify n_batches host batches (independent joins: own collections,
 * thresholds, functions) synchronously in batched launches: one plan and
 * one verify kernel cover every batch of a group.  A call with fewer than
 * 2^25 candidates is one group, its inputs copied to the device first.  A
 * larger call is cut into two consecutive groups of batches with about
 * equal candidate counts (one group if it holds a single batch): its inputs in pinned host memory are read by the
 * kernels directly over the host link (SSJ_HOST_DIRECT) unless a batch sets
 * SSJ_HOST_STAGED, and the inputs that are copied are copied for the second
 * group on a second stream while the first group's kernels run.  Then the
 * counts and results come back.  outs[i] / caps[i]: host room for batch i's
 * triples; n_outs[i] receives its result count.  Host pointers
 * only (SSJ_DEVICE_PTRS is rejected; see ssj_multi_create for device
 * batches).  Flags per batch as for ssj_verify_batch.  If a count exceeds
 * its cap, the first caps[i] triples are written and SSJ_ENOMEM is returned
 * after every batch is done.  Errors as for ssj_verify_batch.
 */
ssj_status ssj_verify_batches(ssj_ctx* ctx, const ssj_batch* batches, uint32_t n_batches, ssj_triple* const* outs,
                              const uint64_t* caps, uint64_t* n_outs);

/*
 * Enqueue the verification of a batch on `stream` (a cudaStream_t, or NULL
 * for the context's stream) and return without waiting.  All batch arrays,
 * d_out (cap triples) and d_count (one uint64, receives the number of
 * result pairs, which may exceed cap) are DEVICE pointers that must stay
 * valid until the stream reaches this work; SSJ_DEVICE_PTRS is implied
 * (with its alignment rule: d_count 8 bytes, d_out 4).
 * The work queue is taken from the context's workspace, which grows (with
 * a device allocation) only when a batch is larger than any before; call
 * ssj_reserve first to keep allocations out of a timed or captured region.
 * Calls on the same context must not overlap on different streams, since
 * they share the workspace.  Invalid ids or offsets are detected on the
 * device: the affected pairs are skipped and ssj_device_error reports it.
 */
ssj_status ssj_verify_batch_async(ssj_ctx* ctx, const ssj_batch* batch, ssj_triple* d_out,
                                  uint64_t cap, uint64_t* d_count, void* stream);

/*
 * Same verification as ssj_verify_batch_async, for callers that cannot let
 * the library allocate device memory during a call: callers whose device
 * memory all goes through their own arena or a framework's caching
 * allocator, and callers on latency-critical paths where cudaMalloc or
 * cudaFree may synchronise the device and stall unrelated streams.  The
 * paper has no counterpart to this entry point.
 * It never allocates: the work queue lives in a fixed 32 MiB block of device
 * memory that belongs to the loaded library (every GPU that loads the
 * library holds it until the process exits).  A batch whose work queue
 * would need more is rejected with SSJ_EINVAL and a message (roughly
 * 800,000 candidates for small batches; split larger batches).  The caller
 * passes every input and output as device memory, as for
 * ssj_verify_batch_async (SSJ_DEVICE_PTRS is implied).
 * Every call looks up the scratch block's device address with the
 * context's device current (so no address outlives a device reset); the
 * first call on a device may also load the library's device code, so make
 * that first call before any stream capture.  A NULL stream means the
 * context's stream, as for ssj_verify_batch_async.  All calls share the
 * one block and it keeps the last call's contents (the counters that must
 * start at zero are cleared on the stream by each call), so calls whose
 * work overlaps on the GPU race:
 * issue them on one stream, or wait for one before starting the next.
 * Device-side checks are read with ssj_device_error.
 */
ssj_status ssj_verify_batch_noalloc(ssj_ctx* ctx, const ssj_batch* batch, ssj_triple* d_out, uint64_t cap,
                                    uint64_t* d_count, void* stream);

/* ------------------------------------------------------------------------
 * Self-join with candidate generation on the device (the paper's future
 * work, Section 6: the filtering phase on the GPU as well)
 * ------------------------------------------------------------------------ */

/*
 * Join a loaded collection with itself at threshold t = p/q (flags may
 * select the similarity function, SSJ_SIM_*): the prefix filter and
 * inverted-index probing of algorithm ALL (Sections 2.2.3, 2.2.4, 3.1) run
 * on the device (sets ordered by size; each set's prefix indexed; each
 * probe matched against the earlier sets' prefix entries that pass the
 * length filter, SSJ_JOIN_POSITIONAL adding the positional bound;
 * candidates deduplicated), then the candidates are verified by the same
 * launch as ssj_verify_batch, without a host round trip.  The candidates
 * are those of the CPU feeder (ssj_feeder.h) for the same function and
 * threshold.  Results as for ssj_verify_batch of a self-join: (min id, max
 * id, overlap) triples in the caller's ids, to out (host memory, or device
 * memory with SSJ_DEVICE_PTRS), at most cap; *n_out receives the count
 * (SSJ_ENOMEM if it exceeds cap), *n_candidates (may be NULL) the number
 * of candidates verified.  Flags: SSJ_SIM_*, SSJ_JOIN_POSITIONAL,
 * SSJ_COUNT_ONLY, SSJ_SORTED, SSJ_DEVICE_PTRS, SSJ_FORCE_*.  Token values
 * must stay below 2^30 (load with SSJ_RENUMBER_BY_FREQ, which the prefix
 * filter wants anyway).  Allocates its scratch (the prefix index, a hash
 * set of candidate pairs and the candidate list) for the call.
 * Errors: SSJ_EINVAL, SSJ_ENOTFOUND, SSJ_ENOMEM, SSJ_EDEVICE.
 */
ssj_status ssj_self_join(ssj_ctx* ctx, ssj_coll coll, uint32_t p, uint32_t q, uint32_t flags, ssj_triple* out,
                         uint64_t cap, uint64_t* n_out, uint64_t* n_candidates);

/* ------------------------------------------------------------------------
 * GroupJoin: group candidates (ssj_groups_create in ssj_feeder.h) expanded
 * and verified on the device (the paper's GroupJoin split, Section 4.1.3,
 * leaves the expanded pairs to the host; here the whole verification runs
 * on the device)
 * ------------------------------------------------------------------------ */

typedef struct {
    ssj_coll coll;                  /* self-join of this collection (ids are its set ids) */
    uint32_t p, q;                  /* threshold, as for ssj_batch */
    uint32_t flags;                 /* SSJ_SIM_*, SSJ_COUNT_ONLY, SSJ_SORTED, SSJ_DEVICE_PTRS (out only), SSJ_FORCE_* */
    uint32_t n_groups;
    const uint64_t* group_offsets;  /* n_groups + 1, host; group g holds members[group_offsets[g] ..
                                       group_offsets[g+1]), every group non-empty */
    const uint32_t* members;        /* set ids, host */
    uint32_t n_probe_groups;
    const uint32_t* probe_groups;   /* host group ids */
    const uint64_t* cand_offsets;   /* n_probe_groups + 1, host, from 0 */
    const uint32_t* cand_groups;    /* host group ids */
} ssj_group_batch;

/*
 * Expand the groups on the device into member pairs (every member of probe
 * group k against every member of its candidate groups, and every pair of
 * members inside a group whose prefix for this threshold is not empty) and
 * verify them with the launch of ssj_verify_batch.  Results as for a
 * self-join batch: to out (host, or device with SSJ_DEVICE_PTRS), at most
 * cap, *n_out the count (SSJ_ENOMEM above cap), *n_pairs (may be NULL) the
 * expanded pairs verified.  Errors: SSJ_EINVAL (layout or ids), SSJ_ENOTFOUND,
 * SSJ_ENOMEM, SSJ_EDEVICE.
 */
ssj_status ssj_verify_groups(ssj_ctx* ctx, const ssj_group_batch* gb, ssj_triple* out, uint64_t cap, uint64_t* n_out,
                             uint64_t* n_pairs);

/* ------------------------------------------------------------------------
 * Batched instances: many independent joins in one launch
 * ------------------------------------------------------------------------ */

typedef struct ssj_multi ssj_multi;  /* opaque, owned by the library */

/*
 * Prepare one launch that verifies n_batches independent batches (each with
 * its own collections and threshold) together: one plan kernel and one
 * persistent verify kernel whose work queue is binned by |r|+|s| across all
 * instances (the granularity rule of Section 5.4 applied per probe).
 * All batch arrays are DEVICE pointers (SSJ_DEVICE_PTRS is implied) and each
 * batch's n_cands is required.  Batch i writes up to caps[i] triples to
 * d_outs[i] (device) and its result count to d_counts[i] (a device array of
 * n_batches uint64); d_outs and caps are host arrays read here.
 * The workspace is allocated and the instance table uploaded here, once; the
 * arrays' contents may change between launches, their addresses and sizes
 * may not.  Collections used by a prepared launch cannot be unloaded until
 * it is destroyed.  Errors: SSJ_EINVAL (a batch is invalid, see
 * ssj_verify_batch), SSJ_ENOTFOUND, SSJ_ENOMEM, SSJ_EDEVICE.
 */
ssj_status ssj_multi_create(ssj_ctx* ctx, const ssj_batch* batches, uint32_t n_batches, ssj_triple* const* d_outs,
                            const uint64_t* caps, uint64_t* d_counts, ssj_multi** out);

/* Enqueue the prepared launch on `stream` (NULL: the context's stream):
 * a counter clear, the plan kernel and the verify kernel.  Allocates
 * nothing and reads no host memory.  Launches of one ssj_multi must not
 * overlap on the GPU (they share its workspace). */
ssj_status ssj_multi_launch(ssj_ctx* ctx, ssj_multi* m, void* stream);

/* Same work through a CUDA graph: the first call captures the launch into a
 * graph owned by m (on an internal stream), every call then launches that
 * graph on `stream`. */
ssj_status ssj_multi_graph_launch(ssj_ctx* ctx, ssj_multi* m, void* stream);

/* Free a prepared launch (waits for its work). NULL is ignored. */
void ssj_multi_destroy(ssj_ctx* ctx, ssj_multi* m);

typedef struct {
    uint32_t thread_max_key;  /* chosen bins (see ssj_set_granularity); 0xFFFFFFFF */
    uint32_t lane_max_key;    /*   for warp_max_key sends no probe to the block bin, */
    uint32_t warp_max_key;    /*   lane_max_key <= thread_max_key means no lane bin */
    uint32_t block_threads;   /* chosen block size (the block path's window is 8 steps per thread),
                                 | SSJ_WIDE_REGISTERS for the wide-register variant,
                                 | SSJ_BULK_STAGING for bulk-copy staging */
    uint32_t drain_min_live;  /* short pairs still merging that keep a warp on them before the rest
                                 are parked again and lanes refilled (8 .. 24) */
    uint32_t settings_tried;  /* distinct settings timed */
    float best_ms;            /* median device time of one launch with the chosen setting */
    float initial_ms;         /* the same for the setting m had before the call */
    uint32_t index_min_cands; /* chosen index-item threshold (0: no index items) */
} ssj_tune_result;

/*
 * Autotune the granularity of a prepared launch on its own inputs: time
 * (CUDA events on `stream`, NULL: the context's stream; median of reps >= 3
 * launches after one untimed launch each) settings of the thread, lane and
 * warp bins' upper keys, of the block size and of the short-pair refill
 * threshold (drain_min_live), by coordinate descent
 * and of the index-item threshold (ssj_set_index_items)
 * from m's current setting, and keep the fastest in m (later launches, and
 * graphs captured later, use it).  Every setting computes the same results
 * (Section 3.3.2 Alternatives A-C differ in speed only, Section 5.4); the
 * outputs and counts of m hold those of the last timed launch.  Synchronises
 * the stream.  Errors: SSJ_EINVAL, SSJ_EDEVICE (a launch failed or the
 * device-side batch checks fired).
 */
ssj_status ssj_multi_autotune(ssj_ctx* ctx, ssj_multi* m, void* stream, uint32_t reps, ssj_tune_result* out);

/* Size the workspace for batches of up to n_probes probes and n_cands
 * candidates (device allocation happens here, not in later calls).
 * Errors: SSJ_EINVAL (n_probes of 2^31 or more, n_cands of 2^40 or more),
 * SSJ_ENOMEM. */
ssj_status ssj_reserve(ssj_ctx* ctx, uint32_t n_probes, uint64_t n_cands);

/* Read and clear the device-side error word of the last stream-ordered or
 * synchronous verification (synchronises the context's stream; call it
 * only after that stream has seen the work).  *code = 0 when no check fired;
 * bit 0: probe id out of range, bit 1: candidate id out of range, bit 2:
 * offsets decreasing or past the candidate array, bit 3: an internal loop
 * bound was reached (a library bug, reported instead of hanging), bit 4:
 * (libssj_checked.so, the build with -DSSJ_CHECKED, only) an index of the
 * plan or verify kernels was out of its array's bounds and the access was
 * skipped (a library bug, reported instead of faulting). */
ssj_status ssj_device_error(ssj_ctx* ctx, uint32_t* code);

/* ------------------------------------------------------------------------
 * Serving: continuous batching (Section 3.2, Fig. executionoverlap: the
 * filtering thread keeps producing chunks while the device verifies earlier
 * ones; a chunk is admitted when device memory M_c allows).
 * ------------------------------------------------------------------------ */

/*
 * Admit a batch.  Host inputs are copied to the device before the call
 * returns (pinned arrays straight from the caller's memory, pageable ones
 * through the slot's pinned staging), so the caller may reuse its arrays at
 * once; with SSJ_KEEP_INPUTS the caller instead keeps pinned arrays
 * unchanged until the ticket is done and the call does not wait for their
 * copies (with SSJ_DEVICE_PTRS the caller keeps the arrays alive until
 * ssj_poll reports done).
 * The batch runs on its own stream, overlapping with other admitted
 * batches.  Returns SSJ_EAGAIN when every slot is busy or the batch does not
 * fit the remaining memory budget; SSJ_EINVAL when it could never fit.
 * *ticket identifies the batch for ssj_poll / ssj_results.
 * Thread-safe with respect to ssj_poll and ssj_results.
 */
ssj_status ssj_submit(ssj_ctx* ctx, const ssj_batch* batch, uint64_t* ticket);

/* Wait up to timeout_ms (0: just test, <0: forever) for a ticket.  *done is
 * 1 when its results are ready.  SSJ_ETIMEDOUT when the wait ran out,
 * SSJ_ENOTFOUND for an unknown or collected ticket. */
ssj_status ssj_poll(ssj_ctx* ctx, uint64_t ticket, int timeout_ms, int* done);

/* Collect a finished ticket.  out == NULL: only report the count in *n_out
 * and keep the ticket.  Otherwise copy min(count, cap) triples to out
 * (host), set *n_out to the count and release the ticket and its slot;
 * SSJ_ENOMEM (ticket kept) if cap < count.  SSJ_EAGAIN if not finished. */
ssj_status ssj_results(ssj_ctx* ctx, uint64_t ticket, ssj_triple* out, uint64_t cap,
                       uint64_t* n_out);

/* ------------------------------------------------------------------------
 * Tuning and measurement
 * ------------------------------------------------------------------------ */

/* For a context created with SSJ_CTX_PROFILE: wait for the verifications
 * launched since the last read and return how many there were and the
 * summed device time of their plan kernels and of their verify kernels
 * (milliseconds, CUDA events recorded on each launch's stream).  Batches
 * run through ssj_submit are not recorded.  SSJ_EINVAL without the flag. */
ssj_status ssj_profile_read(ssj_ctx* ctx, uint32_t* launches, double* plan_ms, double* verify_ms);

/* Granularity bins keyed by |r|+|s| (estimated per probe as 2|r|, since the
 * length filter keeps |s| within [t|r|, |r|/t]): a probe whose key is <=
 * thread_max_key is verified one pair per thread; <= lane_max_key, with
 * |r| <= 1,020 and at least 16 candidates, one pair per lane with r held in
 * the warp's shared memory (Alternative B of Section 3.3.2); <= warp_max_key
 * one pair per warp; otherwise one pair per thread block (the rule of
 * Section 5.4: per-thread work for small sets, cooperative Intersect Path
 * for large ones).  Defaults 128, 2048, 2048; any values are valid (every
 * granularity verifies pairs of any length), they change the speed only;
 * lane_max_key <= thread_max_key leaves the lane bin empty.
 * block_threads is 128, 256 or 512 (default 256), optionally
 * | SSJ_WIDE_REGISTERS for the verify kernel compiled for fewer CTAs per SM
 * (7 instead of 8 of 128 threads, 3 instead of 4 of 256, 1 instead of 2 of
 * 512: more registers per thread, fewer spills) and
 * | SSJ_BULK_STAGING (below).  Zero leaves a value unchanged. */
ssj_status ssj_set_granularity(ssj_ctx* ctx, uint32_t thread_max_key, uint32_t lane_max_key, uint32_t warp_max_key,
                               uint32_t block_threads);
#define SSJ_WIDE_REGISTERS 0x10000u
/* block_threads flag: thread-block and warp items stage their sets in shared
 * memory by one-dimensional bulk copies on the copy engine (cp.async.bulk,
 * completion counted on an mbarrier) instead of 16-byte loads by every
 * thread: the probe set once per item; for thread-block items each
 * candidate's whole set (when it fits the window buffer) while the previous
 * candidate merges; for warp items each merge window of the candidate. */
#define SSJ_BULK_STAGING 0x20000u

/* Index items of later launches of the context (prepared launches take the
 * value at ssj_multi_create; ssj_multi_autotune tunes it per launch): a probe
 * with at least min_cands candidates is verified by a whole thread block
 * that holds the probe set r as a bitmap over the token values in shared
 * memory (one bit per value: the launch's token values must stay below
 * 786,432, which frequency renumbering gives for vocabularies of that size;
 * otherwise the probe keeps its other granularity).  Every thread then
 * merges one candidate s at a time from s's side, each token of s tested
 * against r by one bit lookup, with the positional bound on s's remainder
 * after every 16-byte block (Sections 2.2.3, 3.1; r's tokens are read once
 * per probe instead of once per pair).  0 turns index items off; the
 * default is 256.  Every value computes the same results. */
ssj_status ssj_set_index_items(ssj_ctx* ctx, uint32_t min_cands);

/* Short-pair refill threshold of later launches of the context (prepared
 * launches take it at ssj_multi_create; ssj_multi_autotune tunes it per
 * launch).  Pairs verified one per thread are merged three block steps each,
 * then the undecided ones are parked in shared memory and merged by full
 * warps that park them again once fewer than drain_min_live (1 .. 24) lanes
 * are still merging, refilling the lanes from later pairs.  0 restores the
 * default (16).  Every value computes the same results.  Errors: SSJ_EINVAL. */
ssj_status ssj_set_short_pairs(ssj_ctx* ctx, uint32_t drain_min_live);

/* Measurement aid (the paper has no counterpart): device read bandwidth in
 * GB/s (1e9 bytes/s), streaming a zero-filled device buffer of `bytes`
 * (rounded down to a multiple of 16; allocated and freed here) `passes` times
 * in one kernel launch with 128-bit loads cached in L2 only, after one
 * warm-up pass, timed with CUDA events on the context's stream.  A buffer well below the L2 size
 * gives the L2 read rate that bounds token reads from a resident collection
 * (the L2-aware roofline); one well above it the HBM read rate.
 * Errors: SSJ_EINVAL, SSJ_ENOMEM, SSJ_EDEVICE. */
ssj_status ssj_read_bandwidth(ssj_ctx* ctx, uint64_t bytes, uint32_t passes, double* gbs);

#ifdef __cplusplus
}
#endif

#endif /* SSJ_H */
