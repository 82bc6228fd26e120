/*
 * ssj_serve.h - native drivers of the serving path (ssj_submit / ssj_poll /
 * ssj_results in ssj.h): an open-loop request replayer that measures batch
 * latency under continuous batching, and the filter/verify co-process of
 * Section 3.2 (Fig. executionoverlap), where the CPU filter keeps producing
 * candidate chunks while the GPU verifies earlier ones.
 */
#ifndef SSJ_SERVE_H
#define SSJ_SERVE_H

#include <stdint.h>

#include "ssj.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One request: a host batch (layout of ssj_batch) and its arrival time in
 * seconds from the start of the replay. */
typedef struct {
    ssj_batch batch;      /* host pointers; flags may hold SSJ_COUNT_ONLY */
    double arrival_s;
} ssj_request;

typedef struct {
    double wall_s;        /* first arrival to last completion */
    uint64_t pairs;       /* candidate pairs of all requests */
    uint64_t results;     /* result pairs returned */
    uint32_t eagain;      /* submissions refused for lack of a slot or budget (then retried) */
    uint32_t max_inflight;/* most requests admitted at once */
} ssj_serve_stats;

/*
 * Replay n requests against ctx.  A submitter thread waits for each arrival
 * time, then submits the request (queueing it on the client side and
 * retrying while the library answers SSJ_EAGAIN, requests kept in arrival
 * order); a collector thread polls admitted tickets and collects their
 * results.  latency_s (n entries, host) receives, per request, the time
 * from its arrival to the moment its results were collected.  Requests are
 * admitted while slots and the memory budget allow, so their work overlaps
 * on the device (continuous batching).  Returns the first error of a
 * request, or SSJ_OK.
 */
ssj_status ssj_serve_replay(ssj_ctx* ctx, const ssj_request* reqs, uint32_t n, double* latency_s,
                            ssj_serve_stats* stats);

typedef struct {
    double filter_only_s;   /* the CPU filter run alone (candidates produced and dropped) */
    double join_s;          /* filter and verification overlapped, to the last result */
    double gpu_busy_s;      /* sum over chunks of submit-to-done time */
    uint64_t candidates;    /* candidate pairs verified */
    uint64_t results;       /* result pairs */
    uint32_t chunks;        /* chunks submitted */
} ssj_coprocess_stats;

/*
 * Self-join of a host collection with the CPU filter (ssj_feeder.h, n_threads
 * worker threads) feeding the GPU in chunks of at most chunk_cands
 * candidates, as in Section 3.2: the filter thread builds a chunk and hands
 * it to the device (ssj_submit) while it builds the next; finished chunks
 * are collected by another thread.  coll is the same collection loaded in
 * ctx.  Also times the filter alone, so that join_s can be compared with
 * filter_only_s (the paper's Table overlap reports that the join time falls
 * to the filtering time once verification is hidden).
 */
ssj_status ssj_serve_coprocess(ssj_ctx* ctx, ssj_coll coll, const uint64_t* offsets, const uint32_t* tokens,
                               uint32_t n_sets, uint32_t p, uint32_t q, uint32_t n_threads, uint64_t chunk_cands,
                               ssj_coprocess_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* SSJ_SERVE_H */
