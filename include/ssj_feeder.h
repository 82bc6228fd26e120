/*
 * ssj_feeder.h - CPU candidate generation for a self-join or an R x S join
 * (Jaccard, Dice, Cosine or a plain overlap threshold), the
 * filtering half of the paper's filter-verification framework (thread H0 of
 * Section 3.2) that feeds the GPU verification in include/ssj.h.
 *
 * Algorithm ALL (AllPairs, Section 3.1) as an index nested loop
 * (Section 2.2.4): tokens are renumbered by ascending frequency and sets
 * ordered by (size, lexicographic) (Section 2.2.1); each probe looks up its
 * prefix tokens in the inverted index of the sets before it (prefix filter,
 * Section 2.2.3), keeps those that pass the length filter, deduplicates
 * them, and is then added to the index.  The prefix of a set x is its first
 * |x| - ceil(t|x|) + 1 tokens; every set s that reaches Jaccard t with a
 * probe r (|s| <= |r|) shares a token with r inside both prefixes, so no
 * result pair is lost.
 *
 * Output is the grouped batch layout of ssj_batch (Section 3.3.1): probe ids,
 * candidate offsets, candidate ids, all in the caller's original set ids.
 * Candidates of one probe are contiguous; a probe whose list does not fit
 * the remaining room of a chunk continues in the next chunk (its id then
 * appears in both).
 */
#ifndef SSJ_FEEDER_H
#define SSJ_FEEDER_H

#include <stdint.h>

#include "ssj.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssj_feeder ssj_feeder;

/* Prepare a self-join of n_sets sets (host offsets / tokens as for
 * ssj_load_collection; copied) at Jaccard t = p/q, 0 < p <= q < 2^31.
 * n_threads > 1 generates candidates of consecutive probe ranges in
 * parallel (results identical to one thread).
 * Errors: SSJ_EINVAL (bad threshold or offsets, unsorted set),
 * SSJ_ENOMEM. */
ssj_status ssj_feeder_create(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets, uint32_t p,
                             uint32_t q, uint32_t n_threads, ssj_feeder** out);

#define SSJ_FEEDER_PPJOIN 0x1u  /* PPJoin's positional filter at candidate time: a candidate
                                   is dropped once the prefix matches found so far plus
                                   1 + min(|r|-i-1, |s|-j-1) (i, j: positions of the current
                                   common prefix token) fall below the pair's equivalent
                                   overlap; fewer candidates, the same join */

typedef struct {
    uint32_t sim;        /* 0 Jaccard, 1 Dice, 2 Cosine, 3 plain overlap (SSJ_SIM_* >> 8) */
    uint32_t p, q;       /* threshold t = p/q, as for ssj_batch */
    uint32_t flags;      /* SSJ_FEEDER_PPJOIN */
    uint32_t n_threads;  /* worker threads (results identical to one) */
} ssj_feeder_opts;

/* General form.  s_offsets == NULL: self-join of R, as ssj_feeder_create.
 * Otherwise an R x S join: every set of S is indexed (prefixes as below,
 * one token order for both collections, renumbered by their joint
 * frequency), and each set r of R, in id order, is probed against it with
 * the two-sided length filter (a partner's size lies where the threshold is
 * reachable) and the prefix filter; probe ids are ids of R, candidate ids
 * ids of S.  Errors: SSJ_EINVAL, SSJ_ENOMEM. */
ssj_status ssj_feeder_create_ex(const uint64_t* r_offsets, const uint32_t* r_tokens, uint32_t n_r,
                                const uint64_t* s_offsets, const uint32_t* s_tokens, uint32_t n_s,
                                const ssj_feeder_opts* opts, ssj_feeder** out);

/* The same for another similarity function of Table "Similarity Functions"
 * (sim: 0 Jaccard, 1 Dice, 2 Cosine, 3 plain overlap o >= p/q; the values
 * of SSJ_SIM_* shifted right by 8).  The prefix of a set x is its first
 * |x| - a + 1 tokens, where a is the least overlap x shares with any
 * partner that can reach t (t|x|, t|x|/(2-t), t^2|x| or t, rounded up),
 * and a probe r keeps indexed sets of at least a(|r|) tokens (the length
 * filter).  Thresholds as for ssj_batch. */
ssj_status ssj_feeder_create_sim(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets, uint32_t sim,
                                 uint32_t p, uint32_t q, uint32_t n_threads, ssj_feeder** out);

/* Fill the next chunk: at most max_probes entries in probe_ids (and
 * max_probes+1 in cand_offsets) and at most max_cands candidate ids
 * (max_probes >= 1, max_cands >= 1).  *n_probes and *n_cands receive the
 * chunk's size; *done becomes 1 once every probe has been emitted (the
 * chunk may still hold data).  SSJ_EINVAL for NULL arrays or zero limits. */
ssj_status ssj_feeder_next(ssj_feeder* f, uint32_t max_probes, uint64_t max_cands, uint32_t* probe_ids,
                           uint64_t* cand_offsets, uint32_t* cand_ids, uint32_t* n_probes, uint64_t* n_cands,
                           int* done);

/* Total candidates emitted so far, and probes processed out of n_sets. */
ssj_status ssj_feeder_progress(ssj_feeder* f, uint64_t* n_cands, uint32_t* probed, uint32_t* n_sets);

void ssj_feeder_destroy(ssj_feeder* f);

/* ------------------------------------------------------------------------
 * GroupJoin candidates (the GRP algorithm of the paper's evaluation): sets
 * of equal size and equal prefix form a group, filtering and indexing work
 * on groups, and a candidate group pair stands for every pair of their
 * members; ssj_verify_groups (ssj.h) expands them on the device.
 * ------------------------------------------------------------------------ */

typedef struct ssj_groups ssj_groups;

/* Group the n_sets sets (host offsets / tokens as for ssj_feeder_create;
 * copied) and generate group candidates of a self-join for opts->sim,
 * opts->p / opts->q (opts->flags must be 0, n_threads is ignored).
 * Groups are formed in (size, lexicographic) order of the frequency-
 * renumbered sets; group k's members are set ids; probe group k is paired
 * with the earlier groups that share a prefix token and pass the length
 * filter.  The member pairs the groups stand for (every pair of a probe
 * group's member with a candidate group's member, and every pair inside a
 * group with a non-empty prefix) are exactly algorithm ALL's candidates.
 * Errors: SSJ_EINVAL, SSJ_ENOMEM. */
ssj_status ssj_groups_create(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets,
                             const ssj_feeder_opts* opts, ssj_groups** out);

/* Sizes: groups, probe groups, candidate group entries, and the member pairs
 * they stand for.  Any pointer may be NULL. */
ssj_status ssj_groups_info(ssj_groups* g, uint32_t* n_groups, uint32_t* n_probe_groups, uint64_t* n_cand_groups,
                           uint64_t* n_pairs);

/* Copy the groups out (host arrays): group_offsets (n_groups + 1, into
 * members), members (n_sets set ids), probe_groups (n_probe_groups group
 * ids), cand_offsets (n_probe_groups + 1), cand_groups (n_cand_groups
 * group ids). */
ssj_status ssj_groups_copy(ssj_groups* g, uint64_t* group_offsets, uint32_t* members, uint32_t* probe_groups,
                           uint64_t* cand_offsets, uint32_t* cand_groups);

void ssj_groups_destroy(ssj_groups* g);

#ifdef __cplusplus
}
#endif

#endif /* SSJ_FEEDER_H */
