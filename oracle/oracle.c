/*
 * CPU oracle for the verification phase of exact set similarity joins
 * (Bellas & Gounaris, "Speeding-up the Verification Phase of Set Similarity
 * Joins in the GPGPU paradigm").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the test suite, the smoke check and the
 * bench's CPU-baseline leg and reference arm do.  It shares no code, header or table with the
 * CUDA library.
 *
 * Plain, single-threaded, slow on purpose: every function is the textbook
 * definition or the paper's step written out, in exact integer arithmetic.
 * The Jaccard threshold t is the exact rational p/q (0 < p <= q); products
 * are formed in unsigned 128-bit so no size/threshold combination overflows.
 *
 * The same steps serve the Dice and Cosine functions of Table "Similarity
 * Functions" and the plain overlap threshold (the *_sim entry points); the
 * Jaccard entry points are those with sim = 0.
 *
 * Pins (see tests/test_oracle_pins.py and tests/test_oracle_sim_pins.py):
 * the worked example of Section 2.2.2
 * (two 10-token sets at Jaccard 0.8 need overlap 9), the closed-form
 * equivalence with the ceiling formula of Table "Similarity Functions" in
 * exact rationals, Python set intersection, brute force against the
 * prefix-filter join, and the invariants (symmetry, monotonicity in t,
 * overlap <= min size, renumbering and id permutation).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------
 * Similarity test.
 * ------------------------------------------------------------------------ */

/*
 * Jaccard's equivalent overlap, Table "Similarity Functions" (Section 2.2.2):
 * ceil(t/(1+t) * (|r|+|s|)).  With t = p/q, t/(1+t) = p/(p+q), so this is
 * ceil(p*(|r|+|s|) / (p+q)), computed exactly.
 */
uint64_t oracle_required_overlap(uint64_t nr, uint64_t ns, uint64_t p, uint64_t q) {
    u128 num = (u128)p * (u128)(nr + ns);
    u128 den = (u128)p + (u128)q;
    return (uint64_t)((num + den - 1) / den);
}

/*
 * Jaccard similarity |r n s| / |r u s| >= t (Table "Similarity Functions";
 * the problem definition of Section 3).  With o = |r n s| and
 * |r u s| = |r|+|s|-o, the test o/(|r|+|s|-o) >= p/q is, after multiplying
 * out the (positive) denominators, q*o >= p*(|r|+|s|-o), i.e.
 * o*(p+q) >= p*(|r|+|s|).  An empty union (both sets empty) never matches.
 */
int oracle_jaccard_pass(uint64_t o, uint64_t nr, uint64_t ns, uint64_t p, uint64_t q) {
    if (nr + ns == 0) return 0;
    return (u128)o * ((u128)p + (u128)q) >= (u128)p * (u128)(nr + ns);
}

/*
 * Length filter (Section 2.2.3): a pair can only pass if
 * t*|r| <= |s| <= |r|/t, i.e. p*|r| <= q*|s| and p*|s| <= q*|r|.
 */
int oracle_length_ok(uint64_t nr, uint64_t ns, uint64_t p, uint64_t q) {
    return (u128)p * nr <= (u128)q * ns && (u128)p * ns <= (u128)q * nr;
}

/* ------------------------------------------------------------------------
 * The other normalized similarity functions of Table "Similarity
 * Functions" (Section 2.2.2), and the plain overlap threshold, all with
 * t = p/q exact.  sim: 0 Jaccard, 1 Dice, 2 Cosine, 3 Overlap (o >= t).
 * ------------------------------------------------------------------------ */

enum { ORACLE_SIM_JACCARD = 0, ORACLE_SIM_DICE = 1, ORACLE_SIM_COSINE = 2, ORACLE_SIM_OVERLAP = 3 };

/*
 * The similarity of two sets with sizes nr, ns and overlap o reaches t:
 *   Jaccard  o / (nr + ns - o) >= t   (oracle_jaccard_pass)
 *   Dice     2o / (nr + ns) >= t      <=>  2*q*o >= p*(nr+ns)
 *   Cosine   o / sqrt(nr*ns) >= t     <=>  (q*o)^2 >= p^2*nr*ns   (o >= 0)
 *   Overlap  o >= t                   <=>  q*o >= p
 * An empty denominator (empty sets) never matches.  Products fit in 128
 * bits for sizes below 2^32 and p, q below 2^31.
 */
int oracle_sim_pass(int sim, uint64_t o, uint64_t nr, uint64_t ns, uint64_t p, uint64_t q) {
    switch (sim) {
        case ORACLE_SIM_JACCARD:
            return oracle_jaccard_pass(o, nr, ns, p, q);
        case ORACLE_SIM_DICE:
            if (nr + ns == 0) return 0;
            return (u128)2 * q * o >= (u128)p * (nr + ns);
        case ORACLE_SIM_COSINE: {
            if (nr == 0 || ns == 0) return 0;
            u128 lhs = (u128)q * o;
            return lhs * lhs >= (u128)p * p * nr * ns;
        }
        case ORACLE_SIM_OVERLAP:
            return (u128)q * o >= (u128)p;
        default:
            return 0;
    }
}

/* Smallest y with y*y >= x (x < 2^126), by bisection over 64-bit y. */
static uint64_t ceil_sqrt_u128(u128 x) {
    uint64_t lo = 0, hi = (uint64_t)1 << 63;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if ((u128)mid * mid >= x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/*
 * Equivalent overlap (Table "Similarity Functions"): the least o that
 * reaches the threshold for sizes nr, ns.
 *   Jaccard  ceil(p(nr+ns) / (p+q))
 *   Dice     ceil(t(nr+ns)/2)        = ceil(p(nr+ns) / (2q))
 *   Cosine   ceil(t sqrt(nr ns))     = ceil(ceil(sqrt(p^2 nr ns)) / q)
 *   Overlap  ceil(t)                 = ceil(p / q)
 * (For Cosine, q*o >= sqrt(X) with X = p^2 nr ns holds iff q*o >= ceil(sqrt(X)).)
 */
uint64_t oracle_required_overlap_sim(int sim, uint64_t nr, uint64_t ns, uint64_t p, uint64_t q) {
    switch (sim) {
        case ORACLE_SIM_JACCARD:
            return oracle_required_overlap(nr, ns, p, q);
        case ORACLE_SIM_DICE: {
            u128 num = (u128)p * (nr + ns), den = (u128)2 * q;
            return (uint64_t)((num + den - 1) / den);
        }
        case ORACLE_SIM_COSINE: {
            uint64_t y = ceil_sqrt_u128((u128)p * p * nr * ns);
            return (y + q - 1) / q;
        }
        case ORACLE_SIM_OVERLAP:
            return (p + q - 1) / q;
        default:
            return ~(uint64_t)0;
    }
}

/*
 * Length filter (Section 2.2.3) of each function: the size ratio bounds
 * under which the threshold is reachable at all (o <= min(nr, ns)).
 *   Jaccard  t nr <= ns <= nr / t                (oracle_length_ok)
 *   Dice     t/(2-t) nr <= ns <= (2-t)/t nr      <=>  p nr <= (2q-p) ns, p ns <= (2q-p) nr
 *   Cosine   t^2 nr <= ns <= nr / t^2            <=>  p^2 nr <= q^2 ns, p^2 ns <= q^2 nr
 *   Overlap  min(nr, ns) >= t                    <=>  q min(nr, ns) >= p
 */
int oracle_length_ok_sim(int sim, uint64_t nr, uint64_t ns, uint64_t p, uint64_t q) {
    switch (sim) {
        case ORACLE_SIM_JACCARD:
            return oracle_length_ok(nr, ns, p, q);
        case ORACLE_SIM_DICE:
            return (u128)p * nr <= (u128)(2 * q - p) * ns && (u128)p * ns <= (u128)(2 * q - p) * nr;
        case ORACLE_SIM_COSINE:
            return (u128)p * p * nr <= (u128)q * q * ns && (u128)p * p * ns <= (u128)q * q * nr;
        case ORACLE_SIM_OVERLAP:
            return (u128)q * (nr < ns ? nr : ns) >= (u128)p;
        default:
            return 0;
    }
}

/* ------------------------------------------------------------------------
 * Intersection by merging two sorted lists (Section 4.2.2: the intersection
 * of two sets is derived from a list merge).
 * ------------------------------------------------------------------------ */

/* |a n b| for ascending, duplicate-free a and b: the two-pointer merge. */
uint32_t oracle_overlap(const uint32_t* a, uint32_t na, const uint32_t* b, uint32_t nb) {
    uint32_t i = 0, j = 0, o = 0;
    while (i < na && j < nb) {
        if (a[i] == b[j]) { ++o; ++i; ++j; }
        else if (a[i] < b[j]) ++i;
        else ++j;
    }
    return o;
}

/*
 * Verification of one candidate pair (Section 3.1): a merge-like loop that
 * counts the overlap and stops as soon as the threshold can no longer be
 * reached.  The stopping rule is the positional filter of Section 2.2.3:
 * with o matches found and i tokens of r and j tokens of s consumed, at most
 * min(|r|-i, |s|-j) more matches are possible, so the pair is rejected once
 * o + min(|r|-i, |s|-j) < required overlap.  This is checked before every
 * comparison (with i = j = 0 it is the length filter).  A pair that is not
 * rejected runs to the end of the merge, so its reported overlap is exactly
 * |r n s| (true positives need the full overlap, Section 3.1).
 *
 * early = 0 disables the stopping rule (full merge for every pair).
 * Returns 1 if the pair passes the similarity test (oracle_sim_pass with
 * the required overlap of oracle_required_overlap_sim).  *o is the overlap counted
 * (exact when the pair passes or early = 0); *ci, *cj are the numbers of
 * tokens of r and s consumed when the loop stopped.
 */
int oracle_verify_pair_sim(int sim, const uint32_t* r, uint32_t nr, const uint32_t* s, uint32_t ns,
                           uint64_t p, uint64_t q, int early,
                           uint32_t* o_out, uint32_t* ci, uint32_t* cj) {
    uint64_t req = oracle_required_overlap_sim(sim, nr, ns, p, q);
    uint32_t i = 0, j = 0, o = 0;
    int rejected = 0;
    while (i < nr && j < ns) {
        if (early) {
            uint32_t left_r = nr - i, left_s = ns - j;
            uint32_t left = left_r < left_s ? left_r : left_s;
            if ((uint64_t)o + left < req) { rejected = 1; break; }
        }
        if (r[i] == s[j]) { ++o; ++i; ++j; }
        else if (r[i] < s[j]) ++i;
        else ++j;
    }
    if (o_out) *o_out = o;
    if (ci) *ci = i;
    if (cj) *cj = j;
    if (rejected) return 0;
    return oracle_sim_pass(sim, o, nr, ns, p, q);
}

/* The same for the Jaccard threshold. */
int oracle_verify_pair(const uint32_t* r, uint32_t nr, const uint32_t* s, uint32_t ns,
                       uint64_t p, uint64_t q, int early,
                       uint32_t* o_out, uint32_t* ci, uint32_t* cj) {
    return oracle_verify_pair_sim(ORACLE_SIM_JACCARD, r, nr, s, ns, p, q, early, o_out, ci, cj);
}

/* ------------------------------------------------------------------------
 * Brute force: the problem definition of Section 3 over every pair.
 * ------------------------------------------------------------------------ */

static void put_triple(uint32_t* out, uint64_t cap, uint64_t k, uint32_t r, uint32_t s, uint32_t o) {
    if (out && k < cap) { out[3 * k] = r; out[3 * k + 1] = s; out[3 * k + 2] = o; }
}

/*
 * Self-join: every pair r < s of one collection whose similarity reaches
 * p/q (oracle_sim_pass), as (r, s, |r n s|) triples in (r, s) order.
 * Returns the number of result pairs; at most cap triples are written.
 * Returns -2 if the threshold is invalid (p = 0, q = 0, or p > q for a
 * normalized function).
 */
int64_t oracle_bruteforce_self_sim(int sim, const uint64_t* offs, const uint32_t* toks, uint32_t n,
                                   uint64_t p, uint64_t q, uint32_t* out, uint64_t cap) {
    if (p == 0 || q == 0 || (sim != ORACLE_SIM_OVERLAP && p > q)) return -2;
    uint64_t k = 0;
    for (uint32_t r = 0; r < n; ++r) {
        for (uint32_t s = r + 1; s < n; ++s) {
            uint32_t nr = (uint32_t)(offs[r + 1] - offs[r]), ns = (uint32_t)(offs[s + 1] - offs[s]);
            uint32_t o = oracle_overlap(toks + offs[r], nr, toks + offs[s], ns);
            if (oracle_sim_pass(sim, o, nr, ns, p, q)) put_triple(out, cap, k++, r, s, o);
        }
    }
    return (int64_t)k;
}

int64_t oracle_bruteforce_self(const uint64_t* offs, const uint32_t* toks, uint32_t n,
                               uint64_t p, uint64_t q, uint32_t* out, uint64_t cap) {
    return oracle_bruteforce_self_sim(ORACLE_SIM_JACCARD, offs, toks, n, p, q, out, cap);
}

/* R x S join: every (r in R, s in S) whose similarity reaches p/q, in (r, s) order. */
int64_t oracle_bruteforce_rs_sim(int sim, const uint64_t* r_offs, const uint32_t* r_toks, uint32_t n_r,
                                 const uint64_t* s_offs, const uint32_t* s_toks, uint32_t n_s,
                                 uint64_t p, uint64_t q, uint32_t* out, uint64_t cap) {
    if (p == 0 || q == 0 || (sim != ORACLE_SIM_OVERLAP && p > q)) return -2;
    uint64_t k = 0;
    for (uint32_t r = 0; r < n_r; ++r) {
        for (uint32_t s = 0; s < n_s; ++s) {
            uint32_t nr = (uint32_t)(r_offs[r + 1] - r_offs[r]), ns = (uint32_t)(s_offs[s + 1] - s_offs[s]);
            uint32_t o = oracle_overlap(r_toks + r_offs[r], nr, s_toks + s_offs[s], ns);
            if (oracle_sim_pass(sim, o, nr, ns, p, q)) put_triple(out, cap, k++, r, s, o);
        }
    }
    return (int64_t)k;
}

int64_t oracle_bruteforce_rs(const uint64_t* r_offs, const uint32_t* r_toks, uint32_t n_r,
                             const uint64_t* s_offs, const uint32_t* s_toks, uint32_t n_s,
                             uint64_t p, uint64_t q, uint32_t* out, uint64_t cap) {
    return oracle_bruteforce_rs_sim(ORACLE_SIM_JACCARD, r_offs, r_toks, n_r, s_offs, s_toks, n_s, p, q, out, cap);
}

/* ------------------------------------------------------------------------
 * Verification of a given candidate batch (Section 3.3.1: probe ids, the
 * candidate offsets that delimit each probe's candidates, and candidate ids).
 * ------------------------------------------------------------------------ */

enum { ORACLE_EARLY = 1, ORACLE_EMIT_ALL = 2 };

/*
 * Each listed pair (probe_ids[k], cand_ids[m]), cand_offsets[k] <= m <
 * cand_offsets[k+1], is verified with oracle_verify_pair.  For a self-join a
 * pair whose two ids are equal is skipped, and a result is written as
 * (min id, max id, overlap); otherwise as (r, s, overlap).  Results keep the
 * input pair order.  With ORACLE_EMIT_ALL every (non-skipped) pair is written
 * with its exact overlap, whatever the threshold (a debugging aid to compare
 * every overlap).  consumed_r / consumed_s (one entry per listed pair, may be
 * NULL) receive the tokens read from each side before the merge stopped.
 *
 * Returns the number of results (at most cap written), -1 if an id is out of
 * range or the offsets decrease, -2 if the threshold is invalid.
 */
int64_t oracle_verify_batch_sim(int sim, const uint64_t* r_offs, const uint32_t* r_toks, uint32_t n_r,
                                const uint64_t* s_offs, const uint32_t* s_toks, uint32_t n_s,
                                int self_join, uint64_t p, uint64_t q,
                                uint32_t n_probes, const uint32_t* probe_ids,
                                const uint64_t* cand_offsets, const uint32_t* cand_ids,
                                int flags, uint32_t* out, uint64_t cap,
                                uint32_t* consumed_r, uint32_t* consumed_s) {
    if (p == 0 || q == 0 || (sim != ORACLE_SIM_OVERLAP && p > q)) return -2;
    int early = (flags & ORACLE_EARLY) != 0;
    int emit_all = (flags & ORACLE_EMIT_ALL) != 0;
    if (emit_all) early = 0;
    uint64_t k_out = 0;
    for (uint32_t k = 0; k < n_probes; ++k) {
        if (cand_offsets[k + 1] < cand_offsets[k]) return -1;
        uint32_t r = probe_ids[k];
        if (r >= n_r) return -1;
        const uint32_t* rt = r_toks + r_offs[r];
        uint32_t nr = (uint32_t)(r_offs[r + 1] - r_offs[r]);
        for (uint64_t m = cand_offsets[k]; m < cand_offsets[k + 1]; ++m) {
            uint32_t s = cand_ids[m];
            if (s >= n_s) return -1;
            uint32_t o = 0, ci = 0, cj = 0;
            if (self_join && s == r) {
                if (consumed_r) consumed_r[m] = 0;
                if (consumed_s) consumed_s[m] = 0;
                continue;
            }
            uint32_t ns = (uint32_t)(s_offs[s + 1] - s_offs[s]);
            int pass = oracle_verify_pair_sim(sim, rt, nr, s_toks + s_offs[s], ns, p, q, early, &o, &ci, &cj);
            if (consumed_r) consumed_r[m] = ci;
            if (consumed_s) consumed_s[m] = cj;
            if (pass || emit_all) {
                uint32_t a = r, b = s;
                if (self_join && b < a) { a = s; b = r; }
                put_triple(out, cap, k_out++, a, b, o);
            }
        }
    }
    return (int64_t)k_out;
}

int64_t oracle_verify_batch(const uint64_t* r_offs, const uint32_t* r_toks, uint32_t n_r,
                            const uint64_t* s_offs, const uint32_t* s_toks, uint32_t n_s,
                            int self_join, uint64_t p, uint64_t q,
                            uint32_t n_probes, const uint32_t* probe_ids,
                            const uint64_t* cand_offsets, const uint32_t* cand_ids,
                            int flags, uint32_t* out, uint64_t cap,
                            uint32_t* consumed_r, uint32_t* consumed_s) {
    return oracle_verify_batch_sim(ORACLE_SIM_JACCARD, r_offs, r_toks, n_r, s_offs, s_toks, n_s, self_join, p, q,
                                   n_probes, probe_ids, cand_offsets, cand_ids, flags, out, cap, consumed_r,
                                   consumed_s);
}

/* ------------------------------------------------------------------------
 * Preprocessing of Section 2.2.1 and the AllPairs join (Sections 2.2.3,
 * 2.2.4 and 3.1, algorithm ALL).
 * ------------------------------------------------------------------------ */

static int cmp_u32(const void* x, const void* y) {
    uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
    return (a > b) - (a < b);
}

typedef struct { uint32_t tok; uint32_t cnt; } tokcnt_t;

static int cmp_tokcnt(const void* x, const void* y) {
    const tokcnt_t* a = (const tokcnt_t*)x;
    const tokcnt_t* b = (const tokcnt_t*)y;
    if (a->cnt != b->cnt) return (a->cnt > b->cnt) - (a->cnt < b->cnt);
    return (a->tok > b->tok) - (a->tok < b->tok);
}

/*
 * Token renumbering of Section 2.2.1: tokens are replaced by integers in
 * increasing order of their frequency in the collection (ties by original
 * id), so that infrequent tokens come first; each set is re-sorted under the
 * new ids.  Writes new_toks (same layout as toks).  Returns the number of
 * distinct tokens, or -1 on allocation failure.
 */
int64_t oracle_renumber(const uint64_t* offs, const uint32_t* toks, uint32_t n, uint32_t* new_toks) {
    uint64_t total = offs[n];
    if (total == 0) return 0;
    uint32_t* sorted = (uint32_t*)malloc(sizeof(uint32_t) * total);
    if (!sorted) return -1;
    memcpy(sorted, toks, sizeof(uint32_t) * total);
    qsort(sorted, total, sizeof(uint32_t), cmp_u32);
    uint64_t u = 0;
    for (uint64_t i = 0; i < total; ++i) if (i == 0 || sorted[i] != sorted[i - 1]) ++u;
    tokcnt_t* tc = (tokcnt_t*)malloc(sizeof(tokcnt_t) * u);
    uint32_t* distinct = (uint32_t*)malloc(sizeof(uint32_t) * u);
    uint32_t* rank_of = (uint32_t*)malloc(sizeof(uint32_t) * u);
    if (!tc || !distinct || !rank_of) { free(sorted); free(tc); free(distinct); free(rank_of); return -1; }
    uint64_t d = 0;
    for (uint64_t i = 0; i < total; ++i) {
        if (i == 0 || sorted[i] != sorted[i - 1]) { tc[d].tok = sorted[i]; tc[d].cnt = 0; distinct[d] = sorted[i]; ++d; }
        tc[d - 1].cnt++;
    }
    qsort(tc, u, sizeof(tokcnt_t), cmp_tokcnt);
    /* rank_of[index of token in distinct] = position in frequency order */
    for (uint64_t rnk = 0; rnk < u; ++rnk) {
        uint32_t t = tc[rnk].tok;
        uint64_t lo = 0, hi = u;
        while (lo < hi) { uint64_t mid = (lo + hi) / 2; if (distinct[mid] < t) lo = mid + 1; else hi = mid; }
        rank_of[lo] = (uint32_t)rnk;
    }
    for (uint64_t i = 0; i < total; ++i) {
        uint32_t t = toks[i];
        uint64_t lo = 0, hi = u;
        while (lo < hi) { uint64_t mid = (lo + hi) / 2; if (distinct[mid] < t) lo = mid + 1; else hi = mid; }
        new_toks[i] = rank_of[lo];
    }
    for (uint32_t s = 0; s < n; ++s)
        qsort(new_toks + offs[s], offs[s + 1] - offs[s], sizeof(uint32_t), cmp_u32);
    free(sorted); free(tc); free(distinct); free(rank_of);
    return (int64_t)u;
}

/* Set order of Section 2.2.1: by size, then lexicographically, then by id. */
static const uint64_t* g_offs;
static const uint32_t* g_toks;

static int cmp_sets(const void* x, const void* y) {
    uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
    uint64_t na = g_offs[a + 1] - g_offs[a], nb = g_offs[b + 1] - g_offs[b];
    if (na != nb) return (na > nb) - (na < nb);
    const uint32_t* ta = g_toks + g_offs[a];
    const uint32_t* tb = g_toks + g_offs[b];
    for (uint64_t i = 0; i < na; ++i)
        if (ta[i] != tb[i]) return (ta[i] > tb[i]) - (ta[i] < tb[i]);
    return (a > b) - (a < b);
}

/*
 * Least overlap a set of size len has with any partner that can reach the
 * threshold (the partner's size within the length filter): Jaccard t|x|,
 * Dice t|x|/(2-t), Cosine t^2|x|, Overlap t, rounded up.
 */
static uint64_t min_overlap(int sim, uint32_t len, uint64_t p, uint64_t q) {
    switch (sim) {
        case ORACLE_SIM_DICE: return (uint64_t)(((u128)p * len + (2 * q - p) - 1) / (2 * q - p));
        case ORACLE_SIM_COSINE: return (uint64_t)(((u128)p * p * len + (u128)q * q - 1) / ((u128)q * q));
        case ORACLE_SIM_OVERLAP: return (p + q - 1) / q;
        default: return (uint64_t)(((u128)p * len + q - 1) / q);
    }
}

/* prefix length |x| - alpha + 1 with alpha = min_overlap (0 if alpha > |x|,
 * at most |x|): a set that shares at least alpha tokens with x shares one
 * within this prefix. */
static uint32_t prefix_len(int sim, uint32_t len, uint64_t p, uint64_t q) {
    uint64_t need = min_overlap(sim, len, p, q);
    if (need > len) return 0;
    uint64_t pl = (uint64_t)len + 1 - need;
    return pl > len ? len : (uint32_t)pl;
}

typedef struct { uint32_t* v; uint32_t n, cap; } vec_t;

static int vec_push(vec_t* a, uint32_t x) {
    if (a->n == a->cap) {
        uint32_t nc = a->cap ? 2 * a->cap : 4;
        uint32_t* nv = (uint32_t*)realloc(a->v, sizeof(uint32_t) * nc);
        if (!nv) return -1;
        a->v = nv; a->cap = nc;
    }
    a->v[a->n++] = x;
    return 0;
}

/*
 * AllPairs self-join (algorithm ALL of Section 3.1, index nested loop of
 * Section 2.2.4).  Steps, in the paper's order:
 *   1. preprocessing (Section 2.2.1): renumber tokens by ascending
 *      frequency and sort sets by (size, lexicographic);
 *   2. for each probe r in that order: look up its prefix tokens in the
 *      inverted index (prefix filter, prefix length from min_overlap), keep
 *      indexed sets s that pass the function's length filter (for Jaccard
 *      t*|r| <= |s|; |s| <= |r| holds by the order), deduplicate
 *      (pre-candidates -> candidates);
 *   3. verify each candidate with the early-terminating merge;
 *   4. insert r's prefix into the index (incremental self-join,
 *      Section 2.2.4).
 * Results are (min id, max id, overlap) in the caller's original ids, in
 * the order found.  *n_candidates receives the number of candidates
 * verified.  Returns the number of results, -2 on an invalid threshold, -3
 * on allocation failure.
 */
int64_t oracle_allpairs_self_sim(int sim, const uint64_t* offs, const uint32_t* toks, uint32_t n,
                                 uint64_t p, uint64_t q, uint32_t* out, uint64_t cap,
                                 uint64_t* n_candidates) {
    if (p == 0 || q == 0 || (sim != ORACLE_SIM_OVERLAP && p > q)) return -2;
    uint64_t total = offs[n];
    uint32_t* nt = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
    uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!nt || !order) { free(nt); free(order); return -3; }
    int64_t u = oracle_renumber(offs, toks, n, nt);
    if (u < 0) { free(nt); free(order); return -3; }
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    g_offs = offs; g_toks = nt;
    qsort(order, n, sizeof(uint32_t), cmp_sets);

    vec_t* index = (vec_t*)calloc(u ? (size_t)u : 1, sizeof(vec_t));   /* token -> indexed sets */
    uint32_t* seen = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1)); /* dedup marker per set */
    vec_t cands = {0, 0, 0};
    if (!index || !seen) { free(nt); free(order); free(index); free(seen); return -3; }
    for (uint32_t i = 0; i < n; ++i) seen[i] = 0xFFFFFFFFu;

    uint64_t k_out = 0, n_c = 0;
    int oom = 0;
    for (uint32_t pos = 0; pos < n && !oom; ++pos) {
        uint32_t r = order[pos];
        uint32_t nr = (uint32_t)(offs[r + 1] - offs[r]);
        const uint32_t* rt = nt + offs[r];
        uint32_t pl = prefix_len(sim, nr, p, q);
        cands.n = 0;
        for (uint32_t a = 0; a < pl; ++a) {
            vec_t* lst = &index[rt[a]];
            for (uint32_t b = 0; b < lst->n; ++b) {
                uint32_t s = lst->v[b];
                uint32_t ns = (uint32_t)(offs[s + 1] - offs[s]);
                if (!oracle_length_ok_sim(sim, nr, ns, p, q)) continue;  /* length filter */
                if (seen[s] == pos) continue;                     /* deduplicate */
                seen[s] = pos;
                if (vec_push(&cands, s)) { oom = 1; break; }
            }
        }
        for (uint32_t c = 0; c < cands.n; ++c) {
            uint32_t s = cands.v[c];
            uint32_t ns = (uint32_t)(offs[s + 1] - offs[s]);
            uint32_t o;
            ++n_c;
            if (oracle_verify_pair_sim(sim, rt, nr, nt + offs[s], ns, p, q, 1, &o, NULL, NULL)) {
                uint32_t a = r < s ? r : s, b = r < s ? s : r;
                put_triple(out, cap, k_out++, a, b, o);
            }
        }
        for (uint32_t a = 0; a < pl; ++a)
            if (vec_push(&index[rt[a]], r)) { oom = 1; break; }
    }
    for (int64_t t = 0; t < u; ++t) free(index[t].v);
    free(index); free(seen); free(cands.v); free(nt); free(order);
    if (oom) return -3;
    if (n_candidates) *n_candidates = n_c;
    return (int64_t)k_out;
}

int64_t oracle_allpairs_self(const uint64_t* offs, const uint32_t* toks, uint32_t n,
                             uint64_t p, uint64_t q, uint32_t* out, uint64_t cap,
                             uint64_t* n_candidates) {
    return oracle_allpairs_self_sim(ORACLE_SIM_JACCARD, offs, toks, n, p, q, out, cap, n_candidates);
}
