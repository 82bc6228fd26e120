/*
 * Seeded synthetic collections of token sets.
 *
 * This file produces INPUTS only: set sizes, token draws and candidate id
 * lists.  It contains none of the join's arithmetic (no overlap, no
 * threshold, no filter, no renumbering).  Both the CPU oracle and the CUDA
 * library are fed from here, and neither is linked into this file.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.
 *
 * Token draws follow a Zipf law over ranks 1..V, P(k) ~ k^-s, sampled by
 * inverse CDF.  A drawn rank is mapped to a raw token id by a fixed bijection
 * on uint32 so that raw ids carry no frequency order; renumbering by
 * frequency is the consumer's job.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t* g, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) g->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* g) {
    uint64_t* s = g->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* uniform double in [0,1) with 53 random bits */
static double rng_unif(rng_t* g) { return (double)(rng_next(g) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) by 128-bit multiply-shift (n >= 1) */
static uint64_t rng_below(rng_t* g, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(g) * n) >> 64);
}

static double rng_normal(rng_t* g) {
    /* Box-Muller; u1 in (0,1] */
    double u1 = 1.0 - rng_unif(g);
    double u2 = rng_unif(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* rank (0-based) -> raw token id: odd multiplier and xor, a bijection on uint32 */
static inline uint32_t rank_to_raw(uint64_t rank, uint32_t mask) {
    return ((uint32_t)rank * 0x9E3779B1u) ^ mask;
}

enum { SIZE_UNIFORM = 0, SIZE_LOGNORMAL = 1 };

/*
 * Set sizes.  kind SIZE_UNIFORM: integer uniform in [lo, hi] (a, b unused).
 * kind SIZE_LOGNORMAL: exp(N(mu, sigma)) with mu = ln(a) - sigma^2/2 so the
 * arithmetic mean is a; sigma = b; rounded to nearest and clipped to [lo, hi].
 * Writes n sizes; returns the total.
 */
uint64_t synth_sizes(uint64_t seed, uint32_t n, int kind, double a, double b,
                     uint32_t lo, uint32_t hi, uint32_t* sizes) {
    rng_t g; rng_seed(&g, seed ^ 0x51AE5EEDULL);
    uint64_t total = 0;
    double mu = (kind == SIZE_LOGNORMAL) ? log(a) - 0.5 * b * b : 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t k;
        if (kind == SIZE_UNIFORM) {
            k = lo + rng_below(&g, (uint64_t)hi - lo + 1);
        } else {
            double v = exp(mu + b * rng_normal(&g));
            double r = floor(v + 0.5);
            if (r < (double)lo) r = lo;
            if (r > (double)hi) r = hi;
            k = (uint64_t)r;
        }
        sizes[i] = (uint32_t)k;
        total += k;
    }
    return total;
}

/* Zipf inverse-CDF table over ranks 1..V (cdf[k-1] = sum_{i<=k} i^-s / Z). */
static double* zipf_table(double s, uint32_t V) {
    double* cdf = (double*)malloc(sizeof(double) * (size_t)V);
    if (!cdf) return NULL;
    double acc = 0.0;
    for (uint32_t k = 1; k <= V; ++k) {
        double w = (s == 1.0) ? 1.0 / (double)k : pow((double)k, -s);
        acc += w;
        cdf[k - 1] = acc;
    }
    for (uint32_t k = 0; k < V; ++k) cdf[k] /= acc;
    cdf[V - 1] = 1.0;
    return cdf;
}

static uint32_t zipf_draw(rng_t* g, const double* cdf, uint32_t V) {
    double u = rng_unif(g);
    uint32_t lo = 0, hi = V - 1; /* first index with cdf >= u */
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] < u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int cmp_u32(const void* x, const void* y) {
    uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
    return (a > b) - (a < b);
}

/*
 * Tokens for n sets whose sizes are given: each set draws Zipf(s, V) ranks
 * until it holds sizes[i] distinct ones, maps them to raw ids and sorts them
 * ascending.  offsets (n+1) is written as the exclusive prefix sum of sizes.
 * Returns 0, or -1 if a size exceeds V or memory runs out.
 */
int synth_tokens(uint64_t seed, uint32_t n, const uint32_t* sizes, double zipf_s,
                 uint32_t V, uint64_t* offsets, uint32_t* tokens) {
    rng_t g; rng_seed(&g, seed);
    uint32_t mask = (uint32_t)splitmix64_next(&seed);
    double* cdf = zipf_table(zipf_s, V);
    if (!cdf) return -1;
    uint32_t maxk = 0;
    for (uint32_t i = 0; i < n; ++i) if (sizes[i] > maxk) maxk = sizes[i];
    if (maxk > V) { free(cdf); return -1; }
    /* open-addressing membership table, power of two >= 4*maxk */
    uint32_t cap = 16;
    while (cap < 4 * maxk) cap <<= 1;
    uint32_t* tab = (uint32_t*)malloc(sizeof(uint32_t) * cap);
    if (!tab) { free(cdf); return -1; }
    uint64_t off = 0;
    offsets[0] = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t k = sizes[i];
        memset(tab, 0xFF, sizeof(uint32_t) * cap);
        uint32_t* out = tokens + off;
        uint32_t have = 0;
        while (have < k) {
            uint32_t r = zipf_draw(&g, cdf, V);
            uint32_t h = (r * 0x9E3779B1u) & (cap - 1);
            int seen = 0;
            while (tab[h] != 0xFFFFFFFFu) {
                if (tab[h] == r) { seen = 1; break; }
                h = (h + 1) & (cap - 1);
            }
            if (seen) continue;
            tab[h] = r;
            out[have++] = rank_to_raw(r, mask);
        }
        qsort(out, k, sizeof(uint32_t), cmp_u32);
        off += k;
        offsets[i + 1] = off;
    }
    free(tab);
    free(cdf);
    return 0;
}

/*
 * Planted near-duplicates: for each set i chosen with probability frac
 * (and i > 0), overwrite it with a copy of a random earlier set j of the
 * same size whose first `edits` tokens (in draw order of a random
 * permutation) are replaced by fresh uniform raw ids not in the set.
 * Sizes are unchanged, so offsets stay valid.  Returns the number planted.
 */
uint32_t synth_plant(uint64_t seed, uint32_t n, const uint64_t* offsets, uint32_t* tokens,
                     double frac, uint32_t edits) {
    rng_t g; rng_seed(&g, seed ^ 0xD0D0D0D0ULL);
    uint32_t planted = 0;
    for (uint32_t i = 1; i < n; ++i) {
        if (rng_unif(&g) >= frac) continue;
        uint32_t k = (uint32_t)(offsets[i + 1] - offsets[i]);
        /* look for an earlier set of the same size (bounded tries) */
        uint32_t j = n;
        for (int t = 0; t < 64; ++t) {
            uint32_t c = (uint32_t)rng_below(&g, i);
            if (offsets[c + 1] - offsets[c] == k) { j = c; break; }
        }
        if (j == n) continue;
        uint32_t* dst = tokens + offsets[i];
        const uint32_t* src = tokens + offsets[j];
        memcpy(dst, src, sizeof(uint32_t) * k);
        uint32_t e = edits < k ? edits : k;
        for (uint32_t m = 0; m < e; ++m) {
            uint32_t pos = (uint32_t)rng_below(&g, k);
            for (;;) {
                uint32_t v = (uint32_t)rng_next(&g);
                int dup = 0;
                for (uint32_t z = 0; z < k; ++z) if (dst[z] == v) { dup = 1; break; }
                if (!dup) { dst[pos] = v; break; }
            }
        }
        qsort(dst, k, sizeof(uint32_t), cmp_u32);
        ++planted;
    }
    return planted;
}

/*
 * Random grouped candidate lists: n_probes probe ids uniform in [0, n_r),
 * each with a count uniform in [0, max_per_probe], candidate ids uniform in
 * [0, n_s).  Pass 1 (cand_ids == NULL) writes probe ids and offsets and
 * returns the total; pass 2 fills cand_ids.  Same seed -> same lists.
 */
uint64_t synth_random_batch(uint64_t seed, uint32_t n_r, uint32_t n_s, uint32_t n_probes,
                            uint32_t max_per_probe, uint32_t* probe_ids,
                            uint64_t* cand_offsets, uint32_t* cand_ids) {
    rng_t g; rng_seed(&g, seed ^ 0xBA7C4ULL);
    uint64_t off = 0;
    if (cand_offsets) cand_offsets[0] = 0;
    for (uint32_t k = 0; k < n_probes; ++k) {
        uint32_t pr = (uint32_t)rng_below(&g, n_r);
        uint32_t c = (uint32_t)rng_below(&g, (uint64_t)max_per_probe + 1);
        if (probe_ids) probe_ids[k] = pr;
        for (uint32_t m = 0; m < c; ++m) {
            uint32_t s = (uint32_t)rng_below(&g, n_s);
            if (cand_ids) cand_ids[off + m] = s;
        }
        off += c;
        if (cand_offsets) cand_offsets[k + 1] = off;
    }
    return off;
}

/* log-uniform double in [lo, hi] and uniform double in [lo, hi], for instance specs */
double synth_loguniform(uint64_t seed, uint64_t idx, double lo, double hi) {
    uint64_t x = seed * 0x100000001B3ULL + idx;
    rng_t g; rng_seed(&g, x);
    return exp(log(lo) + (log(hi) - log(lo)) * rng_unif(&g));
}

double synth_uniform(uint64_t seed, uint64_t idx, double lo, double hi) {
    uint64_t x = seed * 0x100000001B3ULL + idx + 0x7777ULL;
    rng_t g; rng_seed(&g, x);
    return lo + (hi - lo) * rng_unif(&g);
}
