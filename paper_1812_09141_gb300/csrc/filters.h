// Host-side threshold arithmetic of the CPU candidate generators (feeder.cpp,
// groups.cpp): the per-function prefix and length filters of Section 2.2.3
// for the similarity functions of Table "Similarity Functions", t = p/q.
#pragma once

#include <algorithm>
#include <cstdint>

#include "arith.h"

namespace ssj {

struct Filters {
    uint32_t sim = 0, p = 1, q = 1;  // sim: 0 Jaccard, 1 Dice, 2 Cosine, 3 plain overlap

    // 0 < p <= q < 2^31 for the normalized functions, 0 < p, q < 2^31 for overlap
    static bool valid(uint32_t sim, uint32_t p, uint32_t q) {
        if (sim > 3) return false;
        if (sim == 3) return p > 0 && q > 0 && p < (1u << 31) && q < (1u << 31);
        return p > 0 && p <= q && q < (1u << 31);
    }

    static uint64_t ceil_mul_div(uint64_t x, uint64_t a, uint64_t b) {
        return (uint64_t)(((unsigned __int128)a * x + b - 1) / b);
    }
    static uint32_t floor_mul_div_sat(uint64_t x, uint64_t a, uint64_t b) {
        const unsigned __int128 v = (unsigned __int128)a * x / b;
        return v > 0xFFFFFFFFu ? 0xFFFFFFFFu : (uint32_t)v;
    }

    // Least overlap a set of size len shares with any partner that can reach
    // the threshold: Jaccard t|x|, Dice t|x|/(2-t), Cosine t^2|x|, plain
    // overlap t (rounded up).  It is also the smallest partner size the
    // length filter admits for a probe of size len.
    uint64_t min_overlap(uint64_t len) const {
        switch (sim) {
            case 1: return ceil_mul_div(len, p, 2ull * q - p);
            case 2: return (uint64_t)(((unsigned __int128)p * p * len + (unsigned __int128)q * q - 1) /
                                      ((unsigned __int128)q * q));
            case 3: return ((uint64_t)p + q - 1) / q;
            default: return ceil_mul_div(len, p, q);
        }
    }

    // Largest partner size the length filter admits for a probe of size len.
    uint32_t max_partner(uint64_t len) const {
        switch (sim) {
            case 1: return floor_mul_div_sat(len, 2ull * q - p, p);
            case 2: return (uint32_t)std::min<unsigned __int128>(
                        (unsigned __int128)q * q * len / ((unsigned __int128)p * p), 0xFFFFFFFFu);
            case 3: return 0xFFFFFFFFu;
            default: return floor_mul_div_sat(len, q, p);
        }
    }

    // Equivalent overlap of a pair of sizes nr, ns.
    uint32_t required(uint32_t nr, uint32_t ns) const {
        switch (sim) {
            case 1: return required_overlap_magic(nr, ns, p, 2 * q, div_magic(2ull * q));
            case 2: return required_overlap_cosine(p, q, nr, ns);
            case 3: return (uint32_t)(((uint64_t)p + q - 1) / q);
            default: return required_overlap_magic(nr, ns, p, p + q, div_magic((uint64_t)p + q));
        }
    }

    // Prefix of len - min_overlap + 1 tokens (none if no partner can reach t).
    uint32_t prefix_len(uint32_t len) const {
        if (len == 0) return 0;
        const uint64_t need = min_overlap(len);
        if (need > len) return 0;
        const uint64_t pl = (uint64_t)len + 1 - need;
        return pl > len ? len : (uint32_t)pl;
    }
};

}  // namespace ssj
