// Exact integer arithmetic of the similarity tests, shared by host and
// device code of the library (Table "Similarity Functions": Jaccard's
// equivalent overlap ceil(t/(1+t) * (|r|+|s|)), Dice's ceil(t(|r|+|s|)/2),
// Cosine's ceil(t sqrt(|r||s|)), with t = p/q).
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define SSJ_HD __host__ __device__ __forceinline__
#else
#define SSJ_HD inline
#endif

namespace ssj {

// High 64 bits of a 64x64-bit product.
SSJ_HD uint64_t mul_hi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Reciprocal of the divisor d = p + q (d >= 2): m = floor((2^64 - 1) / d).
SSJ_HD uint64_t div_magic(uint64_t d) { return ~0ull / d; }

// floor(x / d) for any 64-bit x, given m = div_magic(d).  With e = 2^64 - d*m
// (1 <= e <= d), x*m / 2^64 = x/d - x*e/(d*2^64) lies in (x/d - 1, x/d], so
// the high product is floor(x/d) or one less; one comparison fixes it.
SSJ_HD uint64_t div_by_magic(uint64_t x, uint64_t d, uint64_t m) {
    uint64_t q0 = mul_hi64(x, m);
    if (x - q0 * d >= d) ++q0;
    return q0;
}

// Required overlap ceil(p * (nr + ns) / d) for the divisor d = p + q
// (Jaccard) or d = 2q (Dice, ceil(t(|r|+|s|)/2)); nr, ns < 2^31 and
// p, q < 2^31, so p * (nr + ns) + d - 1 < 2^63.
SSJ_HD uint32_t required_overlap_magic(uint32_t nr, uint32_t ns, uint32_t p, uint32_t d, uint64_t m) {
    const uint64_t x = (uint64_t)p * (uint64_t)(nr + ns) + d - 1;
    return (uint32_t)div_by_magic(x, d, m);
}

// Cosine test o / sqrt(nr * ns) >= p / q, multiplied out: (q o)^2 >= p^2 nr ns
// in 128 bits (q o < 2^63, p^2 < 2^62, nr ns < 2^64).
SSJ_HD bool cosine_pass(uint64_t o, uint32_t p, uint32_t q, uint32_t nr, uint32_t ns) {
    const uint64_t qo = (uint64_t)q * o;
    const uint64_t pp = (uint64_t)p * p, nn = (uint64_t)nr * ns;
    const uint64_t lh = mul_hi64(qo, qo), ll = qo * qo;
    const uint64_t rh = mul_hi64(pp, nn), rl = pp * nn;
    return lh > rh || (lh == rh && ll >= rl);
}

// Cosine's equivalent overlap ceil(t sqrt(nr ns)) (Table "Similarity
// Functions"), capped at min(nr, ns) + 1 (any larger value rejects the pair
// the same way); 0xFFFFFFFF when a set is empty (never similar).  A
// floating-point estimate is corrected by the exact test in both
// directions, so the result is exact whatever the estimate's rounding.
SSJ_HD uint32_t required_overlap_cosine(uint32_t p, uint32_t q, uint32_t nr, uint32_t ns) {
    if (nr == 0 || ns == 0) return 0xFFFFFFFFu;
    const uint64_t cap = (uint64_t)(nr < ns ? nr : ns) + 1;
    const double est = (double)p / (double)q * sqrt((double)nr * (double)ns);
    uint64_t o = est >= (double)cap ? cap : (uint64_t)est;
    while (o > 0 && cosine_pass(o - 1, p, q, nr, ns)) --o;
    while (o < cap && !cosine_pass(o, p, q, nr, ns)) ++o;
    return (uint32_t)o;
}

}  // namespace ssj
