// Exact integer arithmetic of the Jaccard test, shared by host and device
// code of the library (Table "Similarity Functions": Jaccard's equivalent
// overlap ceil(t/(1+t) * (|r|+|s|)), with t = p/q).
#pragma once

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

// Required overlap ceil(p * (nr + ns) / (p + q)); nr, ns < 2^31, p, q < 2^31,
// so p * (nr + ns) + p + q - 1 < 2^63.
SSJ_HD uint32_t required_overlap_magic(uint32_t nr, uint32_t ns, uint32_t p, uint32_t d, uint64_t m) {
    const uint64_t x = (uint64_t)p * (uint64_t)(nr + ns) + d - 1;
    return (uint32_t)div_by_magic(x, d, m);
}

}  // namespace ssj
