// Read-bandwidth probe.  Streams a device buffer with 128-bit loads that are
// cached in L2 only, so that repeated passes over a buffer smaller than L2
// measure the L2 read rate, and passes over a larger one the HBM read rate.
// The L2 figure is the denominator of the L2-aware roofline of verification,
// whose token reads hit L2 once a collection is resident.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "ssj_internal.h"

namespace ssj {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeUnroll = 4;

// passes sweeps over the buffer in one launch, so that a buffer that one
// pass reads in a few microseconds is not timed against launch latency.
__global__ void __launch_bounds__(kProbeThreads) read_probe_kernel(const uint4* __restrict__ p, uint64_t n,
                                                                   uint32_t passes, uint32_t* __restrict__ sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * kProbeThreads;
    const uint64_t i0 = (uint64_t)blockIdx.x * kProbeThreads + threadIdx.x;
    for (uint32_t pass = 0; pass < passes; ++pass) {
        uint64_t i = i0;
        // kProbeUnroll independent loads in flight per thread
        for (; i + (kProbeUnroll - 1) * stride < n; i += kProbeUnroll * stride) {
            uint4 v[kProbeUnroll];
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) v[u] = __ldcg(p + i + u * stride);
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        for (; i < n; i += stride) {
            const uint4 v = __ldcg(p + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        acc = acc * 3u + pass;  // keeps each pass's loads (the buffer holds zeros)
    }
    // practically never taken; the stored value depends on every load
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

}  // namespace

cudaError_t read_probe(const void* buf, uint64_t bytes, uint32_t passes, uint32_t* sink, int num_sms,
                       cudaStream_t st) {
    const uint64_t n = bytes / sizeof(uint4);
    if (n == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, read_probe_kernel, kProbeThreads, 0);
    if (e != cudaSuccess) return e;
    const uint64_t want = (n + kProbeThreads - 1) / kProbeThreads;
    const uint64_t grid = std::min<uint64_t>(want, (uint64_t)num_sms * (uint64_t)(per_sm > 0 ? per_sm : 1));
    read_probe_kernel<<<(unsigned)grid, kProbeThreads, 0, st>>>(static_cast<const uint4*>(buf), n, passes, sink);
    return cudaGetLastError();
}

}  // namespace ssj
