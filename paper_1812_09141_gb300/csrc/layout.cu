// Collection layout on the device (Section 3.3.1, Fig. datasetslayout: all
// tokens of a collection in one linear array plus an offsets array that
// delimits the sets, transferred once).
//
// GB300 layout: every set starts on a 16-byte boundary so that verification
// reads sets with aligned 128-bit loads; the gap after a set repeats its
// last token; desc[i] = (first 16-byte chunk of set i, |set i|).
//
// Steps, all on the device after one host-to-device copy of the raw
// offsets and tokens:
//   1. len_kernel   - per set: length, 16-byte chunk count, sortedness check
//   2. scan         - exclusive prefix sum of chunk counts (three kernels)
//   3. scatter_kernel - one warp per set copies its tokens and the padding
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "ssj_internal.h"

namespace ssj {

namespace {

constexpr int kScanBlock = 1024;

__global__ void len_kernel(const uint64_t* __restrict__ offs, const uint32_t* __restrict__ toks, uint32_t n,
                           int validate, uint64_t* __restrict__ chunks, uint32_t* __restrict__ err) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t a = offs[i], b = offs[i + 1];
        if (b < a || b - a >= (1ull << 31)) {
            atomicOr(err, 1u);
            chunks[i] = 0;
            continue;
        }
        chunks[i] = (b - a + 3) >> 2;
        if (validate) {
            for (uint64_t t = a + 1; t < b; ++t)
                if (toks[t - 1] >= toks[t]) { atomicOr(err, 2u); break; }
        }
    }
}

// Block-level inclusive scan of 64-bit values (Hillis-Steele over warps).
__device__ uint64_t block_inclusive_scan(uint64_t v, uint64_t* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += sh[warp - 1];
    __syncthreads();
    return v;
}

// in-place exclusive scan per block; block totals to sums[blockIdx.x]
__global__ void scan_blocks(uint64_t* data, uint64_t n, uint64_t* sums) {
    __shared__ uint64_t sh[32];
    const uint64_t i = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint64_t v = i < n ? data[i] : 0;
    const uint64_t inc = block_inclusive_scan(v, sh);
    if (i < n) data[i] = inc - v;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = inc;
}

// exclusive scan of the block totals by one block, looping over tiles
__global__ void scan_sums(uint64_t* sums, uint64_t n, uint64_t* total) {
    __shared__ uint64_t sh[32];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < n; base += kScanBlock) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t v = i < n ? sums[i] : 0;
        const uint64_t inc = block_inclusive_scan(v, sh);
        if (i < n) sums[i] = carry + inc - v;
        __shared__ uint64_t tile_total;
        if (threadIdx.x == kScanBlock - 1) tile_total = inc;
        __syncthreads();
        carry += tile_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_add(uint64_t* data, uint64_t n, const uint64_t* sums) {
    const uint64_t i = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) data[i] += sums[blockIdx.x];
}

// one warp per set: tokens to their 16-byte aligned slot, padding after
__global__ void scatter_kernel(const uint64_t* __restrict__ offs, const uint32_t* __restrict__ toks, uint32_t n,
                               const uint64_t* __restrict__ start_chunk, uint32_t* __restrict__ dst,
                               uint2* __restrict__ desc) {
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const uint64_t a = offs[i], b = offs[i + 1];
        const uint64_t len = b >= a ? b - a : 0;
        const uint64_t sc = start_chunk[i];
        const uint64_t padded = ((len + 3) >> 2) << 2;
        uint32_t* d = dst + (sc << 2);
        // the padding repeats the set's last token (the verify kernel's block
        // compare relies on it: a repeated token neither adds a match on the
        // candidate side nor changes the block's last token)
        for (uint64_t t = lane; t < padded; t += 32) d[t] = toks[a + (t < len ? t : len - 1)];
        if (lane == 0) desc[i] = make_uint2((uint32_t)sc, (uint32_t)len);
    }
}

}  // namespace

// Build the padded device layout from raw device copies of offsets/tokens.
// Returns the number of 16-byte chunks via *n_chunks (host), after a sync.
// scratch must hold (n + 1) + ceil(n/1024) + 1 uint64 values.
cudaError_t layout_lengths(const uint64_t* d_offs, const uint32_t* d_toks, uint32_t n, int validate,
                           uint64_t* d_scratch, uint32_t* d_err, uint64_t* n_chunks_host, cudaStream_t st,
                           int num_sms) {
    uint64_t* chunks = d_scratch;
    const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
    uint64_t* sums = d_scratch + n + 1;
    uint64_t* total = sums + nb;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        unsigned blocks = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms * 8);
        len_kernel<<<blocks, 256, 0, st>>>(d_offs, d_toks, n, validate, chunks, d_err);
        scan_blocks<<<(unsigned)nb, kScanBlock, 0, st>>>(chunks, n, sums);
        scan_sums<<<1, kScanBlock, 0, st>>>(sums, nb, total);
        scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(chunks, n, sums);
    } else {
        e = cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
        if (e != cudaSuccess) return e;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(n_chunks_host, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t layout_scatter(const uint64_t* d_offs, const uint32_t* d_toks, uint32_t n, const uint64_t* d_scratch,
                           uint32_t* d_dst, uint2* d_desc, cudaStream_t st, int num_sms) {
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)std::min<uint64_t>(((uint64_t)n * 32 + 255) / 256, (uint64_t)num_sms * 16);
    scatter_kernel<<<blocks, 256, 0, st>>>(d_offs, d_toks, n, d_scratch, d_dst, d_desc);
    return cudaGetLastError();
}

size_t layout_scratch_words(uint32_t n) {
    return (size_t)n + 1 + (n + kScanBlock - 1) / kScanBlock + 1;
}

size_t scan_scratch_words(uint64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t exclusive_scan_u64(uint64_t* data, uint64_t n, uint64_t* scratch, uint64_t* total, cudaStream_t st) {
    if (n == 0) return cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
    const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
    scan_blocks<<<(unsigned)nb, kScanBlock, 0, st>>>(data, n, scratch);
    scan_sums<<<1, kScanBlock, 0, st>>>(scratch, nb, total);
    scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(data, n, scratch);
    return cudaGetLastError();
}

}  // namespace ssj
