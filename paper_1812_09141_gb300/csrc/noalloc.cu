// Verification without any allocation by the library: the work queue lives in
// a fixed block of device memory that is part of the loaded library itself.
//
// Who needs this: callers that cannot let a library allocate device memory
// during a call.  Some run every allocation through their own arena or a
// framework's caching allocator and forbid side allocations; others sit on a
// latency-critical path where cudaMalloc / cudaFree may synchronise the
// device and stall unrelated streams.  ssj_verify_batch_async grows its
// workspace with cudaMalloc when a batch is larger than any before; this entry
// point instead uses the static scratch array below and never allocates.
// The paper has no counterpart to this; it is an interface convenience.
#include <cstdint>

#include <cuda_runtime.h>

#include "ssj_internal.h"

namespace ssj {
ssj_status resolve_device_batch(ssj_ctx* ctx, const ssj_batch* batch, const void* out, const void* count,
                                VerifyArgs* a, int* device, int* num_sms, uint32_t* block_threads,
                                cudaStream_t* ctx_stream);
ssj_status report(ssj_ctx* ctx, ssj_status st, const char* msg);
void remember_counters(ssj_ctx* ctx, Counters* c);
}  // namespace ssj

using namespace ssj;

namespace {

// 32 MiB of scratch, held by every GPU that loads the library until the
// process exits.  Sizes that need more are rejected.
constexpr size_t kNoallocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name only stands in for the symbol, so the address is looked
// up with cudaGetSymbolAddress, with the target device current.  The lookup
// runs on every call (it costs far less than the launch) so that no address
// outlives the context it belongs to, e.g. after a device reset.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" ssj_status ssj_verify_batch_noalloc(ssj_ctx* ctx, const ssj_batch* batch, ssj_triple* d_out,
                                               uint64_t cap, uint64_t* d_count, void* stream) {
    if (!ctx || !batch) return SSJ_EINVAL;
    if (!d_count) return report(ctx, SSJ_EINVAL, "d_count is required");
    VerifyArgs a;
    int device = 0, num_sms = 0;
    uint32_t block_threads = 0;
    cudaStream_t ctx_stream = nullptr;
    ssj_status st = resolve_device_batch(ctx, batch, d_out, d_count, &a, &device, &num_sms, &block_threads, &ctx_stream);
    if (st != SSJ_OK) return st;
    if (cap && !d_out && !(batch->flags & SSJ_COUNT_ONLY)) return report(ctx, SSJ_EINVAL, "NULL output");
    if (workspace_bytes(batch->n_probes, batch->n_cands, num_sms) > kNoallocScratchBytes)
        return report(ctx, SSJ_EINVAL,
                      "batch too large for ssj_verify_batch_noalloc: its work queue needs more than the "
                      "32 MiB of static scratch; split the batch or use ssj_verify_batch_async");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return report(ctx, SSJ_EDEVICE, "cudaGetDevice failed");
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return report(ctx, SSJ_EDEVICE, "cudaSetDevice failed");
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e == cudaSuccess) {
        a.single.out = d_out;
        a.single.cap = (batch->flags & SSJ_COUNT_ONLY) ? 0 : cap;
        a.single.count = reinterpret_cast<unsigned long long*>(d_count);
        bind_workspace(a, scratch, batch->n_probes, batch->n_cands, num_sms);
        remember_counters(ctx, a.ctr);
        // launch_verify clears the counters and the count before the kernels run
        // a NULL stream means the context's stream, as for ssj_verify_batch_async, so that
        // ssj_device_error (which reads on the context's stream) sees this call's checks
        const cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx_stream;
        e = launch_verify(a, s, num_sms, block_threads, nullptr);
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return report(ctx, SSJ_EDEVICE, cudaGetErrorString(e));
    return SSJ_OK;
}
