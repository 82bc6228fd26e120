// Host side of the C ABI declared in include/ssj.h: contexts, collection
// store, batch validation, synchronous and stream-ordered verification, and
// the continuous-batching serving loop (submit / poll / results).
//
// The co-process scheme of Section 3.2 (Fig. executionoverlap) maps onto
// this file as follows: the caller's filtering thread (H0) submits chunks;
// each admitted chunk gets a slot with its own CUDA stream, so its copies
// and kernels overlap with other chunks on the device (H1); a completion
// thread reads the result count, copies back exactly that many triples and
// releases device memory (H2).  Admission is by a device-memory budget
// (M_c, Section 4.1.2) and a slot count.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "arith.h"
#include "ssj_internal.h"

namespace ssj {
cudaError_t layout_lengths(const uint64_t* d_offs, const uint32_t* d_toks, uint32_t n, int validate,
                           uint64_t* d_scratch, uint32_t* d_err, uint64_t* n_chunks_host, cudaStream_t st,
                           int num_sms);
cudaError_t layout_scatter(const uint64_t* d_offs, const uint32_t* d_toks, uint32_t n, const uint64_t* d_scratch,
                           uint32_t* d_dst, uint2* d_desc, cudaStream_t st, int num_sms);
size_t layout_scratch_words(uint32_t n);
void renumber_by_frequency(const uint64_t* offsets, const uint32_t* tokens, uint32_t n, std::vector<uint32_t>& out);
}  // namespace ssj

using namespace ssj;

namespace {

// An NVTX range over a scope: names the API calls and the serving phases on
// a profiler's timeline (a no-op when no tool is attached).
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

}  // namespace

namespace {

// Default of the context's index-item threshold (ssj_set_index_items).
constexpr uint32_t kIndexMinCandsDefault = 256;
// ssj_verify_batches runs a call as one launch per kSplitCands candidates, up to kMaxGroups
// (on the 256-instance workload, four groups measured slower than two: 1.39e10 against
// 1.45e10 pairs/s end to end; each launch adds its own fill and drain).
constexpr uint64_t kSplitCands = 1ull << 24;
constexpr uint32_t kMaxGroups = 2;
// ...and reads inputs in pinned host memory directly over the host link (no staging copy) in
// calls of at least this many candidates: on the 256-instance workload, 1.62e10-1.67e10 pairs/s
// end to end against 1.09e10-1.45e10 with staged copies.
constexpr uint64_t kDirectCands = 1ull << 25;
// Candidates of one batch, and of one call or prepared launch: 2^40 ids are 4 TiB, beyond any
// device's memory, and keep every workspace size computed from the count far from 64-bit wrap.
constexpr uint64_t kMaxCands = 1ull << 40;

struct Collection {
    uint32_t n_sets = 0;
    uint64_t n_tokens = 0;
    uint64_t n_chunks = 0;
    uint32_t* d_toks = nullptr;  // n_chunks * 4 tokens
    uint2* d_desc = nullptr;
    bool renumbered = false;
    uint32_t max_len = 0;        // longest set
    uint32_t vocab = 0;          // largest token on the device + 1
    uint32_t busy = 0;           // submitted batches not yet collected
    size_t l2_window = 0;        // SSJ_PIN_L2: bytes of the token array kept in the persisting L2 set-aside
    float l2_hit_ratio = 0.f;    // share of the window the set-aside holds
    DevColl dev() const {
        DevColl d;
        d.toks4 = reinterpret_cast<const uint4*>(d_toks);
        d.desc = d_desc;
        d.n_sets = n_sets;
        return d;
    }
};

enum class TicketState { kRunning, kDone, kFailed };

struct Ticket {
    uint64_t id = 0;
    ssj_coll R = 0, S = 0;
    uint32_t flags = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t kernel_done = nullptr;
    void* d_mem = nullptr;           // one stream-ordered allocation for the whole batch
    uint64_t bytes = 0;              // charged to the budget
    ssj_triple* d_out = nullptr;
    uint64_t out_cap = 0;
    uint64_t* h_count = nullptr;     // pinned
    uint32_t* h_err = nullptr;       // pinned
    ssj_triple* h_out = nullptr;     // pinned, grown as needed
    uint64_t count = 0;
    TicketState state = TicketState::kRunning;
    std::string error;
    uint32_t derr = 0;  // device check bits of a failed batch
    int slot = -1;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t copied = nullptr;   // host-to-device copies of a submission done
    // pinned staging for host inputs
    uint32_t* h_probe = nullptr;
    uint64_t* h_offs = nullptr;
    uint32_t* h_cand = nullptr;
    uint64_t h_probe_cap = 0, h_offs_cap = 0, h_cand_cap = 0;
    ssj_triple* h_out = nullptr;
    uint64_t h_out_cap = 0;
    uint64_t* h_count = nullptr;
    uint32_t* h_err = nullptr;
    bool busy = false;          // reserved by a ticket until ssj_results collects it
    struct Ticket* pending = nullptr;  // launched, waiting for the completion thread
    std::thread completer;
};

}  // namespace

struct ssj_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t budget = 0;
    uint32_t max_inflight = 0;
    uint32_t thread_max_key = 128;
    uint32_t drain_min_live = 0;  // short-pair policy (0: default)
    uint32_t lane_max_key = 2048;
    uint32_t warp_max_key = 2048;
    uint32_t block_threads = 256;
    uint32_t index_min_cands = kIndexMinCandsDefault;  // probes with this many candidates become index items
    // SSJ_PIN_L2: the context's persisting-L2 set-aside as found (restored when the last pinned
    // collection is unloaded), whether the library raised it, and the pinned collections
    size_t l2_limit_found = 0;
    bool l2_limit_raised = false;
    uint32_t n_pinned = 0;
    std::string err;

    std::map<ssj_coll, Collection> colls;
    ssj_coll next_coll = 1;

    // workspace for synchronous/stream-ordered calls
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // device staging for synchronous host-pointer calls
    void* io = nullptr;
    size_t io_bytes = 0;
    uint64_t* h_count = nullptr;  // pinned
    uint32_t* h_err = nullptr;    // pinned, kMaxGroups words
    // ssj_verify_batches: the stream and event that carry the second group's input copies
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_done[kMaxGroups] = {};
    cudaEvent_t call_start = nullptr;
    Counters* last_ctr = nullptr;
    // kernel timing (SSJ_CTX_PROFILE): events around plan and verify of each launch
    bool profile = false;
    std::vector<cudaEvent_t> prof_ev;  // 3 per recorded launch
    size_t prof_used = 0;             // launches recorded since the last read

    // serving
    std::mutex mu;
    std::condition_variable cv;
    cudaMemPool_t pool = nullptr;
    std::vector<Slot> slots;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_ticket = 1;
    uint64_t used_bytes = 0;
    bool pool_grown = false;   // the pool holds the whole budget (first submission)
    bool stopping = false;
};

namespace {

ssj_status fail(ssj_ctx* ctx, ssj_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

ssj_status cuda_fail(ssj_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, SSJ_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

ssj_status ensure_device_buffer(ssj_ctx* ctx, void** buf, size_t* have, size_t need) {
    if (*have >= need && *buf) return SSJ_OK;
    if (*buf) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    size_t sz = std::max<size_t>(need, 1 << 20);
    cudaError_t e = cudaMalloc(buf, sz);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return fail(ctx, SSJ_ENOMEM, "cudaMalloc(%zu): %s", sz, cudaGetErrorString(e));
    }
    *have = sz;
    return SSJ_OK;
}

template <class T>
ssj_status ensure_pinned(ssj_ctx* ctx, T** buf, uint64_t* have, uint64_t need) {
    if (*have >= need && *buf) return SSJ_OK;
    if (*buf) cudaFreeHost(*buf);
    *buf = nullptr;
    uint64_t n = std::max<uint64_t>(need, std::max<uint64_t>(*have * 2, 1024));
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(buf), n * sizeof(T));
    if (e != cudaSuccess) {
        *buf = nullptr;
        *have = 0;
        return fail(ctx, SSJ_ENOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
    }
    *have = n;
    return SSJ_OK;
}

// The kernels load probe ids and candidate ids as 4-byte words and offsets
// and counts as 8-byte words, and store result triples field by field (4
// bytes).  An address the device reads or writes off that alignment would
// fault the context, so such arrays are refused (device memory) or staged
// (pinned host memory).
bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

ssj_status check_device_alignment(ssj_ctx* ctx, const ssj_batch* b, const void* out, const void* count) {
    if (!aligned_to(b->probe_ids, 4) || !aligned_to(b->cand_offsets, 8) || !aligned_to(b->cand_ids, 4) ||
        !aligned_to(out, 4) || !aligned_to(count, 8))
        return fail(ctx, SSJ_EINVAL,
                    "device arrays must be aligned to their element size (4 bytes for ids and triples, 8 for "
                    "cand_offsets and counts)");
    return SSJ_OK;
}

// Device address of pinned host memory the device can read directly, or
// NULL (pageable memory, no mapping, or an address off the element alignment
// a, which is then staged by a copy).
const void* device_view(const void* p, uintptr_t a) {
    if (!p || !aligned_to(p, a)) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Host-side checks of a host batch.  Only what the host needs is read here
// (the first and last offsets); ids and the monotonicity of the offsets are
// checked on the device by the plan and verify kernels, which report
// violations through the error word.
// Status of a launch's device check bits: the caller's input errors (ids,
// offsets) are SSJ_EINVAL even when a capacity guard fired as their
// consequence; a guard or bounds check alone is a library bug, SSJ_EDEVICE.
ssj_status device_check_status(ssj_ctx* ctx, uint32_t derr) {
    if (derr & (ERR_PROBE_ID | ERR_CAND_ID | ERR_OFFSETS))
        return fail(ctx, SSJ_EINVAL, "batch rejected by the device checks (code %u: %s%s%s)", derr,
                    (derr & ERR_PROBE_ID) ? "probe id out of range " : "",
                    (derr & ERR_CAND_ID) ? "candidate id out of range " : "",
                    (derr & ERR_OFFSETS) ? "offsets not nondecreasing from 0 to n_cands" : "");
    if (derr)
        return fail(ctx, SSJ_EDEVICE, "internal device check fired (code %u: %s%s)", derr,
                    (derr & ERR_GUARD) ? "loop bound reached " : "", (derr & ERR_BOUNDS) ? "index out of bounds" : "");
    return SSJ_OK;
}

ssj_status validate_host_batch(ssj_ctx* ctx, const ssj_batch* b, uint64_t* n_cands) {
    if (b->n_probes && (!b->probe_ids || !b->cand_offsets)) return fail(ctx, SSJ_EINVAL, "NULL batch arrays");
    if (!b->cand_offsets) {
        *n_cands = 0;
        return SSJ_OK;
    }
    if (b->cand_offsets[0] != 0) return fail(ctx, SSJ_EINVAL, "cand_offsets[0] must be 0");
    const uint64_t nc = b->cand_offsets[b->n_probes];
    if (nc >= kMaxCands) return fail(ctx, SSJ_EINVAL, "n_cands must be below 2^40");
    if (b->n_cands && b->n_cands != nc) return fail(ctx, SSJ_EINVAL, "n_cands != cand_offsets[n_probes]");
    if (nc && !b->cand_ids) return fail(ctx, SSJ_EINVAL, "NULL cand_ids");
    *n_cands = nc;
    return SSJ_OK;
}

ssj_status resolve(ssj_ctx* ctx, const ssj_batch* b, Collection** R, Collection** S) {
    if (!ctx || !b) return fail(ctx, SSJ_EINVAL, "NULL argument");
    const uint32_t sim = (b->flags & SSJ_SIM_MASK) >> 8;
    if (sim == SIM_OVERLAP) {
        if (b->p == 0 || b->q == 0 || b->p >= (1u << 31) || b->q >= (1u << 31))
            return fail(ctx, SSJ_EINVAL, "overlap threshold must be 0 < p, q < 2^31");
    } else if (b->p == 0 || b->p > b->q || b->q >= (1u << 31)) {
        return fail(ctx, SSJ_EINVAL, "threshold must be 0 < p <= q < 2^31");
    }
    // sizes derived from n_probes (n_probes + 1 offsets, 32-probe tiles) stay within 32 bits
    if (b->n_probes >= (1u << 31)) return fail(ctx, SSJ_EINVAL, "n_probes must be below 2^31");
    if (b->n_cands >= kMaxCands) return fail(ctx, SSJ_EINVAL, "n_cands must be below 2^40");
    auto ir = ctx->colls.find(b->R);
    auto is = ctx->colls.find(b->S);
    if (ir == ctx->colls.end() || is == ctx->colls.end()) return fail(ctx, SSJ_ENOTFOUND, "unknown collection");
    if (b->R != b->S && (ir->second.renumbered || is->second.renumbered))
        return fail(ctx, SSJ_EINVAL, "renumbered collections can only be self-joined");
    const uint32_t known = SSJ_COUNT_ONLY | SSJ_SORTED | SSJ_DEVICE_PTRS | SSJ_EMIT_ALL | SSJ_FORCE_THREAD |
                           SSJ_FORCE_WARP | SSJ_FORCE_BLOCK | SSJ_FORCE_LANE | SSJ_FORCE_INDEX | SSJ_SIM_MASK |
                           SSJ_KEEP_INPUTS | SSJ_HOST_DIRECT | SSJ_HOST_STAGED;
    if (b->flags & ~known) return fail(ctx, SSJ_EINVAL, "unknown batch flag");
    const uint32_t forced =
        b->flags & (SSJ_FORCE_THREAD | SSJ_FORCE_WARP | SSJ_FORCE_BLOCK | SSJ_FORCE_LANE | SSJ_FORCE_INDEX);
    if (forced & (forced - 1)) return fail(ctx, SSJ_EINVAL, "at most one SSJ_FORCE_* flag");
    *R = &ir->second;
    *S = &is->second;
    return SSJ_OK;
}

uint32_t vflags(uint32_t f) {
    uint32_t v = 0;
    if (f & SSJ_COUNT_ONLY) v |= VF_COUNT_ONLY;
    if (f & SSJ_EMIT_ALL) v |= VF_EMIT_ALL;
    if (f & SSJ_FORCE_THREAD) v |= VF_FORCE_THREAD;
    if (f & SSJ_FORCE_WARP) v |= VF_FORCE_WARP;
    if (f & SSJ_FORCE_BLOCK) v |= VF_FORCE_BLOCK;
    if (f & SSJ_FORCE_LANE) v |= VF_FORCE_LANE;
    if (f & SSJ_FORCE_INDEX) v |= VF_FORCE_INDEX;
    return v;
}

// The instance of one batch (arrays, output and count are filled by the caller).
Instance make_instance(const ssj_batch* b, const Collection& R, const Collection& S, uint64_t n_cands) {
    Instance I;
    memset(&I, 0, sizeof(I));
    I.r_toks4 = reinterpret_cast<const uint4*>(R.d_toks);
    I.r_desc = R.d_desc;
    I.r_n_sets = R.n_sets;
    I.s_toks4 = reinterpret_cast<const uint4*>(S.d_toks);
    I.s_desc = S.d_desc;
    I.s_n_sets = S.n_sets;
    I.r_n_chunks = R.n_chunks;
    I.s_n_chunks = S.n_chunks;
    I.p = b->p;
    I.sim = (b->flags & SSJ_SIM_MASK) >> 8;
    switch (I.sim) {
        case SIM_DICE: I.den = 2 * b->q; break;
        case SIM_COSINE: I.den = b->q; break;
        case SIM_OVERLAP: I.den = (uint32_t)(((uint64_t)b->p + b->q - 1) / b->q); break;
        default: I.den = b->p + b->q; break;
    }
    I.magic = (I.sim == SIM_JACCARD || I.sim == SIM_DICE) ? div_magic(I.den) : 0;
    I.flags = vflags(b->flags) | (b->R == b->S ? VF_SELF_JOIN : 0u);
    I.n_probes = b->n_probes;
    I.n_cands = n_cands;
    I.tile_base = 0;
    return I;
}

// The context's granularity policy for a launch whose collections' token
// values are all below vocab_bound; the probe bitmap of index items is sized
// when index items are on or a batch forces them (and the values fit).
void apply_policy(const ssj_ctx* ctx, VerifyArgs& a, uint64_t vocab_bound, bool force_index) {
    a.thread_max_key = ctx->thread_max_key;
    a.drain_min_live = ctx->drain_min_live;
    a.lane_max_key = ctx->lane_max_key;
    a.warp_max_key = ctx->warp_max_key;
    a.index_min_cands = ctx->index_min_cands;
    a.index_words = (ctx->index_min_cands || force_index) ? index_words_for(vocab_bound) : 0u;
}

// The persisting-L2 window of a pinned collection on the launch (none if c is not pinned).
void set_l2_window(VerifyArgs& a, const Collection& c) {
    a.l2_base = c.l2_window ? c.d_toks : nullptr;
    a.l2_bytes = c.l2_window;
    a.l2_hit_ratio = c.l2_hit_ratio;
}

uint64_t vocab_bound(const Collection& R, const Collection& S) {
    return std::max<uint64_t>(std::max<uint64_t>(R.vocab, S.vocab), 1);
}

VerifyArgs make_args(ssj_ctx* ctx, const ssj_batch* b, const Collection& R, const Collection& S, uint64_t n_cands) {
    VerifyArgs a;
    memset(&a, 0, sizeof(a));
    a.single = make_instance(b, R, S, n_cands);
    a.table = nullptr;
    apply_policy(ctx, a, vocab_bound(R, S), (b->flags & SSJ_FORCE_INDEX) != 0);
    set_l2_window(a, R.l2_window ? R : S);
    return a;
}

// Three timing events for the next launch of a profiling context (else NULL).
cudaEvent_t* profile_events(ssj_ctx* ctx) {
    if (!ctx->profile) return nullptr;
    const size_t need = 3 * (ctx->prof_used + 1);
    while (ctx->prof_ev.size() < need) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
        ctx->prof_ev.push_back(ev);
    }
    cudaEvent_t* evs = &ctx->prof_ev[3 * ctx->prof_used];
    ctx->prof_used++;
    return evs;
}

bool triple_less(const ssj_triple& x, const ssj_triple& y) { return x.r != y.r ? x.r < y.r : x.s < y.s; }

void completion_loop(ssj_ctx* ctx, int slot);

}  // namespace

// ===========================================================================
// Context
// ===========================================================================

extern "C" ssj_status ssj_create(const ssj_config* config, ssj_ctx** out) {
    if (!config || !out) return SSJ_EINVAL;
    if (config->flags & ~SSJ_CTX_PROFILE) return SSJ_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || config->device < 0 || config->device >= ndev) return SSJ_EINVAL;
    std::unique_ptr<ssj_ctx> ctx(new ssj_ctx());
    ctx->device = config->device;
    ctx->profile = (config->flags & SSJ_CTX_PROFILE) != 0;
    DeviceGuard g(ctx->device);
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return SSJ_EDEVICE;
    ctx->budget = config->mem_budget_bytes ? config->mem_budget_bytes : (4ull << 30);
    ctx->max_inflight = config->max_inflight ? config->max_inflight : 4;
    if (config->stream) {
        ctx->stream = static_cast<cudaStream_t>(config->stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return SSJ_EDEVICE;
        ctx->own_stream = true;
    }
    if (cudaMallocHost(reinterpret_cast<void**>(&ctx->h_count), sizeof(uint64_t)) != cudaSuccess) return SSJ_EDEVICE;
    if (cudaMallocHost(reinterpret_cast<void**>(&ctx->h_err), kMaxGroups * sizeof(uint32_t)) != cudaSuccess)
        return SSJ_EDEVICE;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) return SSJ_EDEVICE;
    uint64_t threshold = ctx->budget;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    ctx->slots.resize(ctx->max_inflight);
    for (auto& s : ctx->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return SSJ_EDEVICE;
        // the completion threads sleep on their events instead of spinning, so that many
        // slots do not take the host cores the submitting threads need
        if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess)
            return SSJ_EDEVICE;
        if (cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming) != cudaSuccess) return SSJ_EDEVICE;
        if (cudaMallocHost(reinterpret_cast<void**>(&s.h_count), sizeof(uint64_t)) != cudaSuccess) return SSJ_EDEVICE;
        if (cudaMallocHost(reinterpret_cast<void**>(&s.h_err), sizeof(uint32_t)) != cudaSuccess) return SSJ_EDEVICE;
    }
    ssj_ctx* raw = ctx.release();
    for (size_t i = 0; i < raw->slots.size(); ++i) raw->slots[i].completer = std::thread(completion_loop, raw, (int)i);
    *out = raw;
    return SSJ_OK;
}

// The persisting-L2 set-aside back to what the context had before SSJ_PIN_L2
// raised it, with the persisting lines released.
void release_l2(ssj_ctx* ctx) {
    if (!ctx->l2_limit_raised) return;
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, ctx->l2_limit_found);
    cudaGetLastError();
    ctx->l2_limit_raised = false;
}

extern "C" void ssj_destroy(ssj_ctx* ctx) {
    if (!ctx) return;
    {
        std::unique_lock<std::mutex> lk(ctx->mu);
        ctx->stopping = true;
    }
    ctx->cv.notify_all();
    for (auto& s : ctx->slots)
        if (s.completer.joinable()) s.completer.join();
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& s : ctx->slots) {
        cudaStreamSynchronize(s.stream);
        cudaStreamDestroy(s.stream);
        cudaEventDestroy(s.ev);
        cudaEventDestroy(s.copied);
        cudaFreeHost(s.h_probe);
        cudaFreeHost(s.h_offs);
        cudaFreeHost(s.h_cand);
        cudaFreeHost(s.h_out);
        cudaFreeHost(s.h_count);
        cudaFreeHost(s.h_err);
    }
    for (auto& kv : ctx->tickets)
        if (kv.second->d_mem) {
            cudaFreeAsync(kv.second->d_mem, kv.second->stream);
            cudaStreamSynchronize(kv.second->stream);
        }
    if (ctx->n_pinned) release_l2(ctx);
    for (auto& kv : ctx->colls) {
        cudaFree(kv.second.d_toks);
        cudaFree(kv.second.d_desc);
    }
    cudaFree(ctx->ws);
    cudaFree(ctx->io);
    cudaFreeHost(ctx->h_count);
    cudaFreeHost(ctx->h_err);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t ev : ctx->copy_done)
        if (ev) cudaEventDestroy(ev);
    if (ctx->call_start) cudaEventDestroy(ctx->call_start);

    for (cudaEvent_t ev : ctx->prof_ev) cudaEventDestroy(ev);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" const char* ssj_last_error(ssj_ctx* ctx) {
    if (!ctx) return "NULL context";
    return ctx->err.c_str();
}

extern "C" ssj_status ssj_set_granularity(ssj_ctx* ctx, uint32_t thread_max_key, uint32_t lane_max_key,
                                          uint32_t warp_max_key, uint32_t block_threads) {
    if (!ctx) return SSJ_EINVAL;
    const uint32_t bt = block_threads & ~(SSJ_WIDE_REGISTERS | SSJ_BULK_STAGING);
    if (block_threads && bt != 128 && bt != 256 && bt != 512)
        return fail(ctx, SSJ_EINVAL,
                    "block_threads must be 128, 256 or 512 (optionally | SSJ_WIDE_REGISTERS | SSJ_BULK_STAGING)");
    if (thread_max_key) ctx->thread_max_key = thread_max_key;
    if (lane_max_key) ctx->lane_max_key = lane_max_key;
    if (warp_max_key) ctx->warp_max_key = warp_max_key;
    if (block_threads) ctx->block_threads = block_threads;
    return SSJ_OK;
}

extern "C" ssj_status ssj_set_index_items(ssj_ctx* ctx, uint32_t min_cands) {
    if (!ctx) return SSJ_EINVAL;
    ctx->index_min_cands = min_cands;
    return SSJ_OK;
}

extern "C" ssj_status ssj_set_short_pairs(ssj_ctx* ctx, uint32_t drain_min_live) {
    if (!ctx) return SSJ_EINVAL;
    if (drain_min_live > 24) return fail(ctx, SSJ_EINVAL, "drain_min_live must be 0 .. 24");
    ctx->drain_min_live = drain_min_live;
    return SSJ_OK;
}

// ===========================================================================
// Collections
// ===========================================================================

extern "C" ssj_status ssj_load_collection(ssj_ctx* ctx, const uint64_t* offsets, const uint32_t* tokens,
                                          uint32_t n_sets, uint32_t flags, ssj_coll* out) {
    NvtxScope nvtx_scope("ssj_load_collection");
    if (!ctx || !offsets || !out) return fail(ctx, SSJ_EINVAL, "NULL argument");
    if (flags & ~(SSJ_RENUMBER_BY_FREQ | SSJ_VALIDATE | SSJ_PIN_L2)) return fail(ctx, SSJ_EINVAL, "unknown load flag");
    // a self-join probes every set, and batches hold fewer than 2^31 probes
    if (n_sets >= (1u << 31)) return fail(ctx, SSJ_EINVAL, "n_sets must be below 2^31");
    if (offsets[0] != 0) return fail(ctx, SSJ_EINVAL, "offsets[0] must be 0");
    for (uint32_t i = 0; i < n_sets; ++i)
        if (offsets[i + 1] < offsets[i]) return fail(ctx, SSJ_EINVAL, "offsets decrease at set %u", i);
    const uint64_t total = offsets[n_sets];
    if (total && !tokens) return fail(ctx, SSJ_EINVAL, "NULL tokens");
    DeviceGuard g(ctx->device);

    std::vector<uint32_t> renum;
    const uint32_t* src = tokens;
    if ((flags & SSJ_RENUMBER_BY_FREQ) && total) {
        if (flags & SSJ_VALIDATE) {  // validate the caller's order before it is rewritten
            for (uint32_t s = 0; s < n_sets; ++s)
                for (uint64_t t = offsets[s] + 1; t < offsets[s + 1]; ++t)
                    if (tokens[t - 1] >= tokens[t]) return fail(ctx, SSJ_EINVAL, "set %u is not strictly increasing", s);
        }
        renumber_by_frequency(offsets, tokens, n_sets, renum);
        src = renum.data();
    }

    // raw copies on the device, then the padded layout built there
    uint64_t* d_offs = nullptr;
    uint32_t* d_raw = nullptr;
    uint64_t* d_scratch = nullptr;
    uint32_t* d_err = nullptr;
    Collection c;
    c.n_sets = n_sets;
    c.n_tokens = total;
    c.renumbered = (flags & SSJ_RENUMBER_BY_FREQ) != 0;
    for (uint32_t i = 0; i < n_sets; ++i)
        c.max_len = std::max<uint32_t>(c.max_len, (uint32_t)std::min<uint64_t>(offsets[i + 1] - offsets[i], 0xFFFFFFFFu));
    for (uint64_t t = 0; t < total; ++t) c.vocab = std::max<uint32_t>(c.vocab, src[t] == 0xFFFFFFFFu ? src[t] : src[t] + 1);
    auto cleanup = [&]() {
        cudaFree(d_offs);
        cudaFree(d_raw);
        cudaFree(d_scratch);
        cudaFree(d_err);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&d_offs, sizeof(uint64_t) * (n_sets + 1))) != cudaSuccess ||
        (e = cudaMalloc(&d_raw, sizeof(uint32_t) * std::max<uint64_t>(total, 1))) != cudaSuccess ||
        (e = cudaMalloc(&d_scratch, sizeof(uint64_t) * layout_scratch_words(n_sets))) != cudaSuccess ||
        (e = cudaMalloc(&d_err, sizeof(uint32_t))) != cudaSuccess) {
        cleanup();
        return fail(ctx, SSJ_ENOMEM, "collection staging: %s", cudaGetErrorString(e));
    }
    cudaStream_t st = ctx->stream;
    if ((e = cudaMemcpyAsync(d_offs, offsets, sizeof(uint64_t) * (n_sets + 1), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (total && (e = cudaMemcpyAsync(d_raw, src, sizeof(uint32_t) * total, cudaMemcpyHostToDevice, st)) !=
                      cudaSuccess)) {
        cleanup();
        return cuda_fail(ctx, e, "collection upload");
    }
    const int validate = (flags & SSJ_VALIDATE) && !(flags & SSJ_RENUMBER_BY_FREQ);
    e = layout_lengths(d_offs, d_raw, n_sets, validate, d_scratch, d_err, ctx->h_count, st, ctx->num_sms);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(ctx, e, "layout_lengths");
    }
    c.n_chunks = *ctx->h_count;
    cudaMemcpy(ctx->h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (*ctx->h_err) {
        cleanup();
        return fail(ctx, SSJ_EINVAL, (*ctx->h_err & 1u) ? "a set holds 2^31 tokens or more" : "a set is not strictly increasing");
    }
    if ((e = cudaMalloc(&c.d_toks, 16 * std::max<uint64_t>(c.n_chunks, 1) + 16)) != cudaSuccess ||
        (e = cudaMalloc(&c.d_desc, sizeof(uint2) * std::max<uint32_t>(n_sets, 1))) != cudaSuccess) {
        cudaFree(c.d_toks);
        cleanup();
        return fail(ctx, SSJ_ENOMEM, "collection: %s", cudaGetErrorString(e));
    }
    e = layout_scatter(d_offs, d_raw, n_sets, d_scratch, c.d_toks, c.d_desc, st, ctx->num_sms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
        cudaFree(c.d_toks);
        cudaFree(c.d_desc);
        return cuda_fail(ctx, e, "layout_scatter");
    }
    if (flags & SSJ_PIN_L2) {
        // Persisting-L2 window over the token array, attached to every verify launch that reads
        // this collection.  The context's persisting set-aside (a limit of this context only, gone
        // with it) is raised to the array's size, up to the device's maximum, and restored when
        // the last pinned collection is unloaded.
        int max_persist = 0, max_window = 0;
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device);
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device);
        size_t setaside = 0;
        cudaDeviceGetLimit(&setaside, cudaLimitPersistingL2CacheSize);
        const size_t bytes = 16 * c.n_chunks;
        const size_t want = std::min(bytes, (size_t)std::max(max_persist, 0));
        if (setaside < want) {
            if (!ctx->l2_limit_raised) ctx->l2_limit_found = setaside;
            if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) {
                ctx->l2_limit_raised = true;
                setaside = want;
            }
            cudaGetLastError();  // a refused limit leaves the window smaller, not an error
        }
        c.l2_window = std::min(bytes, (size_t)std::max(max_window, 0));
        if (setaside == 0) c.l2_window = 0;
        c.l2_hit_ratio = c.l2_window ? std::min(1.0f, (float)((double)setaside / (double)c.l2_window)) : 0.f;
        if (c.l2_window) ctx->n_pinned++;
    }
    const ssj_coll h = ctx->next_coll++;
    ctx->colls[h] = c;
    *out = h;
    return SSJ_OK;
}

extern "C" ssj_status ssj_unload_collection(ssj_ctx* ctx, ssj_coll coll) {
    if (!ctx) return SSJ_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->colls.find(coll);
    if (it == ctx->colls.end()) return fail(ctx, SSJ_ENOTFOUND, "unknown collection %u", coll);
    if (it->second.busy) return fail(ctx, SSJ_EBUSY, "collection %u is used by submitted batches", coll);
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(it->second.d_toks);
    cudaFree(it->second.d_desc);
    if (it->second.l2_window && --ctx->n_pinned == 0) release_l2(ctx);
    ctx->colls.erase(it);
    return SSJ_OK;
}

extern "C" ssj_status ssj_collection_info(ssj_ctx* ctx, ssj_coll coll, uint32_t* n_sets, uint64_t* n_tokens) {
    if (!ctx) return SSJ_EINVAL;
    auto it = ctx->colls.find(coll);
    if (it == ctx->colls.end()) return fail(ctx, SSJ_ENOTFOUND, "unknown collection %u", coll);
    if (n_sets) *n_sets = it->second.n_sets;
    if (n_tokens) *n_tokens = it->second.n_tokens;
    return SSJ_OK;
}

// ===========================================================================
// Stream-ordered and synchronous verification
// ===========================================================================

extern "C" ssj_status ssj_reserve(ssj_ctx* ctx, uint32_t n_probes, uint64_t n_cands) {
    if (!ctx) return SSJ_EINVAL;
    if (n_probes >= (1u << 31) || n_cands >= kMaxCands)
        return fail(ctx, SSJ_EINVAL, "n_probes must be below 2^31 and n_cands below 2^40");
    DeviceGuard g(ctx->device);
    return ensure_device_buffer(ctx, &ctx->ws, &ctx->ws_bytes, workspace_bytes(n_probes, n_cands, ctx->num_sms));
}

extern "C" ssj_status ssj_verify_batch_async(ssj_ctx* ctx, const ssj_batch* batch, ssj_triple* d_out, uint64_t cap,
                                             uint64_t* d_count, void* stream) {
    Collection *R, *S;
    ssj_status st = resolve(ctx, batch, &R, &S);
    if (st != SSJ_OK) return st;
    if (!d_count) return fail(ctx, SSJ_EINVAL, "d_count is required");
    if (batch->n_probes && (!batch->probe_ids || !batch->cand_offsets))
        return fail(ctx, SSJ_EINVAL, "NULL batch arrays");
    if (batch->n_cands && !batch->cand_ids) return fail(ctx, SSJ_EINVAL, "NULL cand_ids");
    if (cap && !d_out && !(batch->flags & SSJ_COUNT_ONLY)) return fail(ctx, SSJ_EINVAL, "NULL output");
    st = check_device_alignment(ctx, batch, d_out, d_count);
    if (st != SSJ_OK) return st;
    DeviceGuard g(ctx->device);
    st = ensure_device_buffer(ctx, &ctx->ws, &ctx->ws_bytes, workspace_bytes(batch->n_probes, batch->n_cands, ctx->num_sms));
    if (st != SSJ_OK) return st;
    VerifyArgs a = make_args(ctx, batch, *R, *S, batch->n_cands);
    a.single.probe_ids = batch->probe_ids;
    a.single.cand_offsets = batch->cand_offsets;
    a.single.cand_ids = batch->cand_ids;
    a.single.out = d_out;
    a.single.cap = (batch->flags & SSJ_COUNT_ONLY) ? 0 : cap;
    a.single.count = reinterpret_cast<unsigned long long*>(d_count);
    bind_workspace(a, ctx->ws, batch->n_probes, batch->n_cands, ctx->num_sms);
    ctx->last_ctr = a.ctr;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    cudaError_t e = launch_verify(a, s, ctx->num_sms, ctx->block_threads, profile_events(ctx));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch_verify");
    return SSJ_OK;
}

extern "C" ssj_status ssj_device_error(ssj_ctx* ctx, uint32_t* code) {
    if (!ctx || !code) return SSJ_EINVAL;
    *code = 0;
    if (!ctx->last_ctr) return SSJ_OK;
    DeviceGuard g(ctx->device);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_err, &ctx->last_ctr->err, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    *code = *ctx->h_err;
    CUDA_TRY(ctx, cudaMemsetAsync(&ctx->last_ctr->err, 0, sizeof(uint32_t), ctx->stream));
    return SSJ_OK;
}

extern "C" ssj_status ssj_verify_batch(ssj_ctx* ctx, const ssj_batch* batch, ssj_triple* out, uint64_t cap,
                                       uint64_t* n_out) {
    NvtxScope nvtx_scope("ssj_verify_batch");
    Collection *R, *S;
    ssj_status st = resolve(ctx, batch, &R, &S);
    if (st != SSJ_OK) return st;
    if (!n_out) return fail(ctx, SSJ_EINVAL, "n_out is required");
    if (cap && !out && !(batch->flags & SSJ_COUNT_ONLY)) return fail(ctx, SSJ_EINVAL, "NULL output with cap > 0");
    DeviceGuard g(ctx->device);
    const bool dev = (batch->flags & SSJ_DEVICE_PTRS) != 0;
    const bool count_only = (batch->flags & SSJ_COUNT_ONLY) != 0;
    cudaStream_t s = ctx->stream;
    uint64_t n_cands = 0;
    VerifyArgs a;
    uint64_t* d_count = nullptr;
    if (!dev) {
        st = validate_host_batch(ctx, batch, &n_cands);
        if (st != SSJ_OK) return st;
        a = make_args(ctx, batch, *R, *S, n_cands);
        // device staging: probe ids, offsets, candidates, count, output
        const uint64_t out_cap = count_only ? 0 : std::min<uint64_t>(cap, n_cands);
        size_t off = 0;
        const size_t o_probe = off; off += align256(4ull * std::max<uint32_t>(batch->n_probes, 1));
        const size_t o_offs = off;  off += align256(8ull * (batch->n_probes + 1));
        const size_t o_cand = off;  off += align256(4ull * std::max<uint64_t>(n_cands, 1));
        const size_t o_cnt = off;   off += 256;
        const size_t o_out = off;   off += align256(sizeof(ssj_triple) * std::max<uint64_t>(out_cap, 1));
        st = ensure_device_buffer(ctx, &ctx->io, &ctx->io_bytes, off);
        if (st != SSJ_OK) return st;
        char* base = static_cast<char*>(ctx->io);
        uint32_t* d_probe = reinterpret_cast<uint32_t*>(base + o_probe);
        uint64_t* d_offs = reinterpret_cast<uint64_t*>(base + o_offs);
        uint32_t* d_cand = reinterpret_cast<uint32_t*>(base + o_cand);
        d_count = reinterpret_cast<uint64_t*>(base + o_cnt);
        ssj_triple* d_out = reinterpret_cast<ssj_triple*>(base + o_out);
        if (batch->n_probes) {
            CUDA_TRY(ctx, cudaMemcpyAsync(d_probe, batch->probe_ids, 4ull * batch->n_probes, cudaMemcpyHostToDevice, s));
            CUDA_TRY(ctx, cudaMemcpyAsync(d_offs, batch->cand_offsets, 8ull * (batch->n_probes + 1),
                                          cudaMemcpyHostToDevice, s));
        }
        if (n_cands)
            CUDA_TRY(ctx, cudaMemcpyAsync(d_cand, batch->cand_ids, 4ull * n_cands, cudaMemcpyHostToDevice, s));
        a.single.probe_ids = d_probe;
        a.single.cand_offsets = d_offs;
        a.single.cand_ids = d_cand;
        a.single.out = d_out;
        a.single.cap = out_cap;
    } else {
        n_cands = batch->n_cands;
        if (batch->n_probes && (!batch->probe_ids || !batch->cand_offsets))
            return fail(ctx, SSJ_EINVAL, "NULL batch arrays");
        if (n_cands && !batch->cand_ids) return fail(ctx, SSJ_EINVAL, "NULL cand_ids");
        st = check_device_alignment(ctx, batch, out, nullptr);
        if (st != SSJ_OK) return st;
        a = make_args(ctx, batch, *R, *S, n_cands);
        a.single.probe_ids = batch->probe_ids;
        a.single.cand_offsets = batch->cand_offsets;
        a.single.cand_ids = batch->cand_ids;
        a.single.out = out;
        a.single.cap = count_only ? 0 : cap;
        st = ensure_device_buffer(ctx, &ctx->io, &ctx->io_bytes, 256);
        if (st != SSJ_OK) return st;
        d_count = static_cast<uint64_t*>(ctx->io);
    }
    st = ensure_device_buffer(ctx, &ctx->ws, &ctx->ws_bytes, workspace_bytes(batch->n_probes, n_cands, ctx->num_sms));
    if (st != SSJ_OK) return st;
    a.single.count = reinterpret_cast<unsigned long long*>(d_count);
    bind_workspace(a, ctx->ws, batch->n_probes, n_cands, ctx->num_sms);
    ctx->last_ctr = a.ctr;
    cudaError_t e = launch_verify(a, s, ctx->num_sms, ctx->block_threads, profile_events(ctx));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch_verify");
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_count, d_count, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_err, &a.ctr->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const uint64_t count = *ctx->h_count;
    const uint32_t derr = *ctx->h_err;
    *n_out = count;
    if (derr) return device_check_status(ctx, derr);
    if (count_only) return SSJ_OK;
    const uint64_t n_copy = std::min(count, cap);
    if (!dev) {
        if (n_copy) CUDA_TRY(ctx, cudaMemcpy(out, a.single.out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost));
        if (batch->flags & SSJ_SORTED) std::sort(out, out + n_copy, triple_less);
    } else if ((batch->flags & SSJ_SORTED) && n_copy) {
        std::vector<ssj_triple> h(n_copy);
        CUDA_TRY(ctx, cudaMemcpy(h.data(), out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost));
        std::sort(h.begin(), h.end(), triple_less);
        CUDA_TRY(ctx, cudaMemcpy(out, h.data(), sizeof(ssj_triple) * n_copy, cudaMemcpyHostToDevice));
    }
    if (count > cap) return fail(ctx, SSJ_ENOMEM, "%llu result pairs, room for %llu", (unsigned long long)count,
                                 (unsigned long long)cap);
    return SSJ_OK;
}

extern "C" ssj_status ssj_verify_batches(ssj_ctx* ctx, const ssj_batch* batches, uint32_t n_batches,
                                         ssj_triple* const* outs, const uint64_t* caps, uint64_t* n_outs) {
    NvtxScope nvtx_scope("ssj_verify_batches");
    if (!ctx || (n_batches && (!batches || !outs || !caps || !n_outs))) return fail(ctx, SSJ_EINVAL, "NULL argument");
    if (n_batches == 0) return SSJ_OK;
    std::vector<Instance> table(n_batches);
    std::vector<uint64_t> n_cands(n_batches), io_off(n_batches);
    LaunchShape sh;
    sh.n_inst = n_batches;
    sh.n_tiles = 0;
    sh.total_probes = 0;
    sh.total_cands = 0;
    size_t off = align256(sizeof(uint64_t) * n_batches);  // counts first
    uint64_t launch_vocab = 1;
    bool launch_force_index = false;
    const Collection* pinned = nullptr;  // the first pinned collection: its L2 window
    for (uint32_t i = 0; i < n_batches; ++i) {
        const ssj_batch* b = &batches[i];
        if (b->flags & SSJ_DEVICE_PTRS) return fail(ctx, SSJ_EINVAL, "batch %u: host pointers expected", i);
        Collection *R, *S;
        ssj_status st = resolve(ctx, b, &R, &S);
        if (st != SSJ_OK) return st;
        st = validate_host_batch(ctx, b, &n_cands[i]);
        if (st != SSJ_OK) return st;
        if (caps[i] && !outs[i] && !(b->flags & SSJ_COUNT_ONLY)) return fail(ctx, SSJ_EINVAL, "batch %u: NULL output", i);
        table[i] = make_instance(b, *R, *S, n_cands[i]);
        if (!pinned) pinned = R->l2_window ? R : (S->l2_window ? S : nullptr);
        launch_vocab = std::max(launch_vocab, vocab_bound(*R, *S));
        launch_force_index = launch_force_index || (b->flags & SSJ_FORCE_INDEX) != 0;
        table[i].tile_base = sh.n_tiles;
        const uint64_t tiles = ((uint64_t)b->n_probes + 31) / 32;
        if ((uint64_t)sh.n_tiles + tiles > 0x7FFFFFFull) return fail(ctx, SSJ_EINVAL, "too many probes in one call");
        sh.n_tiles += (uint32_t)tiles;
        sh.total_probes += b->n_probes;
        sh.total_cands += n_cands[i];
        if (sh.total_cands >= kMaxCands) return fail(ctx, SSJ_EINVAL, "2^40 or more candidates in one call");
        // device staging of this batch: probe ids, offsets, candidate ids, output
        io_off[i] = off;
        off += align256(4ull * std::max<uint32_t>(b->n_probes, 1)) + align256(8ull * (b->n_probes + 1)) +
               align256(4ull * std::max<uint64_t>(n_cands[i], 1));
        const uint64_t cap = (b->flags & SSJ_COUNT_ONLY) ? 0 : std::min(caps[i], n_cands[i]);
        off += align256(sizeof(ssj_triple) * std::max<uint64_t>(cap, 1));
    }
    // Large calls run as up to kMaxGroups launches over consecutive groups of batches with about
    // equal candidate counts: each later group's host-to-device copies, on a second stream,
    // overlap the earlier groups' kernels.
    uint32_t groups = (uint32_t)std::min<uint64_t>(
        {(uint64_t)kMaxGroups, (uint64_t)n_batches, std::max<uint64_t>(sh.total_cands / kSplitCands, 1)});
    uint32_t gstart[kMaxGroups + 1];
    {
        uint32_t g = 0;
        uint64_t acc = 0;
        gstart[0] = 0;
        for (uint32_t i = 0; i < n_batches && g + 1 < groups; ++i) {
            acc += n_cands[i];
            if (acc * groups >= (uint64_t)(g + 1) * sh.total_cands && i + 1 < n_batches) gstart[++g] = i + 1;
        }
        groups = g + 1;  // (a group is never empty)
        gstart[groups] = n_batches;
    }
    LaunchShape shp[kMaxGroups];
    size_t ws_off[kMaxGroups + 1];
    ws_off[0] = 0;
    for (uint32_t gi = 0; gi < groups; ++gi) {
        LaunchShape& q = shp[gi];
        q.n_inst = 0;
        q.n_tiles = 0;
        q.total_probes = 0;
        q.total_cands = 0;
        for (uint32_t i = gstart[gi]; i < gstart[gi + 1]; ++i) {
            table[i].tile_base = q.n_tiles;
            q.n_inst += 1;
            q.n_tiles += (uint32_t)(((uint64_t)batches[i].n_probes + 31) / 32);
            q.total_probes += batches[i].n_probes;
            q.total_cands += n_cands[i];
        }
        ws_off[gi + 1] = ws_off[gi] + align256(workspace_bytes(q, ctx->num_sms));
    }
    const size_t ws_total = ws_off[groups];
    DeviceGuard g(ctx->device);
    ssj_status st = ensure_device_buffer(ctx, &ctx->io, &ctx->io_bytes, off);
    if (st != SSJ_OK) return st;
    st = ensure_device_buffer(ctx, &ctx->ws, &ctx->ws_bytes, ws_total);
    if (st != SSJ_OK) return st;
    cudaStream_t s = ctx->stream;
    cudaStream_t cs = s;  // the later groups' copies
    if (groups > 1) {
        if (!ctx->copy_stream) CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (uint32_t gi = 0; gi < kMaxGroups; ++gi)
            if (!ctx->copy_done[gi]) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->copy_done[gi], cudaEventDisableTiming));
        if (!ctx->call_start) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->call_start, cudaEventDisableTiming));
        cs = ctx->copy_stream;
        // the copy stream starts after everything already queued on the context's stream
        CUDA_TRY(ctx, cudaEventRecord(ctx->call_start, s));
        CUDA_TRY(ctx, cudaStreamWaitEvent(cs, ctx->call_start, 0));
    }
    char* base = static_cast<char*>(ctx->io);
    uint64_t* d_counts = reinterpret_cast<uint64_t*>(base);
    for (uint32_t i = 0, gi = 0; i < n_batches; ++i) {
        if (i == gstart[gi + 1]) {  // group gi's copies are all queued
            if (gi > 0) CUDA_TRY(ctx, cudaEventRecord(ctx->copy_done[gi], cs));
            ++gi;
        }
        const cudaStream_t cp = gi == 0 ? s : cs;
        const ssj_batch* b = &batches[i];
        char* p = base + io_off[i];
        uint32_t* d_probe = reinterpret_cast<uint32_t*>(p); p += align256(4ull * std::max<uint32_t>(b->n_probes, 1));
        uint64_t* d_offs = reinterpret_cast<uint64_t*>(p);  p += align256(8ull * (b->n_probes + 1));
        uint32_t* d_cand = reinterpret_cast<uint32_t*>(p);  p += align256(4ull * std::max<uint64_t>(n_cands[i], 1));
        // SSJ_HOST_DIRECT: pinned arrays the device can address are read by the kernels
        // themselves (over the host link), with no staging copy
        // (calls of 2^25+ candidates read pinned inputs directly unless the batch asks for staging)
        const bool direct = (b->flags & SSJ_HOST_DIRECT) ||
                            (sh.total_cands >= kDirectCands && !(b->flags & SSJ_HOST_STAGED));
        const void* dv_probe = direct ? device_view(b->probe_ids, 4) : nullptr;
        const void* dv_offs = direct ? device_view(b->cand_offsets, 8) : nullptr;
        const void* dv_cand = direct ? device_view(b->cand_ids, 4) : nullptr;
        if (b->n_probes && !dv_probe)
            CUDA_TRY(ctx, cudaMemcpyAsync(d_probe, b->probe_ids, 4ull * b->n_probes, cudaMemcpyHostToDevice, cp));
        if (b->n_probes && !dv_offs)
            CUDA_TRY(ctx, cudaMemcpyAsync(d_offs, b->cand_offsets, 8ull * (b->n_probes + 1), cudaMemcpyHostToDevice, cp));
        if (n_cands[i] && !dv_cand)
            CUDA_TRY(ctx, cudaMemcpyAsync(d_cand, b->cand_ids, 4ull * n_cands[i], cudaMemcpyHostToDevice, cp));
        Instance& I = table[i];
        I.probe_ids = dv_probe ? static_cast<const uint32_t*>(dv_probe) : d_probe;
        I.cand_offsets = dv_offs ? static_cast<const uint64_t*>(dv_offs) : d_offs;
        I.cand_ids = dv_cand ? static_cast<const uint32_t*>(dv_cand) : d_cand;
        I.out = reinterpret_cast<ssj_triple*>(p);
        I.cap = (b->flags & SSJ_COUNT_ONLY) ? 0 : std::min(caps[i], n_cands[i]);
        I.count = reinterpret_cast<unsigned long long*>(d_counts + i);
    }
    if (groups > 1) CUDA_TRY(ctx, cudaEventRecord(ctx->copy_done[groups - 1], cs));
    for (uint32_t gi = 0; gi < groups; ++gi) {
        const uint32_t lo = gstart[gi], hi = gstart[gi + 1];
        VerifyArgs a;
        memset(&a, 0, sizeof(a));
        apply_policy(ctx, a, launch_vocab, launch_force_index);
        if (pinned) set_l2_window(a, *pinned);
        bind_workspace(a, static_cast<char*>(ctx->ws) + ws_off[gi], shp[gi], ctx->num_sms);
        a.table = a.table_out;
        if (gi > 0) CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->copy_done[gi], 0));  // the group's inputs are in
        CUDA_TRY(ctx, cudaMemcpyAsync(a.table_out, table.data() + lo, sizeof(Instance) * (hi - lo),
                                      cudaMemcpyHostToDevice, s));
        ctx->last_ctr = a.ctr;
        cudaError_t e = launch_verify(a, s, ctx->num_sms, ctx->block_threads, profile_events(ctx));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "launch_verify");
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_err + gi, &a.ctr->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    std::vector<uint64_t> counts(n_batches);
    CUDA_TRY(ctx, cudaMemcpyAsync(counts.data(), d_counts, sizeof(uint64_t) * n_batches, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    uint32_t derr = 0;
    for (uint32_t gi = 0; gi < groups; ++gi) derr |= ctx->h_err[gi];
    if (derr) return device_check_status(ctx, derr);
    bool short_cap = false;
    for (uint32_t i = 0; i < n_batches; ++i) {
        n_outs[i] = counts[i];
        if (batches[i].flags & SSJ_COUNT_ONLY) continue;
        const uint64_t n_copy = std::min(counts[i], caps[i]);
        if (n_copy)
            CUDA_TRY(ctx, cudaMemcpyAsync(outs[i], table[i].out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost, s));
        short_cap |= counts[i] > caps[i];
    }
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (uint32_t i = 0; i < n_batches; ++i)
        if ((batches[i].flags & SSJ_SORTED) && !(batches[i].flags & SSJ_COUNT_ONLY))
            std::sort(outs[i], outs[i] + std::min(counts[i], caps[i]), triple_less);
    if (short_cap) return fail(ctx, SSJ_ENOMEM, "a batch has more result pairs than its capacity (see n_outs)");
    return SSJ_OK;
}

// ===========================================================================
// Self-join with candidates generated on the device
// ===========================================================================

extern "C" ssj_status ssj_self_join(ssj_ctx* ctx, ssj_coll coll, uint32_t p, uint32_t q, uint32_t flags,
                                    ssj_triple* out, uint64_t cap, uint64_t* n_out, uint64_t* n_candidates) {
    NvtxScope nvtx_scope("ssj_self_join");
    if (!ctx || !n_out) return fail(ctx, SSJ_EINVAL, "NULL argument");
    const uint32_t known = SSJ_COUNT_ONLY | SSJ_SORTED | SSJ_DEVICE_PTRS | SSJ_SIM_MASK | SSJ_JOIN_POSITIONAL |
                           SSJ_FORCE_THREAD | SSJ_FORCE_WARP | SSJ_FORCE_BLOCK | SSJ_FORCE_LANE | SSJ_FORCE_INDEX;
    if (flags & ~known) return fail(ctx, SSJ_EINVAL, "unknown flag");
    if (cap && !out && !(flags & SSJ_COUNT_ONLY)) return fail(ctx, SSJ_EINVAL, "NULL output with cap > 0");
    if ((flags & SSJ_DEVICE_PTRS) && !aligned_to(out, 4))
        return fail(ctx, SSJ_EINVAL, "device output must be aligned to 4 bytes");
    // threshold and collection checks through the batch path's resolve()
    ssj_batch probe_b;
    memset(&probe_b, 0, sizeof(probe_b));
    probe_b.R = probe_b.S = coll;
    probe_b.p = p;
    probe_b.q = q;
    probe_b.flags = flags & (SSJ_SIM_MASK | SSJ_FORCE_THREAD | SSJ_FORCE_WARP | SSJ_FORCE_BLOCK | SSJ_FORCE_LANE |
                             SSJ_FORCE_INDEX);
    Collection *R, *S;
    ssj_status st = resolve(ctx, &probe_b, &R, &S);
    if (st != SSJ_OK) return st;
    const Collection& C = *R;
    if (C.vocab > (1u << 30)) return fail(ctx, SSJ_EINVAL, "token values above 2^30: load with SSJ_RENUMBER_BY_FREQ");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const uint32_t n = C.n_sets;
    std::vector<void*> mem;
    auto release = [&]() {
        for (void* m : mem) cudaFree(m);
        mem.clear();
    };
    auto alloc = [&](size_t bytes) -> void* {
        void* m = nullptr;
        if (cudaMalloc(&m, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        mem.push_back(m);
        return m;
    };
    CandgenIndex ix;
    const uint64_t scan_n = std::max<uint64_t>((uint64_t)C.max_len + 2, (uint64_t)C.vocab + 1);
    ix.size_hist = static_cast<uint64_t*>(alloc(8ull * (C.max_len + 2)));
    ix.order = static_cast<uint32_t*>(alloc(4ull * n));
    ix.rank = static_cast<uint32_t*>(alloc(4ull * n));
    ix.tcnt = static_cast<uint64_t*>(alloc(8ull * (C.vocab + 1)));
    ix.toff = static_cast<uint64_t*>(alloc(8ull * (C.vocab + 1)));
    ix.scan_scratch = static_cast<uint64_t*>(alloc(8ull * scan_scratch_words(scan_n)));
    ix.total = static_cast<uint64_t*>(alloc(8));
    ix.post = nullptr;
    uint32_t* d_err = static_cast<uint32_t*>(alloc(4));
    if (!ix.size_hist || !ix.order || !ix.rank || !ix.tcnt || !ix.toff || !ix.scan_scratch || !ix.total || !d_err) {
        release();
        return fail(ctx, SSJ_ENOMEM, "candidate generation index");
    }
    CandgenInput in;
    memset(&in, 0, sizeof(in));
    in.toks4 = reinterpret_cast<const uint4*>(C.d_toks);
    in.desc = C.d_desc;
    in.n = n;
    in.max_len = C.max_len;
    in.vocab = C.vocab;
    in.sim = (flags & SSJ_SIM_MASK) >> 8;
    in.p = p;
    in.q = q;
    in.positional = (flags & SSJ_JOIN_POSITIONAL) ? 1u : 0u;
    cudaError_t e = cudaMemsetAsync(d_err, 0, 4, s);
    in.stage = 0;
    if (e == cudaSuccess) e = candgen_run(in, s, ctx->num_sms, &ix, ctx->h_count);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "candidate generation (index)");
    }
    const uint64_t entries = *ctx->h_count;
    ix.post = static_cast<uint4*>(alloc(16ull * entries));
    if (!ix.post) {
        release();
        return fail(ctx, SSJ_ENOMEM, "prefix index of %llu entries", (unsigned long long)entries);
    }
    in.stage = 1;
    e = candgen_run(in, s, ctx->num_sms, &ix, ctx->h_count);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "candidate generation (count)");
    }
    const uint64_t bound = *ctx->h_count;  // entries that can yield a candidate
    uint64_t tsize = 1024;
    while (tsize < 2 * bound) tsize <<= 1;
    const uint64_t group_cap = (uint64_t)n + bound / 224 + 1;
    in.table = static_cast<unsigned long long*>(alloc(8ull * tsize));
    in.table_mask = tsize - 1;
    in.out.probe_ids = static_cast<uint32_t*>(alloc(4ull * group_cap));
    in.out.cand_offsets = static_cast<uint64_t*>(alloc(8ull * (group_cap + 1)));
    in.out.cand_ids = static_cast<uint32_t*>(alloc(4ull * std::max<uint64_t>(bound, 1)));
    in.out.packed = static_cast<unsigned long long*>(alloc(8));
    in.out.group_cap = group_cap;
    in.out.cand_cap = bound;
    in.out.err = d_err;
    if (!in.table || !in.out.probe_ids || !in.out.cand_offsets || !in.out.cand_ids || !in.out.packed) {
        release();
        return fail(ctx, SSJ_ENOMEM, "candidate generation output (%llu entries)", (unsigned long long)bound);
    }
    in.stage = 2;
    e = candgen_run(in, s, ctx->num_sms, &ix, ctx->h_count);
    uint32_t derr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&derr, d_err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "candidate generation (probe)");
    }
    if (derr) {
        release();
        return fail(ctx, SSJ_EDEVICE, "candidate generation: an output capacity was exceeded or the candidate hash set was full (code %u)", derr);
    }
    const uint64_t packed = *ctx->h_count;
    const uint64_t groups = packed >> 40, total = packed & ((1ull << 40) - 1);
    if (n_candidates) *n_candidates = total;
    e = cudaMemcpy(in.out.cand_offsets + groups, &total, 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "candidate offsets");
    }
    // index and hash table are no longer needed; verify the generated batch
    ssj_batch b;
    memset(&b, 0, sizeof(b));
    b.R = b.S = coll;
    b.p = p;
    b.q = q;
    b.n_probes = (uint32_t)groups;
    b.probe_ids = in.out.probe_ids;
    b.cand_offsets = in.out.cand_offsets;
    b.cand_ids = in.out.cand_ids;
    b.n_cands = total;
    b.flags = (flags & ~(SSJ_JOIN_POSITIONAL | SSJ_DEVICE_PTRS | SSJ_SORTED)) | SSJ_DEVICE_PTRS;
    if (groups > 0xFFFFFFFFull) {
        release();
        return fail(ctx, SSJ_EINVAL, "too many candidate groups");
    }
    const bool count_only = (flags & SSJ_COUNT_ONLY) != 0;
    const bool dev_out = (flags & SSJ_DEVICE_PTRS) != 0;
    ssj_triple* d_out = nullptr;
    uint64_t d_cap = 0;
    if (!count_only) {
        if (dev_out) {
            d_out = out;
            d_cap = cap;
        } else {
            d_cap = std::min<uint64_t>(cap, total);
            d_out = static_cast<ssj_triple*>(alloc(sizeof(ssj_triple) * std::max<uint64_t>(d_cap, 1)));
            if (!d_out) {
                release();
                return fail(ctx, SSJ_ENOMEM, "join output");
            }
        }
    }
    uint64_t count = 0;
    st = ssj_verify_batch(ctx, &b, d_out, d_cap, &count);
    *n_out = count;
    if (st != SSJ_OK && st != SSJ_ENOMEM) {
        release();
        return st;
    }
    if (!count_only) {
        const uint64_t n_copy = std::min(count, cap);
        if (dev_out) {
            if ((flags & SSJ_SORTED) && n_copy) {
                std::vector<ssj_triple> h(n_copy);
                e = cudaMemcpy(h.data(), out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost);
                std::sort(h.begin(), h.end(), triple_less);
                if (e == cudaSuccess) e = cudaMemcpy(out, h.data(), sizeof(ssj_triple) * n_copy, cudaMemcpyHostToDevice);
            }
        } else if (n_copy) {
            e = cudaMemcpy(out, d_out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && (flags & SSJ_SORTED)) std::sort(out, out + n_copy, triple_less);
        }
        if (e != cudaSuccess) {
            release();
            return cuda_fail(ctx, e, "join results");
        }
    }
    release();
    if (count > cap && !count_only)
        return fail(ctx, SSJ_ENOMEM, "%llu result pairs, room for %llu", (unsigned long long)count,
                    (unsigned long long)cap);
    return SSJ_OK;
}

// ===========================================================================
// GroupJoin: group candidates expanded on the device
// ===========================================================================

extern "C" ssj_status ssj_verify_groups(ssj_ctx* ctx, const ssj_group_batch* gb, ssj_triple* out, uint64_t cap,
                                        uint64_t* n_out, uint64_t* n_pairs) {
    NvtxScope nvtx_scope("ssj_verify_groups");
    if (!ctx || !gb || !n_out) return fail(ctx, SSJ_EINVAL, "NULL argument");
    const uint32_t known = SSJ_COUNT_ONLY | SSJ_SORTED | SSJ_DEVICE_PTRS | SSJ_SIM_MASK | SSJ_FORCE_THREAD |
                           SSJ_FORCE_WARP | SSJ_FORCE_BLOCK | SSJ_FORCE_LANE | SSJ_FORCE_INDEX;
    if (gb->flags & ~known) return fail(ctx, SSJ_EINVAL, "unknown flag");
    if (cap && !out && !(gb->flags & SSJ_COUNT_ONLY)) return fail(ctx, SSJ_EINVAL, "NULL output with cap > 0");
    if ((gb->flags & SSJ_DEVICE_PTRS) && !aligned_to(out, 4))
        return fail(ctx, SSJ_EINVAL, "device output must be aligned to 4 bytes");
    if (!gb->group_offsets || (gb->n_groups && !gb->members) || (gb->n_probe_groups && (!gb->probe_groups ||
        !gb->cand_offsets)))
        return fail(ctx, SSJ_EINVAL, "NULL group arrays");
    ssj_batch probe_b;
    memset(&probe_b, 0, sizeof(probe_b));
    probe_b.R = probe_b.S = gb->coll;
    probe_b.p = gb->p;
    probe_b.q = gb->q;
    probe_b.flags = gb->flags & (SSJ_SIM_MASK | SSJ_FORCE_THREAD | SSJ_FORCE_WARP | SSJ_FORCE_BLOCK | SSJ_FORCE_LANE |
                                SSJ_FORCE_INDEX);
    Collection *R, *S;
    ssj_status st = resolve(ctx, &probe_b, &R, &S);
    if (st != SSJ_OK) return st;
    const Collection& C = *R;
    // host-side checks of the group layout (ids are the collection's)
    const uint64_t n_members = gb->group_offsets[gb->n_groups];
    if (gb->group_offsets[0] != 0) return fail(ctx, SSJ_EINVAL, "group_offsets[0] must be 0");
    for (uint32_t g = 0; g < gb->n_groups; ++g)
        if (gb->group_offsets[g + 1] <= gb->group_offsets[g]) return fail(ctx, SSJ_EINVAL, "group %u is empty", g);
    for (uint64_t i = 0; i < n_members; ++i)
        if (gb->members[i] >= C.n_sets) return fail(ctx, SSJ_EINVAL, "member id out of range");
    const uint64_t n_cg = gb->n_probe_groups ? gb->cand_offsets[gb->n_probe_groups] : 0;
    if (gb->n_probe_groups && gb->cand_offsets[0] != 0) return fail(ctx, SSJ_EINVAL, "cand_offsets[0] must be 0");
    for (uint32_t k = 0; k < gb->n_probe_groups; ++k) {
        if (gb->probe_groups[k] >= gb->n_groups || gb->cand_offsets[k + 1] < gb->cand_offsets[k])
            return fail(ctx, SSJ_EINVAL, "probe group entry %u invalid", k);
    }
    for (uint64_t c = 0; c < n_cg; ++c)
        if (gb->cand_groups[c] >= gb->n_groups) return fail(ctx, SSJ_EINVAL, "candidate group id out of range");
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    std::vector<void*> mem;
    auto release = [&]() {
        for (void* m : mem) cudaFree(m);
        mem.clear();
    };
    auto alloc = [&](size_t bytes) -> void* {
        void* m = nullptr;
        if (cudaMalloc(&m, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        mem.push_back(m);
        return m;
    };
    const uint64_t n_entries = (uint64_t)gb->n_groups + gb->n_probe_groups;
    GroupExpand x;
    memset(&x, 0, sizeof(x));
    x.toks4 = reinterpret_cast<const uint4*>(C.d_toks);
    x.desc = C.d_desc;
    x.sim = (gb->flags & SSJ_SIM_MASK) >> 8;
    x.p = gb->p;
    x.q = gb->q;
    x.n_groups = gb->n_groups;
    x.n_probe_groups = gb->n_probe_groups;
    uint64_t* d_goff = static_cast<uint64_t*>(alloc(8ull * (gb->n_groups + 1)));
    uint32_t* d_mem = static_cast<uint32_t*>(alloc(4ull * n_members));
    uint32_t* d_pg = static_cast<uint32_t*>(alloc(4ull * gb->n_probe_groups));
    uint64_t* d_coff = static_cast<uint64_t*>(alloc(8ull * (gb->n_probe_groups + 1)));
    uint32_t* d_cg = static_cast<uint32_t*>(alloc(4ull * n_cg));
    x.probe_off = static_cast<uint64_t*>(alloc(8ull * (n_entries + 1)));
    x.pair_off = static_cast<uint64_t*>(alloc(8ull * (n_entries + 1)));
    x.per_probe = static_cast<uint64_t*>(alloc(8ull * (n_entries + 1)));
    x.scan_scratch = static_cast<uint64_t*>(alloc(8ull * scan_scratch_words(n_entries + 1)));
    x.total = static_cast<uint64_t*>(alloc(8));
    if (!d_goff || !d_mem || !d_pg || !d_coff || !d_cg || !x.probe_off || !x.pair_off || !x.per_probe ||
        !x.scan_scratch || !x.total) {
        release();
        return fail(ctx, SSJ_ENOMEM, "group expansion");
    }
    cudaError_t e = cudaMemcpyAsync(d_goff, gb->group_offsets, 8ull * (gb->n_groups + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_members) e = cudaMemcpyAsync(d_mem, gb->members, 4ull * n_members, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && gb->n_probe_groups) {
        e = cudaMemcpyAsync(d_pg, gb->probe_groups, 4ull * gb->n_probe_groups, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_coff, gb->cand_offsets, 8ull * (gb->n_probe_groups + 1), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess && n_cg) e = cudaMemcpyAsync(d_cg, gb->cand_groups, 4ull * n_cg, cudaMemcpyHostToDevice, s);
    x.group_offsets = d_goff;
    x.members = d_mem;
    x.probe_groups = d_pg;
    x.cand_offsets = d_coff;
    x.cand_groups = d_cg;
    uint64_t words[2] = {0, 0};
    x.stage = 0;
    if (e == cudaSuccess) e = expand_groups(x, s, ctx->num_sms, words);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "group expansion (count)");
    }
    const uint64_t probes = words[0], pairs = words[1];
    if (n_pairs) *n_pairs = pairs;
    if (probes > 0xFFFFFFFFull) {
        release();
        return fail(ctx, SSJ_EINVAL, "too many expanded probes");
    }
    x.probe_ids = static_cast<uint32_t*>(alloc(4ull * probes));
    x.cand_offsets_out = static_cast<uint64_t*>(alloc(8ull * (probes + 1)));
    x.cand_ids = static_cast<uint32_t*>(alloc(4ull * pairs));
    if (!x.probe_ids || !x.cand_offsets_out || !x.cand_ids) {
        release();
        return fail(ctx, SSJ_ENOMEM, "expanded candidates (%llu pairs)", (unsigned long long)pairs);
    }
    x.stage = 1;
    e = expand_groups(x, s, ctx->num_sms, words);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "group expansion (write)");
    }
    ssj_batch b;
    memset(&b, 0, sizeof(b));
    b.R = b.S = gb->coll;
    b.p = gb->p;
    b.q = gb->q;
    b.n_probes = (uint32_t)probes;
    b.probe_ids = x.probe_ids;
    b.cand_offsets = x.cand_offsets_out;
    b.cand_ids = x.cand_ids;
    b.n_cands = pairs;
    b.flags = (gb->flags & ~(SSJ_DEVICE_PTRS | SSJ_SORTED)) | SSJ_DEVICE_PTRS;
    const bool count_only = (gb->flags & SSJ_COUNT_ONLY) != 0;
    const bool dev_out = (gb->flags & SSJ_DEVICE_PTRS) != 0;
    ssj_triple* d_out = nullptr;
    uint64_t d_cap = 0;
    if (!count_only) {
        if (dev_out) {
            d_out = out;
            d_cap = cap;
        } else {
            d_cap = std::min<uint64_t>(cap, pairs);
            d_out = static_cast<ssj_triple*>(alloc(sizeof(ssj_triple) * std::max<uint64_t>(d_cap, 1)));
            if (!d_out) {
                release();
                return fail(ctx, SSJ_ENOMEM, "group join output");
            }
        }
    }
    uint64_t count = 0;
    st = ssj_verify_batch(ctx, &b, d_out, d_cap, &count);
    *n_out = count;
    if (st != SSJ_OK && st != SSJ_ENOMEM) {
        release();
        return st;
    }
    if (!count_only) {
        const uint64_t n_copy = std::min(count, cap);
        if (dev_out) {
            if ((gb->flags & SSJ_SORTED) && n_copy) {
                std::vector<ssj_triple> h(n_copy);
                e = cudaMemcpy(h.data(), out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost);
                std::sort(h.begin(), h.end(), triple_less);
                if (e == cudaSuccess) e = cudaMemcpy(out, h.data(), sizeof(ssj_triple) * n_copy, cudaMemcpyHostToDevice);
            }
        } else if (n_copy) {
            e = cudaMemcpy(out, d_out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && (gb->flags & SSJ_SORTED)) std::sort(out, out + n_copy, triple_less);
        }
        if (e != cudaSuccess) {
            release();
            return cuda_fail(ctx, e, "group join results");
        }
    }
    release();
    if (count > cap && !count_only)
        return fail(ctx, SSJ_ENOMEM, "%llu result pairs, room for %llu", (unsigned long long)count,
                    (unsigned long long)cap);
    return SSJ_OK;
}

// ===========================================================================
// Serving: continuous batching
// ===========================================================================

namespace {

uint64_t batch_device_bytes(uint32_t n_probes, uint64_t n_cands, bool count_only, bool dev_ptrs, int num_sms) {
    uint64_t b = 0;
    if (!dev_ptrs) {
        b += align256(4ull * std::max<uint32_t>(n_probes, 1));
        b += align256(8ull * (n_probes + 1));
        b += align256(4ull * std::max<uint64_t>(n_cands, 1));
    }
    b += 256;  // count
    b += align256(workspace_bytes(n_probes, n_cands, num_sms));
    if (!count_only) b += align256(sizeof(ssj_triple) * std::max<uint64_t>(n_cands, 1));
    return b;
}

// True if p lies in page-locked host memory (cudaMallocHost, cudaHostAlloc,
// cudaHostRegister), which the copy engines read directly.
bool is_pinned(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// memcpy of pageable input into pinned staging; a large copy is split over a
// few threads, since one core's copy rate is well below the host-to-device
// link's.
void staged_copy(void* dst, const void* src, size_t bytes) {
    constexpr size_t kPart = size_t(8) << 20;
    const size_t hw = std::max(2u, std::thread::hardware_concurrency());
    const size_t parts = std::min<size_t>(std::min<size_t>(bytes / kPart, 8), hw / 2);
    if (parts <= 1) {
        memcpy(dst, src, bytes);
        return;
    }
    const size_t step = ((bytes + parts - 1) / parts + 63) & ~size_t(63);
    std::vector<std::thread> th;
    for (size_t i = 1; i < parts; ++i) {
        const size_t b0 = std::min(bytes, i * step), b1 = std::min(bytes, b0 + step);
        if (b1 > b0)
            th.emplace_back([=] { memcpy(static_cast<char*>(dst) + b0, static_cast<const char*>(src) + b0, b1 - b0); });
    }
    memcpy(dst, src, std::min(bytes, step));
    for (auto& t : th) t.join();
}

void completion_loop(ssj_ctx* ctx, int slot) {
    cudaSetDevice(ctx->device);
    Slot& sl = ctx->slots[slot];
    for (;;) {
        Ticket* t = nullptr;
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            ctx->cv.wait(lk, [&] { return ctx->stopping || sl.pending != nullptr; });
            if (!sl.pending) return;  // stopping with nothing in flight
            t = sl.pending;
        }
        std::string err;
        NvtxScope nvtx_scope("ssj serving: wait for the batch's kernels, copy its results");
        cudaError_t e = cudaEventSynchronize(t->kernel_done);
        uint64_t count = 0;
        if (e == cudaSuccess) {
            count = *sl.h_count;
            if (*sl.h_err) {
                err = "device-side batch check failed";
                t->derr = *sl.h_err;
            }
        } else {
            err = std::string("batch failed: ") + cudaGetErrorString(e);
        }
        if (err.empty() && !(t->flags & SSJ_COUNT_ONLY)) {
            const uint64_t n_copy = std::min(count, t->out_cap);
            if (n_copy) {
                if (ensure_pinned(nullptr, &sl.h_out, &sl.h_out_cap, n_copy) != SSJ_OK) err = "pinned output";
                if (err.empty()) {
                    e = cudaMemcpyAsync(sl.h_out, t->d_out, sizeof(ssj_triple) * n_copy, cudaMemcpyDeviceToHost,
                                        sl.stream);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
                    if (e != cudaSuccess) err = std::string("result copy: ") + cudaGetErrorString(e);
                }
            }
        }
        if (t->d_mem) {
            cudaFreeAsync(t->d_mem, sl.stream);
            t->d_mem = nullptr;
        }
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            t->count = count;
            t->h_out = sl.h_out;
            t->error = err;
            t->state = err.empty() ? TicketState::kDone : TicketState::kFailed;
            ctx->used_bytes -= t->bytes;
            t->bytes = 0;
            sl.pending = nullptr;
        }
        ctx->cv.notify_all();
    }
}

}  // namespace

extern "C" ssj_status ssj_submit(ssj_ctx* ctx, const ssj_batch* batch, uint64_t* ticket) {
    NvtxScope nvtx_scope("ssj_submit");
    if (!ctx || !batch || !ticket) return fail(ctx, SSJ_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(ctx->mu);
    Collection *R, *S;
    ssj_status st = resolve(ctx, batch, &R, &S);
    if (st != SSJ_OK) return st;
    const bool dev = (batch->flags & SSJ_DEVICE_PTRS) != 0;
    const bool count_only = (batch->flags & SSJ_COUNT_ONLY) != 0;
    uint64_t n_cands = batch->n_cands;
    if (dev) {
        st = check_device_alignment(ctx, batch, nullptr, nullptr);
        if (st != SSJ_OK) return st;
    } else {
        lk.unlock();  // validation reads only the caller's arrays and immutable collection sizes
        st = validate_host_batch(ctx, batch, &n_cands);
        lk.lock();
        if (st != SSJ_OK) return st;
    }
    const uint64_t bytes = batch_device_bytes(batch->n_probes, n_cands, count_only, dev, ctx->num_sms);
    if (bytes > ctx->budget) return fail(ctx, SSJ_EINVAL, "batch needs %llu bytes, budget is %llu",
                                         (unsigned long long)bytes, (unsigned long long)ctx->budget);
    if (!ctx->pool_grown) {
        // reserve the budget in the pool once, so that later submissions never wait on the
        // driver for memory (the release threshold keeps it there)
        DeviceGuard g0(ctx->device);
        void* tmp = nullptr;
        cudaStream_t s0 = ctx->slots.empty() ? ctx->stream : ctx->slots[0].stream;
        if (cudaMallocFromPoolAsync(&tmp, ctx->budget, ctx->pool, s0) == cudaSuccess) {
            cudaFreeAsync(tmp, s0);
            cudaStreamSynchronize(s0);
        } else {
            cudaGetLastError();  // not reserved up front; allocations grow the pool as they come
        }
        ctx->pool_grown = true;
    }
    int slot = -1;
    for (size_t i = 0; i < ctx->slots.size(); ++i)
        if (!ctx->slots[i].busy) { slot = (int)i; break; }
    if (slot < 0 || ctx->used_bytes + bytes > ctx->budget) return SSJ_EAGAIN;
    // reserve the slot, the budget and the collections, then work without the lock
    Slot& sl = ctx->slots[slot];
    sl.busy = true;
    ctx->used_bytes += bytes;
    R->busy++;
    S->busy++;
    std::unique_ptr<Ticket> t(new Ticket());
    t->id = ctx->next_ticket++;
    VerifyArgs a = make_args(ctx, batch, *R, *S, n_cands);
    lk.unlock();

    auto unreserve = [&](ssj_status code) {
        std::unique_lock<std::mutex> l2(ctx->mu);
        sl.busy = false;
        ctx->used_bytes -= bytes;
        R->busy--;
        S->busy--;
        return code;
    };
    DeviceGuard g(ctx->device);
    cudaStream_t s = sl.stream;
    t->R = batch->R;
    t->S = batch->S;
    t->flags = batch->flags;
    t->stream = s;
    t->kernel_done = sl.ev;
    t->slot = slot;
    t->bytes = bytes;
    cudaError_t e = cudaMallocFromPoolAsync(&t->d_mem, bytes, ctx->pool, s);
    if (e != cudaSuccess) return unreserve(fail(ctx, SSJ_ENOMEM, "pool allocation: %s", cudaGetErrorString(e)));
    bool direct_copy = false;
    char* base = static_cast<char*>(t->d_mem);
    size_t off = 0;
    if (!dev) {
        // Inputs in pinned memory are copied straight from the caller's arrays,
        // and the call waits for those copies before it returns; pageable
        // inputs go through this slot's pinned staging.  Either way the caller
        // may reuse its arrays once ssj_submit returns.
        const uint64_t offs_n = batch->n_probes ? batch->n_probes + 1ull : 0;
        const bool pin_probe = batch->n_probes && is_pinned(batch->probe_ids);
        const bool pin_offs = offs_n && is_pinned(batch->cand_offsets);
        const bool pin_cand = n_cands && is_pinned(batch->cand_ids);
        direct_copy = pin_probe || pin_offs || pin_cand;
        if ((!pin_probe && (st = ensure_pinned(ctx, &sl.h_probe, &sl.h_probe_cap, std::max<uint64_t>(batch->n_probes, 1))) != SSJ_OK) ||
            (!pin_offs && (st = ensure_pinned(ctx, &sl.h_offs, &sl.h_offs_cap, batch->n_probes + 1ull)) != SSJ_OK) ||
            (!pin_cand && (st = ensure_pinned(ctx, &sl.h_cand, &sl.h_cand_cap, std::max<uint64_t>(n_cands, 1))) != SSJ_OK)) {
            cudaFreeAsync(t->d_mem, s);
            return unreserve(st);
        }
        const void* src_probe = batch->probe_ids;
        const void* src_offs = batch->cand_offsets;
        const void* src_cand = batch->cand_ids;
        if (batch->n_probes && !pin_probe) {
            staged_copy(sl.h_probe, batch->probe_ids, 4ull * batch->n_probes);
            src_probe = sl.h_probe;
        }
        if (offs_n && !pin_offs) {
            staged_copy(sl.h_offs, batch->cand_offsets, 8ull * offs_n);
            src_offs = sl.h_offs;
        }
        if (n_cands && !pin_cand) {
            staged_copy(sl.h_cand, batch->cand_ids, 4ull * n_cands);
            src_cand = sl.h_cand;
        }
        uint32_t* d_probe = reinterpret_cast<uint32_t*>(base + off); off += align256(4ull * std::max<uint32_t>(batch->n_probes, 1));
        uint64_t* d_offs = reinterpret_cast<uint64_t*>(base + off);  off += align256(8ull * (batch->n_probes + 1));
        uint32_t* d_cand = reinterpret_cast<uint32_t*>(base + off);  off += align256(4ull * std::max<uint64_t>(n_cands, 1));
        if (batch->n_probes) e = cudaMemcpyAsync(d_probe, src_probe, 4ull * batch->n_probes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && offs_n) e = cudaMemcpyAsync(d_offs, src_offs, 8ull * offs_n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && n_cands) e = cudaMemcpyAsync(d_cand, src_cand, 4ull * n_cands, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && direct_copy) e = cudaEventRecord(sl.copied, s);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);  // no copy may still read the caller's arrays
            cudaFreeAsync(t->d_mem, s);
            return unreserve(cuda_fail(ctx, e, "submit copy"));
        }
        a.single.probe_ids = d_probe;
        a.single.cand_offsets = d_offs;
        a.single.cand_ids = d_cand;
    } else {
        a.single.probe_ids = batch->probe_ids;
        a.single.cand_offsets = batch->cand_offsets;
        a.single.cand_ids = batch->cand_ids;
    }
    uint64_t* d_count = reinterpret_cast<uint64_t*>(base + off); off += 256;
    void* ws = base + off; off += align256(workspace_bytes(batch->n_probes, n_cands, ctx->num_sms));
    ssj_triple* d_out = count_only ? nullptr : reinterpret_cast<ssj_triple*>(base + off);
    a.single.out = d_out;
    a.single.cap = count_only ? 0 : n_cands;
    a.single.count = reinterpret_cast<unsigned long long*>(d_count);
    bind_workspace(a, ws, batch->n_probes, n_cands, ctx->num_sms);
    e = launch_verify(a, s, ctx->num_sms, ctx->block_threads, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_count, d_count, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_err, &a.ctr->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, s);
    // pinned inputs: wait for their copies unless the caller keeps them until the ticket is done
    if (e == cudaSuccess && direct_copy && !(batch->flags & SSJ_KEEP_INPUTS)) e = cudaEventSynchronize(sl.copied);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        cudaFreeAsync(t->d_mem, s);
        return unreserve(cuda_fail(ctx, e, "submit"));
    }
    t->d_out = d_out;
    t->out_cap = a.single.cap;
    lk.lock();
    Ticket* raw = t.get();
    ctx->tickets[raw->id] = std::move(t);
    sl.pending = raw;
    *ticket = raw->id;
    lk.unlock();
    ctx->cv.notify_all();
    return SSJ_OK;
}

extern "C" ssj_status ssj_poll(ssj_ctx* ctx, uint64_t ticket, int timeout_ms, int* done) {
    if (!ctx || !done) return SSJ_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, SSJ_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Ticket* t = it->second.get();
    auto ready = [&] { return t->state != TicketState::kRunning; };
    if (timeout_ms < 0) {
        ctx->cv.wait(lk, ready);
    } else if (timeout_ms > 0) {
        ctx->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    }
    *done = ready() ? 1 : 0;
    if (!*done) return SSJ_ETIMEDOUT;
    if (t->state == TicketState::kFailed)
        return t->derr ? device_check_status(ctx, t->derr) : fail(ctx, SSJ_EDEVICE, "%s", t->error.c_str());
    return SSJ_OK;
}

extern "C" ssj_status ssj_results(ssj_ctx* ctx, uint64_t ticket, ssj_triple* out, uint64_t cap, uint64_t* n_out) {
    NvtxScope nvtx_scope("ssj_results");
    if (!ctx || !n_out) return SSJ_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, SSJ_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Ticket* t = it->second.get();
    if (t->state == TicketState::kRunning) return SSJ_EAGAIN;
    *n_out = t->count;
    if (!out && t->state == TicketState::kDone) return SSJ_OK;
    ssj_status st = SSJ_OK;
    if (t->state == TicketState::kFailed) {
        st = t->derr ? device_check_status(ctx, t->derr) : fail(ctx, SSJ_EDEVICE, "%s", t->error.c_str());
    } else if (!(t->flags & SSJ_COUNT_ONLY)) {
        if (cap < t->count) return fail(ctx, SSJ_ENOMEM, "%llu result pairs, room for %llu",
                                        (unsigned long long)t->count, (unsigned long long)cap);
        if (t->count) memcpy(out, t->h_out, sizeof(ssj_triple) * t->count);
        if (t->flags & SSJ_SORTED) std::sort(out, out + t->count, triple_less);
    }
    ctx->slots[t->slot].busy = false;
    auto ir = ctx->colls.find(t->R);
    if (ir != ctx->colls.end() && ir->second.busy) ir->second.busy--;
    auto is = ctx->colls.find(t->S);
    if (is != ctx->colls.end() && is->second.busy) is->second.busy--;
    ctx->tickets.erase(it);
    return st;
}

extern "C" ssj_status ssj_profile_read(ssj_ctx* ctx, uint32_t* launches, double* plan_ms, double* verify_ms) {
    if (!ctx || !launches || !plan_ms || !verify_ms) return SSJ_EINVAL;
    *launches = 0;
    *plan_ms = 0;
    *verify_ms = 0;
    if (!ctx->profile) return fail(ctx, SSJ_EINVAL, "context was created without SSJ_CTX_PROFILE");
    DeviceGuard g(ctx->device);
    for (size_t i = 0; i < ctx->prof_used; ++i) {
        cudaEvent_t* ev = &ctx->prof_ev[3 * i];
        CUDA_TRY(ctx, cudaEventSynchronize(ev[2]));
        float a = 0, b = 0;
        CUDA_TRY(ctx, cudaEventElapsedTime(&a, ev[0], ev[1]));
        CUDA_TRY(ctx, cudaEventElapsedTime(&b, ev[1], ev[2]));
        *plan_ms += a;
        *verify_ms += b;
    }
    *launches = (uint32_t)ctx->prof_used;
    ctx->prof_used = 0;
    return SSJ_OK;
}

// ===========================================================================
// Helpers for the scratch-free entry point (noalloc.cu): they read the
// context and never allocate.
// ===========================================================================

namespace ssj {

ssj_status resolve_device_batch(ssj_ctx* ctx, const ssj_batch* batch, const void* out, const void* count,
                                VerifyArgs* a, int* device, int* num_sms, uint32_t* block_threads,
                                cudaStream_t* ctx_stream) {
    Collection *R, *S;
    ssj_status st = resolve(ctx, batch, &R, &S);
    if (st != SSJ_OK) return st;
    if (batch->n_probes && (!batch->probe_ids || !batch->cand_offsets))
        return fail(ctx, SSJ_EINVAL, "NULL batch arrays");
    if (batch->n_cands && !batch->cand_ids) return fail(ctx, SSJ_EINVAL, "NULL cand_ids");
    st = check_device_alignment(ctx, batch, out, count);
    if (st != SSJ_OK) return st;
    *a = make_args(ctx, batch, *R, *S, batch->n_cands);
    a->single.probe_ids = batch->probe_ids;
    a->single.cand_offsets = batch->cand_offsets;
    a->single.cand_ids = batch->cand_ids;
    *device = ctx->device;
    *num_sms = ctx->num_sms;
    *block_threads = ctx->block_threads;
    *ctx_stream = ctx->stream;
    return SSJ_OK;
}

ssj_status report(ssj_ctx* ctx, ssj_status st, const char* msg) { return fail(ctx, st, "%s", msg); }

void remember_counters(ssj_ctx* ctx, Counters* c) { ctx->last_ctr = c; }

}  // namespace ssj

// ===========================================================================
// Batched instances
// ===========================================================================

struct ssj_multi {
    VerifyArgs a;
    LaunchShape shape;
    uint32_t block_threads = 256;
    uint32_t index_words_fit = 0;  // probe bitmap words the instances' token values need (0: too many)
    bool force_index = false;      // an instance forces index items
    void* ws = nullptr;
    std::vector<ssj_coll> colls;  // collections marked busy
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" ssj_status ssj_multi_create(ssj_ctx* ctx, const ssj_batch* batches, uint32_t n_batches,
                                       ssj_triple* const* d_outs, const uint64_t* caps, uint64_t* d_counts,
                                       ssj_multi** out) {
    if (!ctx || !out || (n_batches && (!batches || !d_outs || !caps || !d_counts)))
        return fail(ctx, SSJ_EINVAL, "NULL argument");
    std::vector<Instance> table(n_batches);
    LaunchShape sh;
    sh.n_inst = n_batches;
    sh.n_tiles = 0;
    sh.total_probes = 0;
    sh.total_cands = 0;
    std::unique_ptr<ssj_multi> m(new ssj_multi());
    uint64_t vocab = 1;
    const Collection* pinned = nullptr;  // the first pinned collection: its L2 window
    for (uint32_t i = 0; i < n_batches; ++i) {
        const ssj_batch* b = &batches[i];
        Collection *R, *S;
        ssj_status st = resolve(ctx, b, &R, &S);
        if (st != SSJ_OK) return st;
        if (b->n_probes && (!b->probe_ids || !b->cand_offsets)) return fail(ctx, SSJ_EINVAL, "batch %u: NULL arrays", i);
        if (b->n_cands && !b->cand_ids) return fail(ctx, SSJ_EINVAL, "batch %u: NULL cand_ids", i);
        if (caps[i] && !d_outs[i] && !(b->flags & SSJ_COUNT_ONLY)) return fail(ctx, SSJ_EINVAL, "batch %u: NULL output", i);
        st = check_device_alignment(ctx, b, d_outs[i], d_counts + i);
        if (st != SSJ_OK) return st;
        Instance I = make_instance(b, *R, *S, b->n_cands);
        I.probe_ids = b->probe_ids;
        I.cand_offsets = b->cand_offsets;
        I.cand_ids = b->cand_ids;
        I.out = d_outs[i];
        I.cap = (b->flags & SSJ_COUNT_ONLY) ? 0 : caps[i];
        I.count = reinterpret_cast<unsigned long long*>(d_counts + i);
        I.tile_base = sh.n_tiles;
        const uint64_t tiles = ((uint64_t)b->n_probes + 31) / 32;
        if ((uint64_t)sh.n_tiles + tiles > 0x7FFFFFFull) return fail(ctx, SSJ_EINVAL, "too many probes in one launch");
        sh.n_tiles += (uint32_t)tiles;
        sh.total_probes += b->n_probes;
        sh.total_cands += b->n_cands;
        if (sh.total_cands >= kMaxCands) return fail(ctx, SSJ_EINVAL, "2^40 or more candidates in one launch");
        table[i] = I;
        m->colls.push_back(b->R);
        m->colls.push_back(b->S);
        vocab = std::max(vocab, vocab_bound(*R, *S));
        m->force_index = m->force_index || (b->flags & SSJ_FORCE_INDEX) != 0;
        if (!pinned) pinned = R->l2_window ? R : (S->l2_window ? S : nullptr);
    }
    DeviceGuard g(ctx->device);
    const size_t bytes = workspace_bytes(sh, ctx->num_sms);
    cudaError_t e = cudaMalloc(&m->ws, bytes);
    if (e != cudaSuccess) return fail(ctx, SSJ_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    memset(&m->a, 0, sizeof(m->a));
    apply_policy(ctx, m->a, vocab, m->force_index);
    if (pinned) set_l2_window(m->a, *pinned);
    m->index_words_fit = index_words_for(vocab);
    m->block_threads = ctx->block_threads;
    bind_workspace(m->a, m->ws, sh, ctx->num_sms);
    m->a.table = m->a.table_out;
    m->shape = sh;
    if (n_batches) {
        e = cudaMemcpy(m->a.table_out, table.data(), sizeof(Instance) * n_batches, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(m->ws);
            return cuda_fail(ctx, e, "instance table upload");
        }
    }
    e = prepare_verify(ctx->block_threads, m->a.index_words);
    if (e != cudaSuccess) {
        cudaFree(m->ws);
        return cuda_fail(ctx, e, "prepare_verify");
    }
    {
        std::unique_lock<std::mutex> lk(ctx->mu);
        for (ssj_coll c : m->colls) ctx->colls[c].busy++;
    }
    *out = m.release();
    return SSJ_OK;
}

extern "C" ssj_status ssj_multi_launch(ssj_ctx* ctx, ssj_multi* m, void* stream) {
    NvtxScope nvtx_scope("ssj_multi_launch");
    if (!ctx || !m) return SSJ_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->last_ctr = m->a.ctr;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    cudaError_t e = launch_verify(m->a, s, ctx->num_sms, m->block_threads, profile_events(ctx));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch_verify");
    return SSJ_OK;
}

extern "C" ssj_status ssj_multi_graph_launch(ssj_ctx* ctx, ssj_multi* m, void* stream) {
    if (!ctx || !m) return SSJ_EINVAL;
    DeviceGuard g(ctx->device);
    if (!m->exec) {
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
        CUDA_TRY(ctx, cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_verify(m->a, m->capture_stream, ctx->num_sms, m->block_threads, nullptr);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(m->capture_stream, &graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "capture launch_verify");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
        m->graph = graph;
        CUDA_TRY(ctx, cudaGraphInstantiate(&m->exec, m->graph, 0));
    }
    ctx->last_ctr = m->a.ctr;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    CUDA_TRY(ctx, cudaGraphLaunch(m->exec, s));
    return SSJ_OK;
}

extern "C" void ssj_multi_destroy(ssj_ctx* ctx, ssj_multi* m) {
    if (!m) return;
    if (ctx) {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        std::unique_lock<std::mutex> lk(ctx->mu);
        for (ssj_coll c : m->colls) {
            auto it = ctx->colls.find(c);
            if (it != ctx->colls.end() && it->second.busy) it->second.busy--;
        }
        if (ctx->last_ctr == m->a.ctr) ctx->last_ctr = nullptr;
    }
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->graph) cudaGraphDestroy(m->graph);
    if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
    cudaFree(m->ws);
    delete m;
}

// ===========================================================================
// Autotuning of a batched launch
// ===========================================================================

namespace {

// Median device time (ms) of reps launches of m with the given granularity,
// after one untimed launch; negative on a CUDA error (*err receives it).
float time_setting(ssj_ctx* ctx, const ssj_multi* m, uint32_t tmax, uint32_t lmax, uint32_t wmax, uint32_t bt,
                   uint32_t dml, uint32_t imin, uint32_t reps, cudaStream_t s, cudaEvent_t* ev, cudaError_t* err) {
    VerifyArgs a = m->a;
    a.thread_max_key = tmax;
    a.lane_max_key = lmax;
    a.warp_max_key = wmax;
    a.drain_min_live = dml;
    a.index_min_cands = imin;
    a.index_words = (imin || m->force_index) ? m->index_words_fit : 0u;
    cudaError_t e = prepare_verify(bt, a.index_words);
    if (e == cudaSuccess) e = launch_verify(a, s, ctx->num_sms, bt, nullptr);
    std::vector<float> ms;
    for (uint32_t i = 0; e == cudaSuccess && i < reps; ++i) {
        e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess) e = launch_verify(a, s, ctx->num_sms, bt, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float t = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        ms.push_back(t);
    }
    if (e != cudaSuccess) {
        *err = e;
        return -1.0f;
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

}  // namespace

extern "C" ssj_status ssj_multi_autotune(ssj_ctx* ctx, ssj_multi* m, void* stream, uint32_t reps,
                                         ssj_tune_result* out) {
    NvtxScope nvtx_scope("ssj_multi_autotune");
    if (!ctx || !m || !out) return fail(ctx, SSJ_EINVAL, "NULL argument");
    reps = std::max<uint32_t>(reps, 3);
    DeviceGuard g(ctx->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    CUDA_TRY(ctx, cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(ctx, SSJ_EDEVICE, "cudaEventCreate");
    }
    // Candidate values per coordinate: the thread bin's upper key, the lane
    // bin's upper key (1: no lane bin), the warp bin's upper key (the largest
    // value sends no probe to the block bin) and the block size, which also
    // sets the block path's window (8 merge steps per thread).
    static const uint32_t kThread[] = {32, 64, 128, 256, 512, 1024, 2048, 4096};
    static const uint32_t kLane[] = {1, 256, 512, 1024, 2048};
    static const uint32_t kWarp[] = {256, 512, 1024, 2048, 4096, 0xFFFFFFFFu};
    static const uint32_t kBlock[] = {128, 256, 512, 128 | SSJ_WIDE_REGISTERS, 256 | SSJ_WIDE_REGISTERS,
                                      512 | SSJ_WIDE_REGISTERS, 256 | SSJ_BULK_STAGING, 512 | SSJ_BULK_STAGING,
                                      256 | SSJ_WIDE_REGISTERS | SSJ_BULK_STAGING,
                                      512 | SSJ_WIDE_REGISTERS | SSJ_BULK_STAGING};
    static const uint32_t kMinLive[] = {8, 12, 16, 20, 24};
    // index-item threshold: 0 sends no probe to index items
    static const uint32_t kIndexMin[] = {0, 32, 64, 128, 256, 512, 1024, 4096};
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>, float> seen;
    cudaError_t err = cudaSuccess;
    uint32_t bd = m->a.drain_min_live ? m->a.drain_min_live : 16;
    uint32_t bi = m->index_words_fit ? m->a.index_min_cands : 0u;
    auto cost = [&](uint32_t t, uint32_t l, uint32_t w, uint32_t b) -> float {
        auto key = std::make_tuple(t, l, w, b, bd, bi);
        auto it = seen.find(key);
        if (it != seen.end()) return it->second;
        const float v = time_setting(ctx, m, t, l, w, b, bd, bi, reps, s, ev, &err);
        seen[key] = v;
        return v;
    };
    uint32_t bt = m->a.thread_max_key, bl = m->a.lane_max_key, bw = m->a.warp_max_key, bb = m->block_threads;
    const float first = cost(bt, bl, bw, bb);
    float best = first;
    // coordinate descent: thread bin, lane bin, warp bin, block size; repeated while it improves
    for (int sweep = 0; sweep < 3 && err == cudaSuccess; ++sweep) {
        const float before = best;
        for (uint32_t t : kThread) {
            if (err != cudaSuccess) break;
            const uint32_t w = std::max(bw, t);  // a thread bin above the warp bin empties the latter
            const float v = cost(t, bl, w, bb);
            if (v < best) best = v, bt = t, bw = w;
        }
        for (uint32_t l : kLane) {
            if (err != cudaSuccess) break;
            if (l != 1 && l <= bt) continue;  // empty lane bin, same as 1
            const float v = cost(bt, l, bw, bb);
            if (v < best) best = v, bl = l;
        }
        for (uint32_t w : kWarp) {
            if (w < bt || err != cudaSuccess) continue;
            const float v = cost(bt, bl, w, bb);
            if (v < best) best = v, bw = w;
        }
        for (uint32_t b : kBlock) {
            if (err != cudaSuccess) break;
            const float v = cost(bt, bl, bw, b);
            if (v < best) best = v, bb = b;
        }
        for (uint32_t d : kMinLive) {
            if (err != cudaSuccess) break;
            const uint32_t keep = bd;
            bd = d;
            const float v = cost(bt, bl, bw, bb);
            if (v < best) best = v; else bd = keep;
        }
        for (uint32_t x : kIndexMin) {
            if (err != cudaSuccess || (x && !m->index_words_fit)) break;
            const uint32_t keep = bi;
            bi = x;
            const float v = cost(bt, bl, bw, bb);
            if (v < best) best = v; else bi = keep;
        }
        if (!(best < 0.98f * before)) break;  // no gain worth another sweep
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "autotune launch");
    uint32_t derr = 0;
    CUDA_TRY(ctx, cudaMemcpy(&derr, &m->a.ctr->err, sizeof(derr), cudaMemcpyDeviceToHost));
    if (derr) return fail(ctx, SSJ_EDEVICE, "device checks fired during tuning (code %u)", derr);
    // The multi keeps the best setting; a captured graph holds the old one.
    m->a.thread_max_key = bt;
    m->a.lane_max_key = bl;
    m->a.warp_max_key = bw;
    m->a.drain_min_live = bd;
    m->a.index_min_cands = bi;
    m->a.index_words = (bi || m->force_index) ? m->index_words_fit : 0u;
    m->block_threads = bb;
    CUDA_TRY(ctx, prepare_verify(bb, m->a.index_words));
    if (m->exec) {
        cudaGraphExecDestroy(m->exec);
        m->exec = nullptr;
    }
    if (m->graph) {
        cudaGraphDestroy(m->graph);
        m->graph = nullptr;
    }
    out->thread_max_key = bt;
    out->lane_max_key = bl;
    out->warp_max_key = bw;
    out->block_threads = bb;
    out->drain_min_live = bd;
    out->index_min_cands = bi;
    out->best_ms = best;
    out->initial_ms = first;
    out->settings_tried = (uint32_t)seen.size();
    return SSJ_OK;
}

// ===========================================================================
// Read-bandwidth probe
// ===========================================================================

extern "C" ssj_status ssj_read_bandwidth(ssj_ctx* ctx, uint64_t bytes, uint32_t passes, double* gbs) {
    if (!ctx || !gbs) return fail(ctx, SSJ_EINVAL, "NULL argument");
    bytes &= ~uint64_t(15);
    if (bytes == 0 || passes == 0) return fail(ctx, SSJ_EINVAL, "bytes must be >= 16 and passes > 0");
    DeviceGuard g(ctx->device);
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes + 256);
    if (e != cudaSuccess) return fail(ctx, SSJ_ENOMEM, "cudaMalloc(%llu): %s", (unsigned long long)bytes,
                                      cudaGetErrorString(e));
    uint32_t* sink = reinterpret_cast<uint32_t*>(static_cast<char*>(buf) + bytes);
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMemsetAsync(buf, 0, bytes + 256, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = read_probe(buf, bytes, 1, sink, ctx->num_sms, s);  // warm-up pass
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = read_probe(buf, bytes, passes, sink, ctx->num_sms, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read probe");
    *gbs = ms > 0 ? (double)bytes * passes / (ms * 1e-3) / 1e9 : 0.0;
    return SSJ_OK;
}
