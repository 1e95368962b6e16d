// Context, error reporting, the device memory pool and descriptors.
#include "common.cuh"

#include <stdarg.h>
#include <string.h>

namespace gbx {

static thread_local char g_last_error[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

gb_info fail(gb_info code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

gb_info cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "CUDA error %d (%s) in %s at %s:%d", (int)e,
             cudaGetErrorString(e), what, file, line);
    if (e == cudaErrorMemoryAllocation) return GB_OUT_OF_MEMORY;
    return GB_PANIC;
}

size_t type_size(gb_type t) {
    switch (t) {
    case GB_BOOL: return 1;
    case GB_INT32: return 4;
    case GB_UINT32: return 4;
    case GB_UINT64: return 8;
    case GB_FP32: return 4;
    case GB_FP64: return 8;
    }
    return 0;
}

bool valid_type(int t) { return t >= GB_BOOL && t <= GB_FP64; }

int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x > (1ull << b))) ++b;
    return b;
}

gb_info dalloc(gb_context *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->inject_failures > 0) {
            ctx->inject_failures--;
            return fail(GB_OUT_OF_MEMORY, "injected allocation failure (%zu bytes)", bytes);
        }
    }
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(GB_OUT_OF_MEMORY, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->live[*p] = bytes;
    ctx->held += bytes;
    if (ctx->held > ctx->peak) ctx->peak = ctx->held;
    return GB_SUCCESS;
}

void dfree(gb_context *ctx, void *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->live.find(p);
        if (it != ctx->live.end()) {
            ctx->held -= it->second;
            ctx->live.erase(it);
        }
    }
    cudaFreeAsync(p, ctx->stream);
}

gb_info memset_async(gb_context *ctx, void *p, int v, size_t bytes) {
    if (bytes) GB_CUDA(cudaMemsetAsync(p, v, bytes, ctx->stream));
    return GB_SUCCESS;
}

gb_info copy_in(gb_context *ctx, void *dst_dev, const void *src, size_t bytes, gb_mem mem) {
    if (!bytes) return GB_SUCCESS;
    GB_CUDA(cudaMemcpyAsync(dst_dev, src, bytes, mem == GB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            ctx->stream));
    return GB_SUCCESS;
}

gb_info copy_out(gb_context *ctx, void *dst, const void *src_dev, size_t bytes, gb_mem mem) {
    if (!bytes) return GB_SUCCESS;
    GB_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, mem == GB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            ctx->stream));
    if (mem == GB_HOST) GB_CUDA(cudaStreamSynchronize(ctx->stream));
    return GB_SUCCESS;
}

gb_info sync(gb_context *ctx) {
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    return GB_SUCCESS;
}

static bool pool_event(gb_context *ctx, cudaEvent_t *e) {
    if (!ctx->event_pool.empty()) {
        *e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return true;
    }
    if (cudaEventCreate(e) != cudaSuccess) { cudaGetLastError(); return false; }
    return true;
}

int prof_begin(gb_context *ctx, const char *name) {
    if (!ctx->profiling) return -1;
    gb_context::Span sp;
    sp.name = name;
    if (!pool_event(ctx, &sp.a)) return -1;
    if (!pool_event(ctx, &sp.b)) { ctx->event_pool.push_back(sp.a); return -1; }
    cudaEventRecord(sp.a, ctx->stream);
    ctx->spans.push_back(sp);
    return (int)ctx->spans.size() - 1;
}

void prof_end(gb_context *ctx, int slot) {
    if (slot < 0 || slot >= (int)ctx->spans.size()) return;
    cudaEventRecord(ctx->spans[slot].b, ctx->stream);
}

static void prof_clear(gb_context *ctx) {
    for (auto &sp : ctx->spans) { ctx->event_pool.push_back(sp.a); ctx->event_pool.push_back(sp.b); }
    ctx->spans.clear();
}

static void prof_destroy(gb_context *ctx) {
    prof_clear(ctx);
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    ctx->event_pool.clear();
}

}  // namespace gbx

using namespace gbx;

extern "C" {

const char *gb_version(void) { return "gbx 0.1 sm_103a"; }

gb_info gb_last_error(char *buf, size_t len) {
    if (!buf) return GB_NULL_POINTER;
    if (len == 0) return GB_INVALID_VALUE;
    strncpy(buf, g_last_error, len - 1);
    buf[len - 1] = 0;
    return GB_SUCCESS;
}

gb_info gb_init(int device, gb_context **ctx) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_init: ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    GB_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(GB_INVALID_VALUE, "gb_init: no CUDA device %d", device);
    GB_CUDA(cudaSetDevice(device));
    gb_context *c = new gb_context();
    c->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__); }
    c->own_stream = true;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, device);
    // keep freed pool memory cached instead of returning it to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *ctx = c;
    return GB_SUCCESS;
}

gb_info gb_context_set_stream(gb_context *ctx, void *stream) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_context_set_stream: ctx is NULL");
    GB_CUDA(cudaSetDevice(ctx->device));
    if (ctx->own_stream) {
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        cudaStreamDestroy(ctx->stream);
        ctx->own_stream = false;
    }
    ctx->stream = (cudaStream_t)stream;
    return GB_SUCCESS;
}

gb_info gb_context_synchronize(gb_context *ctx) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_context_synchronize: ctx is NULL");
    GB_CUDA(cudaSetDevice(ctx->device));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    // a timeout of a BFS that was launched without waiting for it
    return bfs_collect_status(ctx);
}

gb_info gb_context_pool_stats(gb_context *ctx, uint64_t *held, uint64_t *peak) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_context_pool_stats: ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->mu);
    if (held) *held = ctx->held;
    if (peak) *peak = ctx->peak;
    return GB_SUCCESS;
}

gb_info gb_context_inject_alloc_failures(gb_context *ctx, uint32_t count) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_context_inject_alloc_failures: ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->inject_failures = count;
    return GB_SUCCESS;
}

namespace {
struct WaitProbe {
    gbx::dev::GridBarrier bar;
    int err;
};
// One block waiting at a barrier of two: the bounded wait must run out.
__global__ void k_selftest_wait(WaitProbe *p, uint64_t limit_ns) {
    gbx::dev::grid_sync(&p->bar, 2u, &p->err, limit_ns);
}
}  // namespace

gb_info gb_context_selftest_wait(gb_context *ctx, uint32_t limit_us, int32_t *status) {
    if (!ctx || !status) return fail(GB_NULL_POINTER, "gb_context_selftest_wait: NULL argument");
    if (limit_us < 1) limit_us = 1;
    if (limit_us > 1000000u) limit_us = 1000000u;
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch probe(ctx);
    GB_CHECK(probe.alloc(sizeof(WaitProbe)));
    GB_CHECK(memset_async(ctx, probe.p, 0, sizeof(WaitProbe)));
    k_selftest_wait<<<1, 32, 0, ctx->stream>>>(probe.as<WaitProbe>(), (uint64_t)limit_us * 1000ull);
    GB_LAUNCH_CHECK();
    int32_t err = 0;
    GB_CUDA(cudaMemcpyAsync(&err, &probe.as<WaitProbe>()->err, sizeof(err), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    *status = err;
    return GB_SUCCESS;
}

gb_info gb_context_profile(gb_context *ctx, int enable) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_context_profile: ctx is NULL");
    GB_CUDA(cudaSetDevice(ctx->device));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    prof_clear(ctx);
    ctx->profiling = enable != 0;
    return GB_SUCCESS;
}

gb_info gb_context_profile_get(gb_context *ctx, const char *kernel, double *total_ms, uint64_t *launches) {
    if (!ctx || !kernel || !total_ms || !launches) return fail(GB_NULL_POINTER, "gb_context_profile_get: NULL");
    GB_CUDA(cudaSetDevice(ctx->device));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    double tot = 0;
    uint64_t k = 0;
    for (auto &sp : ctx->spans) {
        if (sp.name != kernel) continue;
        float ms = 0;
        GB_CUDA(cudaEventElapsedTime(&ms, sp.a, sp.b));
        tot += ms;
        ++k;
    }
    *total_ms = tot;
    *launches = k;
    return GB_SUCCESS;
}

gb_info gb_finalize(gb_context *ctx) {
    if (!ctx) return fail(GB_NULL_POINTER, "gb_finalize: ctx is NULL");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    prof_destroy(ctx);
    bfs_workspace_release(ctx);
    ms_workspace_release(ctx);
    for (auto &kv : ctx->live) cudaFreeAsync(kv.first, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return GB_SUCCESS;
}

// ------------------------------------------------------------ descriptor
gb_info gb_desc_new(gb_desc **d) {
    if (!d) return fail(GB_NULL_POINTER, "gb_desc_new: NULL");
    *d = new gb_desc();
    return GB_SUCCESS;
}

gb_info gb_desc_set(gb_desc *d, gb_field field, int value) {
    if (!d) return fail(GB_NULL_POINTER, "gb_desc_set: NULL");
    switch (field) {
    case GB_MASK:
        if (value < 0 || value > (GB_SCMP | GB_STRUCTURE)) return fail(GB_INVALID_VALUE, "bad GB_MASK value %d", value);
        d->mask = value; break;
    case GB_OUTP:
        if (value != GB_DEFAULT && value != GB_REPLACE) return fail(GB_INVALID_VALUE, "bad GB_OUTP value %d", value);
        d->outp = value; break;
    case GB_INP0:
    case GB_INP1:
        if (value != GB_DEFAULT && value != GB_TRAN) return fail(GB_INVALID_VALUE, "bad GB_INP value %d", value);
        (field == GB_INP0 ? d->inp0 : d->inp1) = value; break;
    case GB_DIRECTION:
        if (value < GB_AUTO || value > GB_PULL) return fail(GB_INVALID_VALUE, "bad GB_DIRECTION value %d", value);
        d->direction = value; break;
    case GB_SWITCH_BETA:
        if (value < 0) return fail(GB_INVALID_VALUE, "bad GB_SWITCH_BETA value %d", value);
        d->beta = value; break;
    case GB_SCHEDULE:
        if (value < GB_SCHED_AUTO || value > GB_SCHED_ASYNC)
            return fail(GB_INVALID_VALUE, "bad GB_SCHEDULE value %d", value);
        d->schedule = value; break;
    case GB_SSSP_DELTA:
        if (value < 0) return fail(GB_INVALID_VALUE, "bad GB_SSSP_DELTA value %d", value);
        d->sssp_delta = value; break;
    default:
        return fail(GB_INVALID_VALUE, "unknown descriptor field %d", (int)field);
    }
    return GB_SUCCESS;
}

gb_info gb_desc_get(const gb_desc *d, gb_field field, int *value) {
    if (!d || !value) return fail(GB_NULL_POINTER, "gb_desc_get: NULL");
    switch (field) {
    case GB_MASK: *value = d->mask; break;
    case GB_OUTP: *value = d->outp; break;
    case GB_INP0: *value = d->inp0; break;
    case GB_INP1: *value = d->inp1; break;
    case GB_DIRECTION: *value = d->direction; break;
    case GB_SCHEDULE: *value = d->schedule; break;
    case GB_SWITCH_BETA: *value = d->beta; break;
    case GB_SSSP_DELTA: *value = d->sssp_delta; break;
    default: return fail(GB_INVALID_VALUE, "unknown descriptor field %d", (int)field);
    }
    return GB_SUCCESS;
}

gb_info gb_desc_toggle(gb_desc *d, gb_field field) {
    if (!d) return fail(GB_NULL_POINTER, "gb_desc_toggle: NULL");
    switch (field) {
    case GB_MASK: d->mask ^= GB_SCMP; break;
    case GB_OUTP: d->outp ^= GB_REPLACE; break;
    case GB_INP0: d->inp0 ^= GB_TRAN; break;
    case GB_INP1: d->inp1 ^= GB_TRAN; break;
    default: return fail(GB_INVALID_VALUE, "field %d cannot be toggled", (int)field);
    }
    return GB_SUCCESS;
}

gb_info gb_desc_free(gb_desc **d) {
    if (!d) return fail(GB_NULL_POINTER, "gb_desc_free: NULL");
    delete *d;
    *d = nullptr;
    return GB_SUCCESS;
}

}  // extern "C"
