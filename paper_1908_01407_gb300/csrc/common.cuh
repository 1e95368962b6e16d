// Internal definitions shared by the library's translation units: object
// layouts, error plumbing, the device memory pool, and small device helpers
// (warp/block primitives, a bounded grid barrier).
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/gbx.h"

#define GBX_MAX_LEVEL_LOG 64

// ------------------------------------------------------------------ errors
namespace gbx {

void set_error(const char *fmt, ...);
gb_info fail(gb_info code, const char *fmt, ...);
gb_info cuda_fail(cudaError_t e, const char *what, const char *file, int line);

}  // namespace gbx

#define GB_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) return gbx::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define GB_CHECK(call)                           \
    do {                                         \
        gb_info _r = (call);                     \
        if (_r != GB_SUCCESS) return _r;         \
    } while (0)

#define GB_LAUNCH_CHECK() GB_CUDA(cudaGetLastError())

// ------------------------------------------------------------------ objects
struct gb_context_t {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int l2_bytes = 0;
    std::mutex mu;
    uint64_t held = 0, peak = 0;
    uint32_t inject_failures = 0;
    std::unordered_map<void *, size_t> live;
    // kernel timing (gb_context_profile): event pairs recorded around the
    // main kernel launch of each operation, on the context stream
    bool profiling = false;
    struct Span { std::string name; cudaEvent_t a, b; };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> event_pool;   // reused across enable/disable cycles
    // upper bound on the blocks of a persistent (cooperative) launch, counted
    // in blocks of 256 threads (a kernel with larger blocks launches
    // proportionally fewer); 0 = the whole GPU. Contexts that share a GPU
    // concurrently split it this way.
    int grid_limit = 0;
};

// One pull candidate (a vertex with an in-edge), as a BFS pull reads it:
// one 32-byte sector holding everything the pull needs before the row
// itself. head = its four in-neighbours of largest out-degree
// (0xffffffff = none), b and len = its CSC row, deg = its out-degree.
struct PullRec {
    uint32_t v, len, b, deg;
    uint4 head;
};
static_assert(sizeof(PullRec) == 32, "a pull record is one 32-byte sector");

// In-rows longer than this are "hubs": the pull kernels (SSSP/CC relaxation,
// multi-source BFS) split their edges over the whole grid instead of giving
// each one to a single warp. The matrix caches the hub list for this length.
constexpr uint32_t GBX_HUB_MIN_LEN = 2048;

struct gb_matrix_t {
    gb_context *ctx = nullptr;
    gb_type type = GB_UINT32;
    uint32_t nrows = 0, ncols = 0;
    uint64_t nvals = 0;
    bool built = false;
    bool has_vals = false;        // false: structural (every stored value is 1)
    bool has_csc = false;
    bool csc_alias = false;       // CSC arrays are the CSR arrays (symmetric)
    uint32_t *rowptr = nullptr;   // [nrows + 1]
    uint32_t *colidx = nullptr;   // [nvals]
    void *vals = nullptr;         // [nvals] of type (nullptr if structural)
    uint32_t *colptr = nullptr;   // [ncols + 1]
    uint32_t *rowidx = nullptr;   // [nvals]
    void *cvals = nullptr;        // [nvals]
    // columns (CSC rows) longer than a threshold and their length prefixes,
    // built on first use by the pull kernels (cached; freed with the matrix)
    uint32_t *hub_list = nullptr, *hub_pre = nullptr;
    uint32_t nhub = 0;
    uint64_t hub_edges = 0;
    bool hub_ready = false;
    // push/pull switch threshold chosen by gb_bfs_autotune (0 = not tuned)
    uint32_t tuned_beta = 0;
    // BFS schedule chosen by gb_bfs_autotune (GB_SCHED_AUTO = not tuned)
    int tuned_schedule = GB_SCHED_AUTO;
    // BFS tile shape (gb_bfs_autotune or gb_bfs_set_shape; 0 = the default):
    // pull candidates per lane in flight (1, 2, 4) and blocks per SM (1..4)
    uint32_t bfs_pull_width = 0;
    uint32_t bfs_blocks_per_sm = 0;
    // PageRank SpMV tile (128-nonzero sub-tiles per warp tile) chosen by
    // gb_pagerank_autotune (0 = not tuned)
    uint32_t tuned_pr_nsub = 0;
    // PageRank vertex order: 1 = run on a copy renamed by decreasing
    // out-degree (pr_view, with pr_new_id[v] the new name of v), whose
    // most-referenced ranks fit in shared memory; 0 = as stored. Chosen by
    // gb_pagerank_autotune or set by hand; the copy is built on first use.
    int pr_order = 0;
    uint32_t pr_staged = 0;           // ranks staged in shared memory (0 = the default)
    gb_matrix_t *pr_view = nullptr;
    uint32_t *pr_new_id = nullptr;
    // vertices with at least one in-edge (nonempty CSC row), ascending,
    // built with the CSC; live_count is a device scalar (live_list[nrows])
    uint32_t *live_list = nullptr;
    uint32_t *live_count = nullptr;
    // per live vertex, in live-list order, its pull record (vertex, CSC row,
    // out-degree and the four in-neighbours of largest out-degree)
    PullRec *live_rec = nullptr;
    // per vertex, the size of its weakly connected component (built by
    // gb_matrix_build for a square matrix with a CSC): a traversal that has
    // reached that many vertices can stop without expanding its last frontier
    uint32_t *comp_size = nullptr;
    // mean stored value (uint32 weights), computed on first use by SSSP; 0 = not yet
    double mean_weight = 0;
    // guards the caches built on first use (hub list, mean weight)
    std::mutex cache_mu;
};

struct gb_vector_t {
    gb_context *ctx = nullptr;
    gb_type type = GB_FP32;
    uint32_t n = 0;
    uint32_t nwords = 0;
    void *vals = nullptr;          // [n] dense value array
    uint32_t *bitmap = nullptr;    // [nwords] presence
    // sparse index list, valid when list_valid (ascending order)
    uint32_t *list = nullptr;      // [n]
    bool list_valid = false;
    uint64_t list_len = 0;
};

struct gb_desc_t {
    int mask = GB_DEFAULT;
    int outp = GB_DEFAULT;
    int inp0 = GB_DEFAULT;
    int inp1 = GB_DEFAULT;
    int direction = GB_AUTO;
    int beta = 0;
    int schedule = GB_SCHED_AUTO;
    int sssp_delta = 0;
};

// ------------------------------------------------------------------ memory
namespace gbx {

size_t type_size(gb_type t);
bool valid_type(int t);

// Stream-ordered pool allocations on the context stream (Section 6.1 keeps
// a pool of device memory; here the CUDA stream-ordered pool backs it).
gb_info dalloc(gb_context *ctx, void **p, size_t bytes);
void dfree(gb_context *ctx, void *p);

template <typename T>
gb_info dalloc_t(gb_context *ctx, T **p, size_t count) {
    return dalloc(ctx, (void **)p, count * sizeof(T) + 16);
}

// RAII scratch buffer freed on scope exit (stream-ordered).
struct Scratch {
    gb_context *ctx;
    void *p = nullptr;
    explicit Scratch(gb_context *c) : ctx(c) {}
    ~Scratch() { if (p) dfree(ctx, p); }
    gb_info alloc(size_t bytes) { return dalloc(ctx, &p, bytes); }
    template <typename T> T *as() const { return (T *)p; }
};

// Device-side helpers implemented in primitives.cu.
gb_info memset_async(gb_context *ctx, void *p, int v, size_t bytes);
gb_info copy_in(gb_context *ctx, void *dst_dev, const void *src, size_t bytes, gb_mem mem);
gb_info copy_out(gb_context *ctx, void *dst, const void *src_dev, size_t bytes, gb_mem mem);
gb_info sync(gb_context *ctx);

// Exclusive prefix sum of n uint32 values (in may equal out); if total is
// non-null the device total is written there (a device pointer).
gb_info scan_exclusive_u32(gb_context *ctx, const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *total);
// Columns of A with more than min_len entries and their length prefix,
// computed on first use and cached on the matrix (matrix.cu).
gb_info matrix_hubs(const gb_matrix *A, uint32_t min_len);
// Per-vertex component sizes (weak components, by FastSV), cached on the
// matrix (fastsv.cu).
gb_info matrix_components(gb_context *ctx, gb_matrix *A);
// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits.
// Results end in keys/vals (the buffers are ping-ponged with the scratch).
gb_info radix_sort_pairs(gb_context *ctx, uint64_t *keys, uint32_t *vals, uint64_t n, int key_bits);

// Builds CSR arrays from tuples already on the device.
gb_info build_csr_from_device_tuples(gb_context *ctx, uint32_t nrows, uint32_t ncols, uint64_t ntup,
                                     const uint32_t *rows, const uint32_t *cols, const void *vals,
                                     gb_type vtype, gb_binop dup, uint32_t **rowptr, uint32_t **colidx,
                                     void **ovals, uint64_t *nnz);

int bits_for(uint64_t x);  // number of bits needed to represent values < x

// Profiling spans: prof_begin records a start event when profiling is on
// and returns its slot (or -1); prof_end records the matching end event.
int prof_begin(gb_context *ctx, const char *name);
void bfs_workspace_release(gb_context *ctx);
gb_info bfs_collect_status(gb_context *ctx);
void ms_workspace_release(gb_context *ctx);
void prof_end(gb_context *ctx, int slot);

}  // namespace gbx

// ------------------------------------------------------------------ device helpers
namespace gbx {
namespace dev {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- TMA bulk copies into shared memory behind an mbarrier (sm_90 and up)
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while the kernel before it in
// the stream drains. grid_dep_wait blocks until that kernel has completed
// and its writes are visible, so a kernel calls it before it reads anything
// the previous one wrote; grid_dep_launch lets the next kernel start
// launching once every block of this one has called it (or exited), so no
// block of this kernel is ever left without an SM. Both are no-ops in a
// kernel launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// one arrival expected (the thread that posts the transaction count)
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive and announce `bytes` of copies that complete the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// [dst, dst + bytes) of this CTA's shared memory <- [src, src + bytes) of
// global memory; both 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// waits for phase `parity` of the barrier to complete, at most limit_ns;
// false when the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

template <typename T>
__device__ __forceinline__ T warp_exclusive_sum(T x, T *total) {
    const int lane = threadIdx.x & 31;
    T v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    *total = __shfl_sync(0xffffffffu, v, 31);
    return v - x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Grid-wide barrier for cooperative launches. Arrival is one
// atom.add.release.gpu on a counter that only grows during a launch (no
// generation word, no reset between barriers): block k of the i-th barrier
// waits until the counter reaches i * nblocks, polling with relaxed loads
// and finishing with one acquire fence. The counter must be 0 (a multiple
// of nblocks) when the launch starts. A block that waits longer than
// limit_ns sets *err = GB_TIMEOUT and leaves; once *err is set every later
// barrier returns false at once.
struct GridBarrier {
    unsigned int count;
    unsigned int exits;    // blocks that have left the kernel (for end-of-launch resets)
};

__device__ __forceinline__ unsigned int atom_add_release_gpu(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_gpu_int(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync(GridBarrier *bar, unsigned int nblocks, int *err, uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_relaxed_gpu_int(err) == 0;
        if (ok) {
            unsigned int old = atom_add_release_gpu(&bar->count, 1u);
            unsigned int target = old - old % nblocks + nblocks;
            unsigned int spins = 0;
            uint64_t t0 = 0;
            while ((int)(ld_relaxed_gpu(&bar->count) - target) < 0) {
                if ((++spins & 255u) == 0) {
                    uint64_t t = globaltimer_ns();
                    if (t0 == 0) {
                        t0 = t;
                    } else if (t - t0 > limit_ns) {
                        atomicCAS(err, 0, (int)GB_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    if (ld_relaxed_gpu_int(err) != 0) { ok = 0; break; }
                }
            }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Waits (thread 0 polls, the block follows) until *err is nonzero or
// limit_ns has passed; in the second case it records GB_TIMEOUT itself.
// Returns false: the caller has left the barrier protocol. Used only by the
// failure-path test in which one block withholds its barrier arrival.
__device__ __forceinline__ bool wait_for_error(int *err, uint64_t limit_ns) {
    if (threadIdx.x == 0) {
        const uint64_t t0 = globaltimer_ns();
        while (ld_relaxed_gpu_int(err) == 0) {
            if (globaltimer_ns() - t0 > limit_ns) {
                atomicCAS(err, 0, (int)GB_TIMEOUT);
                break;
            }
        }
    }
    __syncthreads();
    return false;
}

}  // namespace dev
}  // namespace gbx
