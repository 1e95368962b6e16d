// Connected components by FastSV (Section 7.4: GraphBLAST's CC follows
// Zhang, Azad and Hu's FastSV), as one persistent cooperative kernel. Every
// vertex u keeps a parent f(u) (initially u) and its grandparent
// gf(u) = f(f(u)); an iteration is
//   mngf(u) = min over neighbours v of gf(v)         (min.second mxv)
//   f(f(u)) = min(f(f(u)), mngf(u))                  (stochastic hooking)
//   f(u)    = min(f(u), mngf(u), gf(u))              (aggressive hooking, shortcut)
//   gf(u)   = f(f(u))                                (grandparents)
// until no grandparent changes. Every value written is an id of a vertex in
// u's component and values only decrease, so the updates are atomicMin in
// any order; the fixed point labels every vertex with the smallest id of
// its component (the roots hook to the minimum). For a matrix whose CSC is
// not the CSR, the neighbours are the union of out- and in-neighbours (weak
// components). Rows longer than SV_LONG are scanned by the whole warp.
#include "common.cuh"

using namespace gbx;

namespace gbx {
namespace svk {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;
constexpr uint32_t SV_LONG = 32;
constexpr uint32_t INF = 0xffffffffu;

struct SvState {
    dev::GridBarrier bar;
    int err;
    unsigned int changed[3];   // vertices whose grandparent changed, per iteration slot
    unsigned int iters;
};

struct SvArgs {
    uint32_t n;
    const uint32_t *rp, *ci;     // CSR
    const uint32_t *rp2, *ci2;   // CSC when it is not the CSR (weak components); else null
    uint32_t *f, *gf, *labels;
    SvState *st;
    uint64_t timeout_ns, total_limit_ns;
    uint32_t max_iters;
};

static __device__ __forceinline__ uint32_t ldcg(const uint32_t *p) { return __ldcg(p); }

// min of gf over the row of u in (rp, ci) for the rows a lane takes alone;
// long rows are marked and done by the whole warp afterwards
static __device__ __forceinline__ uint32_t row_min_short(const uint32_t *rp, const uint32_t *ci, const uint32_t *gf,
                                                         uint32_t b, uint32_t e) {
    uint32_t mn = INF;
    uint32_t k = b;
    for (; k + 4 <= e; k += 4) {
        uint32_t v0 = __ldg(&ci[k]), v1 = __ldg(&ci[k + 1]), v2 = __ldg(&ci[k + 2]), v3 = __ldg(&ci[k + 3]);
        uint32_t g0 = ldcg(&gf[v0]), g1 = ldcg(&gf[v1]), g2 = ldcg(&gf[v2]), g3 = ldcg(&gf[v3]);
        mn = min(mn, min(min(g0, g1), min(g2, g3)));
    }
    for (; k < e; ++k) mn = min(mn, ldcg(&gf[__ldg(&ci[k])]));
    return mn;
}

// the warp scans the rows of the lanes in `longm` together
static __device__ __forceinline__ void rows_min_long(const uint32_t *ci, const uint32_t *gf, uint32_t longm, uint32_t b,
                                                     uint32_t e, uint32_t &mn) {
    const int lane = threadIdx.x & 31;
    while (longm) {
        const int l = __ffs(longm) - 1;
        longm &= longm - 1;
        const uint32_t pb = __shfl_sync(0xffffffffu, b, l), pe = __shfl_sync(0xffffffffu, e, l);
        uint32_t m = INF;
        for (uint32_t k = pb + lane; k < pe; k += 32) m = min(m, ldcg(&gf[__ldg(&ci[k])]));
        m = __reduce_min_sync(0xffffffffu, m);
        if (lane == l) mn = min(mn, m);
    }
}

__global__ void __launch_bounds__(BLOCK, 8) k_fastsv(SvArgs a) {
    __shared__ unsigned int s_changed;
    SvState *st = a.st;
    const uint32_t nthreads = gridDim.x * BLOCK;
    const uint32_t tid = blockIdx.x * BLOCK + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwarps = gridDim.x * WARPS;
    for (uint32_t u = tid; u < a.n; u += nthreads) {
        a.f[u] = u;
        a.gf[u] = u;
    }
    bool ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    const uint64_t t_start = dev::globaltimer_ns();
    uint32_t it = 0;
    while (ok) {
        if (tid == 0) st->changed[(it + 1) % 3] = 0;
        // ---- hooking and shortcut (reads gf, lowers f)
        for (uint64_t base = ((uint64_t)blockIdx.x * WARPS + warp) * 32; base < a.n; base += (uint64_t)nwarps * 32) {
            const uint32_t u = (uint32_t)base + lane;
            const bool in = u < a.n;
            uint32_t mn = INF;
            uint32_t b = 0, e = 0;
            if (in) {
                b = __ldg(&a.rp[u]);
                e = __ldg(&a.rp[u + 1]);
            }
            bool lng = e - b > SV_LONG;
            if (in && !lng) mn = row_min_short(a.rp, a.ci, a.gf, b, e);
            rows_min_long(a.ci, a.gf, __ballot_sync(0xffffffffu, lng), b, e, mn);
            if (a.rp2) {
                b = e = 0;
                if (in) {
                    b = __ldg(&a.rp2[u]);
                    e = __ldg(&a.rp2[u + 1]);
                }
                lng = e - b > SV_LONG;
                if (in && !lng) mn = min(mn, row_min_short(a.rp2, a.ci2, a.gf, b, e));
                rows_min_long(a.ci2, a.gf, __ballot_sync(0xffffffffu, lng), b, e, mn);
            }
            if (in) {
                const uint32_t g = ldcg(&a.gf[u]);
                if (mn != INF) {
                    const uint32_t x = ldcg(&a.f[u]);
                    if (mn < ldcg(&a.f[x])) atomicMin(&a.f[x], mn);   // read first: roots are shared
                }
                const uint32_t lo = min(mn, g);
                if (lo < ldcg(&a.f[u])) atomicMin(&a.f[u], lo);
            }
        }
        if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) { ok = false; break; }
        // ---- grandparents
        if (threadIdx.x == 0) s_changed = 0;
        __syncthreads();
        unsigned int ch = 0;
        for (uint32_t u = tid; u < a.n; u += nthreads) {
            const uint32_t g = ldcg(&a.f[ldcg(&a.f[u])]);
            if (g != ldcg(&a.gf[u])) {
                a.gf[u] = g;
                ++ch;
            }
        }
        ch = dev::warp_sum<unsigned int>(ch);
        if (lane == 0 && ch) atomicAdd(&s_changed, ch);
        __syncthreads();
        if (threadIdx.x == 0 && s_changed) atomicAdd(&st->changed[it % 3], s_changed);
        if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) { ok = false; break; }
        const unsigned int any = dev::ld_relaxed_gpu((const unsigned int *)&st->changed[it % 3]);
        ++it;
        if (!any) break;
        if (it >= a.max_iters ||
            (threadIdx.x == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns)) {
            atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
        }
        if (dev::ld_relaxed_gpu_int(&st->err) != 0) { ok = false; break; }
    }
    // ---- labels: the root above each vertex (one hop at the fixed point)
    if (ok) {
        for (uint32_t u = tid; u < a.n; u += nthreads) {
            uint32_t x = ldcg(&a.f[u]);
            for (int k = 0; k < 64; ++k) {
                const uint32_t y = ldcg(&a.f[x]);
                if (y == x) break;
                x = y;
            }
            a.labels[u] = x;
        }
    }
    if (tid == 0) st->iters = it;
}

// size of each vertex's component from its label: a warp adds the lanes
// with equal labels in one atomic (the giant component of an R-MAT graph
// would otherwise take millions of atomics on one word)
__global__ void k_comp_count(uint32_t n, const uint32_t *labels, uint32_t *count) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint32_t lab = i < n ? labels[i] : INF;
    const uint32_t same = __match_any_sync(0xffffffffu, lab);
    if (lab != INF && lane == __ffs(same) - 1) atomicAdd(&count[lab], (uint32_t)__popc(same));
}

__global__ void k_comp_gather(uint32_t n, const uint32_t *labels, const uint32_t *count, uint32_t *csize) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) csize[i] = count[labels[i]];
}

}  // namespace svk

gb_info matrix_components(gb_context *ctx, gb_matrix *A) {
    std::lock_guard<std::mutex> g(A->cache_mu);
    if (A->comp_size || !A->has_csc || A->nrows == 0 || A->nrows != A->ncols) return GB_SUCCESS;
    const uint32_t n = A->nrows;
    Scratch lab(ctx), cnt(ctx);
    GB_CHECK(lab.alloc((size_t)n * 4 + 16));
    GB_CHECK(cnt.alloc((size_t)n * 4 + 16));
    GB_CHECK(gb_cc_fastsv(ctx, A, lab.as<uint32_t>(), GB_DEVICE, nullptr));
    GB_CHECK(memset_async(ctx, cnt.p, 0, (size_t)n * 4));
    uint32_t *cs = nullptr;
    GB_CHECK(dalloc(ctx, (void **)&cs, (size_t)n * 4 + 16));
    const unsigned nb = (unsigned)((n + 255) / 256);
    svk::k_comp_count<<<nb, 256, 0, ctx->stream>>>(n, lab.as<uint32_t>(), cnt.as<uint32_t>());
    svk::k_comp_gather<<<nb, 256, 0, ctx->stream>>>(n, lab.as<uint32_t>(), cnt.as<uint32_t>(), cs);
    if (cudaGetLastError() != cudaSuccess) {
        dfree(ctx, cs);
        return fail(GB_PANIC, "matrix_components: launch failed");
    }
    A->comp_size = cs;
    return GB_SUCCESS;
}

}  // namespace gbx

extern "C" gb_info gb_cc_fastsv(gb_context *ctx, const gb_matrix *A, uint32_t *labels, gb_mem mem,
                                uint32_t *iterations) {
    if (!ctx || !A || !labels) return fail(GB_NULL_POINTER, "gb_cc_fastsv: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_cc_fastsv: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_cc_fastsv: matrix must be square");
    if (!A->has_csc)
        return fail(GB_INVALID_VALUE, "gb_cc_fastsv: needs a symmetric build or a CSC (both edge directions)");
    if (A->nrows == 0) {
        if (iterations) *iterations = 0;
        return GB_SUCCESS;
    }
    GB_CUDA(cudaSetDevice(ctx->device));
    const uint32_t n = A->nrows;
    Scratch fb(ctx), gb(ctx), sb(ctx), ob(ctx);
    GB_CHECK(fb.alloc((size_t)n * 4 + 16));
    GB_CHECK(gb.alloc((size_t)n * 4 + 16));
    GB_CHECK(sb.alloc(sizeof(svk::SvState)));
    uint32_t *out = labels;
    if (mem == GB_HOST) {
        GB_CHECK(ob.alloc((size_t)n * 4 + 16));
        out = ob.as<uint32_t>();
    }
    GB_CHECK(memset_async(ctx, sb.p, 0, sizeof(svk::SvState)));
    svk::SvArgs a;
    a.n = n;
    a.rp = A->rowptr;
    a.ci = A->colidx;
    a.rp2 = A->csc_alias ? nullptr : A->colptr;
    a.ci2 = A->csc_alias ? nullptr : A->rowidx;
    a.f = fb.as<uint32_t>();
    a.gf = gb.as<uint32_t>();
    a.labels = out;
    a.st = sb.as<svk::SvState>();
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 120000000000ull;
    a.max_iters = 100000;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, svk::k_fastsv, svk::BLOCK, 0));
    if (occ < 1) return fail(GB_PANIC, "gb_cc_fastsv: kernel cannot be resident");
    int grid = occ * ctx->num_sms;
    if (ctx->grid_limit > 0 && ctx->grid_limit < grid) grid = ctx->grid_limit;
    uint64_t need = ((uint64_t)n + svk::BLOCK - 1) / svk::BLOCK;
    if ((uint64_t)grid > need) grid = (int)need;
    void *args[] = {&a};
    int span = prof_begin(ctx, "cc_fastsv");
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)svk::k_fastsv, dim3(grid), dim3(svk::BLOCK), args, 0,
                                        ctx->stream));
    prof_end(ctx, span);
    svk::SvState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, sb.p, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    if (mem == GB_HOST)
        GB_CUDA(cudaMemcpyAsync(labels, out, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (iterations) *iterations = hs.iters;
    if (hs.err) return fail(GB_TIMEOUT, "gb_cc_fastsv: a bounded grid barrier wait or the iteration budget ran out");
    return GB_SUCCESS;
}
