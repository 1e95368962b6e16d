// Adaptive PageRank, also called PageRankDelta (Section 5.1 lists it among
// the uses of the output mask; Section 7.3 names it): the PageRank
// recurrence of gb_pagerank,
//   p'(i) = (1 - a)/n + a * ( sum_{j in N(i)} p(j)/deg(j) + D/n ),
// where a vertex whose value moved by at most eps times its new value has
// converged and is masked out of every later iteration: its value stays,
// and the others keep reading it. Only the active rows are recomputed, so
// the work of an iteration shrinks with the active set.
//
// One persistent cooperative kernel runs all iterations. The active
// vertices form a list (the first iteration takes every vertex), and each
// iteration appends the still-active vertices to the next list and the
// newly converged ones to a frozen list; x = p/deg is double-buffered, and
// a vertex frozen in iteration t has its final x copied into the other
// buffer in iteration t+1, so both buffers hold it from then on. Rows of up
// to 32 entries are summed by one lane, longer rows by a warp; the hub rows
// (longer than GBX_HUB_MIN_LEN, the matrix's cached hub list) stay out of
// the lists: they are dealt to the blocks round-robin, with an active flag
// each, so no block ends up with the long rows of others. Each row's sum
// has one fixed order, so the values do not depend on how rows fall to
// threads. The L1
// residual and the change of the dangling mass D are accumulated as 64-bit
// fixed-point integers (every FP32 PageRank value is an integer multiple of
// 2^-61), which makes their sums independent of the list order: runs are
// bit-reproducible. The convergence test |p' - p| <= eps * p' is made in
// FP32 on the FP32 values.
#include "common.cuh"

using namespace gbx;

namespace gbx {
namespace prd {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;
constexpr uint32_t WARP_ROW = 32;     // rows longer than this: a warp
constexpr uint32_t BLOCK_ROW = GBX_HUB_MIN_LEN;   // rows longer than this: hubs, a block each
constexpr double FIX = 2305843009213693952.0;   // 2^61

struct PrdState {
    dev::GridBarrier bar;
    int err;
    unsigned int iters;
    unsigned int cnt[3];                 // active list produced in an iteration (slot = iteration % 3)
    unsigned int fcnt[3];                // frozen list produced in an iteration
    unsigned int hcnt[3];                // hubs still active after an iteration
    unsigned long long dang[3];          // fixed-point change of D in an iteration (two's complement)
};

struct PrdArgs {
    uint32_t n;
    const uint32_t *rp, *ci;             // rows = in-edges of each vertex
    const uint32_t *rp_out;              // out-degrees
    bool rows_are_out;
    float alpha, eps;
    uint32_t max_iters;
    float *p;                            // the ranks (output), updated in place
    float *x[2];                         // p/deg, double-buffered
    uint32_t *act[2], *frz[2];           // active and frozen lists (hubs excluded)
    const uint32_t *hub;                 // hub vertices (rows longer than BLOCK_ROW)
    uint32_t nhub;
    unsigned char *hub_on;               // [nhub] 1 while the hub is active
    unsigned long long ndangling;        // vertices without out-edges
    unsigned long long *res_fix;         // [max_iters] fixed-point L1 residual per iteration (zeroed by the host)
    uint32_t *act_count;                 // [max_iters] active vertices per iteration
    PrdState *st;
    uint64_t timeout_ns, total_limit_ns;
};

__device__ __forceinline__ long long to_fix(float v) { return __double2ll_rn((double)v * FIX); }

__device__ __forceinline__ uint32_t out_degree(const PrdArgs &a, uint32_t i, uint32_t rowlen) {
    return a.rows_are_out ? rowlen : __ldg(&a.rp_out[i + 1]) - __ldg(&a.rp_out[i]);
}

// row i is summed (y): update p, x, the fixed-point partials, and the lists
__device__ __forceinline__ void finish_row(const PrdArgs &a, uint32_t i, float y, float base, float *xw,
                                           uint32_t rowlen, unsigned long long &res, long long &dang, bool &keep) {
    const float pn = base + a.alpha * y;
    const float po = a.p[i];
    a.p[i] = pn;
    const uint32_t deg = out_degree(a, i, rowlen);
    xw[i] = deg ? pn / (float)deg : 0.f;
    res += (unsigned long long)to_fix(fabsf(pn - po));
    if (!deg) dang += to_fix(pn) - to_fix(po);
    keep = !(fabsf(pn - po) <= a.eps * pn);
}

__global__ void __launch_bounds__(BLOCK, 4) k_prd(PrdArgs a) {
    __shared__ float s_red[WARPS];
    __shared__ unsigned long long s_res[WARPS];
    __shared__ long long s_dang[WARPS];
    const uint32_t nthreads = gridDim.x * BLOCK;
    const uint32_t tid = blockIdx.x * BLOCK + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwarps = gridDim.x * WARPS;
    PrdState *st = a.st;
    // ---- init: p = 1/n, x = p/deg in both buffers
    const float p0 = 1.0f / (float)a.n;
    for (uint32_t i = tid; i < a.n; i += nthreads) {
        a.p[i] = p0;
        const uint32_t deg = out_degree(a, i, __ldg(&a.rp[i + 1]) - __ldg(&a.rp[i]));
        const float x0 = deg ? p0 / (float)deg : 0.f;
        a.x[0][i] = x0;
        a.x[1][i] = x0;
    }
    bool ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    const uint64_t t_start = dev::globaltimer_ns();
    long long D = (long long)a.ndangling * to_fix(p0);   // every block keeps the same running D
    uint32_t nlist = a.n, nhub_on = a.nhub, nfrz = 0, it = 0;   // iteration 0's list: every vertex
    while (ok && nlist + nhub_on > 0 && it < a.max_iters) {
        const float *xr = a.x[it & 1];
        float *xw = a.x[(it + 1) & 1];
        const uint32_t *L = it == 0 ? nullptr : a.act[it & 1];
        const uint32_t *Fz = a.frz[it & 1];
        uint32_t *Ln = a.act[(it + 1) & 1], *Fn = a.frz[(it + 1) & 1];
        const float base = (float)((1.0 - (double)a.alpha) / a.n + (double)a.alpha * ((double)D / FIX) / a.n);
        if (tid == 0) {
            st->cnt[(it + 1) % 3] = 0;
            st->fcnt[(it + 1) % 3] = 0;
            st->dang[(it + 1) % 3] = 0;
            st->hcnt[(it + 1) % 3] = 0;
            a.act_count[it] = (it == 0 ? a.n : nlist + nhub_on);
        }
        // vertices frozen in the previous iteration: their final x into this buffer too
        for (uint32_t k = tid; k < nfrz; k += nthreads) {
            const uint32_t i = __ldcg(&Fz[k]);
            xw[i] = __ldcg(&xr[i]);
        }
        unsigned long long res = 0;
        long long dang = 0;
        // active rows of the list: a lane per short row, a warp per longer row
        // (iteration 0 takes every vertex and skips the hubs, done below)
        for (uint32_t g0 = (blockIdx.x * WARPS + warp) * 32; g0 < nlist; g0 += nwarps * 32) {
            const uint32_t k = g0 + lane;
            uint32_t i = 0, b = 0, e = 0;
            bool in = k < nlist;
            if (in) {
                i = L ? __ldcg(&L[k]) : k;
                b = __ldg(&a.rp[i]);
                e = __ldg(&a.rp[i + 1]);
                if (e - b > BLOCK_ROW) in = false;   // a hub
            }
            const uint32_t len = e - b;
            bool keep = false, done = false;
            if (in && len <= WARP_ROW) {
                float y = 0.f;
                for (uint32_t q = b; q < e; q += 4) {
                    float v[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[t] = q + t < e ? __ldcg(&xr[__ldg(&a.ci[q + t])]) : 0.f;
                    y += v[0];
                    y += v[1];
                    y += v[2];
                    y += v[3];
                }
                finish_row(a, i, y, base, xw, len, res, dang, keep);
                done = true;
            }
            uint32_t mid = __ballot_sync(0xffffffffu, in && len > WARP_ROW && len <= BLOCK_ROW);
            while (mid) {
                const int l = __ffs(mid) - 1;
                mid &= mid - 1;
                const uint32_t ri = __shfl_sync(0xffffffffu, i, l);
                const uint32_t rb = __shfl_sync(0xffffffffu, b, l), re = __shfl_sync(0xffffffffu, e, l);
                float y = 0.f;
                for (uint32_t q0 = rb; q0 < re; q0 += 128) {   // four loads per lane in flight
                    float v[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint32_t q = q0 + t * 32 + lane;
                        v[t] = q < re ? __ldcg(&xr[__ldg(&a.ci[q])]) : 0.f;
                    }
                    y += v[0];
                    y += v[1];
                    y += v[2];
                    y += v[3];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
                if (lane == l) {
                    finish_row(a, ri, y, base, xw, re - rb, res, dang, keep);
                    done = true;
                }
            }
            // lists: still active, or frozen now
            const uint32_t km = __ballot_sync(0xffffffffu, done && keep);
            const uint32_t fm = __ballot_sync(0xffffffffu, done && !keep);
            uint32_t kb = 0, fb = 0;
            if (lane == 0) {
                if (km) kb = atomicAdd(&st->cnt[it % 3], (unsigned int)__popc(km));
                if (fm) fb = atomicAdd(&st->fcnt[it % 3], (unsigned int)__popc(fm));
            }
            kb = __shfl_sync(0xffffffffu, kb, 0);
            fb = __shfl_sync(0xffffffffu, fb, 0);
            if (done && keep) Ln[kb + __popc(km & dev::lanemask_lt())] = i;
            if (done && !keep) Fn[fb + __popc(fm & dev::lanemask_lt())] = i;
        }
        __syncthreads();
        // hubs: dealt to the blocks round-robin, the whole block sums each row
        for (uint32_t h = blockIdx.x; h < a.nhub; h += gridDim.x) {
            if (!a.hub_on[h]) continue;   // uniform over the block
            const uint32_t i = __ldg(&a.hub[h]);
            const uint32_t b = __ldg(&a.rp[i]), e = __ldg(&a.rp[i + 1]);
            float y = 0.f;
            for (uint32_t q0 = b; q0 < e; q0 += 4 * BLOCK) {
                float v[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t q = q0 + t * BLOCK + threadIdx.x;
                    v[t] = q < e ? __ldcg(&xr[__ldg(&a.ci[q])]) : 0.f;
                }
                y += v[0];
                y += v[1];
                y += v[2];
                y += v[3];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane == 0) s_red[warp] = y;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.f;
                for (int w = 0; w < WARPS; ++w) t += s_red[w];
                bool keep = false;
                finish_row(a, i, t, base, xw, e - b, res, dang, keep);
                if (keep) atomicAdd(&st->hcnt[it % 3], 1u);
                else {
                    a.hub_on[h] = 0;
                    Fn[atomicAdd(&st->fcnt[it % 3], 1u)] = i;
                }
            }
            __syncthreads();
        }
        // fixed-point partials of the block
        res = dev::warp_sum<unsigned long long>(res);
        unsigned long long ud = dev::warp_sum<unsigned long long>((unsigned long long)dang);
        if (lane == 0) { s_res[warp] = res; s_dang[warp] = (long long)ud; }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long r = 0, dd = 0;
            for (int w = 0; w < WARPS; ++w) { r += s_res[w]; dd += (unsigned long long)s_dang[w]; }
            if (r) atomicAdd(&a.res_fix[it], r);
            if (dd) atomicAdd(&st->dang[it % 3], dd);
        }
        ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
        if (!ok) break;
        D += (long long)__ldcg(&st->dang[it % 3]);
        nlist = __ldcg(&st->cnt[it % 3]);
        nhub_on = __ldcg(&st->hcnt[it % 3]);
        nfrz = __ldcg(&st->fcnt[it % 3]);
        ++it;
        if (threadIdx.x == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns)
            atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
        ok = dev::ld_relaxed_gpu_int(&st->err) == 0;
    }
    if (tid == 0) st->iters = it;
}

__global__ void k_count_dangling(const uint32_t *rp_out, uint32_t n, unsigned long long *cnt) {
    __shared__ unsigned int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    unsigned int c = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        c += rp_out[i + 1] == rp_out[i];
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0 && s) atomicAdd(cnt, (unsigned long long)s);
}

}  // namespace prd
}  // namespace gbx

extern "C" gb_info gb_pagerank_delta(gb_context *ctx, const gb_matrix *A, float damping, float eps,
                                     uint32_t max_iters, float *rank, gb_mem mem, uint32_t *iterations,
                                     double *residuals, uint32_t *active) {
    using namespace gbx::prd;
    if (!ctx || !A || !rank) return fail(GB_NULL_POINTER, "gb_pagerank_delta: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_pagerank_delta: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_pagerank_delta: matrix must be square");
    if (!(damping >= 0.f && damping <= 1.f)) return fail(GB_INVALID_VALUE, "gb_pagerank_delta: damping not in [0, 1]");
    if (eps != eps || (eps >= 0.f && eps < GB_PAGERANK_DELTA_MIN_EPS))
        return fail(GB_INVALID_VALUE,
                    "gb_pagerank_delta: eps = %g is below the FP32 floor %g (a negative eps never freezes)",
                    (double)eps, (double)GB_PAGERANK_DELTA_MIN_EPS);
    const uint32_t n = A->nrows;
    if (n == 0 || max_iters == 0) {
        if (iterations) *iterations = 0;
        return GB_SUCCESS;
    }
    GB_CUDA(cudaSetDevice(ctx->device));
    const bool sym = A->csc_alias;
    if (!sym && !A->has_csc) return fail(GB_INVALID_VALUE, "gb_pagerank_delta: needs the CSC (in-edges) or a symmetric build");
    Scratch pr(ctx), x(ctx), lists(ctx), resf(ctx), actc(ctx), stb(ctx), nd(ctx), hon(ctx);
    GB_CHECK(matrix_hubs(A, GBX_HUB_MIN_LEN));   // rows of the pulled structure (CSC, or CSR if symmetric)
    float *pout = rank;
    if (mem == GB_HOST) {
        GB_CHECK(pr.alloc((size_t)n * 4 + 16));
        pout = pr.as<float>();
    }
    GB_CHECK(x.alloc((size_t)n * 8 + 32));
    GB_CHECK(lists.alloc((size_t)n * 16 + 64));
    GB_CHECK(resf.alloc((size_t)max_iters * 8 + 16));
    GB_CHECK(actc.alloc((size_t)max_iters * 4 + 16));
    GB_CHECK(stb.alloc(sizeof(PrdState)));
    GB_CHECK(nd.alloc(16));
    GB_CHECK(memset_async(ctx, resf.p, 0, (size_t)max_iters * 8));
    GB_CHECK(memset_async(ctx, actc.p, 0, (size_t)max_iters * 4));
    GB_CHECK(memset_async(ctx, stb.p, 0, sizeof(PrdState)));
    GB_CHECK(memset_async(ctx, nd.p, 0, 8));
    k_count_dangling<<<ctx->num_sms * 2, 256, 0, ctx->stream>>>(A->rowptr, n, nd.as<unsigned long long>());
    GB_LAUNCH_CHECK();
    unsigned long long ndang = 0;
    GB_CUDA(cudaMemcpyAsync(&ndang, nd.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    PrdArgs a;
    a.n = n;
    a.rp = sym ? A->rowptr : A->colptr;
    a.ci = sym ? A->colidx : A->rowidx;
    a.rp_out = A->rowptr;
    a.rows_are_out = sym;
    a.alpha = damping;
    a.eps = eps;
    a.max_iters = max_iters;
    a.p = pout;
    a.x[0] = x.as<float>();
    a.x[1] = x.as<float>() + n;
    uint32_t *lb = lists.as<uint32_t>();
    a.act[0] = lb;
    a.act[1] = lb + n;
    a.frz[0] = lb + 2ull * n;
    a.frz[1] = lb + 3ull * n;
    a.ndangling = ndang;
    a.hub = A->hub_list;
    a.nhub = A->nhub;
    GB_CHECK(hon.alloc((size_t)A->nhub + 16));
    GB_CHECK(memset_async(ctx, hon.p, 1, (size_t)A->nhub + 1));
    a.hub_on = hon.as<unsigned char>();
    a.res_fix = resf.as<unsigned long long>();
    a.act_count = actc.as<uint32_t>();
    a.st = stb.as<PrdState>();
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 120000000000ull;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_prd, BLOCK, 0));
    if (occ < 1) return fail(GB_PANIC, "gb_pagerank_delta: kernel cannot be resident");
    int grid = occ * ctx->num_sms;
    if (ctx->grid_limit > 0 && ctx->grid_limit < grid) grid = ctx->grid_limit;
    void *args[] = {&a};
    int span = prof_begin(ctx, "pagerank_delta");
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)k_prd, dim3(grid), dim3(BLOCK), args, 0, ctx->stream));
    prof_end(ctx, span);
    PrdState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, stb.p, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<unsigned long long> rf(max_iters);
    std::vector<uint32_t> ac(max_iters);
    GB_CUDA(cudaMemcpyAsync(rf.data(), resf.p, (size_t)max_iters * 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(ac.data(), actc.p, (size_t)max_iters * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (mem == GB_HOST) GB_CUDA(cudaMemcpyAsync(rank, pout, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (iterations) *iterations = hs.iters;
    for (uint32_t k = 0; k < max_iters; ++k) {
        if (residuals) residuals[k] = k < hs.iters ? (double)rf[k] / FIX : 0.0;
        if (active) active[k] = k < hs.iters ? ac[k] : 0u;
    }
    if (hs.err) return fail(GB_TIMEOUT, "gb_pagerank_delta: a bounded device wait or the time budget ran out");
    return GB_SUCCESS;
}
