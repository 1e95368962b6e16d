// PageRank (Section 7.3), pull formulation, in FP32 with FP32 accumulation:
//   p'(i) = (1 - a)/n + a * ( sum_{j in N(i)} p(j)/deg(j) + D/n ),
// D = sum of p over vertices without edges (spread uniformly), p0 = 1/n,
// a fixed number of iterations. The SpMV is merge-path load balanced
// (Section 6.3.2; Merrill and Garland's 2-D diagonal split of row ends
// against nonzeros): every block gets an equal share of the merged
// sequence, so rows of any length cost the same per item. The update is
// fused into the SpMV's row epilogue, which also writes x' = p'/deg for the
// next iteration. Per-iteration L1 residual sum |p' - p| and the dangling
// mass D are reduced in FP64 in a fixed order, as is the final
// normalisation; no floating-point atomics are used, so a run is
// bit-reproducible.
#include "common.cuh"

using namespace gbx;

namespace gbx {
namespace {

constexpr int PR_BLOCK = 256;
constexpr int PR_IPT = 8;
constexpr int PR_LOAD_BATCH = 8;
constexpr int PR_TILE = PR_BLOCK * PR_IPT;
constexpr int PR_RS_BYTES = ((PR_TILE + 2) * 4 + 15) / 16 * 16;
constexpr int PR_SMEM_BYTES = PR_RS_BYTES + PR_IPT * PR_BLOCK * 4 + PR_TILE * 4;

struct PrRec {
    uint32_t first_row;   // row finished by the block's first row end, if it began earlier
    float first_val;
    uint32_t last_row;    // row still open at the block's end
    float last_val;
    uint32_t flags;       // 1 = has a row end, 2 = starts mid-row, 4 = ends mid-row
};

struct PrArgs {
    uint32_t n;
    uint64_t nnz;
    const uint32_t *rp, *ci;      // rows = in-edges of each vertex
    const uint32_t *rp_out;       // out-degrees
    bool rows_are_out;            // rp is also the out-edge structure (symmetric matrix)
    const float *x;               // p(j)/deg(j), 0 for deg(j) = 0
    const float *p_old;
    float *p_new, *x_new;
    const float *base;            // device scalar: (1-a)/n + a*D/n
    float alpha;
    PrRec *rec;
    double *part_res, *part_dang; // per block
    uint32_t nblocks;
};

// merge-path search: split of diagonal d between row ends a[] (absolute
// offsets) and nonzero indices k0, k0+1, ...; returns x = rows consumed
__device__ __forceinline__ uint32_t merge_search_smem(const uint32_t *a, uint32_t nrows, uint32_t k0, uint32_t nk,
                                                      uint32_t d) {
    uint32_t lo = d > nk ? d - nk : 0;
    uint32_t hi = d < nrows ? d : nrows;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= k0 + d - mid - 1) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// the same on the global row-end array rp[1..n] for an absolute diagonal,
// done by the whole block (one probe per thread per round)
__device__ uint32_t block_merge_search(const uint32_t *rp, uint32_t n, uint64_t nnz, uint64_t d) {
    uint32_t lo = d > nnz ? (uint32_t)(d - nnz) : 0;
    uint32_t hi = d < n ? (uint32_t)d : n;
    // invariant: answer in [lo, hi]; predicate(x) = rp[x+1] <= d - x - 1 is monotone (true then false)
    while (hi > lo) {
        uint32_t span = hi - lo;
        uint32_t step = (span + PR_BLOCK - 1) / PR_BLOCK;
        uint32_t x = lo + threadIdx.x * step;
        int ok = x < hi && (uint64_t)__ldg(&rp[x + 1]) + x + 1 <= d;
        int c = __syncthreads_count(ok);
        if (c == 0) { hi = lo; break; }
        uint32_t last_ok = lo + (uint32_t)(c - 1) * step;   // predicate true here, maybe beyond
        lo = last_ok + 1;
        uint32_t nh = last_ok + step;
        hi = nh < hi ? nh : hi;
    }
    return lo;
}

struct Seg {
    int reset;   // thread (or prefix) contains a row end
    float v;     // partial of the row open at its end
};
__device__ __forceinline__ Seg seg_op(Seg a, Seg b) {
    Seg r;
    r.reset = a.reset | b.reset;
    r.v = b.reset ? b.v : a.v + b.v;
    return r;
}

// row i is complete with sum y: write p'(i), x'(i) = p'(i)/deg(i), and add
// to the residual and dangling partials. rowlen is row i's length in the
// pulled structure; it is the out-degree when that structure is the CSR
// itself (symmetric matrix), otherwise the out-degree is read from rp_out.
__device__ __forceinline__ void epilogue(const PrArgs &a, uint32_t i, float y, float base, float p_old, uint32_t rowlen,
                                         double &res, double &dang) {
    float p = base + a.alpha * y;
    uint32_t deg = a.rows_are_out ? rowlen : __ldg(&a.rp_out[i + 1]) - __ldg(&a.rp_out[i]);
    a.p_new[i] = p;
    a.x_new[i] = deg ? p / (float)deg : 0.f;
    res += fabs((double)p - (double)p_old);
    if (!deg) dang += (double)p;
}

__global__ void __launch_bounds__(PR_BLOCK, 6) k_pr_spmv(PrArgs a) {
    // dynamic shared memory: s_rs[0] = start of the chunk's first row,
    // s_rs[r + 1] = end of its row r; gathered x values and previous ranks
    extern __shared__ __align__(16) unsigned char pr_smem[];
    uint32_t *s_rs = reinterpret_cast<uint32_t *>(pr_smem);
    float (*s_xv)[PR_BLOCK] = reinterpret_cast<float (*)[PR_BLOCK]>(pr_smem + PR_RS_BYTES);
    float *s_sum = reinterpret_cast<float *>(pr_smem + PR_RS_BYTES + PR_IPT * PR_BLOCK * 4);   // finished rows
    __shared__ Seg s_scan[PR_BLOCK / 32];
    __shared__ uint32_t s_x[PR_BLOCK + 1];
    __shared__ double s_red[2][PR_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)a.n + a.nnz;
    const uint64_t D0 = total * blockIdx.x / gridDim.x, D1 = total * (blockIdx.x + 1) / gridDim.x;
    const float base = *a.base;
    double res = 0.0, dang = 0.0;
    uint32_t i0 = block_merge_search(a.rp, a.n, a.nnz, D0);
    uint32_t ic = i0;
    uint64_t kc = D0 - i0;
    const bool start_mid = i0 < a.n && kc > __ldg(&a.rp[i0]);
    bool pending = start_mid;          // the first row end closes a row begun before D0
    bool has_end = false;
    Seg carry = {0, 0.f};
    for (uint64_t c = D0; c < D1; c += PR_TILE) {
        const uint64_t ce = c + PR_TILE < D1 ? c + PR_TILE : D1;
        const uint32_t clen = (uint32_t)(ce - c);
        // stage the row bounds the chunk can reach, PR_BLOCK at a time, until a
        // staged row end lies at or past the chunk's last nonzero: no row
        // beyond it can end inside the chunk, so the merge searches never
        // look further (a chunk of rows of ~30 entries needs one round instead
        // of the clen + 1 bounds a chunk of empty rows would)
        const uint32_t avail = a.n - ic;
        const uint32_t Rmax = avail < clen + 1 ? avail : clen + 1;
        uint32_t R = Rmax;
        for (uint32_t r0 = 0;; r0 += PR_BLOCK) {
            const uint32_t r = r0 + threadIdx.x;
            if (r <= Rmax) s_rs[r] = __ldg(&a.rp[ic + r]);
            __syncthreads();
            const uint32_t last = r0 + PR_BLOCK - 1 < Rmax ? r0 + PR_BLOCK - 1 : Rmax;
            if (last == Rmax || (uint64_t)s_rs[last] >= kc + clen) {
                R = last;
                break;
            }
        }
        const uint32_t *s_re = s_rs + 1;
        const uint64_t nk_left = a.nnz - kc;
        const uint32_t bl = nk_left < clen ? (uint32_t)nk_left : clen;
        // one merge-path search per thread for the start of its items; the
        // last thread also finds the chunk end; neighbours exchange them
        uint32_t d0 = threadIdx.x * PR_IPT < clen ? threadIdx.x * PR_IPT : clen;
        const uint32_t x0 = merge_search_smem(s_re, R, (uint32_t)kc, bl, d0);
        s_x[threadIdx.x] = x0;
        if (threadIdx.x == PR_BLOCK - 1) s_x[PR_BLOCK] = merge_search_smem(s_re, R, (uint32_t)kc, bl, clen);
        __syncthreads();
        const uint32_t nrows = s_x[PR_BLOCK];                  // row ends inside the chunk
        const uint32_t nk = clen - nrows;
        const uint32_t ie = ic + nrows;
        uint32_t d1 = d0 + PR_IPT < clen ? d0 + PR_IPT : clen;
        const uint32_t x1 = s_x[threadIdx.x + 1];
        const uint32_t tk0 = (uint32_t)kc + (d0 - x0), tk1 = (uint32_t)kc + (d1 - x1);
        // all loads of the thread at once: column indices, then the gathers,
        // and the previous ranks of the rows it finishes
#pragma unroll
        for (int j0 = 0; j0 < PR_IPT; j0 += PR_LOAD_BATCH) {
            float xv[PR_LOAD_BATCH];
            uint32_t cidx[PR_LOAD_BATCH];
#pragma unroll
            for (int j = 0; j < PR_LOAD_BATCH; ++j) cidx[j] = tk0 + j0 + j < tk1 ? __ldcs(&a.ci[tk0 + j0 + j]) : 0u;
#pragma unroll
            for (int j = 0; j < PR_LOAD_BATCH; ++j) xv[j] = tk0 + j0 + j < tk1 ? __ldcg(&a.x[cidx[j]]) : 0.f;
#pragma unroll
            for (int j = 0; j < PR_LOAD_BATCH; ++j) s_xv[j0 + j][threadIdx.x] = xv[j];
        }
        // walk the items: a row end stores the row's sum (the first one
        // also needs the partial sums of earlier threads, added after the scan)
        uint32_t ti = x0, tk = tk0, jn = 0;
        float sum = 0.f;
        bool head = false;
        float head_val = 0.f;
        for (uint32_t d = d0; d < d1; ++d) {
            if (ti < nrows && tk >= s_re[ti]) {
                if (!head) { head = true; head_val = sum; }
                else s_sum[ti] = sum;
                sum = 0.f;
                ++ti;
            } else {
                sum += s_xv[jn++][threadIdx.x];
                ++tk;
            }
        }
        // segmented scan over threads: carry into each thread
        Seg me = {head ? 1 : 0, sum};
        Seg incl = me;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Seg y;
            y.reset = __shfl_up_sync(0xffffffffu, incl.reset, o);
            y.v = __shfl_up_sync(0xffffffffu, incl.v, o);
            if (lane >= o) incl = seg_op(y, incl);
        }
        if (lane == 31) s_scan[warp] = incl;
        __syncthreads();
        Seg wpre = carry;                       // chunk carry-in, then earlier warps
        Seg tot_all = carry;
        bool any_head = false;
#pragma unroll
        for (int w = 0; w < PR_BLOCK / 32; ++w) {
            Seg sw = s_scan[w];
            if (w < warp) wpre = seg_op(wpre, sw);
            tot_all = seg_op(tot_all, sw);
            any_head |= sw.reset != 0;
        }
        Seg excl_lane;
        excl_lane.reset = __shfl_up_sync(0xffffffffu, incl.reset, 1);
        excl_lane.v = __shfl_up_sync(0xffffffffu, incl.v, 1);
        Seg into = lane == 0 ? wpre : seg_op(wpre, excl_lane);
        if (head) s_sum[x0] = into.v + head_val;
        __syncthreads();
        // epilogue over the chunk's finished rows [ic, ie): coalesced, one row per thread
        const bool first_pending = pending && nrows > 0;   // row ic began before this block
        for (uint32_t r = threadIdx.x; r < nrows; r += PR_BLOCK) {
            float y = s_sum[r];
            if (r == 0 && first_pending) {
                a.rec[blockIdx.x].first_row = ic;
                a.rec[blockIdx.x].first_val = y;
            } else {
                epilogue(a, ic + r, y, base, __ldg(&a.p_old[ic + r]), s_rs[r + 1] - s_rs[r], res, dang);
            }
        }
        carry.reset = 0;
        carry.v = tot_all.v;
        if (any_head) { pending = false; has_end = true; }
        ic = ie;
        kc = kc + nk;
        __syncthreads();   // the staged arrays and s_scan are rewritten by the next chunk
    }
    // block records
    if (threadIdx.x == 0) {
        uint32_t fl = (has_end ? 1u : 0u) | (start_mid ? 2u : 0u);
        bool end_open = ic < a.n && kc > __ldg(&a.rp[ic]);
        if (end_open) fl |= 4u;
        PrRec &r = a.rec[blockIdx.x];
        r.last_row = ic;
        r.last_val = carry.v;
        r.flags = fl;
        if (!has_end) { r.first_row = i0; r.first_val = 0.f; }
    }
    // fixed-order block reduction of the FP64 partials
    res = dev::warp_sum<double>(res);
    dang = dev::warp_sum<double>(dang);
    if (lane == 0) { s_red[0][warp] = res; s_red[1][warp] = dang; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0, r1 = 0;
        for (int w = 0; w < PR_BLOCK / 32; ++w) { r0 += s_red[0][w]; r1 += s_red[1][w]; }
        a.part_res[blockIdx.x] = r0;
        a.part_dang[blockIdx.x] = r1;
    }
}

// One block: finishes the rows that cross block boundaries (walking
// forward from the block where each one starts, summing in block order),
// then reduces all FP64 partials in a fixed order into the residual and the
// next iteration's dangling mass and base term.
__global__ void __launch_bounds__(PR_BLOCK) k_pr_fix(PrArgs a, double *residual_out, double *dang_io, float *base_out,
                                                    double *fix_res, double *fix_dang, int init) {
    __shared__ double s[2][PR_BLOCK];
    const float base = *a.base;
    if (!init) {
        for (uint32_t b = threadIdx.x; b < a.nblocks; b += PR_BLOCK) {
            double r = 0, dn = 0;
            const PrRec &rb = a.rec[b];
            bool open = rb.flags & 4u;
            bool starts_here = (rb.flags & 1u) || !(rb.flags & 2u);
            if (open && starts_here) {
                uint32_t row = rb.last_row;
                float tot = rb.last_val;
                for (uint32_t b2 = b + 1; b2 < a.nblocks; ++b2) {
                    const PrRec &q = a.rec[b2];
                    if (!(q.flags & 1u)) { tot += q.last_val; continue; }
                    tot += q.first_val;
                    break;
                }
                epilogue(a, row, tot, base, a.p_old[row], __ldg(&a.rp[row + 1]) - __ldg(&a.rp[row]), r, dn);
            }
            fix_res[b] = r;
            fix_dang[b] = dn;
        }
        __syncthreads();
    }
    double r0 = 0, r1 = 0;
    for (uint32_t b = threadIdx.x; b < a.nblocks; b += PR_BLOCK) {
        r0 += a.part_res[b] + (init ? 0.0 : fix_res[b]);
        r1 += a.part_dang[b] + (init ? 0.0 : fix_dang[b]);
    }
    s[0][threadIdx.x] = r0;
    s[1][threadIdx.x] = r1;
    __syncthreads();
    for (int st = PR_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) { s[0][threadIdx.x] += s[0][threadIdx.x + st]; s[1][threadIdx.x] += s[1][threadIdx.x + st]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (residual_out) *residual_out = s[0][0];
        *dang_io = s[1][0];
        double n = (double)a.n;
        *base_out = (float)((1.0 - (double)a.alpha) / n + (double)a.alpha * s[1][0] / n);
    }
}

// p0 = 1/n, x0 = p0/deg; per-block dangling mass
__global__ void __launch_bounds__(PR_BLOCK) k_pr_init(uint32_t n, const uint32_t *rp_out, float *p, float *x,
                                                     double *part_dang, double *part_res) {
    __shared__ double s[PR_BLOCK];
    double dn = 0;
    float p0 = 1.0f / (float)n;
    for (uint32_t i = blockIdx.x * PR_BLOCK + threadIdx.x; i < n; i += gridDim.x * PR_BLOCK) {
        uint32_t deg = rp_out[i + 1] - rp_out[i];
        p[i] = p0;
        x[i] = deg ? p0 / (float)deg : 0.f;
        if (!deg) dn += 1.0 / (double)n;
    }
    s[threadIdx.x] = dn;
    __syncthreads();
    for (int st = PR_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) { part_dang[blockIdx.x] = s[0]; part_res[blockIdx.x] = 0.0; }
}

// final normalisation: S = sum p in FP64 (fixed order), p /= S
__global__ void __launch_bounds__(PR_BLOCK) k_pr_sum(uint32_t n, const float *p, double *part) {
    __shared__ double s[PR_BLOCK];
    double acc = 0;
    uint64_t per = ((uint64_t)n + gridDim.x - 1) / gridDim.x;
    uint64_t b0 = per * blockIdx.x, b1 = b0 + per < n ? b0 + per : n;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += PR_BLOCK) acc += (double)p[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int st = PR_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(PR_BLOCK) k_pr_norm(uint32_t n, const float *p, const double *part, uint32_t nparts,
                                                     float *out) {
    __shared__ double s_tot;
    if (threadIdx.x == 0) {
        double t = 0;
        for (uint32_t b = 0; b < nparts; ++b) t += part[b];
        s_tot = t;
    }
    __syncthreads();
    const double inv = 1.0 / s_tot;
    for (uint32_t i = blockIdx.x * PR_BLOCK + threadIdx.x; i < n; i += gridDim.x * PR_BLOCK)
        out[i] = (float)((double)p[i] * inv);
}

}  // namespace
}  // namespace gbx

extern "C" gb_info gb_pagerank(gb_context *ctx, const gb_matrix *A, float damping, uint32_t iters, float *rank,
                               double *residuals, gb_mem mem) {
    if (!ctx || !A || !rank) return fail(GB_NULL_POINTER, "gb_pagerank: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_pagerank: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_pagerank: matrix must be square");
    if (!A->has_csc) return fail(GB_INVALID_VALUE, "gb_pagerank: needs the CSC copy (in-edges)");
    if (!(damping >= 0.f && damping <= 1.f)) return fail(GB_INVALID_VALUE, "gb_pagerank: damping must be in [0, 1]");
    const uint32_t n = A->nrows;
    if (n == 0) return GB_SUCCESS;
    GB_CUDA(cudaSetDevice(ctx->device));
    int occ = 0;
    GB_CUDA(cudaFuncSetAttribute(k_pr_spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM_BYTES));
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pr_spmv, PR_BLOCK, PR_SMEM_BYTES));
    uint64_t total = (uint64_t)n + A->nvals;
    uint32_t G = (uint32_t)(occ * ctx->num_sms);
    if (G < 1) G = 1;
    // at least a few tiles of work per block
    uint64_t maxg = total / (PR_TILE * 4) + 1;
    if (G > maxg) G = (uint32_t)maxg;
    Scratch p0(ctx), p1(ctx), x0(ctx), x1(ctx), rec(ctx), pres(ctx), pdang(ctx), fres(ctx), fdang(ctx), scal(ctx),
        resid(ctx), outb(ctx);
    GB_CHECK(p0.alloc((size_t)n * 4 + 16));
    GB_CHECK(p1.alloc((size_t)n * 4 + 16));
    GB_CHECK(x0.alloc((size_t)n * 4 + 16));
    GB_CHECK(x1.alloc((size_t)n * 4 + 16));
    uint32_t nrec = G > 1024 ? G : 1024;
    GB_CHECK(rec.alloc((size_t)nrec * sizeof(PrRec)));
    GB_CHECK(pres.alloc((size_t)nrec * 8));
    GB_CHECK(pdang.alloc((size_t)nrec * 8));
    GB_CHECK(fres.alloc((size_t)nrec * 8));
    GB_CHECK(fdang.alloc((size_t)nrec * 8));
    GB_CHECK(scal.alloc(64));
    GB_CHECK(resid.alloc(((size_t)iters + 1) * 8));
    float *out = rank;
    if (mem == GB_HOST) { GB_CHECK(outb.alloc((size_t)n * 4 + 16)); out = outb.as<float>(); }
    double *dang = scal.as<double>();
    float *base = reinterpret_cast<float *>(scal.as<char>() + 16);
    PrArgs a;
    a.n = n;
    a.nnz = A->nvals;
    a.rp = A->colptr;
    a.ci = A->rowidx;
    a.rp_out = A->rowptr;
    a.rows_are_out = A->csc_alias;
    a.alpha = damping;
    a.rec = rec.as<PrRec>();
    a.part_res = pres.as<double>();
    a.part_dang = pdang.as<double>();
    a.base = base;
    // init: p0, x0, D0 -> base
    uint32_t ib = 1024;
    k_pr_init<<<ib, PR_BLOCK, 0, ctx->stream>>>(n, A->rowptr, p0.as<float>(), x0.as<float>(), pdang.as<double>(),
                                              pres.as<double>());
    a.nblocks = ib;
    k_pr_fix<<<1, PR_BLOCK, 0, ctx->stream>>>(a, nullptr, dang, base, fres.as<double>(), fdang.as<double>(), 1);
    GB_LAUNCH_CHECK();
    a.nblocks = G;
    float *pc = p0.as<float>(), *pn = p1.as<float>(), *xc = x0.as<float>(), *xn = x1.as<float>();
    for (uint32_t it = 0; it < iters; ++it) {
        a.p_old = pc; a.x = xc; a.p_new = pn; a.x_new = xn;
        int span = prof_begin(ctx, "pagerank_spmv");
        k_pr_spmv<<<G, PR_BLOCK, PR_SMEM_BYTES, ctx->stream>>>(a);
        prof_end(ctx, span);
        k_pr_fix<<<1, PR_BLOCK, 0, ctx->stream>>>(a, resid.as<double>() + it, dang, base, fres.as<double>(),
                                                 fdang.as<double>(), 0);
        GB_LAUNCH_CHECK();
        float *t = pc; pc = pn; pn = t;
        t = xc; xc = xn; xn = t;
    }
    // final normalisation in FP64
    k_pr_sum<<<1024, PR_BLOCK, 0, ctx->stream>>>(n, pc, pres.as<double>());
    k_pr_norm<<<1024, PR_BLOCK, 0, ctx->stream>>>(n, pc, pres.as<double>(), 1024, out);
    GB_LAUNCH_CHECK();
    if (residuals && iters) GB_CUDA(cudaMemcpyAsync(residuals, resid.p, (size_t)iters * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (mem == GB_HOST) GB_CUDA(cudaMemcpyAsync(rank, out, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (residuals || mem == GB_HOST) GB_CHECK(sync(ctx));
    return GB_SUCCESS;
}
