// Triangle counting (Section 7.5) as the masked SpGEMM C<L> = L (+).(x) L
// over (plus, pair) (Section 6.3.4), reduced on the fly: for every stored
// L(i,j), C(i,j) = |row_i(L) intersect col_j(L)|, computed by binary
// search of the shorter list's entries in the longer one. With L strictly
// lower triangular each triangle {k < j < i} is counted once, at (i, j)
// through its middle vertex k... in the L*L form, at (i,j) with j < k < i.
// The per-entry counts are optionally written (the C of the paper); the
// total is reduced in uint64 without writing C at all (the fusion Section 8.3
// names as the gap to hardwired code). When only the total is asked for, a
// cheaper equivalent count runs instead (k_tc_forward).
#include "common.cuh"
#include "ops_impl.cuh"

using namespace gbx;

namespace gbx {
namespace {

constexpr int TC_BLOCK = 256;

// lower_bound of x in a[lo, hi)
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&a[mid]) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// A warp per row i of L. Lanes take the row's mask entries j in turn; for
// each (i, j) the lane intersects row_i (entries k < i) with col_j
// (entries k > j) by binary searching each entry of the shorter list in the
// longer. Only k in (j, i) can be common, which bounds both searches.
__global__ void __launch_bounds__(TC_BLOCK) k_tc(uint32_t n, const uint32_t *rp, const uint32_t *ci,
                                                 const uint32_t *cp, const uint32_t *ri, uint32_t *cvals,
                                                 unsigned long long *total) {
    __shared__ unsigned long long s_tot;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (TC_BLOCK / 32);
    unsigned long long mine = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * (TC_BLOCK / 32) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const uint32_t rb = __ldg(&rp[i]), re = __ldg(&rp[i + 1]);
        for (uint32_t q = rb + lane; q < re; q += 32) {
            const uint32_t j = __ldg(&ci[q]);
            // row_i restricted to (j, i): entries after q (rows are sorted)
            const uint32_t ab = q + 1, ae = re;
            // col_j restricted to (j, i): entries below i
            const uint32_t bb = __ldg(&cp[j]);
            const uint32_t be = lower_bound_u32(ri, bb, __ldg(&cp[j + 1]), (uint32_t)i);
            uint32_t cnt = 0;
            if (ae - ab <= be - bb) {
                uint32_t lo = bb;
                for (uint32_t x = ab; x < ae && lo < be; ++x) {
                    uint32_t k = __ldg(&ci[x]);
                    lo = lower_bound_u32(ri, lo, be, k);
                    if (lo < be && __ldg(&ri[lo]) == k) ++cnt;
                }
            } else {
                uint32_t lo = ab;
                for (uint32_t x = bb; x < be && lo < ae; ++x) {
                    uint32_t k = __ldg(&ri[x]);
                    lo = lower_bound_u32(ci, lo, ae, k);
                    if (lo < ae && __ldg(&ci[lo]) == k) ++cnt;
                }
            }
            if (cvals) cvals[q] = cnt;
            mine += cnt;
        }
    }
    mine = dev::warp_sum<unsigned long long>(mine);
    if (lane == 0 && mine) atomicAdd(&s_tot, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_tot) atomicAdd(total, s_tot);
}

// Total only: a warp per row i stages row_i (the neighbours of i below i,
// ascending) in shared memory; lane t takes the t-th entry k of the row and
// counts the entries j of row_k (all below k) that row_i also holds: those
// sit in row_i before k's own position, found by a binary search that only
// moves forward. Each triangle j < k < i is counted once, at (i, k). This is
// the L.Lt .* L form of the count; the total equals C<L> = L.L's, and with
// the degree-descending relabel every row is short. Rows longer than
// TC_CAP are searched in global memory instead.
constexpr int TC_CAP = 512;
__global__ void __launch_bounds__(TC_BLOCK) k_tc_forward(uint32_t n, const uint32_t *rp, const uint32_t *ci,
                                                         unsigned long long *total) {
    __shared__ uint32_t s_row[TC_BLOCK / 32][TC_CAP];
    __shared__ unsigned long long s_tot;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (TC_BLOCK / 32);
    uint32_t *row = s_row[warp];
    unsigned long long mine = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * (TC_BLOCK / 32) + warp; i < n; i += nwarps) {
        const uint32_t rb = __ldg(&rp[i]), re = __ldg(&rp[i + 1]);
        const uint32_t li = re - rb;
        if (li < 2) continue;   // warp-uniform
        const bool staged = li <= (uint32_t)TC_CAP;
        if (staged) {
            for (uint32_t t = lane; t < li; t += 32) row[t] = __ldg(&ci[rb + t]);
            __syncwarp();
        }
        for (uint32_t t = 1 + lane; t < li; t += 32) {   // k = row_i[t]; entries before t are below k
            const uint32_t k = staged ? row[t] : __ldg(&ci[rb + t]);
            const uint32_t kb = __ldg(&rp[k]), ke = __ldg(&rp[k + 1]);
            uint32_t lo = 0, cnt = 0;
            for (uint32_t x0 = kb; x0 < ke && lo < t; x0 += 4) {
                uint32_t jj[4];   // four entries of row_k in flight, then their searches
#pragma unroll
                for (int u = 0; u < 4; ++u) jj[u] = x0 + u < ke ? __ldg(&ci[x0 + u]) : 0xffffffffu;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t j = jj[u];
                    if (j == 0xffffffffu || lo >= t) continue;
                    uint32_t a = lo, b = t;   // lower_bound of j in row_i[lo, t)
                    while (a < b) {
                        const uint32_t mid = (a + b) >> 1;
                        const uint32_t r = staged ? row[mid] : __ldg(&ci[rb + mid]);
                        if (r < j) a = mid + 1; else b = mid;
                    }
                    lo = a;
                    if (a < t && (staged ? row[a] : __ldg(&ci[rb + a])) == j) { ++cnt; ++lo; }
                }
            }
            mine += cnt;
        }
        __syncwarp();   // the row buffer is rewritten for the next row
    }
    mine = dev::warp_sum<unsigned long long>(mine);
    if (lane == 0 && mine) atomicAdd(&s_tot, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_tot) atomicAdd(total, s_tot);
}

}  // namespace

gb_info matrix_build_device(gb_matrix *A, const uint32_t *rows, const uint32_t *cols, const void *vals, uint64_t ntup,
                            gb_binop dup, uint32_t flags);
gb_info matrix_expand_rows(const gb_matrix *A, uint32_t *rows);

}  // namespace gbx

extern "C" gb_info gb_tc(gb_context *ctx, const gb_matrix *L, uint64_t *count, gb_matrix *C) {
    if (!ctx || !L || !count) return fail(GB_NULL_POINTER, "gb_tc: NULL argument");
    if (!L->built) return fail(GB_INVALID_VALUE, "gb_tc: L not built");
    if (L->nrows != L->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_tc: L must be square");
    if (!L->has_csc || L->csc_alias) return fail(GB_INVALID_VALUE, "gb_tc: L needs its own CSC copy (build it from tril)");
    if (C && (C->nrows != L->nrows || C->ncols != L->ncols)) return fail(GB_DIMENSION_MISMATCH, "gb_tc: C dims");
    if (C && C->type != GB_UINT32) return fail(GB_DOMAIN_MISMATCH, "gb_tc: C must be GB_UINT32");
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch tot(ctx), cv(ctx), rows(ctx);
    GB_CHECK(tot.alloc(8));
    GB_CHECK(memset_async(ctx, tot.p, 0, 8));
    if (C) GB_CHECK(cv.alloc((L->nvals + 1) * 4));
    uint32_t n = L->nrows;
    if (n) {
        int occ = 0;
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, C ? (const void *)k_tc : (const void *)k_tc_forward,
                                                              TC_BLOCK, 0));
        unsigned blocks = (unsigned)(occ * ctx->num_sms * 4);
        uint64_t need = ((uint64_t)n + 7) / 8;
        if (need < blocks) blocks = (unsigned)need;
        if (blocks < 1) blocks = 1;
        int span = prof_begin(ctx, "tc");
        if (C)   // per-entry C<L> = L.L: the intersection kernel
            k_tc<<<blocks, TC_BLOCK, 0, ctx->stream>>>(n, L->rowptr, L->colidx, L->colptr, L->rowidx,
                                                       cv.as<uint32_t>(), tot.as<unsigned long long>());
        else     // the total alone
            k_tc_forward<<<blocks, TC_BLOCK, 0, ctx->stream>>>(n, L->rowptr, L->colidx, tot.as<unsigned long long>());
        prof_end(ctx, span);
        GB_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    GB_CUDA(cudaMemcpyAsync(&h, tot.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (C) {
        GB_CHECK(rows.alloc((L->nvals + 1) * 4));
        GB_CHECK(matrix_expand_rows(L, rows.as<uint32_t>()));
        GB_CHECK(matrix_build_device(C, rows.as<uint32_t>(), L->colidx, cv.p, L->nvals, GB_FIRST, GB_BUILD_DEFAULT));
    }
    GB_CHECK(sync(ctx));
    *count = h;
    return GB_SUCCESS;
}
