// Triangle counting (Section 7.5) as the masked SpGEMM C<L> = L (+).(pair) L
// (Section 6.3.4): with L strictly lower triangular, C(i,j) counts the k
// with j < k < i and L(i,k), L(k,j), so every triangle {j < k < i} adds one
// to exactly one entry, C(i,j), and the total is the triangle count. The
// per-entry counts are optionally written (the C of the paper); the total is
// reduced in uint64 without writing C at all (the fusion Section 8.3 names as
// the gap to hardwired code).
#include "common.cuh"
#include "ops_impl.cuh"

using namespace gbx;

namespace gbx {
namespace {

constexpr int TC_BLOCK = 256;

// By columns of L: a warp per vertex k puts row_k (the
// neighbours of k below k) in a set in shared memory; its lanes take the
// rows i of column k (the neighbours of k above k, from the CSC) and count
// the entries of row_i below k that the set holds (a prefix of row_i, since
// rows are sorted). Each triangle j < k < i is counted once, at (k, i): this
// is the L.Lt .* L form of the count, Σ over L(i,k) of |row_i ∩ row_k|,
// whose total equals C<L> = L.L's. The set is a bitmap of the ids below k
// while k <= 32 * TC_WORDS (after the degree relabel the rows of small k
// carry most of the work), otherwise a hash table of row_k with linear
// probing at load factor at most one half; rows longer than TC_HROW beyond
// the bitmap's range are probed by binary search in global memory. The
// prefixes are read 16 bytes at a time (the index arrays are 16-byte
// aligned and padded). A hit (i, k, j) is the term L(i,k) L(k,j) of C(i,j),
// and L(i,j) is the probed entry of row i, so when C is asked for the hit
// adds one to that entry's count in place.
constexpr uint32_t TC_WORDS = 1024;   // per warp: a bitmap of 32768 ids or 1024 hash slots
constexpr uint32_t TC_HROW = TC_WORDS / 2;
constexpr uint32_t TC_EMPTY = 0xffffffffu;

// multiplicative hash (Knuth's golden-ratio constant), top `bits` bits
__device__ __forceinline__ uint32_t tc_slot(uint32_t v, int bits) { return (v * 2654435761u) >> (32 - bits); }

template <bool WITH_C>
__global__ void __launch_bounds__(TC_BLOCK) k_tc_hash(uint32_t n, const uint32_t *rp, const uint32_t *ci,
                                                      const uint32_t *cp, const uint32_t *ri, uint32_t *cvals,
                                                      unsigned long long *total) {
    __shared__ uint32_t s_tab[TC_BLOCK / 32][TC_WORDS];
    __shared__ unsigned long long s_tot;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (TC_BLOCK / 32);
    const uint4 *ci4 = reinterpret_cast<const uint4 *>(ci);
    uint32_t *tab = s_tab[warp];
    unsigned long long mine = 0;
    for (uint64_t kk = (uint64_t)blockIdx.x * (TC_BLOCK / 32) + warp; kk < n; kk += nwarps) {
        const uint32_t k = (uint32_t)kk;
        const uint32_t kb = __ldg(&rp[k]), ke = __ldg(&rp[k + 1]);
        const uint32_t cb = __ldg(&cp[k]), ce = __ldg(&cp[k + 1]);
        const uint32_t lk = ke - kb;
        if (lk == 0 || ce == cb) continue;   // warp-uniform
        // 0: bitmap of the ids below k, 1: hash table, 2: binary search of row_k
        const int mode = k <= 32u * TC_WORDS ? 0 : (lk <= TC_HROW ? 1 : 2);
        int bits = 5;
        if (mode == 0) {
            const uint32_t nw = (k + 31) >> 5;
            for (uint32_t s = lane; s < nw; s += 32) tab[s] = 0u;
            __syncwarp();
            for (uint32_t t = lane; t < lk; t += 32) {
                const uint32_t v = __ldg(&ci[kb + t]);
                atomicOr(&tab[v >> 5], 1u << (v & 31));
            }
            __syncwarp();
        } else if (mode == 1) {
            while ((1u << bits) < 2 * lk) ++bits;
            const uint32_t S = 1u << bits;
            for (uint32_t s = lane; s < S; s += 32) tab[s] = TC_EMPTY;
            __syncwarp();
            for (uint32_t t = lane; t < lk; t += 32) {   // the entries are distinct
                const uint32_t v = __ldg(&ci[kb + t]);
                uint32_t h = tc_slot(v, bits);
                while (atomicCAS(&tab[h], TC_EMPTY, v) != TC_EMPTY) h = (h + 1) & (S - 1);
            }
            __syncwarp();
        }
        const uint32_t mask = (1u << bits) - 1;
        for (uint32_t q = cb + lane; q < ce; q += 32) {
            const uint32_t i = __ldg(&ri[q]);
            const uint32_t ib = __ldg(&rp[i]), ie = __ldg(&rp[i + 1]);
            uint32_t cnt = 0;
            bool more = true;
            for (uint32_t x0 = ib & ~3u; x0 < ie && more; x0 += 4) {
                const uint4 w4 = __ldg(&ci4[x0 >> 2]);
                const uint32_t jj[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t x = x0 + u, j = jj[u];
                    if (x < ib) continue;
                    if (!more || x >= ie || j >= k) { more = false; continue; }   // the prefix ends at k
                    bool hit;
                    if (mode == 0) {
                        hit = (tab[j >> 5] >> (j & 31)) & 1u;
                    } else if (mode == 1) {
                        uint32_t h = tc_slot(j, bits), sv;
                        while ((sv = tab[h]) != TC_EMPTY && sv != j) h = (h + 1) & mask;
                        hit = sv == j;
                    } else {
                        uint32_t a = kb, b = ke;   // lower_bound of j in row_k
                        while (a < b) {
                            const uint32_t mid = (a + b) >> 1;
                            if (__ldg(&ci[mid]) < j) a = mid + 1; else b = mid;
                        }
                        hit = a < ke && __ldg(&ci[a]) == j;
                    }
                    // L(i,k) L(k,j) with L(i,j) at position x: one term of C(i,j)
                    if (hit) {
                        ++cnt;
                        if (WITH_C) atomicAdd(&cvals[x], 1u);
                    }
                }
            }
            mine += cnt;
        }
        __syncwarp();   // the set is rebuilt for the next k
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
    if (C) {
        GB_CHECK(cv.alloc((L->nvals + 1) * 4));
        GB_CHECK(memset_async(ctx, cv.p, 0, (L->nvals + 1) * 4));
    }
    uint32_t n = L->nrows;
    if (n) {
        int occ = 0;
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, C ? (const void *)k_tc_hash<true> : (const void *)k_tc_hash<false>, TC_BLOCK, 0));
        unsigned blocks = (unsigned)(occ * ctx->num_sms * 4);
        uint64_t need = ((uint64_t)n + 7) / 8;
        if (need < blocks) blocks = (unsigned)need;
        if (blocks < 1) blocks = 1;
        int span = prof_begin(ctx, "tc");
        if (C)
            k_tc_hash<true><<<blocks, TC_BLOCK, 0, ctx->stream>>>(n, L->rowptr, L->colidx, L->colptr, L->rowidx,
                                                                  cv.as<uint32_t>(), tot.as<unsigned long long>());
        else
            k_tc_hash<false><<<blocks, TC_BLOCK, 0, ctx->stream>>>(n, L->rowptr, L->colidx, L->colptr, L->rowidx,
                                                                   nullptr, tot.as<unsigned long long>());
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
