// Device-wide primitives used by matrix/vector construction: exclusive scan,
// a stable LSD radix sort of (key, value) pairs, and the tuple -> CSR build
// (sort, duplicate combine, row offsets).
#include "common.cuh"
#include "types.cuh"

namespace gbx {

// --------------------------------------------------------------------- scan
namespace {
constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t x, uint32_t *smem_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t wt;
    uint32_t ex = dev::warp_exclusive_sum(x, &wt);
    if (lane == 0) smem_warp[warp] = wt;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < (SCAN_BLOCK / 32) ? smem_warp[lane] : 0u;
        uint32_t t;
        uint32_t e = dev::warp_exclusive_sum(v, &t);
        if (lane < (SCAN_BLOCK / 32)) smem_warp[lane] = e;
        if (lane == 0) smem_warp[SCAN_BLOCK / 32] = t;
    }
    __syncthreads();
    uint32_t r = ex + smem_warp[warp];
    *total = smem_warp[SCAN_BLOCK / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_reduce(const uint32_t *in, uint64_t n, uint32_t *partials) {
    __shared__ uint32_t sw[SCAN_BLOCK / 32 + 1];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
    uint32_t tot;
    block_exclusive_sum(s, sw, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// single block: exclusive scan of the partials in chunks, carrying a running sum
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_partials(uint32_t *partials, uint64_t np, uint32_t *total) {
    __shared__ uint32_t sw[SCAN_BLOCK / 32 + 1];
    uint32_t carry = 0;
    for (uint64_t c = 0; c < np; c += SCAN_TILE) {
        uint64_t base = c + (uint64_t)threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS];
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = base + k < np ? partials[base + k] : 0u;
            s += v[k];
        }
        uint32_t tot;
        uint32_t ex = block_exclusive_sum(s, sw, &tot) + carry;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (base + k < np) partials[base + k] = ex;
            ex += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_down(const uint32_t *in, uint32_t *out, uint64_t n,
                                                        const uint32_t *partials) {
    __shared__ uint32_t sw[SCAN_BLOCK / 32 + 1];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_sum(s, sw, &tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
}
}  // namespace

gb_info scan_exclusive_u32(gb_context *ctx, const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *total) {
    if (n == 0) {
        if (total) GB_CHECK(memset_async(ctx, total, 0, sizeof(uint32_t)));
        return GB_SUCCESS;
    }
    uint64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    Scratch part(ctx);
    GB_CHECK(part.alloc(nb * sizeof(uint32_t)));
    k_scan_reduce<<<(unsigned)nb, SCAN_BLOCK, 0, ctx->stream>>>(in, n, part.as<uint32_t>());
    k_scan_partials<<<1, SCAN_BLOCK, 0, ctx->stream>>>(part.as<uint32_t>(), nb, total);
    k_scan_down<<<(unsigned)nb, SCAN_BLOCK, 0, ctx->stream>>>(in, out, n, part.as<uint32_t>());
    GB_LAUNCH_CHECK();
    return GB_SUCCESS;
}

// --------------------------------------------------------------- radix sort
namespace {
constexpr int RS_BLOCK = 256;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_BLOCK * RS_ROUNDS;  // 2048 keys per tile
constexpr int RS_RADIX = 256;

__global__ void __launch_bounds__(RS_BLOCK) k_rs_hist(const uint64_t *keys, uint64_t n, int shift, uint32_t *counts,
                                                      uint32_t ntiles) {
    __shared__ uint32_t h[RS_RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        uint64_t i = base + (uint64_t)r * RS_BLOCK + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: a tile is split into per-warp runs of 256 keys; within a
// warp keys are ranked round by round with __match_any_sync, then per-digit
// prefix sums across warps give each key's place after all keys of the same
// digit earlier in the tile.
template <bool HAS_VALS>
__global__ void __launch_bounds__(RS_BLOCK) k_rs_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                                         uint32_t *vout, uint64_t n, int shift,
                                                         const uint32_t *offsets, uint32_t ntiles) {
    __shared__ uint32_t wh[RS_WARPS][RS_RADIX];
    __shared__ uint32_t soff[RS_RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_BLOCK) (&wh[0][0])[i] = 0;
    soff[threadIdx.x] = offsets[(uint64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)warp * (RS_ROUNDS * 32);
    uint64_t key[RS_ROUNDS];
    uint32_t val[RS_ROUNDS];
    uint32_t rank[RS_ROUNDS];
    uint32_t dig[RS_ROUNDS];
    const uint32_t lt = dev::lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        uint64_t i = base + (uint64_t)r * 32 + lane;
        bool valid = i < n;
        key[r] = valid ? kin[i] : 0ull;
        if (HAS_VALS) val[r] = valid ? vin[i] : 0u;
        uint32_t d = valid ? (uint32_t)((key[r] >> shift) & 0xff) : 256u;
        dig[r] = d;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (valid) before = wh[warp][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wh[w][threadIdx.x];
            wh[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        if (dig[r] < 256u) {
            uint64_t pos = (uint64_t)soff[dig[r]] + wh[warp][dig[r]] + rank[r];
            kout[pos] = key[r];
            if (HAS_VALS) vout[pos] = val[r];
        }
    }
}
}  // namespace

gb_info radix_sort_pairs(gb_context *ctx, uint64_t *keys, uint32_t *vals, uint64_t n, int key_bits) {
    if (n <= 1 || key_bits <= 0) return GB_SUCCESS;
    if (n >= (1ull << 32)) return fail(GB_INVALID_VALUE, "radix sort: n >= 2^32");
    int passes = (key_bits + 7) / 8;
    uint32_t ntiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    uint64_t ncounts = (uint64_t)ntiles * RS_RADIX;
    Scratch k2(ctx), v2(ctx), counts(ctx);
    GB_CHECK(k2.alloc(n * sizeof(uint64_t)));
    if (vals) GB_CHECK(v2.alloc(n * sizeof(uint32_t)));
    GB_CHECK(counts.alloc(ncounts * sizeof(uint32_t)));
    uint64_t *ka = keys, *kb = k2.as<uint64_t>();
    uint32_t *va = vals, *vb = v2.as<uint32_t>();
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_BLOCK, 0, ctx->stream>>>(ka, n, shift, counts.as<uint32_t>(), ntiles);
        GB_CHECK(scan_exclusive_u32(ctx, counts.as<uint32_t>(), counts.as<uint32_t>(), ncounts, nullptr));
        if (vals)
            k_rs_scatter<true><<<ntiles, RS_BLOCK, 0, ctx->stream>>>(ka, va, kb, vb, n, shift, counts.as<uint32_t>(),
                                                                   ntiles);
        else
            k_rs_scatter<false><<<ntiles, RS_BLOCK, 0, ctx->stream>>>(ka, nullptr, kb, nullptr, n, shift,
                                                                    counts.as<uint32_t>(), ntiles);
        GB_LAUNCH_CHECK();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        GB_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
        if (vals) GB_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return GB_SUCCESS;
}

// ------------------------------------------------------------ CSR building
namespace {
__global__ void k_make_keys(const uint32_t *rows, const uint32_t *cols, uint64_t n, int cbits, uint64_t *keys,
                            uint32_t *idx) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        keys[i] = ((uint64_t)rows[i] << cbits) | cols[i];
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_check_range(const uint32_t *rows, const uint32_t *cols, uint64_t n, uint32_t nrows, uint32_t ncols,
                              uint32_t *bad) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (rows[i] >= nrows || cols[i] >= ncols)) atomicOr(bad, 1u);
}

__global__ void k_heads(const uint64_t *keys, uint64_t n, uint32_t *head) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

template <typename T>
__global__ void k_emit(const uint64_t *keys, const uint32_t *idx, const uint32_t *head, const uint32_t *pos, uint64_t n,
                       int cbits, const T *vals, gb_binop dup, uint32_t *colidx, T *ovals) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !head[i]) return;
    uint32_t p = pos[i];
    uint64_t k = keys[i];
    colidx[p] = (uint32_t)(k & ((1ull << cbits) - 1));
    if (ovals) {
        T acc = vals[idx[i]];
        for (uint64_t j = i + 1; j < n && keys[j] == k; ++j) acc = apply_binop<T>(dup, acc, vals[idx[j]]);
        ovals[p] = acc;
    }
}

__global__ void k_rowptr(const uint64_t *keys, const uint32_t *head, const uint32_t *pos, uint64_t n, int cbits,
                         uint32_t nrows, const uint32_t *total, uint32_t *rowptr) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (head[i]) {
        uint32_t r = (uint32_t)(keys[i] >> cbits);
        int64_t prev = i == 0 ? -1 : (int64_t)(keys[i - 1] >> cbits);
        for (int64_t q = prev + 1; q <= (int64_t)r; ++q) rowptr[q] = pos[i];
    }
    if (i == n - 1) {
        uint32_t r = (uint32_t)(keys[i] >> cbits);
        for (uint64_t q = (uint64_t)r + 1; q <= nrows; ++q) rowptr[q] = *total;
    }
}

inline unsigned nblk(uint64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }
}  // namespace

gb_info build_csr_from_device_tuples(gb_context *ctx, uint32_t nrows, uint32_t ncols, uint64_t ntup,
                                     const uint32_t *rows, const uint32_t *cols, const void *vals, gb_type vtype,
                                     gb_binop dup, uint32_t **rowptr_out, uint32_t **colidx_out, void **vals_out,
                                     uint64_t *nnz_out) {
    *rowptr_out = nullptr; *colidx_out = nullptr; if (vals_out) *vals_out = nullptr;
    uint32_t *rowptr = nullptr, *colidx = nullptr;
    void *ov = nullptr;
    GB_CHECK(dalloc_t(ctx, &rowptr, (size_t)nrows + 1));
    if (ntup == 0) {
        GB_CHECK(memset_async(ctx, rowptr, 0, ((size_t)nrows + 1) * sizeof(uint32_t)));
        GB_CHECK(dalloc_t(ctx, &colidx, 1));
        if (vals) GB_CHECK(dalloc(ctx, &ov, 16));
        *rowptr_out = rowptr; *colidx_out = colidx; if (vals_out) *vals_out = ov; *nnz_out = 0;
        return GB_SUCCESS;
    }
    Scratch bad(ctx);
    GB_CHECK(bad.alloc(sizeof(uint32_t)));
    GB_CHECK(memset_async(ctx, bad.p, 0, sizeof(uint32_t)));
    k_check_range<<<nblk(ntup), 256, 0, ctx->stream>>>(rows, cols, ntup, nrows, ncols, bad.as<uint32_t>());
    uint32_t hbad = 0;
    GB_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (hbad) { dfree(ctx, rowptr); return fail(GB_INVALID_INDEX, "build: an index is outside the dimensions"); }

    int cbits = bits_for(ncols), rbits = bits_for(nrows);
    if (cbits + rbits > 64) { dfree(ctx, rowptr); return fail(GB_INVALID_VALUE, "build: dimensions too large"); }
    Scratch keys(ctx), idx(ctx), head(ctx), pos(ctx), total(ctx);
    GB_CHECK(keys.alloc(ntup * sizeof(uint64_t)));
    GB_CHECK(idx.alloc(ntup * sizeof(uint32_t)));
    GB_CHECK(head.alloc(ntup * sizeof(uint32_t)));
    GB_CHECK(pos.alloc(ntup * sizeof(uint32_t)));
    GB_CHECK(total.alloc(sizeof(uint32_t)));
    k_make_keys<<<nblk(ntup), 256, 0, ctx->stream>>>(rows, cols, ntup, cbits, keys.as<uint64_t>(), idx.as<uint32_t>());
    GB_LAUNCH_CHECK();
    GB_CHECK(radix_sort_pairs(ctx, keys.as<uint64_t>(), idx.as<uint32_t>(), ntup, cbits + rbits));
    k_heads<<<nblk(ntup), 256, 0, ctx->stream>>>(keys.as<uint64_t>(), ntup, head.as<uint32_t>());
    GB_CHECK(scan_exclusive_u32(ctx, head.as<uint32_t>(), pos.as<uint32_t>(), ntup, total.as<uint32_t>()));
    uint32_t nnz = 0;
    GB_CUDA(cudaMemcpyAsync(&nnz, total.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    GB_CHECK(dalloc_t(ctx, &colidx, (size_t)nnz));
    if (vals) GB_CHECK(dalloc(ctx, &ov, (size_t)nnz * type_size(vtype) + 16));
    switch (vals ? vtype : GB_UINT32) {
#define EMIT(GT, T)                                                                                              \
    case GT:                                                                                                     \
        k_emit<T><<<nblk(ntup), 256, 0, ctx->stream>>>(keys.as<uint64_t>(), idx.as<uint32_t>(),                  \
                                                     head.as<uint32_t>(), pos.as<uint32_t>(), ntup, cbits,      \
                                                     (const T *)vals, dup, colidx, (T *)ov);                     \
        break;
        EMIT(GB_BOOL, uint8_t) EMIT(GB_INT32, int32_t) EMIT(GB_UINT32, uint32_t) EMIT(GB_UINT64, uint64_t)
        EMIT(GB_FP32, float) EMIT(GB_FP64, double)
#undef EMIT
    }
    k_rowptr<<<nblk(ntup), 256, 0, ctx->stream>>>(keys.as<uint64_t>(), head.as<uint32_t>(), pos.as<uint32_t>(), ntup,
                                                  cbits, nrows, total.as<uint32_t>(), rowptr);
    GB_LAUNCH_CHECK();
    *rowptr_out = rowptr; *colidx_out = colidx; if (vals_out) *vals_out = ov; *nnz_out = nnz;
    return GB_SUCCESS;
}

}  // namespace gbx
