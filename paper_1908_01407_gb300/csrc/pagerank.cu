// PageRank (Section 7.3), pull formulation, in FP32 with FP32 accumulation:
//   p'(i) = (1 - a)/n + a * ( sum_{j in N(i)} p(j)/deg(j) + D/n ),
// D = sum of p over vertices without edges (spread uniformly), p0 = 1/n,
// a fixed number of iterations.
//
// The SpMV y = A x (x = p/deg) splits the nonzeros, not the rows, evenly
// (Section 6.3.2 balances SpMV by merge-path; here the split is over the
// nonzeros alone, which rows of any length cross freely): every warp takes
// tiles of 512 consecutive nonzeros, each lane 4 consecutive nonzeros of each
// of the tile's four 128-nonzero sub-tiles, so a warp's column-index loads
// are one contiguous 512-byte run per sub-tile and a lane has all 16 of its
// x gathers in flight at once. A bit per nonzero marks the first entry of
// each row (computed once per call), and a per-tile prefix of those bits
// gives the rank of each row start; the k-th row start is row live[k] (the
// ascending list of nonempty rows, which the matrix keeps). Within a tile
// the rows are closed by a lane walk and a warp-level segmented scan (no
// shared memory, no block barrier); a row that crosses tile ends is
// finished by k_pr_span, which adds the tiles' partial sums.
// A separate pass applies the update p' = base + a y, x' = p'/deg and
// reduces the L1 residual sum |p' - p| and the dangling mass D (FP32 over
// 4 consecutive rows, FP64 above that) in a fixed order. Every sum has one fixed order and no floating-point atomics
// are used, so a run is bit-reproducible.
//
// The gathers x[j] are the SpMV's limit: one random 4-byte load per
// nonzero, and the L1 looks up one cache line per cycle, so a warp's
// 32 gathers to 32 lines take 32 cycles however few bytes they move. On a
// graph with a skewed degree distribution the run can instead use a copy
// of the matrix with the vertices renamed by decreasing out-degree: the
// ranks of the first 32,768 vertices, which then take about half of the
// references (52% of the nonzeros of an R-MAT graph with 4M vertices), are
// staged in shared memory by every block and gathered from there, and only
// the rest go through the L1. Staging more leaves too little L1 for the
// rest (57,344 ranks, 224 KB, ran slower than none). The ranks are renamed
// back in the final normalisation. Each warp loads its next tile's column
// indices while it gathers and sums the current one, so the DRAM latency of
// the index stream is hidden behind the gathers.
#include "common.cuh"

using namespace gbx;

namespace gbx {
namespace {

constexpr int PR_BLOCK = 256;
constexpr int PR_WARPS = PR_BLOCK / 32;
constexpr uint32_t PR_SUB = 128;               // nonzeros per sub-tile (4 per lane)
// sub-tiles per warp tile: 2, 4 or 8 (256, 512 or 1,024 nonzeros, 8, 16 or 32
// gathers in flight per lane), picked per matrix by gb_pagerank_autotune
constexpr uint32_t PR_NSUB_DEFAULT = 4;
// the kernel that stages ranks in shared memory: 1,024-thread blocks that
// share up to 224 KB of them (tiles of 256 or 512 nonzeros: within 64
// registers a thread). Fewer staged ranks leave more of the SM's 256 KB of
// L1 + shared memory to the L1 (and room for a second block).
constexpr int PR_HUB_BLOCK = 1024;
constexpr uint32_t PR_HUB_MAX = 57344;
constexpr uint32_t PR_HUB_DEFAULT = 32768;

struct TileArgs {
    uint64_t nnz;
    uint32_t ntiles;
    const uint32_t *ci;       // column indices of the pulled rows (in-edges)
    const uint32_t *flags;    // bit e: nonzero e is the first of its row
    const uint32_t *trank;    // per tile: row starts before it
    const uint32_t *live;     // k-th nonempty row (null: row k, the nonempty rows come first)
    const float *x;           // p(j)/deg(j)
    uint32_t nhub;            // x[0, nhub) is staged in shared memory (a multiple of 4; 0 = none)
    float *y;                 // row sums (rows never written stay 0)
    int *err;                 // set to GB_TIMEOUT when the staging copy did not complete in time
    float *pfirst;            // per tile: partial of the row open at its start (the whole tile without starts)
    float *plast;             // per tile with a start: partial of the row open at its end
    uint32_t *rlast;          // its rank
    uint32_t *tflag;          // 1 if the tile holds a row start
};

__device__ __forceinline__ uint32_t row_of(const TileArgs &a, uint32_t r) {
    return a.live ? __ldg(&a.live[r]) : r;
}

// bit e of flags set where nonzero e starts its row
__global__ void k_pr_flags(const uint32_t *rp, uint32_t n, uint32_t *flags) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t b = __ldg(&rp[i]);
        if (b < __ldg(&rp[i + 1])) atomicOr(&flags[b >> 5], 1u << (b & 31));
    }
}

// row starts per tile (tile / 32 flag words)
__global__ void k_pr_tilecount(const uint32_t *flags, uint32_t nwords, uint32_t ntiles, uint32_t tile, uint32_t *cnt) {
    const uint32_t tw = tile / 32;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        uint32_t c = 0;
        for (uint32_t w = t * tw; w < (t + 1) * tw && w < nwords; ++w) c += __popc(flags[w]);
        cnt[t] = c;
    }
}

template <uint32_t PR_NSUB, bool HUB>
__global__ void __launch_bounds__(HUB ? PR_HUB_BLOCK : PR_BLOCK) k_pr_tiles(TileArgs a) {
    constexpr uint32_t PR_TILE = PR_SUB * PR_NSUB;   // nonzeros per warp tile
    constexpr uint32_t WARPS = (HUB ? PR_HUB_BLOCK : PR_BLOCK) / 32;
    extern __shared__ float4 s_hub4[];
    __shared__ uint64_t s_bar;
    const float *s_hub = reinterpret_cast<const float *>(s_hub4);
    // x was written by the update kernel before this one in the stream
    dev::grid_dep_wait();
    dev::grid_dep_launch();
    if (HUB) {
        // x of the first nhub vertices, once per block: one thread hands the
        // copy to the TMA unit (cp.async.bulk into shared memory, completion
        // counted on an mbarrier) and the block waits on the barrier. x is
        // padded past n to a multiple of 4 and nhub is a multiple of 4, so
        // the copy is whole 16-byte units from a 256-byte aligned start.
        const uint32_t bytes = a.nhub * 4u;
        if (threadIdx.x == 0) {
            // x's writes (generic proxy) before the copy that reads them (async proxy)
            asm volatile("fence.proxy.async.global;" ::: "memory");
            dev::mbar_init(&s_bar, 1);
            dev::mbar_arrive_expect_tx(&s_bar, bytes);
            constexpr uint32_t CHUNK = 32768;   // bytes per bulk copy
            for (uint32_t off = 0; off < bytes; off += CHUNK)
                dev::bulk_copy_g2s(reinterpret_cast<char *>(s_hub4) + off, reinterpret_cast<const char *>(a.x) + off,
                                   bytes - off < CHUNK ? bytes - off : CHUNK, &s_bar);
        }
        __syncthreads();   // the barrier is initialised before anyone waits on it
        if (!dev::mbar_wait_bounded(&s_bar, 0, 1000000000ull)) {
            // never expected: record it, wait once more for the copy in flight,
            // then stage with plain loads so the block's result stays defined
            if (threadIdx.x == 0) atomicExch(a.err, (int)GB_TIMEOUT);
            (void)dev::mbar_wait_bounded(&s_bar, 0, 1000000000ull);
            __syncthreads();
            const float4 *x4 = reinterpret_cast<const float4 *>(a.x);
            for (uint32_t i = threadIdx.x; i < a.nhub / 4; i += blockDim.x) s_hub4[i] = __ldg(&x4[i]);
        }
        __syncthreads();
    }
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * WARPS;
    const uint4 *ci4 = reinterpret_cast<const uint4 *>(a.ci);
    // a tile's own loads: column indices, start bits and the rank of its first row start
    uint32_t col[PR_NSUB][4], fl[PR_NSUB], rank0 = 0;
    auto load_tile = [&](uint32_t tt, uint32_t (&c)[PR_NSUB][4], uint32_t (&fo)[PR_NSUB], uint32_t &r0) {
        const uint64_t b = (uint64_t)tt * PR_TILE;
#pragma unroll
        for (uint32_t k2 = 0; k2 < PR_NSUB; ++k2) {
            const uint64_t e = b + k2 * PR_SUB + 4 * lane;
            uint4 c4 = make_uint4(0, 0, 0, 0);
            uint32_t f = 0;
            if (e < a.nnz) {
                c4 = __ldcs(&ci4[e >> 2]);   // the index array is padded: a partial last chunk is readable
                f = (__ldg(&a.flags[e >> 5]) >> (e & 31)) & 0xfu;
                const uint64_t left = a.nnz - e;
                if (left < 4) f &= (1u << left) - 1u;
            }
            c[k2][0] = c4.x; c[k2][1] = c4.y; c[k2][2] = c4.z; c[k2][3] = c4.w;
            fo[k2] = f;
        }
        r0 = __ldg(&a.trank[tt]);
    };
    uint32_t t = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (t < a.ntiles) load_tile(t, col, fl, rank0);
    for (; t < a.ntiles; t += nwarps) {
        const uint64_t t0 = (uint64_t)t * PR_TILE;
        // the gathers of this tile, then the loads of the warp's next tile,
        // which stream from DRAM while the gathers and the row sums run
        float xv[PR_NSUB][4];
#pragma unroll
        for (uint32_t k2 = 0; k2 < PR_NSUB; ++k2)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t e = t0 + k2 * PR_SUB + 4 * lane + j;
                const uint32_t c = col[k2][j];
                xv[k2][j] = e >= a.nnz ? 0.f : (HUB && c < a.nhub) ? s_hub[c] : __ldg(&a.x[c]);
            }
        const uint32_t R0 = rank0;
        uint32_t R = R0;                   // rank of the next row start
        uint32_t fthis[PR_NSUB];
#pragma unroll
        for (uint32_t k2 = 0; k2 < PR_NSUB; ++k2) fthis[k2] = fl[k2];
        if (t + nwarps < a.ntiles) load_tile(t + nwarps, col, fl, rank0);
        // sub-tiles in order; the row open across them is carried warp-wide
        float carry = 0.f;                 // partial sum of the open row
        bool carry_in_tile = false;        // the open row began inside this tile
#pragma unroll
        for (uint32_t k2 = 0; k2 < PR_NSUB; ++k2) {
            const uint32_t f = fthis[k2];
            const uint32_t nf = __popc(f);
            uint32_t tot;
            const uint32_t excl = dev::warp_exclusive_sum<uint32_t>(nf, &tot);
            const uint32_t Rb = R + excl;
            // lane walk: rows that start and end inside the lane's four entries are done here
            float acc = 0.f, head = 0.f;
            bool seen = false;
            uint32_t r = Rb;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((f >> j) & 1u) {
                    if (seen) {
                        a.y[row_of(a, r)] = acc;
                        ++r;
                    } else {
                        head = acc;
                        seen = true;
                    }
                    acc = 0.f;
                }
                acc += xv[k2][j];
            }
            if (!seen) head = acc;   // no start in the lane: all of it continues the open row
            // segmented inclusive scan over lanes of (value since the lane's last start, start seen)
            float v = seen ? acc : head;
            bool rs = seen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float yv = __shfl_up_sync(full, v, o);
                const bool yr = __shfl_up_sync(full, rs ? 1 : 0, o) != 0;
                if (lane >= o && !rs) {
                    v += yv;
                    rs = yr;
                }
            }
            // what flows into this lane from earlier lanes (and from the carry when none started)
            const uint32_t starts = __ballot_sync(full, seen);
            const bool started_before = (starts & dev::lanemask_lt()) != 0u;
            float inflow = __shfl_up_sync(full, v, 1);
            if (lane == 0) inflow = 0.f;
            if (!started_before) inflow += carry;
            if (seen) {
                // the row this lane's first start closes: rank Rb - 1
                const float total = inflow + head;
                if (started_before || carry_in_tile) a.y[row_of(a, Rb - 1)] = total;
                else a.pfirst[t] = total;   // it began before the tile: finished by k_pr_span
            }
            const float last = __shfl_sync(full, v, 31);
            if (starts) {
                carry = last;
                carry_in_tile = true;
            } else {
                carry += last;
            }
            R += tot;
        }
        if (lane == 0) {
            const bool any = R != R0;
            a.tflag[t] = any ? 1u : 0u;
            if (any) {
                a.plast[t] = carry;
                a.rlast[t] = R - 1;
            } else {
                a.pfirst[t] = carry;
            }
        }
    }
}

// Rows that cross tile ends: the partial at the end of the tile t where
// the row starts, plus the partials of the following tiles up to the first
// one that holds a row start (or the last tile). The first SB blocks take
// a thread per tile and read the next SPAN_SHORT tiles' flags and partials
// at once, adding them in tile order; a row that runs on past those (a row
// of thousands of nonzeros, hundreds of tiles for the largest) is left to
// the warps of the other blocks, a warp per row from the list
// k_pr_long_spans made: each lane adds every 32nd partial after t in tile
// order, the lanes' sums are added by a fixed shuffle tree, then the
// partial of t.
constexpr uint32_t SPAN_SHORT = 8;

// has tile t a row start (t < ntiles - 1)
__device__ __forceinline__ bool tile_has_start(const uint32_t *trank, uint32_t t) {
    return __ldg(&trank[t + 1]) > __ldg(&trank[t]);
}

// once per call: (t, t2) for every row that starts in tile t and crosses
// more than SPAN_SHORT tiles after it, t2 its last tile
__global__ void k_pr_long_spans(const uint32_t *trank, uint32_t ntiles, uint2 *list, uint32_t *count) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        if ((uint64_t)t + SPAN_SHORT + 1 >= ntiles || !tile_has_start(trank, t)) continue;
        bool closed = false;
        for (uint32_t k = 1; k <= SPAN_SHORT && !closed; ++k) closed = tile_has_start(trank, t + k);
        if (closed) continue;
        uint32_t t2 = t + SPAN_SHORT + 1;
        while (t2 < ntiles - 1 && !tile_has_start(trank, t2)) ++t2;
        list[atomicAdd(count, 1u)] = make_uint2(t, t2);
    }
}

__global__ void __launch_bounds__(PR_BLOCK) k_pr_span(TileArgs a, uint32_t short_blocks, const uint2 *long_list,
                                                     const uint32_t *long_count) {
    dev::grid_dep_wait();   // the partial sums of the SpMV kernel before it
    dev::grid_dep_launch();
    if (blockIdx.x < short_blocks) {
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < a.ntiles; t += short_blocks * blockDim.x) {
            if (!a.tflag[t]) continue;
            uint32_t f[SPAN_SHORT];
            float pf[SPAN_SHORT];
#pragma unroll
            for (uint32_t k = 0; k < SPAN_SHORT; ++k) {
                const bool in = (uint64_t)t + 1 + k < a.ntiles;
                f[k] = in ? a.tflag[t + 1 + k] : 1u;
                pf[k] = in ? a.pfirst[t + 1 + k] : 0.f;
            }
            float total = a.plast[t];
            bool done = false;
#pragma unroll
            for (uint32_t k = 0; k < SPAN_SHORT; ++k) {
                if (done) break;
                if ((uint64_t)t + 1 + k < a.ntiles) total += pf[k];
                done = f[k] != 0u;
            }
            if (!done && (uint64_t)t + SPAN_SHORT + 1 < a.ntiles) continue;   // a long row
            a.y[row_of(a, a.rlast[t])] = total;
        }
        return;
    }
    const uint32_t nlong = *long_count;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t w0 = (blockIdx.x - short_blocks) * PR_WARPS + (threadIdx.x >> 5);
    const uint32_t nw = (gridDim.x - short_blocks) * PR_WARPS;
    for (uint32_t e = w0; e < nlong; e += nw) {
        const uint2 sp = long_list[e];
        float acc = 0.f;
        for (uint32_t k = sp.x + 1 + lane; k <= sp.y; k += 32) acc += a.pfirst[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) a.y[row_of(a, a.rlast[sp.x])] = a.plast[sp.x] + acc;
    }
}

struct UpdArgs {
    uint32_t n;
    const float *y, *p_old;
    float *p_new, *x_new;
    const uint32_t *rp_out;   // out-degrees
    const float *base;        // device scalar: (1-a)/n + a*D/n
    float alpha;
    double *part_res, *part_dang;
    uint32_t *done;           // blocks finished (the last one reduces, then resets it)
    double *residual_out;     // this iteration's residual
    float *base_out;          // the next iteration's base term (read by every block first)
};

// One block of PR_BLOCK threads: the FP64 partials in a fixed order -> the
// residual, the dangling mass D and the next base term (1-a)/n + a D/n.
__device__ void reduce_parts(uint32_t n, float alpha, const double *part_res, const double *part_dang,
                             uint32_t nparts, double *residual_out, float *base_out, double (*s)[PR_BLOCK]) {
    double r0 = 0, r1 = 0;
    for (uint32_t b = threadIdx.x; b < nparts; b += PR_BLOCK) {
        r0 += __ldcg(&part_res[b]);
        r1 += __ldcg(&part_dang[b]);
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
        const double nn = (double)n;
        *base_out = (float)((1.0 - (double)alpha) / nn + (double)alpha * s[1][0] / nn);
    }
}

// p' = base + a y, x' = p'/deg; partial sums of |p' - p| and of the
// dangling p' (FP32 over 4 consecutive rows, FP64 above that), each block
// over a fixed contiguous range of rows. The block
// that finishes last adds the partials up (reduce_parts): the order of that
// sum does not depend on which block it is.
__global__ void __launch_bounds__(PR_BLOCK) k_pr_update(UpdArgs a) {
    __shared__ double s_red[2][PR_WARPS];
    __shared__ double s_fin[2][PR_BLOCK];
    __shared__ bool s_last;
    // each block a range of a multiple of 4 rows; each thread takes 4
    // consecutive rows per group with 16-byte loads and stores (the vectors
    // and the row offsets start 256-byte aligned), and loads G groups
    // before it computes any
    constexpr int G = 2;
    dev::grid_dep_wait();   // y of the SpMV and span kernels before it
    dev::grid_dep_launch();
    const uint64_t per = (((uint64_t)a.n + gridDim.x - 1) / gridDim.x + 3) & ~3ull;
    const uint64_t b0 = per * blockIdx.x < a.n ? per * blockIdx.x : a.n;
    const uint64_t b1 = b0 + per < a.n ? b0 + per : a.n;
    const float base = *a.base;
    double res = 0.0, dang = 0.0;
    for (uint64_t i0 = b0 + 4 * threadIdx.x; i0 < b1; i0 += 4 * PR_BLOCK * G) {
        float yv[G][4], po[G][4];
        uint32_t rp[G][5];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint64_t i = i0 + (uint64_t)g * 4 * PR_BLOCK;
            if (i + 4 <= b1) {
                const float4 y4 = __ldg(reinterpret_cast<const float4 *>(a.y + i));
                const float4 o4 = __ldg(reinterpret_cast<const float4 *>(a.p_old + i));
                const uint4 r4 = __ldg(reinterpret_cast<const uint4 *>(a.rp_out + i));
                yv[g][0] = y4.x; yv[g][1] = y4.y; yv[g][2] = y4.z; yv[g][3] = y4.w;
                po[g][0] = o4.x; po[g][1] = o4.y; po[g][2] = o4.z; po[g][3] = o4.w;
                rp[g][0] = r4.x; rp[g][1] = r4.y; rp[g][2] = r4.z; rp[g][3] = r4.w;
                rp[g][4] = __ldg(&a.rp_out[i + 4]);
            } else {
                // a ragged end: rows past b1 read nothing; rp[j] is row i+j's
                // offset for every j up to the row count (b1 <= n, so i+j <= n)
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const bool in = i + j < b1;
                    if (j < 4) {
                        yv[g][j] = in ? __ldg(&a.y[i + j]) : 0.f;
                        po[g][j] = in ? __ldg(&a.p_old[i + j]) : 0.f;
                    }
                    rp[g][j] = i + j <= b1 ? __ldg(&a.rp_out[i + j]) : 0u;
                }
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint64_t i = i0 + (uint64_t)g * 4 * PR_BLOCK;
            float pn[4], xn[4];
            // the group's 4 terms in FP32, the group sums in FP64 (FP64 is
            // slow on this part: one FP64 add per group, not per row)
            float rg = 0.f, dg = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t deg = rp[g][j + 1] - rp[g][j];
                const float p = base + a.alpha * yv[g][j];
                pn[j] = p;
                xn[j] = deg ? p / (float)deg : 0.f;
                if (i + j < b1) {
                    rg += fabsf(p - po[g][j]);
                    if (!deg) dg += p;
                }
            }
            res += (double)rg;
            dang += (double)dg;
            if (i + 4 <= b1) {
                *reinterpret_cast<float4 *>(a.p_new + i) = make_float4(pn[0], pn[1], pn[2], pn[3]);
                *reinterpret_cast<float4 *>(a.x_new + i) = make_float4(xn[0], xn[1], xn[2], xn[3]);
            } else {
                for (int j = 0; j < 4 && i + j < b1; ++j) {
                    a.p_new[i + j] = pn[j];
                    a.x_new[i + j] = xn[j];
                }
            }
        }
    }
    res = dev::warp_sum<double>(res);
    dang = dev::warp_sum<double>(dang);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_red[0][warp] = res; s_red[1][warp] = dang; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0, r1 = 0;
        for (int w = 0; w < PR_WARPS; ++w) { r0 += s_red[0][w]; r1 += s_red[1][w]; }
        a.part_res[blockIdx.x] = r0;
        a.part_dang[blockIdx.x] = r1;
        __threadfence();
        s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    reduce_parts(a.n, a.alpha, a.part_res, a.part_dang, gridDim.x, a.residual_out, a.base_out, s_fin);
    if (threadIdx.x == 0) *a.done = 0u;
}

// One block: reduce_parts of the initial dangling mass
__global__ void __launch_bounds__(PR_BLOCK) k_pr_reduce(uint32_t n, float alpha, const double *part_res,
                                                       const double *part_dang, uint32_t nparts,
                                                       double *residual_out, float *base_out) {
    __shared__ double s[2][PR_BLOCK];
    reduce_parts(n, alpha, part_res, part_dang, nparts, residual_out, base_out, s);
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

// out[v] = p[new_id[v]] / S (new_id null: the identity)
__global__ void __launch_bounds__(PR_BLOCK) k_pr_norm(uint32_t n, const float *p, const double *part, uint32_t nparts,
                                                     const uint32_t *new_id, float *out) {
    __shared__ double s_tot;
    if (threadIdx.x == 0) {
        double t = 0;
        for (uint32_t b = 0; b < nparts; ++b) t += part[b];
        s_tot = t;
    }
    __syncthreads();
    const double inv = 1.0 / s_tot;
    for (uint32_t i = blockIdx.x * PR_BLOCK + threadIdx.x; i < n; i += gridDim.x * PR_BLOCK)
        out[i] = (float)((double)p[new_id ? __ldg(&new_id[i]) : i] * inv);
}

}  // namespace
}  // namespace gbx

// tile kernel with nsub sub-tiles per warp tile (2, 4 or 8), staging ranks in
// shared memory or not (nsub 2 or 4 there)
static const void *tiles_kernel(uint32_t nsub, bool hub) {
    if (hub) return nsub == 2 ? (const void *)k_pr_tiles<2, true> : (const void *)k_pr_tiles<4, true>;
    return nsub == 2 ? (const void *)k_pr_tiles<2, false>
                     : nsub == 8 ? (const void *)k_pr_tiles<8, false> : (const void *)k_pr_tiles<4, false>;
}

// The copy of A with vertices renamed by decreasing out-degree (ties by
// lower id), built on first use and kept on A with the renaming.
static gb_info pagerank_view(const gb_matrix *Ac) {
    gb_matrix *A = const_cast<gb_matrix *>(Ac);
    std::lock_guard<std::mutex> lock(A->cache_mu);
    if (A->pr_view) return GB_SUCCESS;
    gb_context *ctx = A->ctx;
    gb_matrix *B = nullptr;
    uint32_t *nid = nullptr;
    GB_CHECK(gb_matrix_new(&B, ctx, A->type, A->nrows, A->ncols));
    gb_info r = dalloc_t(ctx, &nid, (size_t)A->nrows + 1);
    if (r == GB_SUCCESS) r = gb_matrix_degree_order(B, A, nid, GB_DEVICE);
    if (r != GB_SUCCESS) {
        gb_matrix_free(&B);
        dfree(ctx, nid);
        return r;
    }
    // the copy serves PageRank alone: the BFS pull records are not kept
    dfree(ctx, B->live_rec);
    B->live_rec = nullptr;
    A->pr_view = B;
    A->pr_new_id = nid;
    return GB_SUCCESS;
}

// Launches kernel k on the context stream with programmatic stream
// serialization: its blocks may be scheduled while the kernel before it
// drains (k calls dev::grid_dep_wait before reading that kernel's output),
// which hides most of the launch gap between the three kernels of an
// iteration. Not while the context shares the GPU (a capped context, as in
// the serving loop): blocks placed early wait on the SMs, holding slots that
// concurrent jobs could run in.
static gb_info launch_overlapped(gb_context *ctx, const void *k, dim3 grid, dim3 block, size_t smem, void **args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = ctx->grid_limit > 0 ? 0 : 1;
    GB_CUDA(cudaLaunchKernelExC(&cfg, k, args));
    return GB_SUCCESS;
}

// One PageRank of `iters` iterations with warp tiles of nsub sub-tiles, on A
// as stored (order 0) or on its degree-ordered copy with staged ranks (1).
static gb_info pagerank_run(gb_context *ctx, const gb_matrix *A, float damping, uint32_t iters, float *rank,
                            double *residuals, gb_mem mem, uint32_t nsub, int order, uint32_t staged) {
    if (!ctx || !A || !rank) return fail(GB_NULL_POINTER, "gb_pagerank: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_pagerank: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_pagerank: matrix must be square");
    if (!A->has_csc) return fail(GB_INVALID_VALUE, "gb_pagerank: needs the CSC copy (in-edges)");
    if (!A->live_list) return fail(GB_INVALID_VALUE, "gb_pagerank: the matrix has no list of nonempty rows");
    if (!(damping >= 0.f && damping <= 1.f)) return fail(GB_INVALID_VALUE, "gb_pagerank: damping must be in [0, 1]");
    const uint32_t n = A->nrows;
    if (n == 0) return GB_SUCCESS;
    GB_CUDA(cudaSetDevice(ctx->device));
    const gb_matrix *M = A;               // the matrix the iterations run on
    const uint32_t *new_id = nullptr;     // its renaming of A's vertices
    if (order) {
        GB_CHECK(pagerank_view(A));
        M = A->pr_view;
        new_id = A->pr_new_id;
    }
    const uint64_t m = M->nvals;
    if (nsub != 2 && nsub != 8) nsub = 4;
    const bool hub = order != 0;
    if (hub && nsub == 8) nsub = 4;
    const uint32_t tile = PR_SUB * nsub;
    const uint32_t ntiles = (uint32_t)((m + tile - 1) / tile);
    const uint32_t nfw = (uint32_t)((m + 31) / 32);
    // x is padded to n + 4 floats, so nhub rounded up to a multiple of 4 stays inside it
    if (staged == 0 || staged > PR_HUB_MAX) staged = PR_HUB_DEFAULT;
    const uint32_t nhub = hub ? (((n + 3u) & ~3u) < staged ? ((n + 3u) & ~3u) : staged) : 0u;
    const int block = hub ? PR_HUB_BLOCK : PR_BLOCK;
    const size_t smem = (size_t)nhub * 4;
    const void *kern = tiles_kernel(nsub, hub);
    if (hub) GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(PR_HUB_MAX * 4)));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem));
    // a plain (not cooperative) launch: it needs no co-residency, so it takes the
    // whole GPU even where a context's persistent kernels are capped, and the
    // hardware interleaves its blocks with those of concurrent work
    uint32_t G = (uint32_t)(occ > 0 ? occ : 1) * (uint32_t)ctx->num_sms;
    const uint32_t wpb = (uint32_t)block / 32;
    const uint32_t need = (ntiles + wpb - 1) / wpb;
    if (G > need) G = need > 0 ? need : 1;
    // blocks of the update pass (fixed: the reduction order does not depend on
    // the GPU). Its cost is mostly per block (the FP64 partial sums and the
    // completion count): on R-MAT s22, 512 blocks took 24.9 us, 1,024 took
    // 30.6, 2,048 took 39.5, and 256 to 608 took 25-27.
    const uint32_t UB = 512;
    // blocks of the final normalisation's FP64 sum (its partials share pres)
    const uint32_t NB = 1024;
    Scratch p0(ctx), p1(ctx), x0(ctx), x1(ctx), yb(ctx), fl(ctx), tr(ctx), pf(ctx), pl(ctx), rl(ctx), tf(ctx),
        pres(ctx), pdang(ctx), scal(ctx), resid(ctx), outb(ctx), lsp(ctx);
    GB_CHECK(p0.alloc((size_t)n * 4 + 16));
    GB_CHECK(p1.alloc((size_t)n * 4 + 16));
    GB_CHECK(x0.alloc((size_t)n * 4 + 16));
    GB_CHECK(x1.alloc((size_t)n * 4 + 16));
    GB_CHECK(yb.alloc((size_t)n * 4 + 16));
    GB_CHECK(fl.alloc((size_t)nfw * 4 + 64));
    GB_CHECK(tr.alloc((size_t)ntiles * 4 + 16));
    GB_CHECK(pf.alloc((size_t)ntiles * 4 + 16));
    GB_CHECK(pl.alloc((size_t)ntiles * 4 + 16));
    GB_CHECK(rl.alloc((size_t)ntiles * 4 + 16));
    GB_CHECK(tf.alloc((size_t)ntiles * 4 + 16));
    // each long row takes more than SPAN_SHORT tiles of its own
    GB_CHECK(lsp.alloc(((size_t)ntiles / SPAN_SHORT + 1) * sizeof(uint2)));
    GB_CHECK(pres.alloc((size_t)(UB > NB ? UB : NB) * 8));
    GB_CHECK(pdang.alloc((size_t)UB * 8));
    GB_CHECK(scal.alloc(64));
    GB_CHECK(resid.alloc(((size_t)iters + 1) * 8));
    float *out = rank;
    if (mem == GB_HOST) { GB_CHECK(outb.alloc((size_t)n * 4 + 16)); out = outb.as<float>(); }
    float *base = reinterpret_cast<float *>(scal.as<char>() + 16);
    uint32_t *done = reinterpret_cast<uint32_t *>(scal.as<char>() + 32);
    uint32_t *nlong = reinterpret_cast<uint32_t *>(scal.as<char>() + 48);
    // once per call: the row-start bits, their per-tile prefix, zero row sums
    // (rows without in-edges are never written and keep y = 0), and zero x
    // padding (staged with the ranks, never gathered)
    GB_CHECK(memset_async(ctx, fl.p, 0, (size_t)nfw * 4 + 64));
    GB_CHECK(memset_async(ctx, yb.p, 0, (size_t)n * 4 + 16));
    GB_CHECK(memset_async(ctx, x0.p, 0, (size_t)n * 4 + 16));
    GB_CHECK(memset_async(ctx, x1.p, 0, (size_t)n * 4 + 16));
    GB_CHECK(memset_async(ctx, scal.p, 0, 64));
    k_pr_flags<<<1024, PR_BLOCK, 0, ctx->stream>>>(M->colptr, n, fl.as<uint32_t>());
    if (ntiles) {
        k_pr_tilecount<<<(ntiles + PR_BLOCK - 1) / PR_BLOCK < 4096 ? (ntiles + PR_BLOCK - 1) / PR_BLOCK : 4096,
                         PR_BLOCK, 0, ctx->stream>>>(fl.as<uint32_t>(), nfw, ntiles, tile, tr.as<uint32_t>());
        GB_LAUNCH_CHECK();
        GB_CHECK(scan_exclusive_u32(ctx, tr.as<uint32_t>(), tr.as<uint32_t>(), ntiles, nullptr));
        k_pr_long_spans<<<(ntiles + PR_BLOCK - 1) / PR_BLOCK < 1024 ? (ntiles + PR_BLOCK - 1) / PR_BLOCK : 1024,
                          PR_BLOCK, 0, ctx->stream>>>(tr.as<uint32_t>(), ntiles, lsp.as<uint2>(), nlong);
        GB_LAUNCH_CHECK();
    }
    // init: p0, x0, D0 -> base
    k_pr_init<<<UB, PR_BLOCK, 0, ctx->stream>>>(n, M->rowptr, p0.as<float>(), x0.as<float>(), pdang.as<double>(),
                                             pres.as<double>());
    k_pr_reduce<<<1, PR_BLOCK, 0, ctx->stream>>>(n, damping, pres.as<double>(), pdang.as<double>(), UB, nullptr, base);
    GB_LAUNCH_CHECK();
    TileArgs ta;
    ta.nnz = m;
    ta.ntiles = ntiles;
    ta.ci = M->rowidx;
    ta.flags = fl.as<uint32_t>();
    ta.trank = tr.as<uint32_t>();
    // in the degree-ordered copy of a symmetric matrix the vertices with
    // edges come first, so the k-th nonempty row is row k
    ta.live = (order && M->csc_alias) ? nullptr : M->live_list;
    ta.nhub = nhub;
    ta.err = reinterpret_cast<int *>(scal.as<char>());   // bytes 0-3 of the scalar block
    ta.y = yb.as<float>();
    ta.pfirst = pf.as<float>();
    ta.plast = pl.as<float>();
    ta.rlast = rl.as<uint32_t>();
    ta.tflag = tf.as<uint32_t>();
    UpdArgs ua;
    ua.n = n;
    ua.y = yb.as<float>();
    ua.rp_out = M->rowptr;
    ua.base = base;
    ua.alpha = damping;
    ua.part_res = pres.as<double>();
    ua.part_dang = pdang.as<double>();
    ua.done = done;
    ua.base_out = base;
    const uint32_t SB = (ntiles + PR_BLOCK - 1) / PR_BLOCK < 1024 ? (ntiles + PR_BLOCK - 1) / PR_BLOCK : 1024;
    const uint32_t LB = 256;   // blocks for the long rows (a warp each)
    float *pc = p0.as<float>(), *pn = p1.as<float>(), *xc = x0.as<float>(), *xn = x1.as<float>();
    for (uint32_t it = 0; it < iters; ++it) {
        ta.x = xc;
        ua.p_old = pc; ua.p_new = pn; ua.x_new = xn;
        ua.residual_out = resid.as<double>() + it;
        if (ntiles) {
            int span = prof_begin(ctx, "pagerank_spmv");
            void *args[] = {&ta};
            GB_CHECK(launch_overlapped(ctx, kern, dim3(G), dim3(block), smem, args));
            prof_end(ctx, span);
            int sspan = prof_begin(ctx, "pagerank_span");
            const uint2 *lsp_p = lsp.as<uint2>();
            void *sargs[] = {&ta, (void *)&SB, (void *)&lsp_p, (void *)&nlong};
            GB_CHECK(launch_overlapped(ctx, (const void *)k_pr_span, dim3(SB + LB), dim3(PR_BLOCK), 0, sargs));
            prof_end(ctx, sspan);
        }
        int span = prof_begin(ctx, "pagerank_update");
        void *uargs[] = {&ua};
        GB_CHECK(launch_overlapped(ctx, (const void *)k_pr_update, dim3(UB), dim3(PR_BLOCK), 0, uargs));
        prof_end(ctx, span);
        GB_LAUNCH_CHECK();
        float *t = pc; pc = pn; pn = t;
        t = xc; xc = xn; xn = t;
    }
    // final normalisation in FP64, back to A's vertex names
    k_pr_sum<<<NB, PR_BLOCK, 0, ctx->stream>>>(n, pc, pres.as<double>());
    k_pr_norm<<<NB, PR_BLOCK, 0, ctx->stream>>>(n, pc, pres.as<double>(), NB, new_id, out);
    GB_LAUNCH_CHECK();
    if (residuals && iters) GB_CUDA(cudaMemcpyAsync(residuals, resid.p, (size_t)iters * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (mem == GB_HOST) GB_CUDA(cudaMemcpyAsync(rank, out, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    int herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, scal.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (herr) return fail(GB_TIMEOUT, "gb_pagerank: a bounded wait for a shared-memory staging copy ran out");
    return GB_SUCCESS;
}

extern "C" gb_info gb_pagerank(gb_context *ctx, const gb_matrix *A, float damping, uint32_t iters, float *rank,
                               double *residuals, gb_mem mem) {
    if (!A) return fail(GB_NULL_POINTER, "gb_pagerank: NULL argument");
    return pagerank_run(ctx, A, damping, iters, rank, residuals, mem,
                        A->tuned_pr_nsub ? A->tuned_pr_nsub : PR_NSUB_DEFAULT, A->pr_order, A->pr_staged);
}

extern "C" gb_info gb_pagerank_autotune(gb_context *ctx, gb_matrix *A, uint32_t *tile_nnz, int32_t *degree_order,
                                        uint32_t *staged_ranks, double *ms_per_iteration) {
    if (!ctx || !A || !tile_nnz) return fail(GB_NULL_POINTER, "gb_pagerank_autotune: NULL argument");
    if (!A->built || A->nrows != A->ncols || !A->has_csc)
        return fail(GB_INVALID_VALUE, "gb_pagerank_autotune: needs a built square matrix with its CSC");
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch out(ctx);
    GB_CHECK(out.alloc((size_t)A->nrows * 4 + 16));
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    // (sub-tiles, order, staged ranks): the tiles as stored, and on the
    // degree-ordered copy the tiles that fit the staged-rank kernel's
    // register budget with 16,384 and 32,768 staged ranks (64 or 128 KB:
    // the larger sets leave too little L1 for the other gathers)
    static const uint32_t cand_nsub[] = {2, 4, 8, 2, 4, 2, 4};
    static const int cand_order[] = {0, 0, 0, 1, 1, 1, 1};
    static const uint32_t cand_staged[] = {0, 0, 0, 16384, 16384, 32768, 32768};
    constexpr int NC = 7;
    constexpr uint32_t ITERS = 8;
    double best = 1e30;
    int bc = 1;
    gb_info r = GB_SUCCESS;
    // two passes over the candidates (forward, then backward), each keeping its faster pass
    double tmin[NC];
    for (int c = 0; c < NC; ++c) tmin[c] = 1e30;
    for (int pass = 0; pass < 2 && r == GB_SUCCESS; ++pass) {
        for (int ci = 0; ci < NC && r == GB_SUCCESS; ++ci) {
            const int c = pass == 0 ? ci : NC - 1 - ci;
            r = pagerank_run(ctx, A, 0.85f, 2, out.as<float>(), nullptr, GB_DEVICE, cand_nsub[c], cand_order[c],
                                 cand_staged[c]);   // warm
            if (r == GB_SUCCESS && cudaEventRecord(e0, ctx->stream) != cudaSuccess) r = GB_PANIC;
            if (r == GB_SUCCESS)
                r = pagerank_run(ctx, A, 0.85f, ITERS, out.as<float>(), nullptr, GB_DEVICE, cand_nsub[c], cand_order[c],
                                 cand_staged[c]);
            if (r == GB_SUCCESS && cudaEventRecord(e1, ctx->stream) != cudaSuccess) r = GB_PANIC;
            if (r == GB_SUCCESS && cudaEventSynchronize(e1) != cudaSuccess) r = GB_PANIC;
            float ms = 0;
            if (r == GB_SUCCESS) cudaEventElapsedTime(&ms, e0, e1);
            if (ms < tmin[c]) tmin[c] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GB_SUCCESS) return r == GB_PANIC ? fail(GB_PANIC, "gb_pagerank_autotune: CUDA error") : r;
    for (int c = 0; c < NC; ++c)
        if (tmin[c] < best) { best = tmin[c]; bc = c; }
    A->tuned_pr_nsub = cand_nsub[bc];
    A->pr_order = cand_order[bc];
    A->pr_staged = cand_staged[bc];
    if (!A->pr_order && A->pr_view) {   // the copy is not used: give its memory back
        std::lock_guard<std::mutex> lock(A->cache_mu);
        gb_matrix_free(&A->pr_view);
        dfree(ctx, A->pr_new_id);
        A->pr_new_id = nullptr;
    }
    *tile_nnz = cand_nsub[bc] * PR_SUB;
    if (degree_order) *degree_order = cand_order[bc];
    if (staged_ranks) *staged_ranks = cand_order[bc] ? cand_staged[bc] : 0u;
    if (ms_per_iteration) *ms_per_iteration = best / ITERS;
    return GB_SUCCESS;
}

extern "C" gb_info gb_pagerank_set_tile(gb_matrix *A, uint32_t tile_nnz) {
    if (!A) return fail(GB_NULL_POINTER, "gb_pagerank_set_tile: NULL matrix");
    if (tile_nnz != 0 && tile_nnz != 2 * PR_SUB && tile_nnz != 4 * PR_SUB && tile_nnz != 8 * PR_SUB)
        return fail(GB_INVALID_VALUE, "gb_pagerank_set_tile: tile of %u nonzeros (256, 512, 1024 or 0)", tile_nnz);
    A->tuned_pr_nsub = tile_nnz / PR_SUB;
    return GB_SUCCESS;
}

extern "C" gb_info gb_pagerank_set_order(gb_matrix *A, int32_t degree_order, uint32_t staged_ranks) {
    if (!A) return fail(GB_NULL_POINTER, "gb_pagerank_set_order: NULL matrix");
    if (degree_order != 0 && degree_order != 1)
        return fail(GB_INVALID_VALUE, "gb_pagerank_set_order: %d (0 = as stored, 1 = degree order)", (int)degree_order);
    if (staged_ranks % 1024 != 0 || staged_ranks > PR_HUB_MAX)
        return fail(GB_INVALID_VALUE, "gb_pagerank_set_order: %u staged ranks (a multiple of 1,024 up to %u, 0 = default)",
                    staged_ranks, PR_HUB_MAX);
    A->pr_order = degree_order;
    A->pr_staged = staged_ranks;
    return GB_SUCCESS;
}
