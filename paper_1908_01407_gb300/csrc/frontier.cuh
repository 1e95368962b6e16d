// Frontier machinery shared by the traversal kernels (BFS, SSSP, connected
// components): the list form of a frontier with exclusive out-degree
// prefixes and row starts, appended through one packed 64-bit atomicAdd per
// block tile; a merge-path push over the list's edges; the bitmap -> list
// compaction used when a push follows a pull.
#pragma once
#include "common.cuh"

// Threads per block of the kernels that use this machinery: 256 unless the
// including file sets GBX_FRONTIER_BLOCK before it includes this header
// (the BFS kernel runs 512). Everything here has internal linkage, so each
// file gets its own instance at its own block size.
#ifndef GBX_FRONTIER_BLOCK
#define GBX_FRONTIER_BLOCK 256
#endif

namespace gbx {
namespace fr {
namespace {

constexpr int BLOCK = GBX_FRONTIER_BLOCK;
constexpr int WARPS = BLOCK / 32;
static_assert(BLOCK % 32 == 0 && BLOCK >= 64 && BLOCK <= 1024, "block size");
constexpr int PUSH_ITEMS = 4;
constexpr int PUSH_TILE = BLOCK * PUSH_ITEMS;      // edges per block tile
constexpr int PUSH_OWNERS = PUSH_TILE + 1;          // owner entries staged in smem
constexpr int PULL_WPW = 2;                          // pull candidates per lane in flight
constexpr int PULL_ROUNDS = 2;                       // 16-byte chunks a lane checks alone

struct SmemPush {
    uint32_t P[PUSH_OWNERS];
    uint32_t Q[PUSH_OWNERS];
    uint32_t R[PUSH_OWNERS];
    uint32_t k0, nk;
};
// Per-tile staging of newly discovered vertices: each warp collects up to
// STAGE_CAP (vertex, out-degree) pairs, then one atomicAdd per block tile
// reserves list slots and edge-prefix space for all of them.
constexpr int STAGE_CAP = 128;
static_assert(PUSH_ITEMS * 32 <= STAGE_CAP && PULL_WPW * 32 <= STAGE_CAP, "staging capacity");
struct Stage {
    uint32_t v[WARPS][STAGE_CAP];
    uint32_t deg[WARPS][STAGE_CAP];
    uint32_t r0[WARPS][STAGE_CAP];   // row start (rp_out[v]), loaded with the degree
    uint32_t wcnt[WARPS];
    uint32_t wdeg[WARPS];
    unsigned long long base;
};
// Per-warp queue of pull candidates whose row head had no frontier vertex:
// they are scanned 32 at a time (one per lane), so a long row delays only
// the misses batched with it, not every candidate of its group.
constexpr int MISS_CAP = 96;   // fewer than 32 left over + a group of at most 64
struct MissQueue {
    uint32_t v[WARPS][MISS_CAP];     // vertex
    uint32_t c[WARPS][MISS_CAP];     // candidate (the entry a later pull walks)
    uint32_t len[WARPS][MISS_CAP];   // in-degree
    uint32_t deg[WARPS][MISS_CAP];   // out-degree
};
struct Smem {
    union {
        SmemPush push;      // push levels
        MissQueue miss;     // pull levels
    };
    Stage stage;
    unsigned long long qs;
    unsigned long long ue;   // in-edges of the last pull's leftover candidates
    unsigned int uc;         // their number
};

static __device__ __forceinline__ uint32_t ldcg(const uint32_t *p) { return __ldcg(p); }
// Loads of data a traversal streams through once (adjacency, the live
// table): evict-first in L1 and L2, so the 0.5 GB of column indices does not
// push the small working set out of L2 (bitmaps, frontier lists, and the
// levels/parents lines whose sectors fill up over a traversal).
template <class T>
static __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
static __device__ __forceinline__ int ld_relaxed_gpu_int_(const int *p) { return dev::ld_relaxed_gpu_int(p); }

// largest k in [0, cnt) with P[k] <= e (P[0] == 0 <= e)
static __device__ __forceinline__ uint32_t owner_search_global(const uint32_t *P, uint32_t cnt, uint64_t e) {
    uint32_t lo = 0, hi = cnt;  // invariant: P[lo] <= e, answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)ldcg(&P[mid]) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// warp-level: add this lane's discovery (if win) to the warp's staging row
static __device__ __forceinline__ void stage_add(Stage &sg, uint32_t &staged, uint32_t &wdeg, bool win, uint32_t v,
                                          uint32_t deg, uint32_t r0) {
    const uint32_t full = 0xffffffffu;
    const int warp = threadIdx.x >> 5;
    uint32_t wm = __ballot_sync(full, win);
    if (!wm) return;
    if (win) {
        uint32_t idx = staged + __popc(wm & dev::lanemask_lt());
        sg.v[warp][idx] = v;
        sg.deg[warp][idx] = deg;
        sg.r0[warp][idx] = r0;
    }
    staged += __popc(wm);
    wdeg += dev::warp_sum<uint32_t>(win ? deg : 0u);
}

// block-level (every thread calls it): append all staged discoveries to the
// next list with one atomicAdd on the packed (count, edge-sum) word
template <class Args>
__device__ void stage_flush(const Args &a, Stage &sg, int slot_next, uint32_t *Qn, uint32_t *Pn, uint32_t *Rn,
                            uint32_t staged, uint32_t wdeg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sg.wcnt[warp] = staged;
        sg.wdeg[warp] = wdeg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t cacc = 0, sacc = 0;
        for (int w = 0; w < WARPS; ++w) {
            uint32_t cw = sg.wcnt[w], sw = sg.wdeg[w];
            sg.wcnt[w] = cacc;
            sg.wdeg[w] = sacc;
            cacc += cw;
            sacc += sw;
        }
        unsigned long long base = 0;
        if (cacc) base = atomicAdd(&a.st->qstate[slot_next], ((unsigned long long)cacc << a.ebits) | sacc);
        sg.base = base;
    }
    __syncthreads();
    if (staged) {
        unsigned long long base = sg.base;
        uint32_t pos = (uint32_t)(base >> a.ebits) + sg.wcnt[warp];
        uint32_t pre = (uint32_t)(base & a.emask) + sg.wdeg[warp];
        for (uint32_t c0 = 0; c0 < staged; c0 += 32) {
            uint32_t idx = c0 + lane;
            uint32_t dg = idx < staged ? sg.deg[warp][idx] : 0u;
            uint32_t tot;
            uint32_t ex = dev::warp_exclusive_sum<uint32_t>(dg, &tot);
            if (idx < staged) {
                uint32_t v = sg.v[warp][idx];
                Qn[pos + idx] = v;
                Pn[pos + idx] = pre + ex;
                Rn[pos + idx] = sg.r0[warp][idx];
            }
            pre += tot;
        }
    }
    __syncthreads();
}

// Cooperative search by the whole block: the largest k in [0, cnt) with
// P[k] <= x (P is non-decreasing and P[0] = 0). Each round probes BLOCK
// evenly spaced positions in parallel, so a list of 4M entries needs three
// rounds of one load per thread instead of a 22-step dependent chain.
static __device__ uint32_t block_owner_search(const uint32_t *P, uint32_t cnt, uint64_t x) {
    uint32_t lo = 0, hi = cnt;   // answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t span = hi - lo;
        uint32_t step = (span + BLOCK - 1) / BLOCK;
        uint32_t idx = lo + threadIdx.x * step;
        int ok = (idx < hi) && (uint64_t)ldcg(&P[idx]) <= x;
        int c = __syncthreads_count(ok);      // probes 0..c-1 satisfy (monotone)
        uint32_t nlo = lo + (uint32_t)(c - 1) * step;
        uint32_t nhi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Push: every block takes an equal, contiguous share of the frontier's
// edges (merge-path split over the edge prefixes), stages the owning
// vertices of a tile (prefix, id, row start) in shared memory and maps each
// edge to its owner by binary search there. visit(u, v, p, Fn, &deg) handles
// the edge u -> v stored at position p and returns whether v joins the next
// frontier for the first time (then with its out-degree in deg and its row
// start in r0).
template <class Args, class Visit>
__device__ void push_edges(const Args &a, Smem &sm, int d, uint32_t cnt, uint64_t fe, Visit visit) {
    const int cur = d & 1, nxt = (d + 1) & 1;
    const int slot_next = (d + 1) % 3;
    const uint32_t *Q = a.q[cur];
    const uint32_t *P = a.qp[cur];
    const uint32_t *R = a.qr[cur];
    uint32_t *Qn = a.q[nxt];
    uint32_t *Pn = a.qp[nxt];
    uint32_t *Rn = a.qr[nxt];
    uint32_t *Fn = a.front[(d + 1) % 3];
    const uint64_t Eb0 = fe * blockIdx.x / gridDim.x;
    const uint64_t Eb1 = fe * (blockIdx.x + 1) / gridDim.x;
    if (Eb0 >= Eb1) return;
    uint32_t k = block_owner_search(P, cnt, Eb0);
    uint64_t E = Eb0;
    while (E < Eb1) {
        const uint32_t W = cnt - k < (uint32_t)(PUSH_OWNERS - 1) ? cnt - k : (uint32_t)(PUSH_OWNERS - 1);
        for (uint32_t j = threadIdx.x; j <= W; j += BLOCK) {
            if (j < W) {
                sm.push.Q[j] = ldcg(&Q[k + j]);
                sm.push.P[j] = ldcg(&P[k + j]);
                sm.push.R[j] = ldcg(&R[k + j]);
            } else {
                sm.push.P[j] = k + W < cnt ? ldcg(&P[k + W]) : (uint32_t)fe;   // end of the staged owners' edges
            }
        }
        __syncthreads();
        uint64_t Eend = E + PUSH_TILE;
        if (Eend > Eb1) Eend = Eb1;
        if (Eend > sm.push.P[W]) Eend = sm.push.P[W];
        if (Eend <= E) {          // every staged owner has no out-edges: skip them
            __syncthreads();
            k += W;
            continue;
        }
        uint32_t staged = 0, wdeg = 0;
#pragma unroll
        for (int it = 0; it < PUSH_ITEMS; ++it) {
            uint64_t e = E + (uint64_t)it * BLOCK + threadIdx.x;
            bool win = false;
            uint32_t v = 0, deg = 0, r0 = 0;
            if (e < Eend) {
                uint32_t lo = 0, hi = W;
                while (hi - lo > 1) {
                    uint32_t mid = (lo + hi) >> 1;
                    if ((uint64_t)sm.push.P[mid] <= e) lo = mid; else hi = mid;
                }
                uint32_t u = sm.push.Q[lo];
                uint32_t p = sm.push.R[lo] + (uint32_t)(e - sm.push.P[lo]);
                v = ld_stream(&a.ci_out[p]);
                win = visit(u, v, p, Fn, &deg, &r0);
            }
            stage_add(sm.stage, staged, wdeg, win, v, deg, r0);
        }
        // the owner of the next tile's first edge
        uint32_t knext = k + W;
        if (Eend < sm.push.P[W]) {
            uint32_t lo = 0, hi = W;
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if ((uint64_t)sm.push.P[mid] <= Eend) lo = mid; else hi = mid;
            }
            knext = k + lo;
        }
        stage_flush(a, sm.stage, slot_next, Qn, Pn, Rn, staged, wdeg);
        k = knext;
        E = Eend;
    }
}

// Builds the frontier list (with out-degree prefixes) of level d from its
// bitmap, for a push that follows a pull. Each block compacts a contiguous
// range of words; one atomicAdd per 256-word chunk on the packed
// (count, edge-sum) word places the chunk in the list.
template <class Args>
__device__ void compact_level(const Args &a, Smem &sm, int d) {
    const uint32_t *F = a.front[d % 3];
    uint32_t *Q = a.q[d & 1];
    uint32_t *P = a.qp[d & 1];
    uint32_t *R = a.qr[d & 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t wb0 = (uint64_t)a.nwords * blockIdx.x / gridDim.x;
    const uint64_t wb1 = (uint64_t)a.nwords * (blockIdx.x + 1) / gridDim.x;
    for (uint64_t c = wb0; c < wb1; c += BLOCK) {
        const uint64_t word = c + threadIdx.x;
        uint32_t bits = word < wb1 ? ldcg(&F[word]) : 0u;
        uint32_t cntv = __popc(bits), degv = 0;
        for (uint32_t bb = bits; bb; bb &= bb - 1) {
            uint32_t v = (uint32_t)(word * 32 + (__ffs(bb) - 1));
            degv += __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
        }
        uint32_t tc, td;
        uint32_t ec = dev::warp_exclusive_sum<uint32_t>(cntv, &tc);
        uint32_t ed = dev::warp_exclusive_sum<uint32_t>(degv, &td);
        if (lane == 0) {
            sm.stage.wcnt[warp] = tc;
            sm.stage.wdeg[warp] = td;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t cacc = 0, sacc = 0;
            for (int w = 0; w < WARPS; ++w) {
                uint32_t cw = sm.stage.wcnt[w], sw = sm.stage.wdeg[w];
                sm.stage.wcnt[w] = cacc;
                sm.stage.wdeg[w] = sacc;
                cacc += cw;
                sacc += sw;
            }
            unsigned long long base = 0;
            if (cacc) base = atomicAdd(&a.st->cstate[d % 3], ((unsigned long long)cacc << a.ebits) | sacc);
            sm.stage.base = base;
        }
        __syncthreads();
        uint32_t pos = (uint32_t)(sm.stage.base >> a.ebits) + sm.stage.wcnt[warp] + ec;
        uint32_t pre = (uint32_t)(sm.stage.base & a.emask) + sm.stage.wdeg[warp] + ed;
        for (uint32_t bb = bits; bb; bb &= bb - 1) {
            uint32_t v = (uint32_t)(word * 32 + (__ffs(bb) - 1));
            uint32_t r0 = __ldg(&a.rp_out[v]);
            Q[pos] = v;
            P[pos] = pre;
            R[pos] = r0;
            pre += __ldg(&a.rp_out[v + 1]) - r0;
            ++pos;
        }
        __syncthreads();
    }
}


}  // namespace
}  // namespace fr
}  // namespace gbx
