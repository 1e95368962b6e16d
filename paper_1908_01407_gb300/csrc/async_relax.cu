// Barrier-free relaxation for graphs of high diameter: the asynchronous
// execution model that Section 9 names as future work for the road-network
// gap of Section 8 (road_usa and rgg, where a level-synchronous traversal
// pays one device-wide synchronisation per level over thousands of levels).
//
// The fixed points are the ones of the level-synchronous kernels:
//  * SSSP (min.plus):  dist(v) = min over in-edges (u,v) of dist(u) + w(u,v),
//    dist(src) = 0 (Section 7.2);
//  * BFS (unit weights): level(v) = min over (u,v) of level(u) + 1, with a
//    parent taken afterwards among the in-neighbours one level up;
//  * CC (min.second):  label(v) = min over (u,v) of label(u), labels
//    starting at the vertex ids (Section 7.4's reading of config 3).
// Each is the least solution of monotone min-updates, so any order of
// applying them that applies every improvement reaches it exactly: the
// result is independent of the schedule and bit-identical to Dijkstra /
// queue BFS / union-find.
//
// Schedule. One persistent launch. Work items are (value, vertex) entries
// in a ring of 64-bit slots. A warp owns fixed 32-slot chunks of the ring
// (chunk g, g + W, g + 2W, ... for warp g of W), so taking work needs no
// shared counter: a lane polls its slot until a producer has filled it. A
// producer reserves slots with one atomicAdd on the ring's tail per warp
// round. An entry whose value is no longer its vertex's value is stale and
// skipped (the later improvement has an entry of its own). A warp keeps up to
// 32 of its own new entries as its next batch instead of publishing them, so
// most hops of a long path cost no ring round trip; what does not fit goes
// to the ring, where idle warps pick it up.
// Termination without a barrier: done counts retired ring entries, tail the
// reserved ones; a warp retires what it took only once it holds no local
// entries, so done == tail (done read with acquire first) means nothing is
// in flight and nothing can be produced again.
// Near-far (SSSP): improvements at or beyond a bound go to a far bitmap
// instead of the ring; when the ring is quiescent, one grid barrier, the
// bound grows by delta and the far vertices below it are published. That is
// one barrier pair per distance bucket instead of one per hop.
// Every wait is bounded: a wait that runs out sets GB_TIMEOUT and every warp
// leaves.
#include <cstdlib>

#include "common.cuh"
#include "types.cuh"

using namespace gbx;

namespace gbx {
namespace arx {

constexpr int ABLOCK = 256;
constexpr int AWARPS = ABLOCK / 32;
constexpr unsigned long long EMPTY = ~0ull;
constexpr int KS = 4;                  // edges a lane relaxes per round of a short row
constexpr uint32_t SHORT_MAX = 16;     // rows up to this length are relaxed by one lane

enum { K_SSSP = 0, K_BFS = 1, K_CC = 2 };

struct AState {
    dev::GridBarrier bar;
    int err;
    unsigned int far_cnt;              // vertices with their far bit set
    unsigned int far_min;              // smallest value among them (set at each phase end)
    unsigned int pad0;
    unsigned long long tail;           // ring slots reserved
    unsigned long long done;           // ring entries retired
    unsigned long long items, stale, edges, updates;
    unsigned int phases, pad;
    unsigned long long t_begin, t_end;
    unsigned int reached, maxlev;      // BFS: vertices reached, largest level (the parent pass)
};

struct AArgs {
    const uint32_t *rp, *ci, *w;       // out-edges (CSR) and, for SSSP, their weights
    uint32_t n, nwords;
    uint32_t src;
    uint32_t *val;                     // dist / level / label
    uint32_t *far;                     // SSSP near-far: improved at or beyond the bound
    unsigned long long *ring;
    unsigned long long mask;           // ring slots - 1 (a power of two, >= 32 * warps)
    uint64_t delta;                    // bucket width; 0 = one phase (no bound)
    int local;                         // keep a warp's own new entries as its next batch
    AState *st;
    uint64_t wait_ns;                  // bound on one wait for a free ring slot
    uint64_t total_limit_ns;           // bound on the whole traversal
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long pack(uint32_t value, uint32_t v) {
    return ((unsigned long long)value << 32) | v;
}

template <int KIND>
__device__ __forceinline__ uint32_t cand(uint32_t d, const uint32_t *w, uint32_t p) {
    if (KIND == K_SSSP) return sat_add<uint32_t>(d, __ldcs(&w[p]));
    if (KIND == K_BFS) return d + 1u;
    return d;
}

struct Counts {
    unsigned long long items = 0, stale = 0, edges = 0, updates = 0;
};

// The warp's view of where its new entries go.
struct WarpOut {
    unsigned long long *loc;   // this warp's local batch (32 entries, shared memory)
    uint32_t nloc;             // entries in it (uniform across the warp)
};

// Marks v far (its improvement lies at or beyond the bound).
__device__ __forceinline__ void mark_far(const AArgs &a, uint32_t v) {
    const uint32_t bit = 1u << (v & 31);
    if (!(atomicOr(&a.far[v >> 5], bit) & bit)) atomicAdd(&a.st->far_cnt, 1u);
}

// Writes entry e to ring slot s once the slot is free (its previous entry
// taken); the wait is bounded and sets GB_TIMEOUT when it runs out.
__device__ __forceinline__ void ring_put(const AArgs &a, unsigned long long s, unsigned long long e) {
    unsigned long long *p = &a.ring[s & a.mask];
    if (ld_relaxed_u64(p) != EMPTY) {
        const uint64_t t0 = dev::globaltimer_ns();
        while (ld_relaxed_u64(p) != EMPTY) {
            if (dev::globaltimer_ns() - t0 > a.wait_ns) {
                atomicCAS(&a.st->err, 0, (int)GB_TIMEOUT);
                return;
            }
        }
    }
    st_release_u64(p, e);
}

// Publishes the entries (c[k], u[k]) whose ok[k] is set, warp-collectively:
// the first ones fill the warp's local batch, the rest go to the ring.
template <int K>
__device__ __forceinline__ void emit(const AArgs &a, WarpOut &wo, const bool (&ok)[K], const uint32_t (&u)[K],
                                     const uint32_t (&c)[K]) {
    const int lane = threadIdx.x & 31;
    uint32_t np = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) np += ok[k] ? 1u : 0u;
    uint32_t tot;
    uint32_t r = dev::warp_exclusive_sum<uint32_t>(np, &tot);
    if (tot == 0) return;
    const uint32_t room = a.local ? 32u - wo.nloc : 0u;
    const uint32_t nring = tot > room ? tot - room : 0u;
    unsigned long long base = 0;
    if (nring && lane == 0) base = atomicAdd(&a.st->tail, (unsigned long long)nring);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!ok[k]) continue;
        const unsigned long long e = pack(c[k], u[k]);
        if (r < room) wo.loc[wo.nloc + r] = e;
        else ring_put(a, base + (r - room), e);
        ++r;
    }
    wo.nloc += tot < room ? tot : room;
    __syncwarp();
}

// Relaxes the out-edges of the entries the lanes hold (e == EMPTY: none).
template <int KIND>
__device__ void relax_entries(const AArgs &a, unsigned long long e, uint64_t bound, WarpOut &wo, Counts &cn) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    bool act = e != EMPTY;
    const uint32_t v = (uint32_t)e, d = (uint32_t)(e >> 32);
    uint32_t b = 0, len = 0;
    if (act) {
        // the value check and the row bounds load together (one dependent step
        // per hop fewer; a stale entry wastes two row-pointer reads)
        const uint32_t cur = __ldcg(&a.val[v]);
        b = __ldg(&a.rp[v]);
        len = __ldg(&a.rp[v + 1]) - b;
        if (cur < d) {   // a later improvement of v has an entry of its own
            act = false;
            len = 0;
            cn.stale++;
        } else {
            cn.items++;
            cn.edges += len;
        }
    }
    // short rows: each lane its own row, KS edges per round, every load of a
    // round independent of the others
    const bool sh = act && len <= SHORT_MAX;
    const uint32_t mlen = __reduce_max_sync(full, sh ? len : 0u);
    for (uint32_t j0 = 0; j0 < mlen; j0 += KS) {
        bool ok[KS];
        uint32_t u[KS], c[KS];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            ok[k] = sh && j0 + k < len;
            u[k] = 0;
            c[k] = 0;
            if (ok[k]) {
                u[k] = __ldcs(&a.ci[b + j0 + k]);
                c[k] = cand<KIND>(d, a.w, b + j0 + k);
            }
        }
#pragma unroll
        for (int k = 0; k < KS; ++k)
            if (ok[k]) ok[k] = c[k] < __ldcg(&a.val[u[k]]);
#pragma unroll
        for (int k = 0; k < KS; ++k)
            if (ok[k]) ok[k] = c[k] < atomicMin(&a.val[u[k]], c[k]);
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            if (!ok[k]) continue;
            cn.updates++;
            if (KIND != K_BFS && a.delta && (uint64_t)c[k] >= bound) {
                mark_far(a, u[k]);
                ok[k] = false;
            }
        }
        emit<KS>(a, wo, ok, u, c);
    }
    // long rows: the whole warp, 32 edges per round
    uint32_t coop = __ballot_sync(full, act && len > SHORT_MAX);
    while (coop) {
        const int l = __ffs(coop) - 1;
        coop &= coop - 1;
        const uint32_t pb = __shfl_sync(full, b, l), pl = __shfl_sync(full, len, l), pd = __shfl_sync(full, d, l);
        for (uint32_t j0 = 0; j0 < pl; j0 += 32) {
            bool ok[1];
            uint32_t u[1], c[1];
            ok[0] = j0 + lane < pl;
            u[0] = 0;
            c[0] = 0;
            if (ok[0]) {
                u[0] = __ldcs(&a.ci[pb + j0 + lane]);
                c[0] = cand<KIND>(pd, a.w, pb + j0 + lane);
                ok[0] = c[0] < __ldcg(&a.val[u[0]]) && c[0] < atomicMin(&a.val[u[0]], c[0]);
                if (ok[0]) {
                    cn.updates++;
                    if (KIND != K_BFS && a.delta && (uint64_t)c[0] >= bound) {
                        mark_far(a, u[0]);
                        ok[0] = false;
                    }
                }
            }
            emit<1>(a, wo, ok, u, c);
        }
    }
}

// Works until the ring is quiescent (or an error is set). start_slot is a
// multiple of 32: the first chunk of this phase.
template <int KIND>
__device__ void consume(const AArgs &a, uint64_t bound, unsigned long long start_slot, unsigned long long *loc,
                        Counts &cn, uint64_t t_start) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long W = (unsigned long long)gridDim.x * AWARPS;
    const unsigned long long g = (unsigned long long)blockIdx.x * AWARPS + (threadIdx.x >> 5);
    AState *st = a.st;
    unsigned long long chunk = start_slot / 32 + g;
    uint32_t pend = full;          // lanes of the chunk whose slot is still to be taken
    unsigned long long taken = 0;  // ring entries taken and not yet retired
    WarpOut wo{loc, 0};
    uint32_t idle = 0;
    for (;;) {
        unsigned long long e = EMPTY;
        if (wo.nloc) {
            if ((uint32_t)lane < wo.nloc) e = loc[lane];
            wo.nloc = 0;
            __syncwarp();
        } else {
            // each lane polls its own slot (no shared word is polled while
            // work is pending, so the tail's line stays free for producers)
            const unsigned long long s = chunk * 32 + lane;
            if ((pend >> lane) & 1u) {
                unsigned long long *p = &a.ring[s & a.mask];
                e = ld_acquire_u64(p);
                if (e != EMPTY) st_relaxed_u64(p, EMPTY);
            }
            const uint32_t gm = __ballot_sync(full, e != EMPTY);
            pend &= ~gm;
            taken += __popc(gm);
            if (pend == 0) {
                chunk += W;
                pend = full;
            }
        }
        if (__any_sync(full, e != EMPTY)) {
            relax_entries<KIND>(a, e, bound, wo, cn);
            idle = 0;
            continue;
        }
        // nothing to do: retire what was taken, then test for quiescence
        if (taken) {
            if (lane == 0) red_release_add_u64(&st->done, taken);
            taken = 0;
        }
        // the quiescence test reads two shared words: every 4th idle round
        int stop = 0;
        if (lane == 0 && (idle & 3u) == 0) {
            const unsigned long long dn = ld_acquire_u64(&st->done);
            const unsigned long long tl = ld_relaxed_u64(&st->tail);
            stop = dn == tl || dev::ld_relaxed_gpu_int(&st->err) != 0;
            if (!stop && (idle & 63u) == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns) {
                atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
                stop = 1;
            }
        }
        if (__shfl_sync(full, stop, 0)) break;
        ++idle;
        __nanosleep(idle < 16 ? 64u : (idle < 64 ? 256u : 1024u));
    }
}

template <int KIND>
__global__ void __launch_bounds__(ABLOCK, 4) k_async(AArgs a) {
    __shared__ unsigned long long s_loc[AWARPS][32];
    __shared__ int s_flag;
    AState *st = a.st;
    const uint64_t nth = (uint64_t)gridDim.x * ABLOCK;
    const uint64_t tid = (uint64_t)blockIdx.x * ABLOCK + threadIdx.x;
    // start: values, far bitmap, ring. Components: every vertex is an entry
    // (label = id); with label buckets the vertices whose id is at or beyond
    // the first bound start in the far set instead.
    const uint64_t ncc = KIND == K_CC ? (a.delta && a.delta < a.n ? a.delta : (uint64_t)a.n) : 0;
    for (uint64_t i = tid; i < a.n; i += nth)
        a.val[i] = KIND == K_CC ? (uint32_t)i : (i == a.src ? 0u : UINT32_MAX);
    if (a.far)
        for (uint64_t w = tid; w < a.nwords; w += nth) {
            uint32_t f = 0u;
            if (KIND == K_CC) {   // bits of the ids in [ncc, n)
                const uint64_t lo = w * 32, hi = lo + 32;
                for (uint64_t v = lo < ncc ? ncc : lo; v < hi && v < a.n; ++v) f |= 1u << (v - lo);
            }
            a.far[w] = f;
        }
    for (uint64_t s = tid; s <= a.mask; s += nth) {
        unsigned long long e = EMPTY;
        if (KIND == K_CC) {
            if (s < ncc) e = pack((uint32_t)s, (uint32_t)s);
        } else if (s == 0) {
            e = pack(0u, a.src);
        }
        a.ring[s] = e;
    }
    if (tid == 0) {
        st->tail = KIND == K_CC ? ncc : 1ull;
        st->done = 0;
        st->far_min = UINT32_MAX;
        st->far_cnt = KIND == K_CC ? (unsigned int)(a.n - ncc) : 0u;
    }
    bool ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.wait_ns);
    const uint64_t t_start = dev::globaltimer_ns();
    if (tid == 0) st->t_begin = t_start;
    Counts cn;
    uint64_t bound = a.delta ? a.delta : ~0ull;
    unsigned long long start_slot = 0;
    unsigned int phases = 0;
    while (ok) {
        ++phases;
        consume<KIND>(a, bound, start_slot, s_loc[threadIdx.x >> 5], cn, t_start);
        if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.total_limit_ns)) { ok = false; break; }
        if (!a.delta) break;
        // quiescent: no entry is in flight, far_cnt is stable
        if (threadIdx.x == 0) s_flag = (int)dev::ld_relaxed_gpu(&st->far_cnt);
        __syncthreads();
        const bool far_left = s_flag != 0;
        __syncthreads();
        if (!far_left) break;
        // the next phase starts on a fresh chunk: slots between the tail and
        // the next multiple of 32 stay empty and count as retired
        // (shared state and the far bitmap are read and written in L2 only:
        // atomics updated them there, and this SM's L1 may still hold lines
        // from an earlier phase)
        // Every thread takes the phase's first slot from the tail now, while
        // nothing can change it (after the next barrier the far vertices are
        // published through it): all warps then agree on who owns which chunk.
        start_slot = (ld_relaxed_u64(&st->tail) + 31ull) & ~31ull;
        if (tid == 0) {
            st_relaxed_u64(&st->tail, start_slot);
            st_relaxed_u64(&st->done, start_slot);
            if (dev::globaltimer_ns() - t_start > a.total_limit_ns) atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
        }
        // the smallest far value decides the next bucket
        uint32_t fmin = UINT32_MAX;
        for (uint64_t w = tid; w < a.nwords; w += nth)
            for (uint32_t bb = __ldcg(&a.far[w]); bb; bb &= bb - 1) {
                const uint32_t x = __ldcg(&a.val[(uint32_t)(w * 32 + (__ffs(bb) - 1))]);
                fmin = x < fmin ? x : fmin;
            }
        fmin = __reduce_min_sync(0xffffffffu, fmin);
        if ((threadIdx.x & 31) == 0 && fmin != UINT32_MAX) atomicMin(&st->far_min, fmin);
        if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.wait_ns)) { ok = false; break; }
        const uint64_t fm = dev::ld_relaxed_gpu(&st->far_min);
        const uint64_t next = (fm / a.delta + 1) * a.delta;
        bound = next > bound + a.delta ? next : bound + a.delta;
        // publish the far vertices below the new bound
        uint32_t moved = 0;
        for (uint64_t w0 = tid - (threadIdx.x & 31); w0 < a.nwords; w0 += nth) {
            const uint64_t w = w0 + (threadIdx.x & 31);
            const uint32_t bits = w < a.nwords ? __ldcg(&a.far[w]) : 0u;
            uint32_t take = 0;
            for (uint32_t bb = bits; bb; bb &= bb - 1) {
                const uint32_t v = (uint32_t)(w * 32 + (__ffs(bb) - 1));
                if ((uint64_t)__ldcg(&a.val[v]) < bound) take |= bb & (~bb + 1u);
            }
            const uint32_t cnt = __popc(take);
            uint32_t tot;
            uint32_t r = dev::warp_exclusive_sum<uint32_t>(cnt, &tot);
            if (tot == 0) continue;
            unsigned long long base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(&st->tail, (unsigned long long)tot);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (take) {
                __stcg(&a.far[w], bits & ~take);
                for (uint32_t bb = take; bb; bb &= bb - 1) {
                    const uint32_t v = (uint32_t)(w * 32 + (__ffs(bb) - 1));
                    ring_put(a, base + r, pack(__ldcg(&a.val[v]), v));
                    ++r;
                }
            }
            moved += cnt;
        }
        moved = dev::warp_sum<uint32_t>(moved);
        if ((threadIdx.x & 31) == 0 && moved) atomicSub(&st->far_cnt, moved);
        if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.wait_ns)) { ok = false; break; }
        // far_min is read again only after the next phase's quiescence barrier
        if (tid == 0) atomicExch(&st->far_min, UINT32_MAX);
    }
    // statistics
    unsigned long long v4[4] = {cn.items, cn.stale, cn.edges, cn.updates};
#pragma unroll
    for (int k = 0; k < 4; ++k) v4[k] = dev::warp_sum<unsigned long long>(v4[k]);
    if ((threadIdx.x & 31) == 0) {
        if (v4[0]) atomicAdd(&st->items, v4[0]);
        if (v4[1]) atomicAdd(&st->stale, v4[1]);
        if (v4[2]) atomicAdd(&st->edges, v4[2]);
        if (v4[3]) atomicAdd(&st->updates, v4[3]);
    }
    if (tid == 0) {
        st->phases = phases;
        st->t_end = dev::globaltimer_ns();
    }
}

// BFS parents after the levels: for every reached u and out-edge (u, v)
// with level(v) = level(u) + 1, parent(v) = the smallest such u (any of them
// is a valid BFS-tree parent; the smallest makes the output deterministic).
// A thread per vertex; rows longer than 32 are walked by the whole warp.
// Also counts the vertices reached and the largest level (par == null: the
// count only).
__global__ void k_async_parents(const uint32_t *rp, const uint32_t *ci, uint32_t n, const uint32_t *lv,
                                uint32_t *par, uint32_t src, AState *st) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    uint32_t reached = 0, maxlev = 0;
    for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); u0 < n; u0 += nth) {
        const uint64_t u = u0 + lane;
        uint32_t lu = UINT32_MAX, b = 0, e = 0;
        if (u < n) {
            lu = __ldcg(&lv[u]);
            if (lu != UINT32_MAX) {
                ++reached;
                maxlev = lu > maxlev ? lu : maxlev;
                if (par) {
                    b = __ldg(&rp[u]);
                    e = __ldg(&rp[u + 1]);
                }
            }
            if (par && u == src) par[u] = src;
        }
        if (e - b <= 32) {
            for (uint32_t p = b; p < e; ++p) {
                const uint32_t v = __ldcs(&ci[p]);
                if (v != src && __ldcg(&lv[v]) == lu + 1u) atomicMin(&par[v], (uint32_t)u);
            }
        }
        uint32_t todo = __ballot_sync(full, e - b > 32);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t pb = __shfl_sync(full, b, l), pe = __shfl_sync(full, e, l);
            const uint32_t pl = __shfl_sync(full, lu, l);
            const uint32_t pu = (uint32_t)(u0 + l);
            for (uint32_t p = pb + lane; p < pe; p += 32) {
                const uint32_t v = __ldcs(&ci[p]);
                if (v != src && __ldcg(&lv[v]) == pl + 1u) atomicMin(&par[v], pu);
            }
        }
    }
    reached = dev::warp_sum<uint32_t>(reached);
    maxlev = __reduce_max_sync(full, maxlev);
    if (lane == 0) {
        if (reached) atomicAdd(&st->reached, reached);
        atomicMax(&st->maxlev, maxlev);
    }
}

}  // namespace arx

// Runs the barrier-free relaxation of `kind` (0 SSSP, 1 BFS, 2 CC) on A into
// the device array out (n values). delta = SSSP bucket width (0 = none).
// parents (BFS, device, may be null). Fills stats when given.
gb_info async_relax_run(gb_context *ctx, const gb_matrix *A, int kind, uint32_t src, uint32_t *out,
                        uint32_t *parents, uint64_t delta, gb_bfs_stats *stats, const char *who) {
    using namespace arx;
    const uint32_t n = A->nrows;
    AArgs a;
    a.rp = A->rowptr;
    a.ci = A->colidx;
    a.w = kind == K_SSSP ? (const uint32_t *)A->vals : nullptr;
    a.n = n;
    a.nwords = (n + 31) / 32;
    a.src = src;
    a.val = out;
    a.delta = kind == K_BFS ? 0 : delta;
    a.local = 1;
    a.wait_ns = 4000000000ull;
    a.total_limit_ns = 60000000000ull;
    // failure-path test: GBX_TEST_ASYNC_LIMIT_US bounds the whole traversal by
    // that many microseconds (1 us .. 1 s), so its bounded waits run out
    if (const char *e = getenv("GBX_TEST_ASYNC_LIMIT_US")) {
        long long us = atoll(e);
        if (us > 0) {
            if (us > 1000000) us = 1000000;
            a.total_limit_ns = (uint64_t)us * 1000ull;
        }
    }
    const void *fn = kind == K_SSSP ? (const void *)k_async<K_SSSP>
                     : kind == K_BFS ? (const void *)k_async<K_BFS> : (const void *)k_async<K_CC>;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, ABLOCK, 0));
    if (occ < 1) return fail(GB_PANIC, "%s: kernel cannot be resident", who);
    int grid = occ * ctx->num_sms;
    if (ctx->grid_limit > 0 && ctx->grid_limit < grid) grid = ctx->grid_limit;
    const unsigned long long warps = (unsigned long long)grid * AWARPS;
    // ring: a power of two of at least 2 n (4 n for components, which start
    // with every vertex as an entry) plus two chunks per warp
    unsigned long long slots = 1ull << 16;
    while (slots < (kind == K_CC ? 4ull : 2ull) * n + 64ull * warps) slots <<= 1;
    a.mask = slots - 1;
    Scratch ring(ctx), far(ctx), stb(ctx);
    GB_CHECK(ring.alloc(slots * 8));
    a.ring = ring.as<unsigned long long>();
    a.far = nullptr;
    if (a.delta) {
        GB_CHECK(far.alloc((size_t)a.nwords * 4 + 16));
        a.far = far.as<uint32_t>();
    }
    GB_CHECK(stb.alloc(sizeof(AState)));
    GB_CHECK(memset_async(ctx, stb.p, 0, sizeof(AState)));
    a.st = stb.as<AState>();
    void *args[] = {&a};
    int span = prof_begin(ctx, who);
    GB_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(ABLOCK), args, 0, ctx->stream));
    GB_LAUNCH_CHECK();
    if (kind == K_BFS && (parents || stats)) {
        if (parents) GB_CUDA(cudaMemsetAsync(parents, 0xff, (size_t)n * 4, ctx->stream));
        k_async_parents<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(A->rowptr, A->colidx, n, out, parents, src,
                                                                   a.st);
        GB_LAUNCH_CHECK();
    }
    prof_end(ctx, span);
    AState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, a.st, sizeof(AState), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->depth = kind == K_BFS ? hs.maxlev + 1 : hs.phases;
        stats->push_levels = hs.phases;
        stats->status = (uint32_t)hs.err;
        stats->vertices_reached = kind == K_BFS ? hs.reached : hs.items;
        stats->edges_examined = hs.edges;
        stats->frontier_edges = hs.edges;
        // 4 n value writes; per vertex relaxed 8 (row bounds) + 4 (its value);
        // per edge 4 (index), + 4 (weight) for SSSP; 4 per improved value;
        // 8 per entry read from the ring (stale ones included)
        const double ew = kind == K_SSSP ? 8.0 : 4.0;
        stats->alg_bytes = (uint64_t)(4.0 * n + 12.0 * hs.items + ew * hs.edges + 4.0 * hs.updates +
                                      8.0 * (hs.items + hs.stale));
        stats->trace_len = 0;
        stats->init_us = 0;
        stats->final_us = (float)((hs.t_end - hs.t_begin) * 1e-3);
        stats->schedule = GB_SCHED_ASYNC;
    }
    if (hs.err) return fail(GB_TIMEOUT, "%s: a bounded device wait or the time budget ran out", who);
    return GB_SUCCESS;
}

}  // namespace gbx
