// BFS for graphs of high diameter (long chains of small frontiers, e.g.
// road networks and grids, where Section 8's measurements show a
// level-synchronous traversal spending its time in per-level overhead):
// the whole traversal runs inside ONE thread-block cluster. Its CTAs are
// co-scheduled by the hardware, so levels are separated by the cluster
// barrier instead of a grid-wide one, and the frontier stays in the CTAs'
// shared memory:
//  * level d: the frontier is the concatenation of the CTAs' lists (read
//    through distributed shared memory) and a global overflow list; item i
//    goes to CTA i mod (cluster size), so the work is balanced whichever
//    CTA discovered the vertices. Each vertex is expanded by push, claiming
//    unvisited neighbours with atomicOr on the visited bitmap (the mask is
//    tested before the write); a CTA appends what it claims to its own next
//    list, and past the list's capacity to the global overflow list;
//  * rows longer than HEAVY are queued and expanded warp-cooperatively;
//  * the next frontier's size is summed into CTA 0's shared memory with
//    distributed-shared-memory atomics, read by every CTA after the barrier.
// Levels and parents are those of Algorithm 1 (levels 0-based, -1 for
// unreached vertices), exactly as the persistent-grid kernel writes them.
// The same frontier machinery runs SSSP (Section 7.2) as min.plus
// relaxation: an edge (u, v, w) lowers dist(v) to dist(u) + w (saturating)
// by atomicMin, and v joins the next frontier the first time it improves in
// an iteration (an iteration stamp per vertex); the loop ends when no
// distance changes, the exact fixed point.
#include <cooperative_groups.h>

#include "common.cuh"
#include "bfs_common.cuh"

namespace cg = cooperative_groups;
using namespace gbx;

namespace gbx {
namespace clk {

constexpr int CT = 1024;              // threads per CTA
constexpr uint32_t CAP = 5120;        // frontier entries per CTA and buffer (shared memory)
constexpr uint32_t HEAVY = 32;        // rows longer than this are expanded by a whole warp
constexpr uint32_t HCAP = 1024;       // heavy-row queue per CTA (shared memory)

struct ClState {
    unsigned int ov_cnt[3];   // overflow list length, per level slot
    int err;
    unsigned int depth;
    unsigned int pad;
    unsigned long long reached;
    unsigned long long edges;      // frontier out-edges expanded
    unsigned long long t_begin, t_end;
};

struct ClArgs {
    uint32_t n, nwords;
    uint32_t src;
    const uint32_t *rp, *ci;       // CSR (out-edges)
    int32_t *levels, *parents;
    uint32_t *visited;             // BFS
    uint32_t *dist;                // SSSP: distances (UINT32_MAX = unreached)
    const uint32_t *wt;            // SSSP: edge weights, CSR order
    uint32_t *stamp;               // SSSP: last iteration + 1 in which a vertex joined a frontier
    uint32_t *ov[2];               // overflow frontier lists, n entries each
    ClState *st;
    uint64_t total_limit_ns;
    int *err_sticky;               // optional: a timeout is also max-ed in here (batched runs)
};

struct ClSmem {
    uint32_t list[2][CAP];
    uint32_t heavy[HCAP];
    unsigned int cnt[2];           // claims this CTA made for the next list
    unsigned int nheavy;
    unsigned int tot[3];           // (CTA 0) next-frontier size per level slot, summed over the cluster
    unsigned int stop;             // (CTA 0) 1 = leave after this level (timeout)
    unsigned int pre[17];          // exclusive prefix of the CTAs' list lengths at this level
    unsigned long long edges;
};

// claim v from u at level d: the first atomicOr on v's visited bit wins
__device__ __forceinline__ bool claim(const ClArgs &a, uint32_t u, uint32_t v, int d) {
    const uint32_t bit = 1u << (v & 31);
    if (atomicOr(&a.visited[v >> 5], bit) & bit) return false;
    a.levels[v] = d + 1;
    if (a.parents) a.parents[v] = (int32_t)u;
    return true;
}

__device__ __forceinline__ uint32_t sat_add(uint32_t x, uint32_t w) {
    const uint32_t r = x + w;
    return r < x ? 0xffffffffu : r;
}

template <bool SSSP>
__global__ void __launch_bounds__(CT, 1) k_cluster(ClArgs a) {
    extern __shared__ __align__(16) unsigned char cl_smem_raw[];
    ClSmem &s = *reinterpret_cast<ClSmem *>(cl_smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const unsigned int rank = cl.block_rank(), ncta = cl.num_blocks();
    const uint32_t gtid = rank * CT + threadIdx.x, gthreads = ncta * CT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ClState *st = a.st;
    ClSmem *s0 = cl.map_shared_rank(&s, 0);   // CTA 0's copy: cluster-wide counters
    // ---- init: visited bits (vertices past n are marked visited), the source
    if (SSSP) {
        for (uint32_t i = gtid; i < a.n; i += gthreads) {
            a.dist[i] = i == a.src ? 0u : 0xffffffffu;
            a.stamp[i] = 0u;
        }
    } else {
        const uint32_t tail = (a.n & 31) ? ~((1u << (a.n & 31)) - 1u) : 0u;
        for (uint32_t w = gtid; w < a.nwords; w += gthreads) {
            uint32_t vis = (w == a.nwords - 1) ? tail : 0u;
            if (w == (a.src >> 5)) vis |= 1u << (a.src & 31);
            a.visited[w] = vis;
        }
    }
    if (threadIdx.x == 0) {
        s.cnt[0] = (rank == 0) ? 1u : 0u;
        s.cnt[1] = 0;
        s.nheavy = 0;
        s.edges = 0;
        s.tot[0] = s.tot[1] = s.tot[2] = 0;
        s.stop = 0;
        if (rank == 0) {
            s.list[0][0] = a.src;
            if (!SSSP) {
                a.levels[a.src] = 0;
                if (a.parents) a.parents[a.src] = (int32_t)a.src;
            }
        }
    }
    cl.sync();
    const uint64_t t_start = dev::globaltimer_ns();
    unsigned long long reached = 1;
    int d = 0;
    unsigned int frontier_total = 1;
    while (frontier_total) {
        const int cur = d & 1, nxt = cur ^ 1;
        const uint32_t *ov_cur = cur ? a.ov[1] : a.ov[0];   // selected, not indexed: the
        uint32_t *ov_nxt = cur ? a.ov[0] : a.ov[1];          // parameter array stays in registers
        // the lengths of every CTA's list (distributed shared memory), as a prefix
        if (threadIdx.x < ncta) {
            const unsigned int c = cl.map_shared_rank(&s, threadIdx.x)->cnt[cur];
            s.pre[threadIdx.x + 1] = c < CAP ? c : CAP;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s.pre[0] = 0;
            for (unsigned int r = 1; r <= ncta; ++r) s.pre[r] += s.pre[r - 1];
        }
        const unsigned int nov = __ldcg(&st->ov_cnt[d % 3]);
        __syncthreads();
        if (threadIdx.x == 0) {
            s.cnt[nxt] = 0;
            s.nheavy = 0;
            if (rank == 0) {
                // the slots level d+1 will fill: last read right after the
                // barrier that ended level d-2, which every CTA has passed
                s.tot[(d + 2) % 3] = 0;
                st->ov_cnt[(d + 2) % 3] = 0;
            }
        }
        __syncthreads();
        unsigned long long my_edges = 0;
        // expand: the concatenation of all CTAs' lists and then the overflow
        // list, item i handled by CTA i % ncta (balanced whoever claimed them)
        const unsigned int nlist = s.pre[ncta];
        const unsigned int nitems = nlist + nov;
        for (unsigned int i = rank + threadIdx.x * ncta; i < nitems; i += CT * ncta) {
            uint32_t u;
            if (i < nlist) {
                unsigned int o = 0;
                while (s.pre[o + 1] <= i) ++o;   // owner CTA of item i (at most 16 steps)
                u = cl.map_shared_rank(&s, o)->list[cur][i - s.pre[o]];
            } else {
                u = __ldcg(&ov_cur[i - nlist]);
            }
            const uint32_t b = __ldg(&a.rp[u]), e = __ldg(&a.rp[u + 1]);
            my_edges += e - b;
            if (e - b > HEAVY) {
                const unsigned int h = atomicAdd(&s.nheavy, 1u);
                if (h < HCAP) { s.heavy[h] = u; continue; }
            }
            if (SSSP) {
                const uint32_t du = __ldcg(&a.dist[u]);
                for (uint32_t k0 = b; k0 < e; k0 += 4) {
                    uint32_t v[4], nd[4], cur_d[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool in = k0 + k < e;
                        v[k] = in ? __ldg(&a.ci[k0 + k]) : 0u;
                        nd[k] = in ? sat_add(du, __ldg(&a.wt[k0 + k])) : 0xffffffffu;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) cur_d[k] = nd[k] != 0xffffffffu ? __ldcg(&a.dist[v[k]]) : 0u;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (nd[k] >= cur_d[k]) continue;
                        if (nd[k] >= atomicMin(&a.dist[v[k]], nd[k])) continue;
                        if (atomicExch(&a.stamp[v[k]], (uint32_t)d + 1) == (uint32_t)d + 1) continue;
                        const unsigned int idx = atomicAdd(&s.cnt[nxt], 1u);
                        if (idx < CAP) s.list[nxt][idx] = v[k];
                        else ov_nxt[atomicAdd(&st->ov_cnt[(d + 1) % 3], 1u)] = v[k];
                    }
                }
                continue;
            }
            // four neighbours at a time: their loads, then their claims, in flight together
            for (uint32_t k0 = b; k0 < e; k0 += 4) {
                uint32_t v[4], bit[4], old[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = k0 + k < e ? __ldg(&a.ci[k0 + k]) : 0xffffffffu;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    bit[k] = 1u << (v[k] & 31);
                    old[k] = v[k] != 0xffffffffu ? atomicOr(&a.visited[v[k] >> 5], bit[k]) : bit[k];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (old[k] & bit[k]) continue;
                    a.levels[v[k]] = d + 1;
                    if (a.parents) a.parents[v[k]] = (int32_t)u;
                    const unsigned int idx = atomicAdd(&s.cnt[nxt], 1u);
                    if (idx < CAP) s.list[nxt][idx] = v[k];
                    else ov_nxt[atomicAdd(&st->ov_cnt[(d + 1) % 3], 1u)] = v[k];
                }
            }
        }
        __syncthreads();
        // heavy rows: a warp per row, 32 edges per step
        const unsigned int nh = s.nheavy < HCAP ? s.nheavy : HCAP;
        for (unsigned int h = warp; h < nh; h += CT / 32) {
            const uint32_t u = s.heavy[h];
            const uint32_t b = __ldg(&a.rp[u]), e = __ldg(&a.rp[u + 1]);
            const uint32_t du = SSSP ? __ldcg(&a.dist[u]) : 0u;
            for (uint32_t k = b + lane; k < e; k += 32) {
                const uint32_t v = __ldg(&a.ci[k]);
                bool joins;
                if (SSSP) {
                    const uint32_t nd = sat_add(du, __ldg(&a.wt[k]));
                    joins = nd < __ldcg(&a.dist[v]) && nd < atomicMin(&a.dist[v], nd) &&
                            atomicExch(&a.stamp[v], (uint32_t)d + 1) != (uint32_t)d + 1;
                } else {
                    joins = claim(a, u, v, d);
                }
                if (joins) {
                    const unsigned int idx = atomicAdd(&s.cnt[nxt], 1u);
                    if (idx < CAP) s.list[nxt][idx] = v;
                    else ov_nxt[atomicAdd(&st->ov_cnt[(d + 1) % 3], 1u)] = v;
                }
            }
        }
        my_edges = dev::warp_sum<unsigned long long>(my_edges);
        if (lane == 0 && my_edges) atomicAdd(&s.edges, my_edges);
        __syncthreads();
        // publish this CTA's claims into CTA 0's cluster-wide sum
        if (threadIdx.x == 0) {
            if (s.cnt[nxt]) atomicAdd(&s0->tot[(d + 1) % 3], s.cnt[nxt]);
            if (rank == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns) s.stop = 1;
        }
        cl.sync();
        frontier_total = s0->tot[(d + 1) % 3];
        const unsigned int stop = s0->stop;
        reached += frontier_total;
        ++d;
        if (stop) {
            if (rank == 0 && threadIdx.x == 0) {
                atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
                if (a.err_sticky) atomicMax(a.err_sticky, (int)GB_TIMEOUT);
            }
            break;
        }
    }
    // ---- vertices never reached get level and parent -1
    if (!SSSP && !s0->stop) {
        for (uint32_t w0 = (rank * (CT / 32) + warp) * 32; w0 < a.nwords; w0 += (gthreads / 32) * 32) {
            const uint32_t me = w0 + lane < a.nwords ? __ldcg(&a.visited[w0 + lane]) : ~0u;
            uint32_t todo = __ballot_sync(0xffffffffu, me != ~0u);
            while (todo) {
                const int k = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t bits = __shfl_sync(0xffffffffu, me, k);
                if (!((bits >> lane) & 1u)) {
                    const uint64_t v = (uint64_t)(w0 + k) * 32 + lane;
                    a.levels[v] = -1;
                    if (a.parents) a.parents[v] = -1;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s.edges) atomicAdd(&st->edges, s.edges);
    if (rank == 0 && threadIdx.x == 0) {
        st->depth = (unsigned int)d;
        st->reached = reached;
        st->t_begin = t_start;
        st->t_end = dev::globaltimer_ns();
    }
    cl.sync();   // no CTA leaves while others may still read CTA 0's shared memory
}

}  // namespace clk

// The cluster size this device can co-schedule (16, else 8), 0 if none.
static int cluster_size(gb_context *ctx) {
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(ctx->device);
    if (it != cache.end()) return it->second;
    int best = 0;
    const size_t smem = sizeof(clk::ClSmem);
    bool attrs = true;
    for (const void *fn : {(const void *)clk::k_cluster<false>, (const void *)clk::k_cluster<true>}) {
        attrs = attrs && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
                cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    }
    if (attrs) {
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(clk::CT);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, clk::k_cluster<true>, &cfg) == cudaSuccess && nclusters > 0 &&
                cudaOccupancyMaxActiveClusters(&nclusters, clk::k_cluster<false>, &cfg) == cudaSuccess && nclusters > 0) {
                best = c;
                break;
            }
        }
    }
    cudaGetLastError();
    cache[ctx->device] = best;
    return best;
}

bool bfs_cluster_available(gb_context *ctx) { return cluster_size(ctx) > 0; }

// Runs one BFS in a single cluster; the overflow lists use the BFS
// workspace's frontier lists.
gb_info bfs_cluster_launch(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels, int32_t *parents,
                           uint32_t *visited, uint32_t *ov0, uint32_t *ov1, void *state, int *err_sticky) {
    const int c = cluster_size(ctx);
    if (!c) return fail(GB_NOT_IMPLEMENTED, "gb_bfs: this device cannot co-schedule a thread-block cluster");
    clk::ClArgs a;
    a.n = A->nrows;
    a.nwords = (A->nrows + 31) / 32;
    a.src = src;
    a.rp = A->rowptr;
    a.ci = A->colidx;
    a.levels = levels;
    a.parents = parents;
    a.visited = visited;
    a.dist = nullptr;
    a.wt = nullptr;
    a.stamp = nullptr;
    a.ov[0] = ov0;
    a.ov[1] = ov1;
    a.st = (clk::ClState *)state;
    a.total_limit_ns = 120000000000ull;
    a.err_sticky = err_sticky;
    GB_CHECK(memset_async(ctx, state, 0, sizeof(clk::ClState)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(clk::CT);
    cfg.dynamicSmemBytes = sizeof(clk::ClSmem);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int span = prof_begin(ctx, "bfs");
    GB_CUDA(cudaLaunchKernelEx(&cfg, clk::k_cluster<false>, a));
    prof_end(ctx, span);
    return GB_SUCCESS;
}

// SSSP from src in a single cluster: dist[n] out (device), stamp[n] scratch.
gb_info sssp_cluster_launch(gb_context *ctx, const gb_matrix *A, uint32_t src, uint32_t *dist, uint32_t *stamp,
                            uint32_t *ov0, uint32_t *ov1, void *state) {
    const int c = cluster_size(ctx);
    if (!c) return fail(GB_NOT_IMPLEMENTED, "gb_sssp: this device cannot co-schedule a thread-block cluster");
    clk::ClArgs a;
    a.n = A->nrows;
    a.nwords = (A->nrows + 31) / 32;
    a.src = src;
    a.rp = A->rowptr;
    a.ci = A->colidx;
    a.levels = nullptr;
    a.parents = nullptr;
    a.visited = nullptr;
    a.dist = dist;
    a.wt = (const uint32_t *)A->vals;
    a.stamp = stamp;
    a.ov[0] = ov0;
    a.ov[1] = ov1;
    a.st = (clk::ClState *)state;
    a.total_limit_ns = 300000000000ull;
    a.err_sticky = nullptr;
    GB_CHECK(memset_async(ctx, state, 0, sizeof(clk::ClState)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(clk::CT);
    cfg.dynamicSmemBytes = sizeof(clk::ClSmem);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int span = prof_begin(ctx, "sssp");
    GB_CUDA(cudaLaunchKernelEx(&cfg, clk::k_cluster<true>, a));
    prof_end(ctx, span);
    return GB_SUCCESS;
}

// Iterations and status of a finished cluster traversal (after a sync).
gb_info cluster_iterations(gb_context *ctx, const void *state, uint32_t *iterations) {
    clk::ClState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (iterations) *iterations = hs.depth;
    if (hs.err) return fail(GB_TIMEOUT, "the cluster traversal ran out of its time budget");
    return GB_SUCCESS;
}

size_t bfs_cluster_state_bytes() { return sizeof(clk::ClState); }

// Reads the state a cluster BFS left (after the stream has synchronised).
gb_info bfs_cluster_result(gb_context *ctx, const void *state, gb_bfs_stats *stats) {
    clk::ClState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->depth = hs.depth;
        stats->push_levels = hs.depth;
        stats->status = (uint32_t)hs.err;
        stats->vertices_reached = hs.reached;
        stats->edges_examined = hs.edges;
        stats->frontier_edges = hs.edges;
        stats->init_us = 0.f;
        stats->final_us = 0.f;
    }
    if (hs.err) return fail(GB_TIMEOUT, "gb_bfs: the cluster traversal ran out of its time budget");
    return GB_SUCCESS;
}

}  // namespace gbx
