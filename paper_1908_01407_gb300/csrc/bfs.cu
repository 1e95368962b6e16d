// Direction-optimised BFS (Algorithm 1, Section 6.1) as one persistent
// cooperative kernel: every level runs either
//   push  = SpMSpV over the out-edges (CSR rows) of the sparse frontier list,
//           claiming unvisited vertices with atomicOr on the visited bitmap
//           (the mask is applied before the write, not after: Section 5.3), or
//   pull  = masked SpMV over the in-edges (CSC columns) of unvisited vertices
//           only (mask first), stopping at the first frontier parent (the
//           Boolean semiring's early exit, Table 3) and reading no values
//           (structure only),
// with the assign of the level, the frontier count and the next frontier's
// edge count fused in. The direction rule is Table 8's: pull iff the
// frontier's edge count |E_f| > |E| / beta, with |E_f| exact (each appended
// vertex carries an exclusive prefix of out-degrees, see below).
//
// Frontier representation: both a bitmap (for pull) and a list with edge
// prefixes (for push) are produced every level (operand reuse, Section 6.1).
// Appends use a single 64-bit atomicAdd on a packed (count, edge-sum) word,
// so list positions and edge prefixes come out consistent and monotone: the
// push of the next level balances its edges over the grid by a merge-path
// search over the prefixes, without a separate scan.
//
// Levels are separated by a grid barrier with a wall-clock bound; on timeout
// the kernel records GB_TIMEOUT and exits.
#include "common.cuh"
#include "bfs_common.cuh"

using namespace gbx;

namespace gbx {
namespace bfsk {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;
constexpr int PUSH_ITEMS = 4;
constexpr int PUSH_TILE = BLOCK * PUSH_ITEMS;      // edges per block tile
constexpr int PUSH_OWNERS = PUSH_TILE + 1;          // owner entries staged in smem
constexpr int PULL_WPW = 4;                          // bitmap words per warp per tile
constexpr int PULL_TILE_WORDS = WARPS * PULL_WPW;    // 32 words = 1024 vertices
constexpr int PULL_LANE_LIMIT = 8;                   // neighbours a lane checks alone

struct SmemPush {
    uint32_t P[PUSH_OWNERS];
    uint32_t Q[PUSH_OWNERS];
    uint32_t R[PUSH_OWNERS];
    uint32_t k0, nk;
};
struct SmemPull {
    uint32_t v[WARPS][PULL_WPW * 32];
    uint32_t deg[WARPS][PULL_WPW * 32];
    uint32_t wcnt[WARPS];
    uint32_t wdeg[WARPS];
    unsigned long long base;
};
union Smem {
    SmemPush push;
    SmemPull pull;
};

__device__ __forceinline__ uint32_t ldcg(const uint32_t *p) { return __ldcg(p); }

// largest k in [0, cnt) with P[k] <= e (P[0] == 0 <= e)
__device__ __forceinline__ uint32_t owner_search_global(const uint32_t *P, uint32_t cnt, uint64_t e) {
    uint32_t lo = 0, hi = cnt;  // invariant: P[lo] <= e, answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)ldcg(&P[mid]) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ void append_warp(const BfsArgs &a, int slot_next, uint32_t *Qn, uint32_t *Pn, bool win, uint32_t v,
                            uint32_t deg) {
    const uint32_t full = 0xffffffffu;
    uint32_t wmask = __ballot_sync(full, win);
    if (!wmask) return;
    uint32_t tot;
    uint32_t ex = dev::warp_exclusive_sum<uint32_t>(win ? deg : 0u, &tot);
    unsigned long long base = 0;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        unsigned long long add = ((unsigned long long)__popc(wmask) << a.ebits) | tot;
        base = atomicAdd(&a.st->qstate[slot_next], add);
    }
    base = __shfl_sync(full, base, 0);
    if (win) {
        uint32_t pos = (uint32_t)(base >> a.ebits) + __popc(wmask & dev::lanemask_lt());
        uint32_t pre = (uint32_t)(base & a.emask) + ex;
        Qn[pos] = v;
        Pn[pos] = pre;
    }
}

__device__ __forceinline__ bool claim(const BfsArgs &a, uint32_t v, uint32_t parent, int d, uint32_t *Fn,
                                      uint32_t *deg_out) {
    uint32_t w = v >> 5, bit = 1u << (v & 31);
    if (ldcg(&a.visited[w]) & bit) return false;
    uint32_t old = atomicOr(&a.visited[w], bit);
    if (old & bit) return false;
    a.levels[v] = d + 1;
    if (a.parents) a.parents[v] = (int32_t)parent;
    atomicOr(&Fn[w], bit);
    *deg_out = __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
    return true;
}

__device__ void push_level(const BfsArgs &a, Smem &sm, int d, uint32_t cnt, uint64_t fe) {
    const int cur = d & 1, nxt = (d + 1) & 1;
    const int slot_next = (d + 1) % 3;
    const uint32_t *Q = a.q[cur];
    const uint32_t *P = a.qp[cur];
    uint32_t *Qn = a.q[nxt];
    uint32_t *Pn = a.qp[nxt];
    uint32_t *Fn = a.front[(d + 1) % 3];
    uint64_t ntiles = (fe + PUSH_TILE - 1) / PUSH_TILE;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t E0 = t * PUSH_TILE;
        uint64_t E1 = E0 + PUSH_TILE < fe ? E0 + PUSH_TILE : fe;
        if (threadIdx.x == 0) {
            uint32_t k0 = owner_search_global(P, cnt, E0);
            uint32_t k1 = owner_search_global(P, cnt, E1 - 1);
            sm.push.k0 = k0;
            sm.push.nk = k1 - k0 + 1;
        }
        __syncthreads();
        const uint32_t k0 = sm.push.k0, nk = sm.push.nk;
        const bool staged = nk <= PUSH_OWNERS;
        if (staged) {
            for (uint32_t j = threadIdx.x; j < nk; j += BLOCK) {
                uint32_t u = ldcg(&Q[k0 + j]);
                sm.push.Q[j] = u;
                sm.push.P[j] = ldcg(&P[k0 + j]);
                sm.push.R[j] = __ldg(&a.rp_out[u]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < PUSH_ITEMS; ++it) {
            uint64_t e = E0 + (uint64_t)it * BLOCK + threadIdx.x;
            bool win = false;
            uint32_t v = 0, deg = 0;
            if (e < E1) {
                uint32_t u, p;
                if (staged) {
                    uint32_t lo = 0, hi = nk;
                    while (hi - lo > 1) {
                        uint32_t mid = (lo + hi) >> 1;
                        if ((uint64_t)sm.push.P[mid] <= e) lo = mid; else hi = mid;
                    }
                    u = sm.push.Q[lo];
                    p = sm.push.R[lo] + (uint32_t)(e - sm.push.P[lo]);
                } else {
                    uint32_t k = owner_search_global(P, cnt, e);
                    u = ldcg(&Q[k]);
                    p = __ldg(&a.rp_out[u]) + (uint32_t)(e - ldcg(&P[k]));
                }
                v = __ldg(&a.ci_out[p]);
                win = claim(a, v, u, d, Fn, &deg);
            }
            append_warp(a, slot_next, Qn, Pn, win, v, deg);
        }
        __syncthreads();
    }
}

__device__ void pull_level(const BfsArgs &a, Smem &sm, int d, unsigned long long *examined) {
    const int nxt = (d + 1) & 1;
    const int slot_next = (d + 1) % 3;
    const uint32_t *F = a.front[d % 3];
    uint32_t *Fn = a.front[(d + 1) % 3];
    uint32_t *Qn = a.q[nxt];
    uint32_t *Pn = a.qp[nxt];
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t ntiles = (a.nwords + PULL_TILE_WORDS - 1) / PULL_TILE_WORDS;
    unsigned long long exam = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t staged = 0;
        uint32_t wdegsum = 0;
#pragma unroll 1
        for (int j = 0; j < PULL_WPW; ++j) {
            uint64_t word = t * PULL_TILE_WORDS + (uint64_t)warp * PULL_WPW + j;
            if (word >= a.nwords) break;
            uint32_t vis = ldcg(&a.visited[word]);
            uint32_t cand = ~vis;
            if (cand == 0) continue;
            uint32_t v = (uint32_t)(word * 32 + lane);
            bool active = (cand >> lane) & 1u;
            bool found = false;
            uint32_t par = 0, b = 0, e = 0, p = 0;
            if (active) {
                b = __ldg(&a.rp_in[v]);
                e = __ldg(&a.rp_in[v + 1]);
                uint32_t lim = e - b > PULL_LANE_LIMIT ? b + PULL_LANE_LIMIT : e;
                for (p = b; p < lim; ++p) {
                    uint32_t u = __ldg(&a.ci_in[p]);
                    if ((ldcg(&F[u >> 5]) >> (u & 31)) & 1u) { found = true; par = u; ++p; break; }
                }
                exam += p - b;
            }
            uint32_t coop = __ballot_sync(full, active && !found && p < e);
            while (coop) {
                int l = __ffs(coop) - 1;
                coop &= coop - 1;
                uint32_t pb = __shfl_sync(full, p, l);
                uint32_t pe = __shfl_sync(full, e, l);
                bool got = false;
                uint32_t gpar = 0;
                for (uint32_t q0 = pb; q0 < pe; q0 += 32) {
                    uint32_t q = q0 + lane;
                    uint32_t u = 0;
                    bool hit = false;
                    if (q < pe) {
                        u = __ldg(&a.ci_in[q]);
                        hit = (ldcg(&F[u >> 5]) >> (u & 31)) & 1u;
                    }
                    uint32_t hb = __ballot_sync(full, hit);
                    if (hb) {
                        int f = __ffs(hb) - 1;
                        gpar = __shfl_sync(full, u, f);
                        got = true;
                        if (lane == 0) exam += (q0 - pb) + f + 1;
                        break;
                    }
                    if (lane == 0) exam += (pe - q0 < 32 ? pe - q0 : 32);
                }
                if (lane == l && got) { found = true; par = gpar; }
            }
            uint32_t fm = __ballot_sync(full, found);
            if (fm) {
                if (lane == 0) {
                    a.visited[word] = vis | fm;
                    Fn[word] = fm;
                }
                uint32_t deg = 0;
                if (found) {
                    a.levels[v] = d + 1;
                    if (a.parents) a.parents[v] = (int32_t)par;
                    deg = a.csr_is_csc ? e - b : __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
                    uint32_t idx = staged + __popc(fm & dev::lanemask_lt());
                    sm.pull.v[warp][idx] = v;
                    sm.pull.deg[warp][idx] = deg;
                }
                staged += __popc(fm);
                wdegsum += dev::warp_sum<uint32_t>(deg);
            }
        }
        if (lane == 0) {
            sm.pull.wcnt[warp] = staged;
            sm.pull.wdeg[warp] = wdegsum;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t c = 0, s = 0;
            for (int w = 0; w < WARPS; ++w) {
                uint32_t cw = sm.pull.wcnt[w], sw = sm.pull.wdeg[w];
                sm.pull.wcnt[w] = c;
                sm.pull.wdeg[w] = s;
                c += cw;
                s += sw;
            }
            unsigned long long base = 0;
            if (c) base = atomicAdd(&a.st->qstate[slot_next], ((unsigned long long)c << a.ebits) | s);
            sm.pull.base = base;
        }
        __syncthreads();
        {
            unsigned long long base = sm.pull.base;
            uint32_t pos = (uint32_t)(base >> a.ebits) + sm.pull.wcnt[warp];
            uint32_t pre = (uint32_t)(base & a.emask) + sm.pull.wdeg[warp];
            for (uint32_t c0 = 0; c0 < staged; c0 += 32) {
                uint32_t idx = c0 + lane;
                uint32_t dg = idx < staged ? sm.pull.deg[warp][idx] : 0u;
                uint32_t tot;
                uint32_t ex = dev::warp_exclusive_sum<uint32_t>(dg, &tot);
                if (idx < staged) {
                    Qn[pos + idx] = sm.pull.v[warp][idx];
                    Pn[pos + idx] = pre + ex;
                }
                pre += tot;
            }
        }
        __syncthreads();
    }
    *examined += exam;
}

__device__ __forceinline__ bool choose_pull(const BfsArgs &a, uint64_t fe) {
    if (a.mode == GB_PUSH || !a.rp_in) return false;
    if (a.mode == GB_PULL) return true;
    return fe * (uint64_t)a.beta > a.m;
}

__global__ void __launch_bounds__(BLOCK) k_bfs(BfsArgs a) {
    __shared__ Smem sm;
    __shared__ unsigned long long s_exam;
    const uint32_t nthreads = gridDim.x * BLOCK;
    const uint32_t tid = blockIdx.x * BLOCK + threadIdx.x;
    BfsState *st = a.st;
    // ---- init: levels/parents, bitmaps, the level-0 list
    for (uint64_t i = tid; i < a.n; i += nthreads) {
        a.levels[i] = i == a.src ? 0 : -1;
        if (a.parents) a.parents[i] = i == a.src ? (int32_t)a.src : -1;
    }
    const uint32_t sw = a.src >> 5, sbit = 1u << (a.src & 31);
    const uint32_t tail = (a.n & 31) ? ~((1u << (a.n & 31)) - 1u) : 0u;
    for (uint64_t w = tid; w < a.nwords; w += nthreads) {
        uint32_t vis = (w == sw ? sbit : 0u);
        if (w == a.nwords - 1) vis |= tail;
        a.visited[w] = vis;
        a.front[0][w] = w == sw ? sbit : 0u;
        a.front[1][w] = 0u;
        a.front[2][w] = 0u;
    }
    if (tid == 0) {
        uint32_t deg = __ldg(&a.rp_out[a.src + 1]) - __ldg(&a.rp_out[a.src]);
        a.q[0][0] = a.src;
        a.qp[0][0] = 0;
        st->qstate[0] = (1ull << a.ebits) | deg;
        st->qstate[1] = 0;
        st->qstate[2] = 0;
        st->exam[0] = st->exam[1] = st->exam[2] = 0;
    }
    if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) return;
    const uint64_t t_start = a.t_start_hint ? a.t_start_hint : dev::globaltimer_ns();
    uint64_t reached = 0;
    // previous level's numbers for the algorithmic byte count
    uint32_t prev_dir = 0, prev_cnt = 0;
    uint64_t prev_fe = 0, prev_unvisited = 0;
    double alg = 8.0 * a.n;   // levels + parents initialisation writes
    int d = 0;
    for (;; ++d) {
        unsigned long long qs = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(st->qstate[d % 3])
                                    .load(cuda::memory_order_relaxed);
        uint32_t cnt = (uint32_t)(qs >> a.ebits);
        uint64_t fe = qs & a.emask;
        if (tid == 0 && d > 0) {
            unsigned long long ex = st->exam[(d - 1) % 3];
            if (prev_dir == 0)
                alg += 8.0 * prev_cnt + 4.0 * prev_fe + 12.0 * cnt;
            else
                alg += a.n / 8.0 + 8.0 * prev_unvisited + 4.0 * ex + 12.0 * cnt;
            st->edges_examined += prev_dir == 0 ? prev_fe : ex;
        }
        if (cnt == 0) break;
        // guards: no BFS has more than n levels; the whole kernel has a wall-clock budget
        if (d > (int)a.n || dev::globaltimer_ns() - t_start > a.total_limit_ns) {
            if (tid == 0) atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
            break;
        }
        const bool pull = choose_pull(a, fe);
        if (tid == 0) {
            if (d < GBX_MAX_LEVEL_LOG) st->dir_log[d] = pull ? 2 : 1;
            if (pull) st->pull_levels++; else st->push_levels++;
            st->qstate[(d + 2) % 3] = 0;
            st->exam[(d + 2) % 3] = 0;
            st->frontier_edges += fe;
            prev_unvisited = a.n - reached - cnt;
            prev_dir = pull ? 1u : 0u;
            prev_cnt = cnt;
            prev_fe = fe;
        }
        reached += cnt;
        uint32_t *Fclr = a.front[(d + 2) % 3];
        for (uint64_t w = tid; w < a.nwords; w += nthreads) Fclr[w] = 0u;
        if (pull) {
            if (threadIdx.x == 0) s_exam = 0;
            __syncthreads();
            unsigned long long ex = 0;
            pull_level(a, sm, d, &ex);
            ex = dev::warp_sum<unsigned long long>(ex);
            if ((threadIdx.x & 31) == 0 && ex) atomicAdd(&s_exam, ex);
            __syncthreads();
            if (threadIdx.x == 0 && s_exam) atomicAdd(&st->exam[d % 3], s_exam);
        } else {
            push_level(a, sm, d, cnt, fe);
        }
        if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) return;
    }
    if (tid == 0) {
        st->depth = d;
        st->reached = reached;
        st->alg_bytes = alg;
    }
}

}  // namespace bfsk

struct BfsWorkspace {
    uint32_t n = 0;
    uint32_t *visited = nullptr, *front = nullptr, *q = nullptr, *qp = nullptr;
    BfsState *st = nullptr;
    int grid = 0;
};

static std::mutex g_ws_mu;
static std::unordered_map<gb_context *, BfsWorkspace> g_ws;

gb_info bfs_workspace(gb_context *ctx, uint32_t n, BfsWorkspace **out) {
    std::lock_guard<std::mutex> g(g_ws_mu);
    BfsWorkspace &w = g_ws[ctx];
    if (w.n < n || !w.st) {
        dfree(ctx, w.visited); dfree(ctx, w.front); dfree(ctx, w.q); dfree(ctx, w.qp); dfree(ctx, w.st);
        w = BfsWorkspace();
        uint32_t nw = (n + 31) / 32;
        GB_CHECK(dalloc_t(ctx, &w.visited, nw));
        GB_CHECK(dalloc_t(ctx, &w.front, 3ull * nw));
        GB_CHECK(dalloc_t(ctx, &w.q, 2ull * n + 2));
        GB_CHECK(dalloc_t(ctx, &w.qp, 2ull * n + 2));
        GB_CHECK(dalloc_t(ctx, &w.st, 1));
        w.n = n;
    }
    if (!w.grid) {
        int occ = 0;
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bfsk::k_bfs, bfsk::BLOCK, 0));
        if (occ < 1) return fail(GB_PANIC, "BFS kernel cannot be resident");
        w.grid = occ * ctx->num_sms;
    }
    *out = &w;
    return GB_SUCCESS;
}

void bfs_workspace_release(gb_context *ctx) {
    std::lock_guard<std::mutex> g(g_ws_mu);
    auto it = g_ws.find(ctx);
    if (it == g_ws.end()) return;
    BfsWorkspace &w = it->second;
    dfree(ctx, w.visited); dfree(ctx, w.front); dfree(ctx, w.q); dfree(ctx, w.qp); dfree(ctx, w.st);
    g_ws.erase(it);
}

gb_info bfs_launch(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels, int32_t *parents,
                   const gb_desc *desc, BfsWorkspace *w, int grid_override) {
    BfsArgs a;
    a.n = A->nrows;
    a.nwords = (A->nrows + 31) / 32;
    a.m = A->nvals;
    a.src = src;
    a.rp_out = A->rowptr;
    a.ci_out = A->colidx;
    a.rp_in = A->has_csc ? A->colptr : nullptr;
    a.ci_in = A->has_csc ? A->rowidx : nullptr;
    a.csr_is_csc = A->csc_alias;
    a.levels = levels;
    a.parents = parents;
    a.visited = w->visited;
    for (int k = 0; k < 3; ++k) a.front[k] = w->front + (size_t)k * a.nwords;
    a.q[0] = w->q; a.q[1] = w->q + A->nrows + 1;
    a.qp[0] = w->qp; a.qp[1] = w->qp + A->nrows + 1;
    a.ebits = 64 - bits_for((uint64_t)A->nrows + 1);
    a.emask = (a.ebits >= 64) ? ~0ull : ((1ull << a.ebits) - 1);
    a.mode = desc ? desc->direction : GB_AUTO;
    a.beta = (desc && desc->beta > 0) ? (uint32_t)desc->beta : 10u;
    a.st = w->st;
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 120000000000ull;
    a.t_start_hint = 0;
    GB_CUDA(cudaMemsetAsync(w->st, 0, sizeof(BfsState), ctx->stream));
    int grid = grid_override > 0 && grid_override < w->grid ? grid_override : w->grid;
    void *args[] = {&a};
    int span = prof_begin(ctx, "bfs");
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)bfsk::k_bfs, dim3(grid), dim3(bfsk::BLOCK), args, 0,
                                        ctx->stream));
    prof_end(ctx, span);
    return GB_SUCCESS;
}

}  // namespace gbx

extern "C" gb_info gb_bfs(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels, int32_t *parents,
                          gb_mem mem, const gb_desc *desc, gb_bfs_stats *stats) {
    if (!ctx || !A || !levels) return fail(GB_NULL_POINTER, "gb_bfs: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_bfs: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_bfs: matrix must be square");
    if (A->nrows == 0 || src >= A->nrows) return fail(GB_INVALID_INDEX, "gb_bfs: source %u out of range", src);
    GB_CUDA(cudaSetDevice(ctx->device));
    BfsWorkspace *w = nullptr;
    GB_CHECK(bfs_workspace(ctx, A->nrows, &w));
    int32_t *dl = levels, *dp = parents;
    Scratch tl(ctx), tp(ctx);
    if (mem == GB_HOST) {
        GB_CHECK(tl.alloc((size_t)A->nrows * 4));
        dl = tl.as<int32_t>();
        if (parents) {
            GB_CHECK(tp.alloc((size_t)A->nrows * 4));
            dp = tp.as<int32_t>();
        }
    }
    GB_CHECK(bfs_launch(ctx, A, src, dl, dp, desc, w, 0));
    if (mem == GB_HOST) {
        GB_CUDA(cudaMemcpyAsync(levels, dl, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
        if (parents) GB_CUDA(cudaMemcpyAsync(parents, dp, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (stats || mem == GB_HOST) {
        BfsState hs;
        GB_CUDA(cudaMemcpyAsync(&hs, w->st, sizeof(BfsState), cudaMemcpyDeviceToHost, ctx->stream));
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        if (stats) {
            stats->depth = hs.depth;
            stats->push_levels = hs.push_levels;
            stats->pull_levels = hs.pull_levels;
            stats->status = (uint32_t)hs.err;
            stats->vertices_reached = hs.reached;
            stats->edges_examined = hs.edges_examined;
            stats->frontier_edges = hs.frontier_edges;
            stats->alg_bytes = (uint64_t)hs.alg_bytes;
        }
        if (hs.err) return fail(GB_TIMEOUT, "gb_bfs: a bounded grid barrier wait ran out");
    }
    return GB_SUCCESS;
}
