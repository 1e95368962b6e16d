// Min-relaxation over a frontier of changed vertices, as one persistent
// cooperative kernel (the loop of Section 7.2 run on the device):
//  * SSSP, adaptive Bellman-Ford with sparsification (Section 7.2):
//      dist(v) <- min(dist(v), min_{u in F, (u,v) in E} dist(u) + w(u,v))
//    over the min.plus semiring (saturating add, UINT32_MAX = infinity);
//  * connected components by min-label propagation (min.second):
//      label(v) <- min(label(v), min_{u in F, (u,v) in E} label(u)),
//    labels starting at the vertex ids, every vertex active at first.
// The next frontier is exactly the set of vertices whose value decreased
// (the sparsification step: Section 7.2 keeps only vertices that improved).
// For SSSP the changed set is further split by distance (near-far order,
// the bucket discipline of delta-stepping expressed as a mask): only
// improved vertices below the current bound B form the frontier; the others
// wait in a far bitmap. When the frontier empties, B grows by delta and the
// far vertices below it move into the frontier. Every improvement is still
// relaxed, so the fixed point (Dijkstra's distances) is the same; what
// changes is the order, which on weighted graphs saves most of the repeated
// relaxations of vertices improved many times over.
// Each iteration is a push (merge-path over the frontier's out-edges,
// atomicMin into the target) or a pull (every vertex scans its in-edges,
// taking only frontier sources into account) by the rule of Table 9. The
// loop ends when no value changes, which is the exact fixed point.
#include "common.cuh"
#include "bfs_common.cuh"
#include "frontier.cuh"
#include "types.cuh"

using namespace gbx;

namespace gbx {
namespace rlx {
using namespace fr;

struct RelaxArgs {
    const uint32_t *rp_out, *ci_out, *w_out;   // CSR (+ weights): out-edges, for push
    const uint32_t *rp_in, *ci_in, *w_in;      // CSC (+ weights): in-edges, for pull
    bool weighted;                             // SSSP (true) or components (false)
    bool csr_is_csc;
    uint32_t n, nwords;
    uint64_t m;
    uint32_t src;
    bool all_active;
    uint32_t *val;
    uint32_t *front[3];
    uint32_t *q[2], *qp[2], *qr[2];
    int ebits;
    unsigned long long emask;
    int mode;
    uint32_t beta;
    BfsState *st;
    uint64_t timeout_ns, total_limit_ns;
    const uint32_t *hub_list, *hub_pre;   // pull rows longer than RPULL_HUB
    uint32_t nhub;
    uint64_t hub_edges;
    uint64_t delta;          // SSSP bucket width of the near-far frontier; 0 = no buckets
    uint32_t *far;           // bitmap of the far set (improved, at or beyond the current bound)
};

constexpr int RPULL_WPW = 1;

// weights stream through once per relaxation pass: evict-first, like the
// indices, so they do not push the distances and bitmaps out of L2
__device__ __forceinline__ uint32_t relax_val(const RelaxArgs &a, uint32_t vu, uint32_t p, const uint32_t *w) {
    return a.weighted ? sat_add<uint32_t>(vu, ld_stream(&w[p])) : vu;
}

// pull: lane per vertex, RPULL_WPW vertices per lane in flight. Each round
// reads an aligned 16-byte chunk (up to 4 in-edges) of every pending row
// and tests its sources against the frontier bitmap, all loads of a round
// independent; rows longer than RPULL_LONG are scanned by the whole warp.
constexpr uint32_t RPULL_LONG = 64;
constexpr uint32_t RPULL_HUB = GBX_HUB_MIN_LEN;   // rows longer than this are split over the whole grid

__device__ void relax_pull(const RelaxArgs &a, int d, uint32_t *cnt_out, uint32_t *deg_out) {
    const uint32_t *F = a.front[d % 3];
    uint32_t *Fn = a.front[(d + 1) % 3];
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint4 *ci4 = reinterpret_cast<const uint4 *>(a.ci_in);
    const uint4 *w4 = reinterpret_cast<const uint4 *>(a.w_in);
    const uint64_t ngroups = (a.nwords + RPULL_WPW - 1) / RPULL_WPW;
    const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
    uint32_t mycnt = 0, mydeg = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * WARPS + warp; g < ngroups; g += nwarps) {
        const uint64_t w0 = g * RPULL_WPW;
        uint32_t b[RPULL_WPW], e[RPULL_WPW], p[RPULL_WPW], best[RPULL_WPW], cur[RPULL_WPW];
#pragma unroll
        for (int j = 0; j < RPULL_WPW; ++j) {
            uint32_t v = (uint32_t)((w0 + j) * 32 + lane);
            b[j] = e[j] = 0;
            cur[j] = UINT32_MAX;
            if (v < a.n) {
                b[j] = __ldg(&a.rp_in[v]);
                e[j] = __ldg(&a.rp_in[v + 1]);
                cur[j] = ldcg(&a.val[v]);
            }
            best[j] = cur[j];
            p[j] = b[j];
        }
        for (;;) {
            bool pend[RPULL_WPW];
            bool any = false;
#pragma unroll
            for (int j = 0; j < RPULL_WPW; ++j) {
                pend[j] = p[j] < e[j] && e[j] - b[j] <= RPULL_LONG;
                any |= pend[j];
            }
            if (!__any_sync(full, any)) break;
            // indices and weights of a chunk load together: reading the weights only
            // after the frontier test found a source would add a dependent DRAM step
            // to every round, and in a pull (a dense frontier) most chunks hit anyway
            uint4 c[RPULL_WPW], wv[RPULL_WPW];
#pragma unroll
            for (int j = 0; j < RPULL_WPW; ++j) {
                if (pend[j]) {
                    c[j] = ld_stream(&ci4[p[j] >> 2]);
                    if (a.weighted) wv[j] = ld_stream(&w4[p[j] >> 2]);
                }
            }
            uint32_t fw[RPULL_WPW][4];
#pragma unroll
            for (int j = 0; j < RPULL_WPW; ++j) {
                uint32_t q = p[j] & ~3u;
                uint32_t cc[4] = {c[j].x, c[j].y, c[j].z, c[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    bool in = pend[j] && q + k >= p[j] && q + k < e[j];
                    fw[j][k] = in ? ((ldcg(&F[cc[k] >> 5]) >> (cc[k] & 31)) & 1u) : 0u;
                }
            }
#pragma unroll
            for (int j = 0; j < RPULL_WPW; ++j) {
                if (!pend[j]) continue;
                uint32_t cc[4] = {c[j].x, c[j].y, c[j].z, c[j].w};
                uint32_t ww[4] = {0, 0, 0, 0};
                if (a.weighted) { ww[0] = wv[j].x; ww[1] = wv[j].y; ww[2] = wv[j].z; ww[3] = wv[j].w; }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (fw[j][k]) {
                        uint32_t vu = ldcg(&a.val[cc[k]]);
                        uint32_t cand = a.weighted ? sat_add<uint32_t>(vu, ww[k]) : vu;
                        if (cand < best[j]) best[j] = cand;
                    }
                }
                p[j] = (p[j] & ~3u) + 4;
            }
        }
#pragma unroll
        for (int j = 0; j < RPULL_WPW; ++j) {
            uint32_t coop = __ballot_sync(full, e[j] - b[j] > RPULL_LONG && e[j] - b[j] <= RPULL_HUB);
            while (coop) {
                int l = __ffs(coop) - 1;
                coop &= coop - 1;
                uint32_t pb = __shfl_sync(full, b[j], l), pe = __shfl_sync(full, e[j], l);
                uint32_t mn = UINT32_MAX;
                for (uint32_t q = pb + lane; q < pe; q += 32) {
                    uint32_t u = ld_stream(&a.ci_in[q]);
                    if ((ldcg(&F[u >> 5]) >> (u & 31)) & 1u) {
                        uint32_t c = relax_val(a, ldcg(&a.val[u]), q, a.w_in);
                        if (c < mn) mn = c;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    uint32_t y = __shfl_xor_sync(full, mn, o);
                    mn = y < mn ? y : mn;
                }
                if (lane == l && mn < best[j]) best[j] = mn;
            }
            bool improved = best[j] < cur[j];
            uint32_t fm = __ballot_sync(full, improved);
            if (fm) {
                const uint64_t word = w0 + j;
                if (lane == 0) atomicOr(&Fn[word], fm);    // hub bits of this word come from the hub phase
                if (improved) {
                    uint32_t v = (uint32_t)(word * 32 + lane);
                    a.val[v] = best[j];
                    mydeg += a.csr_is_csc ? e[j] - b[j] : __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
                    mycnt += 1;
                }
            }
        }
    }
    *cnt_out += mycnt;
    *deg_out += mydeg;
}

// pull, hub rows: every in-edge of a row longer than RPULL_HUB is one work
// item, spread evenly over the grid; improvements go through atomicMin (the
// min is order independent, so the result does not depend on the split)
__device__ void relax_pull_hubs(const RelaxArgs &a, int d, uint32_t *cnt_out, uint32_t *deg_out) {
    if (!a.nhub) return;
    const uint32_t *F = a.front[d % 3];
    uint32_t *Fn = a.front[(d + 1) % 3];
    const uint64_t nth = (uint64_t)gridDim.x * BLOCK;
    uint32_t mycnt = 0, mydeg = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; x < a.hub_edges; x += nth) {
        uint32_t lo = 0, hi = a.nhub;   // last h with hub_pre[h] <= x
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if ((uint64_t)__ldg(&a.hub_pre[mid]) <= x) lo = mid; else hi = mid;
        }
        const uint32_t v = __ldg(&a.hub_list[lo]);
        const uint32_t p = __ldg(&a.rp_in[v]) + (uint32_t)(x - __ldg(&a.hub_pre[lo]));
        const uint32_t u = ld_stream(&a.ci_in[p]);
        if (!((ldcg(&F[u >> 5]) >> (u & 31)) & 1u)) continue;
        const uint32_t c = relax_val(a, ldcg(&a.val[u]), p, a.w_in);
        if (c >= ldcg(&a.val[v])) continue;
        if (c >= atomicMin(&a.val[v], c)) continue;
        const uint32_t bit = 1u << (v & 31);
        if (atomicOr(&Fn[v >> 5], bit) & bit) continue;
        mycnt += 1;
        mydeg += __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
    }
    *cnt_out += mycnt;
    *deg_out += mydeg;
}

__global__ void __launch_bounds__(BLOCK, 6) k_relax(RelaxArgs a) {
    __shared__ Smem sm;
    __shared__ uint32_t s_cnt, s_deg, s_far;
    __shared__ unsigned long long s_qs;
    uint64_t bound = a.delta;   // near-far: the frontier holds improved vertices below bound
    const uint32_t nthreads = gridDim.x * BLOCK;
    const uint32_t tid = blockIdx.x * BLOCK + threadIdx.x;
    BfsState *st = a.st;
    BfsResult *res = &st->res;
    const uint32_t tail = (a.n & 31) ? ((1u << (a.n & 31)) - 1u) : ~0u;
    for (uint64_t i = tid; i < a.n; i += nthreads)
        a.val[i] = a.all_active ? (uint32_t)i : (i == a.src ? 0u : UINT32_MAX);
    for (uint64_t w = tid; w < a.nwords; w += nthreads) {
        uint32_t f;
        if (a.all_active) f = (w == a.nwords - 1) ? tail : ~0u;
        else f = (w == (a.src >> 5)) ? (1u << (a.src & 31)) : 0u;
        a.front[0][w] = f;
        a.front[1][w] = 0u;
        a.front[2][w] = 0u;
        if (a.far) a.far[w] = 0u;
    }
    if (tid == 0) {
        memset(res, 0, sizeof(BfsResult));
        if (a.all_active) {
            st->qstate[0] = ((unsigned long long)a.n << a.ebits) | a.m;
        } else {
            uint32_t r0 = __ldg(&a.rp_out[a.src]);
            a.q[0][0] = a.src;
            a.qp[0][0] = 0;
            a.qr[0][0] = r0;
            st->qstate[0] = (1ull << a.ebits) | (__ldg(&a.rp_out[a.src + 1]) - r0);
        }
    }
    bool ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    const uint64_t t_start = dev::globaltimer_ns();
    bool list_valid = !a.all_active;
    // algorithmic bytes (thread 0 of block 0): the initial value writes, then
    // per push 8 per frontier vertex (offsets), 8 (or 4 unweighted) per
    // frontier out-edge (index, weight); per pull the full masked pass:
    // 4 (n + 1) offsets, n / 8 frontier bits, 4 m indices, 4 per weight of an
    // edge out of the frontier; per level 4 per value written (next frontier)
    double alg = 4.0 * a.n;
    uint32_t prev_cnt = 0;
    uint64_t prev_fe = 0;
    bool prev_pull = false;
    int d = 0;
    for (; ok; ++d) {
        if (threadIdx.x == 0)
            sm.qs = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(st->qstate[d % 3])
                        .load(cuda::memory_order_relaxed);
        __syncthreads();
        const unsigned long long qs = sm.qs;
        __syncthreads();
        uint32_t cnt = (uint32_t)(qs >> a.ebits);
        uint64_t fe = qs & a.emask;
        if (tid == 0 && d > 0) {
            const double ew = a.weighted ? 4.0 : 0.0;
            if (prev_pull) alg += 4.0 * (a.n + 1.0) + a.n / 8.0 + 4.0 * a.m + ew * prev_fe;
            else alg += 8.0 * prev_cnt + (4.0 + ew) * prev_fe;
            alg += 4.0 * cnt;
        }
        if (cnt == 0 && a.delta) {
            // the frontier is empty: raise the bound by delta until far vertices
            // fall below it (they become the frontier), or none is left. The far
            // count is read once here, where it is stable (push levels change it,
            // and they are behind the barrier); every block then tracks it
            // identically from the counts it reads after each barrier.
            if (threadIdx.x == 0) s_far = dev::ld_relaxed_gpu((const unsigned int *)&st->far_cnt);
            __syncthreads();
            uint32_t far_left = s_far;
            __syncthreads();
            bool advanced = false;
            while (far_left > 0) {
                bound += a.delta;
                if (tid == 0) alg += a.n / 8.0 + 4.0 * far_left;   // the far bitmap and the far values
                uint32_t *F = a.front[d % 3];
                uint32_t moved = 0, mdeg = 0;
                for (uint64_t w = tid; w < a.nwords; w += nthreads) {
                    // L2 reads and writes: the far bits were set by atomics, and
                    // this SM's L1 may hold the word from an earlier bound step
                    const uint32_t bits = __ldcg(&a.far[w]);
                    if (!bits) continue;
                    uint32_t take = 0;
                    for (uint32_t bb = bits; bb; bb &= bb - 1) {
                        const uint32_t v = (uint32_t)(w * 32 + (__ffs(bb) - 1));
                        if ((uint64_t)ldcg(&a.val[v]) < bound) {
                            take |= bb & (~bb + 1u);
                            mdeg += __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
                        }
                    }
                    if (take) {
                        __stcg(&a.far[w], bits & ~take);
                        F[w] = take;   // F is empty: no improvement reached the frontier this level
                        moved += __popc(take);
                    }
                }
                moved = dev::warp_sum<uint32_t>(moved);
                mdeg = dev::warp_sum<uint32_t>(mdeg);
                if ((threadIdx.x & 31) == 0 && moved)
                    atomicAdd(&st->qstate[d % 3], ((unsigned long long)moved << a.ebits) | mdeg);
                if (threadIdx.x == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns)
                    atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
                if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) { ok = false; break; }
                if (threadIdx.x == 0)
                    s_qs = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(st->qstate[d % 3])
                               .load(cuda::memory_order_relaxed);
                __syncthreads();
                const unsigned long long q2 = s_qs;
                __syncthreads();
                cnt = (uint32_t)(q2 >> a.ebits);
                fe = q2 & a.emask;
                if (cnt) {
                    advanced = true;
                    // the moved vertices leave the far count; it is read again only
                    // after this level's barrier
                    if (tid == 0) atomicSub(&st->far_cnt, cnt);
                    break;
                }
            }
            if (!ok) break;
            if (!advanced) break;
            list_valid = false;   // the moved vertices exist as a bitmap only
        }
        if (cnt == 0) break;
        // guard: every value can decrease only finitely often; a wall-clock budget bounds the loop
        if (threadIdx.x == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns) atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
        bool pull = !a.delta && a.rp_in && a.mode != GB_PUSH && (a.mode == GB_PULL || fe * (uint64_t)a.beta > a.m);
        if (tid == 0) {
            if (d < GBX_MAX_LEVEL_LOG) {
                res->dir_log[d] = pull ? 2 : 1;
                res->lv_cnt[d] = cnt;
                res->lv_fe[d] = fe;
                res->lv_ns[d] = dev::globaltimer_ns();
            }
            if (pull) res->pull_levels++; else res->push_levels++;
            res->frontier_edges += fe;
            st->qstate[(d + 2) % 3] = 0;
            st->cstate[(d + 2) % 3] = 0;
            prev_cnt = cnt;
            prev_fe = fe;
            prev_pull = pull;
        }
        uint32_t *Fclr = a.front[(d + 2) % 3];
        for (uint64_t w = tid; w < a.nwords; w += nthreads) Fclr[w] = 0u;
        if (pull) {
            if (threadIdx.x == 0) { s_cnt = 0; s_deg = 0; }
            __syncthreads();
            uint32_t c = 0, dg = 0;
            relax_pull(a, d, &c, &dg);
            relax_pull_hubs(a, d, &c, &dg);
            c = dev::warp_sum<uint32_t>(c);
            dg = dev::warp_sum<uint32_t>(dg);
            if ((threadIdx.x & 31) == 0 && c) { atomicAdd(&s_cnt, c); atomicAdd(&s_deg, dg); }
            __syncthreads();
            if (threadIdx.x == 0 && s_cnt)
                atomicAdd(&st->qstate[(d + 1) % 3], ((unsigned long long)s_cnt << a.ebits) | s_deg);
            list_valid = false;
        } else {
            if (!list_valid) {
                compact_level(a, sm, d);
                if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) { ok = false; break; }
            }
            uint32_t nfar = 0;
            push_edges(a, sm, d, cnt, fe, [&](uint32_t u, uint32_t v, uint32_t p, uint32_t *Fn, uint32_t *deg, uint32_t *r0) {
                uint32_t c = relax_val(a, ldcg(&a.val[u]), p, a.w_out);
                if (c >= ldcg(&a.val[v])) return false;
                uint32_t old = atomicMin(&a.val[v], c);
                if (c >= old) return false;
                uint32_t bit = 1u << (v & 31);
                if (a.delta && (uint64_t)c >= bound) {   // beyond the bound: the far set
                    if (!(atomicOr(&a.far[v >> 5], bit) & bit)) ++nfar;
                    return false;
                }
                uint32_t o = atomicOr(&Fn[v >> 5], bit);
                if (o & bit) return false;
                *r0 = __ldg(&a.rp_out[v]);
                *deg = __ldg(&a.rp_out[v + 1]) - *r0;
                return true;
            });
            if (a.delta) {
                nfar = dev::warp_sum<uint32_t>(nfar);
                if ((threadIdx.x & 31) == 0 && nfar) atomicAdd(&st->far_cnt, nfar);
            }
            list_valid = true;
        }
        ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    }
    if (tid == 0) {
        res->depth = d;
        if (d < GBX_MAX_LEVEL_LOG) res->lv_ns[d] = dev::globaltimer_ns();
        res->t_begin = t_start;
        res->alg_bytes = alg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int old = atomicAdd(&st->bar.exits, 1u);
        if (old == gridDim.x - 1) {
            __threadfence();
            res->err = ld_relaxed_gpu_int_(&st->err);
            st->err = 0;
            st->bar.count = 0;
            for (int k = 0; k < 3; ++k) { st->qstate[k] = 0; st->exam[k] = 0; st->cstate[k] = 0; }
            st->far_cnt = 0;
            __threadfence();
            st->bar.exits = 0;
        }
    }
}

}  // namespace rlx

struct BfsWorkspace;
gb_info bfs_workspace_raw(gb_context *ctx, uint32_t n, uint32_t **visited, uint32_t **front, uint32_t **q,
                          uint32_t **qp, uint32_t **qr, BfsState **st, void **cl_state);
bool bfs_cluster_available(gb_context *ctx);
gb_info sssp_cluster_launch(gb_context *ctx, const gb_matrix *A, uint32_t src, uint32_t *dist, uint32_t *stamp,
                            uint32_t *ov0, uint32_t *ov1, void *state);
gb_info cluster_iterations(gb_context *ctx, const void *state, uint32_t *iterations);
gb_info async_relax_run(gb_context *ctx, const gb_matrix *A, int kind, uint32_t src, uint32_t *out,
                        uint32_t *parents, uint64_t delta, gb_bfs_stats *stats, const char *who);

namespace {
__global__ void k_weight_sum(const uint32_t *w, uint64_t m, unsigned long long *sum) {
    unsigned long long acc = 0;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (uint64_t)gridDim.x * blockDim.x)
        acc += w[q];
    acc = dev::warp_sum<unsigned long long>(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}
}  // namespace

// Mean stored weight of A (uint32 values), computed once and kept on the matrix.
static gb_info matrix_mean_weight(gb_context *ctx, const gb_matrix *A, double *mean) {
    gb_matrix *M = const_cast<gb_matrix *>(A);
    std::lock_guard<std::mutex> g(M->cache_mu);
    if (M->mean_weight <= 0) {
        Scratch s(ctx);
        GB_CHECK(s.alloc(16));
        GB_CHECK(memset_async(ctx, s.p, 0, 16));
        if (A->nvals)
            k_weight_sum<<<1024, 256, 0, ctx->stream>>>((const uint32_t *)A->vals, A->nvals,
                                                       s.as<unsigned long long>());
        GB_LAUNCH_CHECK();
        unsigned long long sum = 0;
        GB_CUDA(cudaMemcpyAsync(&sum, s.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CHECK(sync(ctx));
        M->mean_weight = A->nvals ? (double)sum / (double)A->nvals : 1.0;
        if (M->mean_weight <= 0) M->mean_weight = 1.0;
    }
    *mean = M->mean_weight;
    return GB_SUCCESS;
}

// Default label-bucket width of the barrier-free components: n / CC_BUCKETS
// (at least 1,024). On the 4096^2 grid (ids row by row) widths of n/16,
// n/64, n/256, n/1024 and n/4096 ran 107 / 106 / 88 / 79 / 83 ms against
// 118 ms for one bucket (132 relaxations per vertex, 68 at n/1024): narrower
// buckets relabel less but pay a phase change (three grid barriers and two
// passes over the far bitmap) per bucket.
constexpr uint64_t CC_BUCKETS = 1024;
static uint64_t cc_async_default_bucket(uint32_t n) {
    const uint64_t b = (uint64_t)n / CC_BUCKETS;
    return b < 1024 ? 1024 : b;
}

// Default SSSP bucket width: a multiple of the mean weight times the mean
// degree (32 for the synchronous schedule, ASYNC_DELTA_FACTOR for the
// barrier-free one), clamped to [1, 2^31 - 2]. The barrier-free schedule
// pays a phase change (three grid barriers and two passes over the far
// bitmap) per bucket, but relaxes more vertices more than once the wider a
// bucket is: on the weighted 4096^2 grid (mean weight 500, degree 3.6)
// widths of 1,000 / 4,000 / 8,000 / 16,000 / 32,000 ran 245 / 117 / 87 / 79 /
// 85 ms with 1.3 / 1.7 / 2.3 / 3.6 / 6.6 relaxations per vertex.
constexpr double ASYNC_DELTA_FACTOR = 8.0;
static gb_info default_delta(gb_context *ctx, const gb_matrix *A, int schedule, uint64_t *delta) {
    double mean = 1.0;
    GB_CHECK(matrix_mean_weight(ctx, A, &mean));
    const double avg_deg = A->nrows ? (double)A->nvals / (double)A->nrows : 1.0;
    const double f = schedule == GB_SCHED_ASYNC ? ASYNC_DELTA_FACTOR : 32.0;
    const double dl = f * mean * (avg_deg > 1.0 ? avg_deg : 1.0);
    *delta = dl < 1.0 ? 1u : (dl > 2147483646.0 ? 2147483646ull : (uint64_t)(dl + 0.5));
    return GB_SUCCESS;
}

static gb_info relax_run(gb_context *ctx, const gb_matrix *A, bool weighted, uint32_t src, uint32_t *out, gb_mem mem,
                         const gb_desc *desc, uint32_t *iterations, gb_bfs_stats *stats, const char *who) {
    if (stats) memset(stats, 0, sizeof(*stats));
    if (!ctx || !A || !out) return fail(GB_NULL_POINTER, "%s: NULL argument", who);
    if (!A->built) return fail(GB_INVALID_VALUE, "%s: matrix not built", who);
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "%s: matrix must be square", who);
    if (A->nrows == 0) return GB_SUCCESS;
    if (weighted) {
        if (src >= A->nrows) return fail(GB_INVALID_INDEX, "%s: source %u out of range", who, src);
        if (!A->has_vals || A->type != GB_UINT32) return fail(GB_DOMAIN_MISMATCH, "%s: needs uint32 edge weights", who);
    }
    GB_CUDA(cudaSetDevice(ctx->device));
    uint32_t *visited, *front, *q, *qp, *qr;
    BfsState *st;
    void *cl_state = nullptr;
    GB_CHECK(bfs_workspace_raw(ctx, A->nrows, &visited, &front, &q, &qp, &qr, &st, &cl_state));
    rlx::RelaxArgs a;
    a.n = A->nrows;
    a.nwords = (A->nrows + 31) / 32;
    a.m = A->nvals;
    a.rp_out = A->rowptr; a.ci_out = A->colidx; a.w_out = weighted ? (const uint32_t *)A->vals : nullptr;
    a.rp_in = A->has_csc ? A->colptr : nullptr;
    a.ci_in = A->has_csc ? A->rowidx : nullptr;
    a.w_in = (weighted && A->has_csc) ? (const uint32_t *)A->cvals : nullptr;
    a.csr_is_csc = A->csc_alias;
    a.weighted = weighted;
    a.src = src;
    a.all_active = !weighted;
    Scratch ob(ctx);
    a.val = out;
    if (mem == GB_HOST) {
        GB_CHECK(ob.alloc((size_t)A->nrows * 4 + 16));
        a.val = ob.as<uint32_t>();
    }
    // SSSP in a single cluster only when the descriptor asks for it: on
    // weighted graphs the frontiers of improved vertices stay large even
    // where BFS frontiers are small, and the whole GPU relaxes them faster
    const int sch = desc ? desc->schedule : GB_SCHED_AUTO;
    if (weighted && sch == GB_SCHED_CLUSTER && bfs_cluster_available(ctx)) {
        Scratch stamp(ctx);
        GB_CHECK(stamp.alloc((size_t)A->nrows * 4 + 16));
        GB_CHECK(sssp_cluster_launch(ctx, A, src, a.val, stamp.as<uint32_t>(), q, q + A->nrows + 1, cl_state));
        if (mem == GB_HOST)
            GB_CUDA(cudaMemcpyAsync(out, a.val, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
        uint32_t it = 0;
        const gb_info r = cluster_iterations(ctx, cl_state, &it);
        if (iterations) *iterations = it;
        if (stats) {
            stats->depth = it;
            stats->push_levels = it;
            stats->schedule = GB_SCHED_CLUSTER;
        }
        return r;
    }
    if (weighted && sch == GB_SCHED_ASYNC) {
        // barrier-free relaxation inside distance buckets (async_relax.cu)
        uint64_t delta = 0;
        const int dd = desc ? desc->sssp_delta : 0;
        if (dd == 0) GB_CHECK(default_delta(ctx, A, GB_SCHED_ASYNC, &delta));
        else if (dd < 0x7fffffff) delta = (uint64_t)dd;
        gb_bfs_stats hs;
        const gb_info r = async_relax_run(ctx, A, 0, src, a.val, nullptr, delta, &hs, who);
        if (stats) *stats = hs;
        if (iterations) *iterations = hs.depth;
        GB_CHECK(r);
        if (mem == GB_HOST) {
            GB_CUDA(cudaMemcpyAsync(out, a.val, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
            GB_CHECK(sync(ctx));
        }
        return GB_SUCCESS;
    }
    for (int k = 0; k < 3; ++k) a.front[k] = front + (size_t)k * a.nwords;
    a.q[0] = q; a.q[1] = q + A->nrows + 1;
    a.qp[0] = qp; a.qp[1] = qp + A->nrows + 1;
    a.qr[0] = qr; a.qr[1] = qr + A->nrows + 1;
    a.ebits = 64 - bits_for((uint64_t)A->nrows + 1);
    a.emask = (a.ebits >= 64) ? ~0ull : ((1ull << a.ebits) - 1);
    a.mode = desc ? desc->direction : GB_AUTO;
    a.beta = (desc && desc->beta > 0) ? (uint32_t)desc->beta : 10u;
    a.st = st;
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 300000000000ull;
    a.hub_list = a.hub_pre = nullptr;
    a.nhub = 0;
    a.hub_edges = 0;
    // SSSP bucket width: the descriptor's, or, by default, 32 times the mean
    // weight times the mean degree. Narrow buckets save repeated relaxations
    // but add synchronous steps (a step per bucket and per hop inside it);
    // measured on the weighted 4096^2 grid (mean weight 500, degree 3.6),
    // widths of 16,000 to 64,000 run 115-122 ms against 353 ms for no buckets
    // and 460 ms for a width of 278, and on R-MAT s22 (weights 1-255, degree
    // 30.6) every width from 16 up is within 15% of no buckets. A forced
    // pull, or a width of 2^31 - 1 or more, is the plain changed-set iteration.
    a.delta = 0;
    a.far = nullptr;
    Scratch farb(ctx);
    if (weighted && a.mode != GB_PULL) {
        const int dd = desc ? desc->sssp_delta : 0;
        if (dd == 0) {
            GB_CHECK(default_delta(ctx, A, GB_SCHED_GRID, &a.delta));
        } else if (dd < 0x7fffffff) {
            a.delta = (uint64_t)dd;
        }
        if (a.delta) {
            GB_CHECK(farb.alloc((size_t)a.nwords * 4 + 16));
            a.far = farb.as<uint32_t>();
        }
    }
    if (A->has_csc) {
        GB_CHECK(matrix_hubs(A, rlx::RPULL_HUB));
        a.hub_list = A->hub_list;
        a.hub_pre = A->hub_pre;
        a.nhub = A->nhub;
        a.hub_edges = A->hub_edges;
    }
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rlx::k_relax, rlx::BLOCK, 0));
    if (occ < 1) return fail(GB_PANIC, "%s: kernel cannot be resident", who);
    void *args[] = {&a};
    int span = prof_begin(ctx, weighted ? "sssp" : "cc");
    int grid = occ * ctx->num_sms;
    if (ctx->grid_limit > 0 && ctx->grid_limit < grid) grid = ctx->grid_limit;
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)rlx::k_relax, dim3(grid), dim3(rlx::BLOCK), args, 0,
                                        ctx->stream));
    prof_end(ctx, span);
    BfsResult hs;
    GB_CUDA(cudaMemcpyAsync(&hs, &st->res, sizeof(BfsResult), cudaMemcpyDeviceToHost, ctx->stream));
    if (mem == GB_HOST) GB_CUDA(cudaMemcpyAsync(out, a.val, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (iterations) *iterations = hs.depth;
    if (stats) {
        stats->depth = hs.depth;
        stats->push_levels = hs.push_levels;
        stats->pull_levels = hs.pull_levels;
        stats->status = (uint32_t)hs.err;
        stats->frontier_edges = hs.frontier_edges;
        stats->alg_bytes = (uint64_t)hs.alg_bytes;
        const uint32_t nl = hs.depth < GB_TRACE_LEVELS ? hs.depth : GB_TRACE_LEVELS;
        stats->trace_len = nl;
        for (uint32_t l = 0; l < nl; ++l) {
            stats->trace_dir[l] = hs.dir_log[l];
            stats->trace_vertices[l] = hs.lv_cnt[l];
            stats->trace_edges[l] = hs.lv_fe[l];
            const uint64_t t1 = (l + 1 < GBX_MAX_LEVEL_LOG) ? hs.lv_ns[l + 1] : hs.lv_ns[l];
            stats->trace_us[l] = (float)((t1 - hs.lv_ns[l]) * 1e-3);
        }
        stats->schedule = GB_SCHED_GRID;
    }
    if (hs.err) return fail(GB_TIMEOUT, "%s: a bounded device wait or the time budget ran out", who);
    return GB_SUCCESS;
}

}  // namespace gbx

extern "C" {

gb_info gb_sssp(gb_context *ctx, const gb_matrix *A, uint32_t src, uint32_t *dist, gb_mem mem, const gb_desc *desc,
                uint32_t *iterations, gb_bfs_stats *stats) {
    return relax_run(ctx, A, true, src, dist, mem, desc, iterations, stats, "gb_sssp");
}

gb_info gb_cc(gb_context *ctx, const gb_matrix *A, uint32_t *labels, gb_mem mem, uint32_t *iterations,
              gb_bfs_stats *stats) {
    return relax_run(ctx, A, false, 0, labels, mem, nullptr, iterations, stats, "gb_cc");
}

gb_info gb_cc_async(gb_context *ctx, const gb_matrix *A, uint32_t *labels, gb_mem mem, uint32_t label_bucket,
                    gb_bfs_stats *stats) {
    if (stats) memset(stats, 0, sizeof(*stats));
    if (!ctx || !A || !labels) return fail(GB_NULL_POINTER, "gb_cc_async: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_cc_async: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_cc_async: matrix must be square");
    if (A->nrows == 0) return GB_SUCCESS;
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch ob(ctx);
    uint32_t *out = labels;
    if (mem == GB_HOST) {
        GB_CHECK(ob.alloc((size_t)A->nrows * 4 + 16));
        out = ob.as<uint32_t>();
    }
    // label buckets: labels below the bound spread first, the others wait as
    // far vertices (the near-far discipline of SSSP on label values)
    uint64_t bucket = label_bucket;
    if (bucket == 0) bucket = cc_async_default_bucket(A->nrows);
    if (bucket >= A->nrows) bucket = 0;   // one phase
    GB_CHECK(async_relax_run(ctx, A, 2, 0, out, nullptr, bucket, stats, "gb_cc_async"));
    if (mem == GB_HOST) {
        GB_CUDA(cudaMemcpyAsync(labels, out, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CHECK(sync(ctx));
    }
    return GB_SUCCESS;
}

}  // extern "C"
