// Multi-source BFS as a Boolean SpMM over 64-bit bit-packed frontiers
// (Section 3.3: mxm is a traversal from several independent sets of active
// vertices at once; Section 9 proposes direction optimisation for it). Up to
// 64 BFS share one launch: bit q of F[v] says that v is on source q's
// frontier. Per level, either
//   push: every vertex u on some frontier ORs F[u] into the next-frontier
//         word of each out-neighbour v, minus the bits v already has
//         (merge-path over the frontier list's out-edges), or
//   pull: every vertex v that some live source has not reached ORs the
//         frontier words of its in-neighbours, stopping as soon as all live
//         sources are covered (the Boolean early exit, per 64 searches),
// chosen by the rule of Table 9 on the union frontier's edge count. The
// visited words are merged one level late (V | F is the visited set), so a
// level needs a single grid barrier. Levels are first recorded per vertex:
// byte q of a vertex's 64-byte record is 1 + its level for source q (0 =
// not reached, 255 = level 254 or more, written to the output directly), so
// the stores of a level stay inside one record per vertex; the last pass
// turns the records into the k x n output with coalesced row stores.
#include "common.cuh"
#include "bfs_common.cuh"
#include "frontier.cuh"

using namespace gbx;

namespace gbx {
namespace msk {
using namespace fr;

struct MsArgs {
    const uint32_t *rp_out, *ci_out;
    const uint32_t *rp_in, *ci_in;
    bool csr_is_csc;
    uint32_t n, nwords;
    uint64_t m;
    uint32_t k;                        // sources of this launch (<= 64 * words per vertex)
    unsigned long long live[4];        // bits of the k sources, word by word
    const uint32_t *srcs;
    int32_t *levels;                   // k x n
    unsigned long long *rec;           // per vertex, 8 words per 64 sources: one level byte per source
    unsigned long long *V;             // visited (NW words per vertex), merged one level late
    unsigned long long *F[3];          // frontier words (NW per vertex), rotating
    uint32_t *mark[3];                 // NW > 1: a bit per vertex set by whoever adds it to the next frontier
    uint32_t *front[3];                // unused by this kernel (frontier helpers' interface)
    uint32_t *q[2], *qp[2], *qr[2];
    int ebits;
    unsigned long long emask;
    int mode;
    uint32_t beta;
    BfsState *st;
    uint64_t timeout_ns, total_limit_ns;
    const uint32_t *hub_list, *hub_pre;   // in-rows longer than GBX_HUB_MIN_LEN and their edge prefix
    uint32_t nhub;
    uint64_t hub_edges;
};

__device__ __forceinline__ unsigned long long ldcg64(const unsigned long long *p) { return __ldcg(p); }

// NW 64-bit words of source bits (bit q of word w: source 64 w + q).
template <int NW>
struct Bits {
    unsigned long long w[NW];
    __device__ __forceinline__ static Bits zero() {
        Bits r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.w[i] = 0ull;
        return r;
    }
    __device__ __forceinline__ bool any() const {
        unsigned long long x = 0;
#pragma unroll
        for (int i = 0; i < NW; ++i) x |= w[i];
        return x != 0ull;
    }
    __device__ __forceinline__ Bits operator|(const Bits &o) const {
        Bits r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.w[i] = w[i] | o.w[i];
        return r;
    }
    __device__ __forceinline__ Bits operator&(const Bits &o) const {
        Bits r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.w[i] = w[i] & o.w[i];
        return r;
    }
    __device__ __forceinline__ Bits andnot(const Bits &o) const {   // this & ~o
        Bits r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.w[i] = w[i] & ~o.w[i];
        return r;
    }
    __device__ __forceinline__ bool operator==(const Bits &o) const {
        unsigned long long x = 0;
#pragma unroll
        for (int i = 0; i < NW; ++i) x |= w[i] ^ o.w[i];
        return x == 0ull;
    }
    __device__ __forceinline__ bool operator!=(const Bits &o) const { return !(*this == o); }
    __device__ __forceinline__ Bits shfl(int l) const {
        Bits r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.w[i] = __shfl_sync(0xffffffffu, w[i], l);
        return r;
    }
    __device__ __forceinline__ Bits warp_or() const {
        Bits r = *this;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < NW; ++i) r.w[i] |= __shfl_xor_sync(0xffffffffu, r.w[i], o);
        return r;
    }
};

// the words of vertex v in an array of NW words per vertex (L2 reads: other
// SMs write them during a level)
template <int NW>
__device__ __forceinline__ Bits<NW> ldbits(const unsigned long long *p, uint64_t v) {
    Bits<NW> r;
    if constexpr (NW == 1) {
        r.w[0] = __ldcg(&p[v]);
    } else {
        const ulonglong2 *p2 = reinterpret_cast<const ulonglong2 *>(p + v * NW);
#pragma unroll
        for (int i = 0; i < NW / 2; ++i) {
            const ulonglong2 x = __ldcg(&p2[i]);
            r.w[2 * i] = x.x;
            r.w[2 * i + 1] = x.y;
        }
    }
    return r;
}
template <int NW>
__device__ __forceinline__ void stbits(unsigned long long *p, uint64_t v, const Bits<NW> &b) {
#pragma unroll
    for (int i = 0; i < NW; ++i) p[v * NW + i] = b.w[i];
}
template <int NW>
__device__ __forceinline__ Bits<NW> live_bits(const MsArgs &a) {
    Bits<NW> r;
#pragma unroll
    for (int i = 0; i < NW; ++i) r.w[i] = a.live[i];
    return r;
}

// ORs nb into the next-frontier words of v; true for exactly one caller per
// vertex and level: the one that added v to the next frontier (with one
// word, the one that turned it nonzero; with more, the one that set v's
// bit in the level's mark bitmap)
template <int NW>
__device__ __forceinline__ bool or_next(const MsArgs &a, unsigned long long *Fn, uint32_t *mark, uint64_t v,
                                        const Bits<NW> &nb) {
    if constexpr (NW == 1) {
        return atomicOr(&Fn[v], nb.w[0]) == 0ull;
    } else {
#pragma unroll
        for (int i = 0; i < NW; ++i)
            if (nb.w[i]) atomicOr(&Fn[v * NW + i], nb.w[i]);
        const uint32_t bit = 1u << (v & 31);
        return !(atomicOr(&mark[v >> 5], bit) & bit);
    }
}

// bit i of m -> 0xff in byte i
__device__ __forceinline__ unsigned long long spread8(unsigned long long m) {
    m &= 0xffull;
    m = (m | (m << 28)) & 0x0000000F0000000Full;
    m = (m | (m << 14)) & 0x0003000300030003ull;
    m = (m | (m << 7)) & 0x0101010101010101ull;
    return m * 0xffull;
}

// records level d for the sources in f at vertex v: one 64-bit atomicOr per
// group of eight sources (the bytes it sets are still zero, each (q, v) is
// reached once); from level 254 on the output is written directly
template <int NW>
__device__ __forceinline__ void record_levels(const MsArgs &a, uint64_t v, const Bits<NW> &f, int d) {
    if (!f.any()) return;
    const unsigned long long b = d < 254 ? (unsigned long long)(d + 1) * 0x0101010101010101ull : ~0ull;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const unsigned long long m = (f.w[i] >> (8 * c)) & 0xffull;
            if (m) atomicOr(&a.rec[(v * NW + i) * 8 + c], spread8(m) & b);
        }
        if (d >= 254)
            for (unsigned long long u = f.w[i]; u; u &= u - 1)
                a.levels[(uint64_t)(64 * i + __ffsll((long long)u) - 1) * a.n + v] = d;
    }
}

// Builds the list form (vertex, out-degree prefix, row start) of the
// frontier F_d from its words; one atomicAdd per 256 vertices.
template <int NW>
__device__ void ms_compact(const MsArgs &a, Smem &sm, int d) {
    const unsigned long long *F = a.F[d % 3];
    uint32_t *Q = a.q[d & 1], *P = a.qp[d & 1], *R = a.qr[d & 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t vb0 = (uint64_t)a.n * blockIdx.x / gridDim.x;
    const uint64_t vb1 = (uint64_t)a.n * (blockIdx.x + 1) / gridDim.x;
    for (uint64_t c = vb0; c < vb1; c += BLOCK) {
        const uint64_t v = c + threadIdx.x;
        bool on = v < vb1 && ldbits<NW>(F, v).any();
        uint32_t r0 = 0, deg = 0;
        if (on) { r0 = __ldg(&a.rp_out[v]); deg = __ldg(&a.rp_out[v + 1]) - r0; }
        uint32_t tc, td;
        uint32_t ec = dev::warp_exclusive_sum<uint32_t>(on ? 1u : 0u, &tc);
        uint32_t ed = dev::warp_exclusive_sum<uint32_t>(deg, &td);
        if (lane == 0) { sm.stage.wcnt[warp] = tc; sm.stage.wdeg[warp] = td; }
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
        if (on) {
            uint32_t pos = (uint32_t)(sm.stage.base >> a.ebits) + sm.stage.wcnt[warp] + ec;
            Q[pos] = (uint32_t)v;
            P[pos] = (uint32_t)(sm.stage.base & a.emask) + sm.stage.wdeg[warp] + ed;
            R[pos] = r0;
        }
        __syncthreads();
    }
}

// pull: lane per vertex, 2 vertices per lane in flight. A lane scans a
// row of up to 32 in-neighbours alone, four independent loads at a time;
// longer rows continue warp-cooperatively (128 neighbours per step), and
// hub rows (longer than GBX_HUB_MIN_LEN) are left to ms_pull_hubs. Every
// vertex also merges its frontier bits into its visited words here, and
// sources whose bits are all covered stop the scan (the Boolean early exit
// per 64 NW searches).
template <int NW>
__device__ void ms_pull(const MsArgs &a, int d, uint32_t *cnt_out, uint32_t *deg_out, unsigned long long *exam_out) {
    const unsigned long long *F = a.F[d % 3];
    unsigned long long *Fn = a.F[(d + 1) % 3];
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
    const uint64_t ngroups = (a.n + 63) / 64;
    const Bits<NW> live = live_bits<NW>(a);
    uint32_t mycnt = 0, mydeg = 0;
    unsigned long long myexam = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * WARPS + warp; g < ngroups; g += nwarps) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint64_t v = g * 64 + j * 32 + lane;
            const bool valid = v < a.n;
            Bits<NW> f = Bits<NW>::zero(), vis = live;
            uint32_t b = 0, e = 0;
            if (valid) {
                f = ldbits<NW>(F, v);
                vis = ldbits<NW>(a.V, v) | f;
                if (f.any()) stbits<NW>(a.V, v, vis);
                b = __ldg(&a.rp_in[v]);
                e = __ldg(&a.rp_in[v + 1]);
            }
            if (valid) record_levels<NW>(a, v, f, d);
            const bool hub = e - b > GBX_HUB_MIN_LEN;
            Bits<NW> acc = Bits<NW>::zero();
            const bool need = valid && vis != live && !hub;
            uint32_t p = b;
            if (need) {
                const uint32_t lim = e - b > 32 ? b + 32 : e;
                for (; p < lim; p += 4) {
                    uint32_t u[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) u[k] = p + k < lim ? fr::ld_stream(&a.ci_in[p + k]) : 0u;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (p + k < lim) acc = acc | ldbits<NW>(F, u[k]);
                    myexam += lim - p < 4 ? lim - p : 4;
                    if ((acc | vis) == live) { p = e; break; }
                }
                if (p > lim) p = lim;
            }
            uint32_t coop = __ballot_sync(full, need && p < e);
            while (coop) {
                const int l = __ffs(coop) - 1;
                coop &= coop - 1;
                const uint32_t pb = __shfl_sync(full, p, l), pe = __shfl_sync(full, e, l);
                const Bits<NW> lv = vis.shfl(l);
                Bits<NW> la = acc.shfl(l);
                for (uint32_t q0 = pb; q0 < pe; q0 += 128) {
                    Bits<NW> x = Bits<NW>::zero();
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t q = q0 + k * 32 + lane;
                        if (q < pe) x = x | ldbits<NW>(F, fr::ld_stream(&a.ci_in[q]));
                    }
                    la = la | x.warp_or();
                    if (lane == 0) myexam += pe - q0 < 128 ? pe - q0 : 128;
                    if ((la | lv) == live) break;
                }
                if (lane == l) acc = la;
            }
            const Bits<NW> nb = acc.andnot(vis);
            if (nb.any()) {
                stbits<NW>(Fn, v, nb);
                mycnt += 1;
                mydeg += a.csr_is_csc ? e - b : __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
            }
        }
    }
    *cnt_out += mycnt;
    *deg_out += mydeg;
    *exam_out += myexam;
}

// pull, hub rows: the hubs' in-edges are cut into one contiguous range per
// warp (equal lengths over the whole grid). A warp finds the hub of its
// range start once, then walks the range 32 edges per step (a step spans at
// most two hubs, as every hub has more than GBX_HUB_MIN_LEN edges), ORs the
// frontier words of the step's edges per hub and sets the new bits of the
// hub's next-frontier words with atomicOr; it jumps past the rest of a
// hub once every live source has reached or found it. A hub is counted by
// the caller that adds it to the next frontier (or_next). The OR over a
// hub's in-edges is the same whichever warps its edges fall to.
template <int NW>
__device__ void ms_pull_hubs(const MsArgs &a, int d, uint32_t *cnt_out, uint32_t *deg_out,
                             unsigned long long *exam_out) {
    if (!a.nhub) return;
    const unsigned long long *F = a.F[d % 3];
    unsigned long long *Fn = a.F[(d + 1) % 3];
    uint32_t *mark = a.mark[(d + 1) % 3];
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
    const uint64_t wid = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    const uint64_t X0 = a.hub_edges * wid / nwarps, X1 = a.hub_edges * (wid + 1) / nwarps;
    const Bits<NW> live = live_bits<NW>(a);
    uint32_t mycnt = 0, mydeg = 0;
    if (X0 < X1) {
        uint32_t h = 0, hi = a.nhub;   // last h with hub_pre[h] <= X0
        while (hi - h > 1) {
            const uint32_t mid = (h + hi) >> 1;
            if ((uint64_t)__ldg(&a.hub_pre[mid]) <= X0) h = mid; else hi = mid;
        }
        uint64_t x0 = X0;
        while (x0 < X1) {
            const uint64_t hb = __ldg(&a.hub_pre[h]);
            const uint64_t he = h + 1 < a.nhub ? (uint64_t)__ldg(&a.hub_pre[h + 1]) : a.hub_edges;
            if (x0 >= he) { ++h; continue; }
            const uint32_t v = __ldg(&a.hub_list[h]);
            const Bits<NW> vis = ldbits<NW>(a.V, v) | ldbits<NW>(F, v);
            if (((ldbits<NW>(Fn, v) | vis) & live) == live) {   // nothing left to find here
                x0 = he;
                ++h;
                continue;
            }
            // one step: the edges [x0, x0+32) of this hub (the part past he is the next hub's)
            const uint64_t x = x0 + lane;
            const bool mine = x < X1 && x < he;
            Bits<NW> bits = Bits<NW>::zero();
            if (mine) {
                const uint32_t p = __ldg(&a.rp_in[v]) + (uint32_t)(x - hb);
                bits = ldbits<NW>(F, fr::ld_stream(&a.ci_in[p]));
            }
            bits = bits.warp_or().andnot(vis) & live;
            if (lane == 0) *exam_out += (X1 < he ? X1 : he) - x0 < 32 ? (X1 < he ? X1 : he) - x0 : 32;
            if (lane == 0 && bits.any()) {
                const Bits<NW> cur = ldbits<NW>(Fn, v);
                if ((cur | bits) != cur && or_next<NW>(a, Fn, mark, v, bits)) {
                    mycnt += 1;
                    mydeg += a.csr_is_csc ? (uint32_t)(he - hb) : __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
                }
            }
            x0 = x0 + 32 < he ? x0 + 32 : he;
        }
    }
    *cnt_out += mycnt;
    *deg_out += mydeg;
}

template <int NW>
__global__ void __launch_bounds__(BLOCK, NW == 1 ? 5 : (NW == 2 ? 4 : 3)) k_msbfs(MsArgs a) {
    __shared__ Smem sm;
    __shared__ uint32_t s_cnt, s_deg;
    __shared__ unsigned long long s_exam;
    const uint32_t nthreads = gridDim.x * BLOCK;
    const uint32_t tid = blockIdx.x * BLOCK + threadIdx.x;
    BfsState *st = a.st;
    BfsResult *res = &st->res;
    for (uint64_t x = tid; x < (uint64_t)a.n * NW; x += nthreads) {
        a.V[x] = 0ull;
        a.F[0][x] = 0ull;
        a.F[1][x] = 0ull;
        a.F[2][x] = 0ull;
    }
    if (NW > 1)
        for (uint64_t w = tid; w < a.nwords; w += nthreads) {
            a.mark[0][w] = 0u;
            a.mark[1][w] = 0u;
            a.mark[2][w] = 0u;
        }
    {
        ulonglong2 *r2 = reinterpret_cast<ulonglong2 *>(a.rec);
        for (uint64_t x = tid; x < (uint64_t)a.n * 4 * NW; x += nthreads) r2[x] = make_ulonglong2(0ull, 0ull);
    }
    bool ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    if (ok && tid == 0) {
        memset(res, 0, sizeof(BfsResult));
        uint32_t cnt = 0, deg = 0;
        for (uint32_t q = 0; q < a.k; ++q) {
            const uint32_t v = a.srcs[q];
            unsigned long long any = 0;
#pragma unroll
            for (int i = 0; i < NW; ++i) any |= a.F[0][(uint64_t)v * NW + i];
            a.F[0][(uint64_t)v * NW + q / 64] |= 1ull << (q % 64);
            if (!any) {
                uint32_t r0 = __ldg(&a.rp_out[v]);
                a.q[0][cnt] = v;
                a.qp[0][cnt] = deg;
                a.qr[0][cnt] = r0;
                deg += __ldg(&a.rp_out[v + 1]) - r0;
                ++cnt;
            }
        }
        st->qstate[0] = ((unsigned long long)cnt << a.ebits) | deg;
    }
    if (ok) ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    const uint64_t t_start = dev::globaltimer_ns();
    bool list_valid = true;
    // algorithmic bytes (thread 0 of block 0): the k x n level writes, then per
    // push level 8 per frontier vertex (list entry, row start), 4 per frontier
    // out-edge (index) + 8 NW per out-edge (the target's visited words), per
    // pull level 8 (n + 1) row offsets + 8 NW n (frontier and visited words)
    // + (4 + 8 NW) per examined in-edge (index, the neighbour's frontier
    // words); per level 8 NW per vertex of the next frontier (its words)
    double alg = 4.0 * a.k * a.n;
    bool prev_pull = false;
    uint32_t prev_cnt = 0;
    uint64_t prev_fe = 0;
    int d = 0;
    for (; ok; ++d) {
        if (threadIdx.x == 0)
            sm.qs = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(st->qstate[d % 3])
                        .load(cuda::memory_order_relaxed);
        __syncthreads();
        const unsigned long long qs = sm.qs;
        __syncthreads();
        const uint32_t cnt = (uint32_t)(qs >> a.ebits);
        const uint64_t fe = qs & a.emask;
        if (tid == 0 && d > 0) {
            const double w8 = 8.0 * NW;
            if (prev_pull) {
                const unsigned long long ex = __ldcg(&st->exam[(d - 1) % 3]);
                res->edges_examined += ex;
                alg += 8.0 * (a.n + 1.0) + w8 * a.n + (4.0 + w8) * (double)ex;
            } else {
                res->edges_examined += prev_fe;
                alg += 8.0 * prev_cnt + (4.0 + w8) * (double)prev_fe;
            }
            alg += w8 * cnt;
        }
        if (cnt == 0) break;
        if (d > (int)a.n || (threadIdx.x == 0 && dev::globaltimer_ns() - t_start > a.total_limit_ns))
            atomicCAS(&st->err, 0, (int)GB_TIMEOUT);
        const bool pull = a.rp_in && a.mode != GB_PUSH && (a.mode == GB_PULL || fe * (uint64_t)a.beta > a.m);
        if (tid == 0) {
            if (d < GBX_MAX_LEVEL_LOG) {
                res->dir_log[d] = pull ? 2 : 1;
                res->lv_cnt[d] = cnt;
                res->lv_fe[d] = fe;
                res->lv_ns[d] = dev::globaltimer_ns();
            }
            if (pull) res->pull_levels++; else res->push_levels++;
            res->frontier_edges += fe;
            res->reached += cnt;
            st->qstate[(d + 2) % 3] = 0;
            st->cstate[(d + 2) % 3] = 0;
            st->exam[(d + 2) % 3] = 0;
            prev_pull = pull;
            prev_cnt = cnt;
            prev_fe = fe;
        }
        unsigned long long *Fclr = a.F[(d + 2) % 3];
        for (uint64_t x = tid; x < (uint64_t)a.n * NW; x += nthreads) Fclr[x] = 0ull;
        if (NW > 1) {
            uint32_t *Mclr = a.mark[(d + 2) % 3];
            for (uint64_t w = tid; w < a.nwords; w += nthreads) Mclr[w] = 0u;
        }
        if (pull) {
            if (threadIdx.x == 0) { s_cnt = 0; s_deg = 0; s_exam = 0; }
            __syncthreads();
            uint32_t c = 0, dg = 0;
            unsigned long long ex = 0;
            ms_pull<NW>(a, d, &c, &dg, &ex);
            ms_pull_hubs<NW>(a, d, &c, &dg, &ex);
            c = dev::warp_sum<uint32_t>(c);
            dg = dev::warp_sum<uint32_t>(dg);
            ex = dev::warp_sum<unsigned long long>(ex);
            if ((threadIdx.x & 31) == 0) {
                if (c) { atomicAdd(&s_cnt, c); atomicAdd(&s_deg, dg); }
                if (ex) atomicAdd(&s_exam, ex);
            }
            __syncthreads();
            if (threadIdx.x == 0 && s_cnt)
                atomicAdd(&st->qstate[(d + 1) % 3], ((unsigned long long)s_cnt << a.ebits) | s_deg);
            if (threadIdx.x == 0 && s_exam) atomicAdd(&st->exam[d % 3], s_exam);
            list_valid = false;
        } else {
            if (!list_valid) {
                ms_compact<NW>(a, sm, d);
                if (!dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns)) { ok = false; break; }
            }
            // merge this level's frontier into the visited words and write its levels
            {
                const uint32_t *Q = a.q[d & 1];
                const uint64_t nw = ((uint64_t)cnt + 31) / 32;
                for (uint64_t wi = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); wi < nw;
                     wi += (uint64_t)gridDim.x * WARPS) {
                    uint64_t x = wi * 32 + (threadIdx.x & 31);
                    bool valid = x < cnt;
                    uint32_t v = valid ? ldcg(&Q[x]) : 0u;
                    if (valid) {
                        const Bits<NW> f = ldbits<NW>(a.F[d % 3], v);
#pragma unroll
                        for (int i = 0; i < NW; ++i)
                            if (f.w[i]) atomicOr(&a.V[(uint64_t)v * NW + i], f.w[i]);
                        record_levels<NW>(a, v, f, d);
                    }
                }
            }
            const unsigned long long *F = a.F[d % 3];
            unsigned long long *Fn = a.F[(d + 1) % 3];
            uint32_t *mark = a.mark[(d + 1) % 3];
            push_edges(a, sm, d, cnt, fe, [&](uint32_t u, uint32_t v, uint32_t, uint32_t *, uint32_t *deg, uint32_t *r0) {
                const Bits<NW> nb = ldbits<NW>(F, u).andnot(ldbits<NW>(a.V, v) | ldbits<NW>(F, v));
                if (!nb.any()) return false;
                const Bits<NW> cur = ldbits<NW>(Fn, v);
                if ((cur | nb) == cur) return false;
                if (!or_next<NW>(a, Fn, mark, v, nb)) return false;
                *r0 = __ldg(&a.rp_out[v]);
                *deg = __ldg(&a.rp_out[v + 1]) - *r0;
                return true;
            });
            list_valid = true;
        }
        ok = dev::grid_sync(&st->bar, gridDim.x, &st->err, a.timeout_ns);
    }
    // ---- the records become the output: lane per vertex, each row q stored
    // for 32 consecutive vertices at once; (source, vertex) pairs never
    // reached get -1, pairs at level 254 or more are already written
    if (ok) {
        const int lane = threadIdx.x & 31;
        const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
        const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(a.rec);
        for (uint64_t g = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); g * 32 < a.n; g += nwarps) {
            const uint64_t v = g * 32 + lane;
            const bool valid = v < a.n;
#pragma unroll 1
            for (int i = 0; i < NW; ++i) {
                if ((uint32_t)(64 * i) >= a.k) break;
                unsigned long long w[8];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const ulonglong2 x = valid ? __ldcg(&r2[(v * NW + i) * 4 + c]) : make_ulonglong2(0ull, 0ull);
                    w[2 * c] = x.x;
                    w[2 * c + 1] = x.y;
                }
#pragma unroll
                for (int q = 0; q < 64; ++q) {
                    if ((uint32_t)(64 * i + q) >= a.k) break;
                    const uint32_t byte = (uint32_t)(w[q >> 3] >> (8 * (q & 7))) & 0xffu;
                    if (valid && byte != 0xffu)
                        a.levels[(uint64_t)(64 * i + q) * a.n + v] = byte ? (int32_t)byte - 1 : -1;
                }
            }
        }
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
            for (int k2 = 0; k2 < 3; ++k2) { st->qstate[k2] = 0; st->exam[k2] = 0; st->cstate[k2] = 0; }
            __threadfence();
            st->bar.exits = 0;
        }
    }
}

}  // namespace msk

struct MsWorkspace {
    uint32_t n = 0, nw = 0;
    unsigned long long *V = nullptr, *F = nullptr, *rec = nullptr;
    uint32_t *mark = nullptr;
    uint32_t *q = nullptr, *qp = nullptr, *qr = nullptr;
    BfsState *st = nullptr;
};
static std::mutex g_ms_mu;
static std::unordered_map<gb_context *, MsWorkspace> g_ms;

static void ms_free(gb_context *ctx, MsWorkspace &w) {
    dfree(ctx, w.V); dfree(ctx, w.F); dfree(ctx, w.q); dfree(ctx, w.qp); dfree(ctx, w.qr); dfree(ctx, w.st);
    dfree(ctx, w.rec); dfree(ctx, w.mark);
    w = MsWorkspace();
}

// Working arrays for n vertices and nw words of source bits per vertex.
static gb_info ms_workspace(gb_context *ctx, uint32_t n, uint32_t nw, MsWorkspace **out) {
    std::lock_guard<std::mutex> g(g_ms_mu);
    MsWorkspace &w = g_ms[ctx];
    if (w.n < n || w.nw < nw || !w.st) {
        const uint32_t nn = n > w.n ? n : w.n, ww = nw > w.nw ? nw : w.nw;
        ms_free(ctx, w);
        const size_t words = (size_t)nn * ww;
        GB_CHECK(dalloc_t(ctx, &w.V, words + 4));
        GB_CHECK(dalloc_t(ctx, &w.rec, 8 * words + 8));
        GB_CHECK(dalloc_t(ctx, &w.F, 3 * words + 12));
        GB_CHECK(dalloc_t(ctx, &w.mark, 3ull * ((nn + 31) / 32) + 3));
        GB_CHECK(dalloc_t(ctx, &w.q, 2ull * nn + 2));
        GB_CHECK(dalloc_t(ctx, &w.qp, 2ull * nn + 2));
        GB_CHECK(dalloc_t(ctx, &w.qr, 2ull * nn + 2));
        GB_CHECK(dalloc_t(ctx, &w.st, 1));
        GB_CHECK(memset_async(ctx, w.st, 0, sizeof(BfsState)));
        w.n = nn;
        w.nw = ww;
    }
    *out = &w;
    return GB_SUCCESS;
}

void ms_workspace_release(gb_context *ctx) {
    std::lock_guard<std::mutex> g(g_ms_mu);
    auto it = g_ms.find(ctx);
    if (it == g_ms.end()) return;
    ms_free(ctx, it->second);
    g_ms.erase(it);
}

// Sources one launch serves: 64 per word of source bits, up to 4 words.
constexpr uint32_t MS_MAX_SOURCES = 256;
static uint32_t msk_max_sources() { return MS_MAX_SOURCES; }

// Launches a multi-source BFS (k <= MS_MAX_SOURCES sources on the device)
// into levels (device, k x n): one word of source bits per vertex for up to
// 64 sources, two for up to 128, four for up to 256.
gb_info msbfs_launch(gb_context *ctx, const gb_matrix *A, const uint32_t *d_srcs, uint32_t k, int32_t *levels,
                     const gb_desc *desc, BfsResult *res_out) {
    if (k == 0 || k > MS_MAX_SOURCES) return fail(GB_INVALID_VALUE, "multi-source BFS launch of %u sources", k);
    const uint32_t nw = k <= 64 ? 1 : (k <= 128 ? 2 : 4);
    MsWorkspace *w = nullptr;
    GB_CHECK(ms_workspace(ctx, A->nrows, nw, &w));
    msk::MsArgs a;
    a.n = A->nrows;
    a.nwords = (A->nrows + 31) / 32;
    a.m = A->nvals;
    a.k = k;
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t lo = 64 * i;
        a.live[i] = k <= lo ? 0ull : (k - lo >= 64 ? ~0ull : ((1ull << (k - lo)) - 1));
    }
    a.srcs = d_srcs;
    a.levels = levels;
    a.rec = w->rec;
    a.rp_out = A->rowptr;
    a.ci_out = A->colidx;
    a.rp_in = A->has_csc ? A->colptr : nullptr;
    a.ci_in = A->has_csc ? A->rowidx : nullptr;
    a.csr_is_csc = A->csc_alias;
    a.V = w->V;
    for (int j = 0; j < 3; ++j) {
        a.F[j] = w->F + (size_t)j * A->nrows * nw;
        a.mark[j] = w->mark + (size_t)j * a.nwords;
        a.front[j] = nullptr;
    }
    a.q[0] = w->q; a.q[1] = w->q + A->nrows + 1;
    a.qp[0] = w->qp; a.qp[1] = w->qp + A->nrows + 1;
    a.qr[0] = w->qr; a.qr[1] = w->qr + A->nrows + 1;
    a.ebits = 64 - bits_for((uint64_t)A->nrows + 1);
    a.emask = (1ull << a.ebits) - 1;
    a.mode = desc ? desc->direction : GB_AUTO;
    a.beta = (desc && desc->beta > 0) ? (uint32_t)desc->beta : 10u;
    a.st = w->st;
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 120000000000ull;
    a.hub_list = a.hub_pre = nullptr;
    a.nhub = 0;
    a.hub_edges = 0;
    if (A->has_csc) {
        GB_CHECK(matrix_hubs(A, GBX_HUB_MIN_LEN));
        a.hub_list = A->hub_list;
        a.hub_pre = A->hub_pre;
        a.nhub = A->nhub;
        a.hub_edges = A->hub_edges;
    }
    const void *fn = nw == 1 ? (const void *)msk::k_msbfs<1>
                     : nw == 2 ? (const void *)msk::k_msbfs<2> : (const void *)msk::k_msbfs<4>;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, msk::BLOCK, 0));
    if (occ < 1) return fail(GB_PANIC, "multi-source BFS kernel cannot be resident");
    void *args[] = {&a};
    int span = prof_begin(ctx, "bfs_multi");
    int grid = occ * ctx->num_sms;
    if (ctx->grid_limit > 0 && ctx->grid_limit < grid) grid = ctx->grid_limit;
    GB_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(msk::BLOCK), args, 0, ctx->stream));
    prof_end(ctx, span);
    if (res_out) GB_CUDA(cudaMemcpyAsync(res_out, &w->st->res, sizeof(BfsResult), cudaMemcpyDeviceToHost, ctx->stream));
    return GB_SUCCESS;
}

}  // namespace gbx

extern "C" gb_info gb_bfs_multi(gb_context *ctx, const gb_matrix *A, const uint32_t *srcs, uint32_t k, int32_t *levels,
                                gb_mem mem, const gb_desc *desc, gb_bfs_stats *stats) {
    if (k == 0) return fail(GB_INVALID_VALUE, "gb_bfs_multi: no sources");
    if (!ctx || !A || !srcs || !levels) return fail(GB_NULL_POINTER, "gb_bfs_multi: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_bfs_multi: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_bfs_multi: matrix must be square");
    for (uint32_t q = 0; q < k; ++q)
        if (srcs[q] >= A->nrows) return fail(GB_INVALID_INDEX, "gb_bfs_multi: source %u out of range", srcs[q]);
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch ds(ctx), dl(ctx);
    GB_CHECK(ds.alloc((size_t)k * 4 + 16));
    GB_CHECK(copy_in(ctx, ds.p, srcs, (size_t)k * 4, GB_HOST));
    int32_t *out = levels;
    size_t bytes = (size_t)k * A->nrows * 4;
    if (mem == GB_HOST) { GB_CHECK(dl.alloc(bytes + 16)); out = dl.as<int32_t>(); }
    // up to 256 sources share one launch (64 per word of source bits); more
    // run as consecutive launches of 256, each with its own push/pull
    // decisions; the trace is the first launch's (depth and counts are
    // summed and maximised over all of them)
    const uint32_t per = msk_max_sources();
    std::vector<BfsResult> parts((k + per - 1) / per);
    for (uint32_t q0 = 0; q0 < k; q0 += per) {
        const uint32_t kc = k - q0 < per ? k - q0 : per;
        GB_CHECK(msbfs_launch(ctx, A, ds.as<uint32_t>() + q0, kc, out + (size_t)q0 * A->nrows, desc,
                              &parts[q0 / per]));
    }
    if (mem == GB_HOST) GB_CUDA(cudaMemcpyAsync(levels, out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    BfsResult hs = parts[0];
    for (size_t c = 1; c < parts.size(); ++c) {
        const BfsResult &hk = parts[c];
        if (hk.depth > hs.depth) hs.depth = hk.depth;
        hs.push_levels += hk.push_levels;
        hs.pull_levels += hk.pull_levels;
        hs.reached += hk.reached;
        hs.frontier_edges += hk.frontier_edges;
        hs.edges_examined += hk.edges_examined;
        hs.alg_bytes += hk.alg_bytes;
        if (!hs.err) hs.err = hk.err;
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->depth = hs.depth;
        stats->push_levels = hs.push_levels;
        stats->pull_levels = hs.pull_levels;
        stats->status = (uint32_t)hs.err;
        stats->vertices_reached = hs.reached;
        stats->frontier_edges = hs.frontier_edges;
        stats->edges_examined = hs.edges_examined;
        stats->alg_bytes = (uint64_t)hs.alg_bytes;
        uint32_t nl = hs.depth < GB_TRACE_LEVELS ? hs.depth : GB_TRACE_LEVELS;
        stats->trace_len = nl;
        for (uint32_t l = 0; l < nl; ++l) {
            stats->trace_dir[l] = hs.dir_log[l];
            stats->trace_vertices[l] = hs.lv_cnt[l];
            stats->trace_edges[l] = hs.lv_fe[l];
            uint64_t t1 = (l + 1 < GBX_MAX_LEVEL_LOG) ? hs.lv_ns[l + 1] : hs.lv_ns[l];
            stats->trace_us[l] = (float)((t1 - hs.lv_ns[l]) * 1e-3);
        }
    }
    if (hs.err) return fail(GB_TIMEOUT, "gb_bfs_multi: a bounded grid barrier wait ran out");
    return GB_SUCCESS;
}
