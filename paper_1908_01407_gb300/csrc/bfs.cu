// Direction-optimised BFS (Algorithm 1, Section 7.1) as one persistent
// cooperative kernel: every level runs either
//   push  = SpMSpV over the out-edges (CSR rows) of the sparse frontier list,
//           claiming unvisited vertices with atomicOr on the visited bitmap
//           (the mask is tested before the write; Section 6.3.1's SpMSpV applies it after the product), or
//   pull  = masked SpMV over the in-edges (CSC columns) of unvisited vertices
//           only (mask first), stopping at the first frontier parent (the
//           Boolean semiring's early exit, Section 7.1) and reading no values
//           (structure only),
// with the assign of the level, the frontier count and the next frontier's
// edge count fused in. The direction rule is Table 9's: pull iff the
// frontier's edge count |E_f| > |E| / beta, with |E_f| exact (each appended
// vertex carries an exclusive prefix of out-degrees, see below).
//
// Frontier representation: both a bitmap (for pull) and a list with edge
// prefixes (for push) are produced every level (operand reuse, Section 7.1).
// Appends use a single 64-bit atomicAdd on a packed (count, edge-sum) word,
// so list positions and edge prefixes come out consistent and monotone: the
// push of the next level balances its edges over the grid by a merge-path
// search over the prefixes, without a separate scan.
//
// Levels are separated by a grid barrier with a wall-clock bound; on timeout
// the kernel records GB_TIMEOUT and exits.
//
// Blocks of 512 threads, two per SM: the same threads per SM as four blocks
// of 256, but half the blocks meet at each grid barrier and each block walks
// twice the candidates between them (0.111 against 0.115 ms per BFS on R-MAT
// scale 22).
#define GBX_FRONTIER_BLOCK 512
#include "common.cuh"
#include "bfs_common.cuh"
#include "frontier.cuh"

using namespace gbx;

namespace gbx {
namespace bfsk {
using namespace fr;

// claim v for the next frontier: the first atomicOr on its visited bit wins.
// On large pushes the bit is read first, which saves the atomic for the
// many targets already visited; on small ones that read would only add a
// dependent memory step.
__device__ __forceinline__ bool claim(const BfsArgs &a, uint32_t v, uint32_t parent, int d, uint32_t *Fn,
                                      uint32_t *deg_out, uint32_t *r0_out, bool precheck) {
    uint32_t w = v >> 5, bit = 1u << (v & 31);
    if (precheck && (ldcg(&a.visited[w]) & bit)) return false;
    uint32_t old = atomicOr(&a.visited[w], bit);
    if (old & bit) return false;
    a.levels[v] = d + 1;
    if (a.parents) a.parents[v] = (int32_t)parent;
    atomicOr(&Fn[w], bit);
    const uint32_t r0 = __ldg(&a.rp_out[v]);
    *deg_out = __ldg(&a.rp_out[v + 1]) - r0;
    *r0_out = r0;
    return true;
}

constexpr uint64_t PRECHECK_MIN_EDGES = 32768;

__device__ void push_level(const BfsArgs &a, Smem &sm, int d, uint32_t cnt, uint64_t fe) {
    const bool precheck = fe >= PRECHECK_MIN_EDGES;
    push_edges(a, sm, d, cnt, fe, [&](uint32_t u, uint32_t v, uint32_t, uint32_t *Fn, uint32_t *deg, uint32_t *r0) {
        return claim(a, v, u, d, Fn, deg, r0, precheck);
    });
}

// OR of `bits` over each run of adjacent lanes holding the same `key`;
// true for the first lane of a run, which then holds the run's OR. A key
// that recurs in a later run gets its own head (both heads then update the
// same word, which an atomicOr tolerates).
static __device__ __forceinline__ bool run_or_head(uint32_t key, uint32_t &bits) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t ob = __shfl_down_sync(full, bits, o);
        uint32_t ok = __shfl_down_sync(full, key, o);
        if (lane + o < 32 && ok == key) bits |= ob;
    }
    uint32_t kp = __shfl_up_sync(full, key, 1);
    return lane == 0 || kp != key;
}

// Shared memory of the pull levels (in a union with the push staging):
// per warp, the candidates it keeps for the next pull, appended to the next
// list PULL_KEEP_CAP at a time (one atomicAdd per flush), and the queue of
// candidates whose head missed.
constexpr int PULL_KEEP_CAP = 64;
constexpr int PULL_MISS_CAP = 64;   // fewer than 32 left over + one lane slot of 32
struct PullSmem {
    PullRec keep[WARPS][PULL_KEEP_CAP];
    PullRec miss[WARPS][PULL_MISS_CAP];
};

// Claims the found vertices of one lane slot across the warp: visited and
// next-frontier bits with one atomicOr per run of lanes in the same word,
// then level, parent and the out-degree count.
static __device__ __forceinline__ void claim_found(const BfsArgs &a, uint32_t *Fn, int d, bool f, uint32_t v,
                                                   uint32_t par, uint32_t dego, uint32_t &mycnt, uint32_t &mydeg) {
    const uint32_t NONE = 0xffffffffu;
    if (!__ballot_sync(0xffffffffu, f)) return;
    uint32_t key = f ? (v >> 5) : NONE;
    uint32_t bits = f ? 1u << (v & 31) : 0u;
    if (run_or_head(key, bits) && f) {
        atomicOr(&a.visited[key], bits);
        atomicOr(&Fn[key], bits);
    }
    if (f) {
        a.levels[v] = d + 1;
        if (a.parents) a.parents[v] = (int32_t)par;
        if (dego == NONE) dego = __ldg(&a.rp_out[v + 1]) - __ldg(&a.rp_out[v]);
        mydeg += dego;
        mycnt += 1;
    }
}

// Writes the warp's staged candidates to the next candidate list: one
// atomicAdd reserves their places, the copy is coalesced (their pull records
// with the live table, their vertex ids without it).
template <bool TABLE>
static __device__ __forceinline__ void flush_kept(PullRec *kbuf, uint32_t &staged, void *Lout,
                                                  unsigned int *lout_cnt) {
    if (!staged) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(lout_cnt, staged);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < staged; i += 32) {
        if (TABLE) static_cast<PullRec *>(Lout)[base + i] = kbuf[i];
        else static_cast<uint32_t *>(Lout)[base + i] = kbuf[i].v;
    }
    staged = 0;
    __syncwarp();
}

// Adds the lanes' kept candidates to the warp's staging buffer, flushing it
// first when they would not fit.
template <bool TABLE>
static __device__ __forceinline__ void keep_candidates(PullRec *kbuf, uint32_t &staged, void *Lout,
                                                       unsigned int *lout_cnt, bool keep, const PullRec &r) {
    const uint32_t km = __ballot_sync(0xffffffffu, keep);
    if (!km) return;
    if (staged + __popc(km) > (uint32_t)PULL_KEEP_CAP) flush_kept<TABLE>(kbuf, staged, Lout, lout_cnt);
    if (keep) kbuf[staged + __popc(km & dev::lanemask_lt())] = r;
    staged += __popc(km);
    __syncwarp();
}

// Scans the rows of the last k (<= 32) entries of the warp's miss queue,
// one per lane: in aligned 16-byte chunks for PULL_ROUNDS chunks, then
// warp-cooperatively (32 entries per step), stopping at the first
// in-neighbour on the frontier. A queued row had no frontier vertex in its
// head: with the live table the head is not a row prefix, so the whole row
// is scanned (its head entries again, harmlessly); without it the scan
// starts after the four head entries.
template <bool TABLE>
static __device__ void scan_misses(const BfsArgs &a, PullRec *mq, uint32_t &nq, uint32_t k, const uint32_t *F,
                                   uint32_t *Fn, int d, PullRec *kbuf, uint32_t &staged, void *Lout,
                                   unsigned int *lout_cnt, uint32_t &exam, uint32_t &lefte, uint32_t &mycnt,
                                   uint32_t &mydeg) {
    const uint32_t full = 0xffffffffu;
    const uint32_t NONE = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint4 *ci4 = reinterpret_cast<const uint4 *>(a.ci_in);
    const uint32_t q0 = nq - k;
    struct { uint32_t v, len, b, deg; } r = {NONE, 0, 0, 0};   // the head is re-read only to keep the record
    if ((uint32_t)lane < k) {
        const uint4 x = *reinterpret_cast<const uint4 *>(&mq[q0 + lane]);
        r.v = x.x; r.len = x.y; r.b = x.z; r.deg = x.w;
    }
    nq = q0;   // the entries stay intact until this warp queues again, after this call
    bool found = false;
    uint32_t par = 0, p = 0, e = 0;
    if (r.v != NONE) {
        p = TABLE ? r.b : r.b + 4;
        e = r.b + r.len;
    }
#pragma unroll 1
    for (int rd = 0; rd < PULL_ROUNDS; ++rd) {
        const bool pend = p < e;
        if (!__any_sync(full, pend)) break;
        uint4 cw = make_uint4(0, 0, 0, 0);
        if (pend) cw = ld_stream(&ci4[p >> 2]);
        const uint32_t q = p & ~3u;
        const uint32_t cc[4] = {cw.x, cw.y, cw.z, cw.w};
        uint32_t f4[4];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            const bool in = pend && q + k2 >= p && q + k2 < e;
            f4[k2] = in ? ldcg(&F[cc[k2] >> 5]) : 0u;
        }
        if (pend) {
            uint32_t stop = q + 4 < e ? q + 4 : e;
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) {
                const uint32_t pos = q + k2;
                if (!found && pos >= p && pos < e && ((f4[k2] >> (cc[k2] & 31)) & 1u)) {
                    found = true;
                    par = cc[k2];
                    stop = pos + 1;
                }
            }
            exam += stop - p;
            p = found ? e : q + 4;
        }
    }
    uint32_t coop = __ballot_sync(full, !found && p < e);
    while (coop) {
        const int l = __ffs(coop) - 1;
        coop &= coop - 1;
        const uint32_t pb = __shfl_sync(full, p, l);
        const uint32_t pe = __shfl_sync(full, e, l);
        bool got = false;
        uint32_t gpar = 0;
        for (uint32_t x0 = pb; x0 < pe; x0 += 32) {
            const uint32_t x = x0 + lane;
            uint32_t u = 0;
            bool hit = false;
            if (x < pe) {
                u = ld_stream(&a.ci_in[x]);
                hit = (ldcg(&F[u >> 5]) >> (u & 31)) & 1u;
            }
            const uint32_t hb = __ballot_sync(full, hit);
            if (hb) {
                const int f = __ffs(hb) - 1;
                gpar = __shfl_sync(full, u, f);
                got = true;
                if (lane == 0) exam += (x0 - pb) + f + 1;
                break;
            }
            if (lane == 0) exam += (pe - x0 < 32 ? pe - x0 : 32);
        }
        if (lane == l && got) { found = true; par = gpar; }
    }
    claim_found(a, Fn, d, found, r.v, par, r.deg, mycnt, mydeg);
    const bool keep = r.v != NONE && !found;
    if (keep) lefte += r.len;
    const uint32_t km = __ballot_sync(full, keep);
    if (km) {
        if (staged + __popc(km) > (uint32_t)PULL_KEEP_CAP) flush_kept<TABLE>(kbuf, staged, Lout, lout_cnt);
        if (keep) kbuf[staged + __popc(km & dev::lanemask_lt())] = mq[q0 + lane];
        staged += __popc(km);
    }
    __syncwarp();
}

// Pull over a list of candidates: for the first pull of a traversal every
// vertex with an in-edge, afterwards the candidates the previous pull left
// unvisited (a push may have claimed some since; their visited bit skips
// them). Vertices without in-edges can never be reached by a pull, and a
// later pull needs only what an earlier one left, so a pull touches
// |candidates| vertices rather than all n. With the matrix's live table a
// candidate is a pull record (vertex, CSC row, out-degree and its four
// in-neighbours of largest out-degree, one 32-byte sector, read with two
// coalesced 16-byte loads): the first pull reads the table itself, a later
// one the records the previous pull kept, contiguous in its list. Without
// the table a candidate is a vertex and its head is the first four entries
// of its row, read through the row pointers. The visited word and the
// frontier words of the four head entries load together (one dependent
// step), so a candidate with a frontier vertex among its head is decided
// there. Warps take groups of 32 WPW consecutive candidates, each lane
// WPW (a tile shape the autotuner picks per matrix: 1, 2 or 4). A candidate whose head has no frontier vertex and whose row is
// longer than four goes to the warp's miss queue, scanned 32 at a time
// (scan_misses). Found vertices set their visited and next-frontier bits
// (one atomicOr per run of lanes in the same bitmap word); the others are
// staged per warp and appended to the next list PULL_KEEP_CAP at a time.
// Pull writes the next frontier as a bitmap and only counts it (vertices,
// out-edges); the list form is built when a push needs it. It also counts
// the unvisited candidates it walked and sums the in-degrees of those it
// leaves (what a later pull over them reads at most).
template <bool TABLE, int WPW>
__device__ void pull_level(const BfsArgs &a, PullSmem &ps, int d, const void *Lin, uint32_t nin, void *Lout,
                           unsigned int *lout_cnt, unsigned long long *examined, uint32_t *cnt_out,
                           uint32_t *deg_out, uint32_t *act_out, unsigned long long *left_edges) {
    const uint32_t *F = a.front[d % 3];
    uint32_t *Fn = a.front[(d + 1) % 3];
    const uint32_t full = 0xffffffffu;
    const uint32_t NONE = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ngroups = (uint32_t)(((uint64_t)nin + (WPW * 32) - 1) / (WPW * 32));
    const uint32_t nwarps = gridDim.x * WARPS;
    const PullRec *recs = TABLE ? (Lin ? static_cast<const PullRec *>(Lin) : a.live_rec) : nullptr;
    PullRec *kbuf = ps.keep[warp];
    PullRec *mq = ps.miss[warp];
    uint32_t exam = 0, lefte = 0;   // per thread and level these stay far below 2^32
    uint32_t mycnt = 0, mydeg = 0, myact = 0;
    uint32_t nq = 0;       // entries in this warp's miss queue
    uint32_t staged = 0;   // candidates staged for the next list
    static_assert(31 + 32 <= PULL_MISS_CAP, "a lane slot's misses fit the queue");
    for (uint32_t g = blockIdx.x * WARPS + warp; g < ngroups; g += nwarps) {
        PullRec r[WPW];
        bool act[WPW], found[WPW];
        uint32_t par[WPW];
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            const uint32_t idx = g * (WPW * 32) + j * 32 + lane;
            r[j].v = NONE;
            r[j].len = r[j].b = r[j].deg = 0;
            r[j].head = make_uint4(NONE, NONE, NONE, NONE);
            if (idx < nin) {
                if (TABLE) {
                    const uint4 *q = reinterpret_cast<const uint4 *>(recs + idx);
                    const uint4 x = ld_stream(q), y = ld_stream(q + 1);
                    r[j].v = x.x; r[j].len = x.y; r[j].b = x.z; r[j].deg = x.w;
                    r[j].head = y;
                } else {
                    const uint32_t v = Lin ? ldcg(&static_cast<const uint32_t *>(Lin)[idx]) : idx;
                    r[j].v = v;
                    r[j].b = __ldg(&a.rp_in[v]);
                    r[j].len = __ldg(&a.rp_in[v + 1]) - r[j].b;
                    r[j].deg = a.csr_is_csc ? r[j].len : NONE;   // read from the CSR once found
                }
            }
        }
        if (!TABLE) {
#pragma unroll
            for (int j = 0; j < WPW; ++j) {
                uint32_t hh[4] = {NONE, NONE, NONE, NONE};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (r[j].v != NONE && (uint32_t)k < r[j].len) hh[k] = ld_stream(&a.ci_in[r[j].b + k]);
                r[j].head = make_uint4(hh[0], hh[1], hh[2], hh[3]);
            }
        }
        // the visited word and the frontier word of the first head entry
        // (the in-neighbour of largest out-degree) together; the other three
        // only where it missed. Every frontier word is a random sector lookup
        // and the lookups' rate bounds a wide pull, so each candidate asks for
        // as few as decide it.
        uint32_t vw[WPW], fw[WPW][4];
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            vw[j] = r[j].v != NONE ? ldcg(&a.visited[r[j].v >> 5]) : full;
            fw[j][0] = r[j].head.x != NONE ? ldcg(&F[r[j].head.x >> 5]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            act[j] = r[j].v != NONE && !((vw[j] >> (r[j].v & 31)) & 1u);
            found[j] = act[j] && r[j].head.x != NONE && ((fw[j][0] >> (r[j].head.x & 31)) & 1u);
            par[j] = found[j] ? r[j].head.x : 0u;
        }
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            const uint32_t h[3] = {r[j].head.y, r[j].head.z, r[j].head.w};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                fw[j][1 + k] = (act[j] && !found[j] && h[k] != NONE) ? ldcg(&F[h[k] >> 5]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            uint32_t ex = r[j].len < 4 ? r[j].len : 4;
            if (act[j] && !found[j]) {
                const uint32_t h[3] = {r[j].head.y, r[j].head.z, r[j].head.w};
#pragma unroll
                for (int k = 2; k >= 0; --k)   // the first frontier neighbour in head order
                    if (h[k] != NONE && ((fw[j][1 + k] >> (h[k] & 31)) & 1u)) {
                        found[j] = true;
                        par[j] = h[k];
                        ex = k + 2;
                    }
            } else if (found[j]) {
                ex = 1;
            }
            if (act[j]) { exam += ex; ++myact; }
        }
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            claim_found(a, Fn, d, found[j], r[j].v, par[j], r[j].deg, mycnt, mydeg);
            // rows longer than four whose head missed: to the miss queue
            const bool miss = act[j] && !found[j] && r[j].len > 4;
            const uint32_t mm = __ballot_sync(full, miss);
            if (miss) mq[nq + __popc(mm & dev::lanemask_lt())] = r[j];
            nq += __popc(mm);
            // rows of at most four entries are done: unvisited ones stay candidates
            const bool keep = act[j] && !found[j] && r[j].len > 0 && r[j].len <= 4;
            if (keep) lefte += r[j].len;
            keep_candidates<TABLE>(kbuf, staged, Lout, lout_cnt, keep, r[j]);
            __syncwarp();
            if (nq >= 32)
                scan_misses<TABLE>(a, mq, nq, 32, F, Fn, d, kbuf, staged, Lout, lout_cnt, exam, lefte, mycnt, mydeg);
        }
    }
    if (nq) scan_misses<TABLE>(a, mq, nq, nq, F, Fn, d, kbuf, staged, Lout, lout_cnt, exam, lefte, mycnt, mydeg);
    flush_kept<TABLE>(kbuf, staged, Lout, lout_cnt);
    *examined += exam;
    *cnt_out += mycnt;
    *deg_out += mydeg;
    *act_out += myact;
    *left_edges += lefte;
}

// Table 9's rule: pull iff |E_f| * beta > |E|. Once a pull has run, the
// next pull would walk only the candidates it left (uc of them, ue in-edges
// in all), so a level also pulls when that walk reads no more than the push
// would: the frontier's out-edges, its list, and, after a pull (the list form
// does not exist yet), one pass over the frontier bitmap to build it. In the
// last levels of a traversal of a low-diameter graph this keeps a frontier of
// many leaves with few unvisited vertices left in pull.
__device__ __forceinline__ bool choose_pull(const BfsArgs &a, uint64_t fe, uint32_t cnt, int npull, bool list_valid,
                                            uint32_t uc, unsigned long long ue) {
    if (a.mode == GB_PUSH || !a.rp_in) return false;
    if (a.mode == GB_PULL) return true;
    if (fe * (uint64_t)a.beta > a.m) return true;
    if (npull == 0) return false;
    const unsigned long long pull_reads = 8ull * uc + ue;
    const unsigned long long push_reads = fe + 4ull * cnt + (list_valid ? 0ull : (unsigned long long)a.nwords);
    return pull_reads <= push_reads;
}

union BfsShared {
    Smem push;       // push levels and the bitmap -> list compaction
    PullSmem pull;   // pull levels
};

// level and parent -1 for the vertices whose bit is set in unreached(w): each
// lane loads one word, then the warp walks its 32 words with one broadcast
// and one coalesced store per word (a single dependent load per warp)
template <class Unreached>
__device__ __forceinline__ void write_unreached(const BfsArgs &ar, Unreached unreached) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
    for (uint64_t w0 = ((uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5)) * 32; w0 < ar.nwords; w0 += nwarps * 32) {
        const uint32_t mine = w0 + lane < ar.nwords ? unreached(w0 + lane) : 0u;
        uint32_t todo = __ballot_sync(0xffffffffu, mine != 0u);
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t bits = __shfl_sync(0xffffffffu, mine, k);
            if ((bits >> lane) & 1u) {
                const uint64_t v = (w0 + k) * 32 + lane;
                ar.levels[v] = -1;
                if (ar.parents) ar.parents[v] = -1;
            }
        }
    }
}

// One traversal from ar.src (Algorithm 1): its start (bitmaps, level-0 list,
// counters), the levels, each ended by a grid barrier on bst, and the final
// pass that gives unreached vertices -1. ar.st holds the traversal's
// counters and result record; bst holds the barrier and the error word.
// Returns false when a barrier wait ran out.
template <int WPW>
__device__ bool bfs_run(const BfsArgs &ar, BfsState *bst, bool first, uint64_t t_entry, BfsShared &shm,
                        unsigned long long *s_box, uint32_t *s_box32) {
    Smem &sm = shm.push;
    unsigned long long &s_exam = s_box[0], &s_left = s_box[1], &s_qs = s_box[2], &s_ue = s_box[3];
    uint32_t &s_cnt = s_box32[0], &s_deg = s_box32[1], &s_act = s_box32[2], &s_uc = s_box32[3];
    const uint32_t nthreads = gridDim.x * BLOCK;
    const uint32_t tid = blockIdx.x * BLOCK + threadIdx.x;
    BfsState *st = ar.st;
    BfsResult *res = &st->res;
    // ---- start: bitmaps and the level-0 list (levels/parents of vertices
    // that stay unreached are written at the end)
    const uint32_t sw = ar.src >> 5, sbit = 1u << (ar.src & 31);
    const uint32_t tail = (ar.n & 31) ? ~((1u << (ar.n & 31)) - 1u) : 0u;
    for (uint64_t w = tid; w < ar.nwords; w += nthreads) {
        uint32_t vis = (w == sw ? sbit : 0u);
        if (w == ar.nwords - 1) vis |= tail;
        ar.visited[w] = vis;
        ar.front[0][w] = w == sw ? sbit : 0u;
        ar.front[1][w] = 0u;
        ar.front[2][w] = 0u;
    }
    if (tid == 0) {
        uint32_t r0 = __ldg(&ar.rp_out[ar.src]);
        uint32_t deg = __ldg(&ar.rp_out[ar.src + 1]) - r0;
        ar.levels[ar.src] = 0;
        if (ar.parents) ar.parents[ar.src] = (int32_t)ar.src;
        ar.q[0][0] = ar.src;
        ar.qp[0][0] = 0;
        ar.qr[0][0] = r0;
        st->qstate[0] = (1ull << ar.ebits) | deg;
    }
    if (blockIdx.x == 0) {
        // block 0 zeroes the result record, then its thread 0 owns it
        unsigned long long *r8 = reinterpret_cast<unsigned long long *>(res);
        for (uint32_t k = threadIdx.x; k < sizeof(BfsResult) / 8; k += BLOCK) r8[k] = 0ull;
        __syncthreads();
        if (threadIdx.x == 0) res->t_entry = t_entry;
    }
    bool ok;
    if (first && ar.withhold && blockIdx.x == 0 && gridDim.x > 1) {
        // failure-path test: this block never arrives, so the bounded wait of
        // the others runs out; it waits (bounded too) until they record it
        ok = dev::wait_for_error(&bst->err, 2 * ar.timeout_ns);
    } else {
        ok = dev::grid_sync(&bst->bar, gridDim.x, &bst->err, ar.timeout_ns);
    }
    const uint64_t t_start = dev::globaltimer_ns();
    uint64_t reached = 0;
    // previous level's numbers for the algorithmic byte count
    uint32_t prev_dir = 0, prev_cnt = 0, prev_nin = 0;
    uint64_t prev_fe = 0;
    double alg = 8.0 * ar.n;   // levels + parents writes
    bool list_valid = true;    // the list form of the current frontier exists
    int npull = 0;             // pull steps so far (selects the candidate lists)
    // the source's component size: once that many vertices are reached the
    // last frontier has nothing left to discover and is not expanded
    const uint32_t csize = ar.comp_size ? __ldg(&ar.comp_size[ar.src]) : 0u;
    bool exhausted = false;
    int d = 0;
    for (; ok; ++d) {
        if (threadIdx.x == 0) {
            s_qs = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(st->qstate[d % 3])
                       .load(cuda::memory_order_relaxed);
            if (npull > 0) {
                s_uc = (uint32_t)dev::ld_relaxed_gpu_int((const int *)&st->ucnt[(npull - 1) % 3]);
                s_ue = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(st->uedg[(npull - 1) % 3])
                           .load(cuda::memory_order_relaxed);
            }
        }
        __syncthreads();
        const unsigned long long qs = s_qs;
        const uint32_t uc = npull > 0 ? s_uc : 0u;
        const unsigned long long ue = npull > 0 ? s_ue : 0ull;
        __syncthreads();
        uint32_t cnt = (uint32_t)(qs >> ar.ebits);
        uint64_t fe = qs & ar.emask;
        if (tid == 0 && d > 0) {
            unsigned long long ex = st->exam[(d - 1) % 3];
            if (prev_dir == 0) {
                alg += 8.0 * prev_cnt + 4.0 * prev_fe + 12.0 * cnt;
            } else {
                // the mask words the pull reads, the row pointers of the unvisited candidates it
                // walked, the adjacency entries it examined and the discoveries it wrote
                const double mask = ar.n / 8.0 < 4.0 * prev_nin ? ar.n / 8.0 : 4.0 * prev_nin;
                alg += mask + 8.0 * (double)st->uact[(d - 1) % 3] + 4.0 * ex + 12.0 * cnt;
            }
            res->edges_examined += prev_dir == 0 ? prev_fe : ex;
        }
        if (cnt == 0) break;
        if (csize && reached + cnt >= csize) {
            reached += cnt;
            exhausted = true;
            break;
        }
        // guard: no BFS has more than n levels; the traversal has a wall-clock budget
        if (d > (int)ar.n || (threadIdx.x == 0 && dev::globaltimer_ns() - t_start > ar.total_limit_ns)) {
            atomicCAS(&bst->err, 0, (int)GB_TIMEOUT);
        }
        const bool pull = choose_pull(ar, fe, cnt, npull, list_valid, uc, ue);
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
            st->exam[(d + 2) % 3] = 0;
            st->uact[(d + 2) % 3] = 0;
            st->cstate[(d + 2) % 3] = 0;
            prev_dir = pull ? 1u : 0u;
            prev_cnt = cnt;
            prev_fe = fe;
        }
        reached += cnt;
        uint32_t *Fclr = ar.front[(d + 2) % 3];
        for (uint64_t w = tid; w < ar.nwords; w += nthreads) Fclr[w] = 0u;
        if (pull) {
            if (threadIdx.x == 0) { s_exam = 0; s_left = 0; s_cnt = 0; s_deg = 0; s_act = 0; }
            __syncthreads();
            // candidates: all live ones for the first pull, then what the previous pull left
            const void *Lin;
            uint32_t nin;
            if (npull == 0) {
                // every candidate once: the live table's records (with the
                // table), otherwise the vertices 0..n-1
                Lin = nullptr;
                nin = ar.live_rec ? ldcg(ar.live_count) : ar.n;
            } else {
                Lin = ar.ul[(npull - 1) & 1];
                nin = (uint32_t)dev::ld_relaxed_gpu_int((const int *)&st->ucnt[(npull - 1) % 3]);
            }
            if (tid == 0) {
                st->ucnt[(npull + 1) % 3] = 0;
                st->uedg[(npull + 1) % 3] = 0;
                prev_nin = nin;
            }
            const int us = npull % 3;
            unsigned long long ex = 0, le = 0;
            uint32_t c = 0, dg = 0, na = 0;
            if (ar.live_rec)
                pull_level<true, WPW>(ar, shm.pull, d, Lin, nin, ar.ul[npull & 1], &st->ucnt[us], &ex, &c, &dg, &na,
                                      &le);
            else
                pull_level<false, WPW>(ar, shm.pull, d, Lin, nin, ar.ul[npull & 1], &st->ucnt[us], &ex, &c, &dg, &na,
                                       &le);
            ++npull;
            ex = dev::warp_sum<unsigned long long>(ex);
            le = dev::warp_sum<unsigned long long>(le);
            c = dev::warp_sum<uint32_t>(c);
            dg = dev::warp_sum<uint32_t>(dg);
            na = dev::warp_sum<uint32_t>(na);
            if ((threadIdx.x & 31) == 0) {
                if (ex) atomicAdd(&s_exam, ex);
                if (le) atomicAdd(&s_left, le);
                if (na) atomicAdd(&s_act, na);
                if (c) { atomicAdd(&s_cnt, c); atomicAdd(&s_deg, dg); }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (s_exam) atomicAdd(&st->exam[d % 3], s_exam);
                if (s_left) atomicAdd(&st->uedg[us], s_left);
                if (s_act) atomicAdd(&st->uact[d % 3], (unsigned long long)s_act);
                if (s_cnt) atomicAdd(&st->qstate[(d + 1) % 3], ((unsigned long long)s_cnt << ar.ebits) | s_deg);
            }
            list_valid = false;
        } else {
            if (!list_valid) {
                compact_level(ar, sm, d);
                if (!dev::grid_sync(&bst->bar, gridDim.x, &bst->err, ar.timeout_ns)) { ok = false; break; }
            }
            push_level(ar, sm, d, cnt, fe);
            list_valid = true;
        }
        ok = dev::grid_sync(&bst->bar, gridDim.x, &bst->err, ar.timeout_ns);
    }
    if (tid == 0) {
        res->t_end = dev::globaltimer_ns();
        if (d < GBX_MAX_LEVEL_LOG) res->lv_ns[d] = res->t_end;
    }
    // ---- vertices never reached get level and parent -1
    if (ok) write_unreached(ar, [&](uint64_t w) -> uint32_t { return ~ldcg(&ar.visited[w]); });
    if (tid == 0) {
        res->depth = d + (exhausted ? 1 : 0);
        res->reached = reached;
        res->alg_bytes = alg;
        res->t_begin = t_start;
    }
    return ok;
}

// The last block to leave resets the working state for the next launch.
__device__ void bfs_leave(const BfsArgs &a) {
    __syncthreads();
    if (threadIdx.x == 0) {
        BfsState *st = a.st;
        __threadfence();
        unsigned int old = atomicAdd(&st->bar.exits, 1u);
        if (old == gridDim.x - 1) {
            __threadfence();
            const int e = ld_relaxed_gpu_int_(&st->err);
            st->res.err = e;
            if (e && a.err_sticky) atomicMax(a.err_sticky, e);
            if (a.status_out) *a.status_out = e;
            st->res.t_exit = dev::globaltimer_ns();
            st->err = 0;
            st->bar.count = 0;
            for (int k = 0; k < 3; ++k) {
                st->qstate[k] = 0; st->exam[k] = 0; st->cstate[k] = 0; st->ucnt[k] = 0;
                st->uedg[k] = 0; st->uact[k] = 0;
            }
            __threadfence();
            st->bar.exits = 0;
        }
    }
}

// WPW: pull candidates per lane in flight (a tile shape tuned per matrix);
// 1,024 threads per SM for widths 1 and 2 (64 registers each), 512 for
// width 4, which needs more
template <int WPW>
__global__ void __launch_bounds__(BLOCK, (WPW == 4 ? 512 : 1024) / BLOCK) k_bfs(BfsArgs a) {
    __shared__ BfsShared shm;
    __shared__ unsigned long long s_box[4];
    __shared__ uint32_t s_box32[4];
    const uint64_t t_entry = dev::globaltimer_ns();
    bfs_run<WPW>(a, a.st, true, t_entry, shm, s_box, s_box32);
    bfs_leave(a);
}

// the k_bfs instance for a pull width (1, 2 or 4; anything else: the default)
static const void *bfs_kernel(uint32_t wpw) {
    if (wpw == 1) return (const void *)k_bfs<1>;
    if (wpw == 4) return (const void *)k_bfs<4>;
    return (const void *)k_bfs<PULL_WPW>;
}

}  // namespace bfsk

// the barrier-free schedule (async_relax.cu)
gb_info async_relax_run(gb_context *ctx, const gb_matrix *A, int kind, uint32_t src, uint32_t *out,
                        uint32_t *parents, uint64_t delta, gb_bfs_stats *stats, const char *who);

// the single-cluster schedule (bfs_cluster.cu)
bool bfs_cluster_available(gb_context *ctx);
gb_info bfs_cluster_launch(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels, int32_t *parents,
                           uint32_t *visited, uint32_t *ov0, uint32_t *ov1, void *state, int *err_sticky);
size_t bfs_cluster_state_bytes();
gb_info bfs_cluster_result(gb_context *ctx, const void *state, gb_bfs_stats *stats);

struct BfsWorkspace {
    uint32_t n = 0;
    uint32_t *visited = nullptr, *front = nullptr, *q = nullptr, *qp = nullptr, *qr = nullptr;
    PullRec *ul = nullptr;   // two candidate lists of pull records
    BfsState *st = nullptr;
    void *cl_state = nullptr;   // state block of the single-cluster schedule
    int grid = 0;               // blocks of the default k_bfs at full occupancy
    int occ[3] = {0, 0, 0};     // resident blocks per SM of k_bfs<1>, <2>, <4>
};

// index of a pull width in BfsWorkspace::occ
static int wpw_slot(uint32_t wpw) { return wpw == 1 ? 0 : (wpw == 4 ? 2 : 1); }

static std::mutex g_ws_mu;
static std::unordered_map<gb_context *, BfsWorkspace> g_ws;

gb_info bfs_workspace(gb_context *ctx, uint32_t n, BfsWorkspace **out) {
    std::lock_guard<std::mutex> g(g_ws_mu);
    BfsWorkspace &w = g_ws[ctx];
    if (w.n < n || !w.st) {
        dfree(ctx, w.visited); dfree(ctx, w.front); dfree(ctx, w.q); dfree(ctx, w.qp); dfree(ctx, w.qr);
        dfree(ctx, w.ul); dfree(ctx, w.st); dfree(ctx, w.cl_state);
        w = BfsWorkspace();
        uint32_t nw = (n + 31) / 32;
        GB_CHECK(dalloc_t(ctx, &w.visited, nw));
        GB_CHECK(dalloc_t(ctx, &w.front, 3ull * nw));
        GB_CHECK(dalloc_t(ctx, &w.q, 2ull * n + 2));
        GB_CHECK(dalloc_t(ctx, &w.qp, 2ull * n + 2));
        GB_CHECK(dalloc_t(ctx, &w.qr, 2ull * n + 2));
        GB_CHECK(dalloc(ctx, (void **)&w.ul, (2ull * n + 2) * sizeof(PullRec) + 16));
        GB_CHECK(dalloc_t(ctx, &w.st, 1));
        GB_CHECK(dalloc(ctx, &w.cl_state, bfs_cluster_state_bytes()));
        // the only reset of the working state: launches leave it zeroed
        GB_CHECK(memset_async(ctx, w.st, 0, sizeof(BfsState)));
        w.n = n;
    }
    if (!w.grid) {
        const uint32_t widths[3] = {1, 2, 4};
        for (int i = 0; i < 3; ++i) {
            GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&w.occ[i], bfsk::bfs_kernel(widths[i]),
                                                                  bfsk::BLOCK, 0));
            if (w.occ[i] < 1) return fail(GB_PANIC, "BFS kernel cannot be resident");
        }
        w.grid = w.occ[wpw_slot(0)] * ctx->num_sms;
    }
    *out = &w;
    return GB_SUCCESS;
}

gb_info bfs_workspace_raw(gb_context *ctx, uint32_t n, uint32_t **visited, uint32_t **front, uint32_t **q,
                          uint32_t **qp, uint32_t **qr, BfsState **st, void **cl_state) {
    BfsWorkspace *w = nullptr;
    GB_CHECK(bfs_workspace(ctx, n, &w));
    *visited = w->visited; *front = w->front; *q = w->q; *qp = w->qp; *qr = w->qr; *st = w->st;
    if (cl_state) *cl_state = w->cl_state;
    return GB_SUCCESS;
}

void bfs_workspace_release(gb_context *ctx) {
    std::lock_guard<std::mutex> g(g_ws_mu);
    auto it = g_ws.find(ctx);
    if (it == g_ws.end()) return;
    BfsWorkspace &w = it->second;
    dfree(ctx, w.visited); dfree(ctx, w.front); dfree(ctx, w.q); dfree(ctx, w.qp); dfree(ctx, w.qr);
    dfree(ctx, w.ul); dfree(ctx, w.st); dfree(ctx, w.cl_state);
    g_ws.erase(it);
}

// The schedule a gb_bfs call runs: the descriptor's, else the matrix's tuned
// one, else the persistent grid; the cluster needs a device that can
// co-schedule it.
static int bfs_schedule(gb_context *ctx, const gb_matrix *A, const gb_desc *desc) {
    int sch = (desc && desc->schedule != GB_SCHED_AUTO) ? desc->schedule : A->tuned_schedule;
    if (sch == GB_SCHED_CLUSTER && !bfs_cluster_available(ctx)) sch = GB_SCHED_GRID;
    if (sch == GB_SCHED_ASYNC) return GB_SCHED_ASYNC;
    return sch == GB_SCHED_CLUSTER ? GB_SCHED_CLUSTER : GB_SCHED_GRID;
}

static gb_info bfs_cluster_run(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels,
                               int32_t *parents, BfsWorkspace *w, int *err_sticky = nullptr) {
    return bfs_cluster_launch(ctx, A, src, levels, parents, w->visited, w->q, w->q + A->nrows + 1, w->cl_state,
                              err_sticky);
}

// Failure-path test hook: when the environment variable
// GBX_TEST_WITHHOLD_BARRIER_US is set to a positive number of microseconds,
// BFS launches bound each grid-barrier wait by that much and block 0
// withholds its arrival at the first barrier, so the wait of the other
// blocks runs out (no fault, no hang) and the launch ends with GB_TIMEOUT.
static uint64_t test_withhold_ns() {
    const char *e = getenv("GBX_TEST_WITHHOLD_BARRIER_US");
    if (!e || !*e) return 0;
    long long us = atoll(e);
    if (us <= 0) return 0;
    if (us > 1000000) us = 1000000;
    return (uint64_t)us * 1000ull;
}

gb_info bfs_launch(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels, int32_t *parents,
                   const gb_desc *desc, BfsWorkspace *w, int grid_override, int *err_sticky = nullptr) {
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
    a.qr[0] = w->qr; a.qr[1] = w->qr + A->nrows + 1;
    a.live_rec = A->has_csc ? A->live_rec : nullptr;
    a.live_count = a.live_rec ? A->live_count : nullptr;
    a.ul[0] = w->ul; a.ul[1] = w->ul + A->nrows + 1;
    a.comp_size = A->comp_size;
    a.ebits = 64 - bits_for((uint64_t)A->nrows + 1);
    a.emask = (a.ebits >= 64) ? ~0ull : ((1ull << a.ebits) - 1);
    a.mode = desc ? desc->direction : GB_AUTO;
    a.beta = (desc && desc->beta > 0) ? (uint32_t)desc->beta : (A->tuned_beta ? A->tuned_beta : 10u);
    a.st = w->st;
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 120000000000ull;
    // without a caller's word, a timeout is kept for gb_context_synchronize
    a.err_sticky = err_sticky ? err_sticky : &w->st->sticky;
    a.status_out = nullptr;
    a.withhold = false;
    if (const uint64_t t = test_withhold_ns()) {
        a.timeout_ns = t;
        a.withhold = true;
    }
    // the matrix's tile shape: pull width (kernel instance) and blocks per SM
    const uint32_t wpw = A->bfs_pull_width;
    int per_sm = w->occ[wpw_slot(wpw)];
    if (A->bfs_blocks_per_sm > 0 && (int)A->bfs_blocks_per_sm < per_sm) per_sm = (int)A->bfs_blocks_per_sm;
    int grid = per_sm * ctx->num_sms;
    // the context's cap counts blocks of 256 threads
    const int cap = ctx->grid_limit > 0 ? std::max(1, ctx->grid_limit * 256 / bfsk::BLOCK) : 0;
    if (cap > 0 && cap < grid) grid = cap;
    if (grid_override > 0 && grid_override < grid) grid = grid_override;
    void *args[] = {&a};
    int span = prof_begin(ctx, "bfs");
    GB_CUDA(cudaLaunchCooperativeKernel(bfsk::bfs_kernel(wpw), dim3(grid), dim3(bfsk::BLOCK), args, 0,
                                        ctx->stream));
    prof_end(ctx, span);
    return GB_SUCCESS;
}

// Reads and clears the context's sticky BFS status word (the largest exit
// code of launches whose caller did not wait for them); GB_TIMEOUT if it
// was set. Called by gb_context_synchronize.
gb_info bfs_collect_status(gb_context *ctx) {
    BfsState *st = nullptr;
    {
        std::lock_guard<std::mutex> g(g_ws_mu);
        auto it = g_ws.find(ctx);
        if (it == g_ws.end() || !it->second.st) return GB_SUCCESS;
        st = it->second.st;
    }
    int e = 0;
    GB_CUDA(cudaMemcpyAsync(&e, &st->sticky, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (!e) return GB_SUCCESS;
    GB_CUDA(cudaMemsetAsync(&st->sticky, 0, sizeof(int), ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    return fail(GB_TIMEOUT, "a BFS launched without waiting for it ran out of a bounded device wait");
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
    if (bfs_schedule(ctx, A, desc) == GB_SCHED_ASYNC) {
        GB_CHECK(async_relax_run(ctx, A, 1, src, (uint32_t *)dl, (uint32_t *)dp, 0, stats, "gb_bfs"));
        if (mem == GB_HOST) {
            GB_CUDA(cudaMemcpyAsync(levels, dl, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
            if (parents)
                GB_CUDA(cudaMemcpyAsync(parents, dp, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
            GB_CHECK(sync(ctx));
        }
        return GB_SUCCESS;
    }
    const int sch = bfs_schedule(ctx, A, desc);
    if (sch == GB_SCHED_CLUSTER) GB_CHECK(bfs_cluster_run(ctx, A, src, dl, dp, w, &w->st->sticky));
    else GB_CHECK(bfs_launch(ctx, A, src, dl, dp, desc, w, 0));
    if (mem == GB_HOST) {
        GB_CUDA(cudaMemcpyAsync(levels, dl, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
        if (parents) GB_CUDA(cudaMemcpyAsync(parents, dp, (size_t)A->nrows * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (sch == GB_SCHED_CLUSTER) {
        if (stats || mem == GB_HOST) {
            const gb_info r = bfs_cluster_result(ctx, w->cl_state, stats);
            if (r == GB_TIMEOUT) (void)bfs_collect_status(ctx);   // reported here, not again
            GB_CHECK(r);
            if (stats) stats->schedule = GB_SCHED_CLUSTER;
        }
        return GB_SUCCESS;
    }
    if (stats || mem == GB_HOST) {
        BfsResult hs;
        GB_CUDA(cudaMemcpyAsync(&hs, &w->st->res, sizeof(BfsResult), cudaMemcpyDeviceToHost, ctx->stream));
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        // this launch's status is in hs.err; its copy in the sticky word is
        // reported here, not again by gb_context_synchronize
        if (hs.err) (void)bfs_collect_status(ctx);
        if (stats) {
            stats->depth = hs.depth;
            stats->push_levels = hs.push_levels;
            stats->pull_levels = hs.pull_levels;
            stats->status = (uint32_t)hs.err;
            stats->vertices_reached = hs.reached;
            stats->edges_examined = hs.edges_examined;
            stats->frontier_edges = hs.frontier_edges;
            stats->alg_bytes = (uint64_t)hs.alg_bytes;
            // the expanded levels (a traversal that exhausted the source's
            // component does not expand its last frontier)
            const uint32_t nexp = hs.push_levels + hs.pull_levels;
            uint32_t nl = nexp < GB_TRACE_LEVELS ? nexp : GB_TRACE_LEVELS;
            stats->trace_len = nl;
            for (uint32_t l = 0; l < nl; ++l) {
                stats->trace_dir[l] = hs.dir_log[l];
                stats->trace_vertices[l] = hs.lv_cnt[l];
                stats->trace_edges[l] = hs.lv_fe[l];
                uint64_t t1 = (l + 1 < GBX_MAX_LEVEL_LOG) ? hs.lv_ns[l + 1] : hs.lv_ns[l];
                stats->trace_us[l] = (float)((t1 - hs.lv_ns[l]) * 1e-3);
            }
            stats->init_us = hs.depth ? (float)((hs.lv_ns[0] - hs.t_entry) * 1e-3) : 0.f;
            stats->final_us = (float)((hs.t_exit - hs.t_end) * 1e-3);
            stats->schedule = GB_SCHED_GRID;
        }
        if (hs.err) return fail(GB_TIMEOUT, "gb_bfs: a bounded grid barrier wait ran out");
    }
    return GB_SUCCESS;
}

// k independent BFS runs. With host outputs, run q writes one of two device
// result buffers and a second stream copies it to row q of the host arrays
// while run q+1 traverses; run q+2 waits for that copy before it reuses the
// buffer. Each kernel max-es a nonzero exit status into one device word.
namespace {
struct CopyPipe {
    cudaStream_t cs = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    ~CopyPipe() {
        // the device buffers are freed after this (declared before): no copy may still read them
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        for (int b = 0; b < 2; ++b) {
            if (done[b]) cudaEventDestroy(done[b]);
            if (copied[b]) cudaEventDestroy(copied[b]);
        }
    }
    gb_info init() {
        GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            GB_CUDA(cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming));
            GB_CUDA(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
        }
        return GB_SUCCESS;
    }
};
}  // namespace

extern "C" gb_info gb_bfs_batch(gb_context *ctx, const gb_matrix *A, const uint32_t *srcs, uint32_t k,
                                int32_t *levels, int32_t *parents, gb_mem mem, const gb_desc *desc) {
    if (!ctx || !A || !srcs || !levels) return fail(GB_NULL_POINTER, "gb_bfs_batch: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_bfs_batch: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_bfs_batch: matrix must be square");
    if (k == 0) return fail(GB_INVALID_VALUE, "gb_bfs_batch: no sources");
    const uint32_t n = A->nrows;
    for (uint32_t q = 0; q < k; ++q)
        if (srcs[q] >= n) return fail(GB_INVALID_INDEX, "gb_bfs_batch: source %u (entry %u) out of range", srcs[q], q);
    GB_CUDA(cudaSetDevice(ctx->device));
    BfsWorkspace *w = nullptr;
    GB_CHECK(bfs_workspace(ctx, n, &w));
    const int sch = bfs_schedule(ctx, A, desc);
    const size_t row = (size_t)n;
    Scratch eb(ctx), lb(ctx), pb(ctx);
    GB_CHECK(eb.alloc(sizeof(int)));
    GB_CHECK(memset_async(ctx, eb.p, 0, sizeof(int)));
    int *err = eb.as<int>();
    auto run = [&](uint32_t q, int32_t *dl, int32_t *dp) -> gb_info {
        if (sch == GB_SCHED_ASYNC)
            return async_relax_run(ctx, A, 1, srcs[q], (uint32_t *)dl, (uint32_t *)dp, 0, nullptr, "gb_bfs_batch");
        if (sch == GB_SCHED_CLUSTER) return bfs_cluster_run(ctx, A, srcs[q], dl, dp, w, err);
        return bfs_launch(ctx, A, srcs[q], dl, dp, desc, w, 0, err);
    };
    if (mem == GB_DEVICE) {
        for (uint32_t q = 0; q < k; ++q)
            GB_CHECK(run(q, levels + q * row, parents ? parents + q * row : nullptr));
    } else {
        GB_CHECK(lb.alloc(2 * row * 4));
        if (parents) GB_CHECK(pb.alloc(2 * row * 4));
        CopyPipe cp;
        GB_CHECK(cp.init());
        for (uint32_t q = 0; q < k; ++q) {
            const int b = q & 1;
            int32_t *dl = lb.as<int32_t>() + b * row;
            int32_t *dp = parents ? pb.as<int32_t>() + b * row : nullptr;
            if (q >= 2) GB_CUDA(cudaStreamWaitEvent(ctx->stream, cp.copied[b], 0));
            GB_CHECK(run(q, dl, dp));
            GB_CUDA(cudaEventRecord(cp.done[b], ctx->stream));
            GB_CUDA(cudaStreamWaitEvent(cp.cs, cp.done[b], 0));
            GB_CUDA(cudaMemcpyAsync(levels + q * row, dl, row * 4, cudaMemcpyDeviceToHost, cp.cs));
            if (dp) GB_CUDA(cudaMemcpyAsync(parents + q * row, dp, row * 4, cudaMemcpyDeviceToHost, cp.cs));
            GB_CUDA(cudaEventRecord(cp.copied[b], cp.cs));
        }
        GB_CUDA(cudaStreamSynchronize(cp.cs));
    }
    int herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (herr) return fail(GB_TIMEOUT, "gb_bfs_batch: a run's bounded device wait ran out");
    return GB_SUCCESS;
}

// ------------------------------------------------------------------------
// BFS without any device allocation: the scratch (bitmaps, frontier lists,
// working state) lives in one array compiled into this library, so the call
// path never calls cudaMalloc/cudaFree. It serves callers that cannot
// allocate device memory when they run a traversal: a process whose device
// memory is owned by another allocator (a framework's caching allocator or
// a fixed arena), a latency-critical loop that cannot afford the device-wide
// synchronisation cudaFree implies, or a deployment that forbids dynamic
// allocation after start-up. The array has room for graphs of up to
// GB_NOALLOC_MAX_VERTICES vertices and stays resident on every GPU that
// loads the library until the process exits.
namespace gbx {
namespace noalloc {
constexpr size_t MAX_N = GB_NOALLOC_MAX_VERTICES;
constexpr size_t NW = (MAX_N + 31) / 32;
constexpr size_t LIST = 2 * (MAX_N + 1) * sizeof(uint32_t);
constexpr size_t OFF_VISITED = 0;
constexpr size_t OFF_FRONT = OFF_VISITED + NW * 4;
constexpr size_t OFF_Q = ((OFF_FRONT + 3 * NW * 4) + 255) / 256 * 256;
constexpr size_t OFF_QP = OFF_Q + (LIST + 255) / 256 * 256;
constexpr size_t OFF_QR = OFF_QP + (LIST + 255) / 256 * 256;
constexpr size_t OFF_UL = OFF_QR + (LIST + 255) / 256 * 256;
constexpr size_t OFF_ST = OFF_UL + (LIST + 255) / 256 * 256;
constexpr size_t BYTES = OFF_ST + (sizeof(BfsState) + 255) / 256 * 256;

struct Device {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of the scratch array on this device
    int grid = 0;
};
constexpr int MAX_DEVICES = 64;
std::mutex mu;
Device devices[MAX_DEVICES];
}  // namespace noalloc

// The scratch array. In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress (done once per device).
static __device__ __align__(256) unsigned char g_bfs_scratch[noalloc::BYTES];

}  // namespace gbx

extern "C" gb_info gb_bfs_noalloc(const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *colptr,
                                  const uint32_t *rowidx, uint32_t n, uint64_t nnz, uint32_t src, int32_t *levels,
                                  int32_t *parents, int32_t *status, void *stream) {
    using namespace gbx::noalloc;
    if (!rowptr || !colidx || !levels) return fail(GB_NULL_POINTER, "gb_bfs_noalloc: NULL argument");
    if ((colptr == nullptr) != (rowidx == nullptr))
        return fail(GB_NULL_POINTER, "gb_bfs_noalloc: colptr and rowidx must both be given or both be NULL");
    if (n == 0 || n > MAX_N)
        return fail(GB_INVALID_VALUE, "gb_bfs_noalloc: n = %u vertices, but the built-in scratch holds 1..%u",
                    n, (unsigned)MAX_N);
    if (nnz >= (1ull << 32)) return fail(GB_INVALID_VALUE, "gb_bfs_noalloc: nnz must be < 2^32");
    if (src >= n) return fail(GB_INVALID_INDEX, "gb_bfs_noalloc: source %u out of range", src);
    if (((uintptr_t)colidx & 15) || ((uintptr_t)rowidx & 15))
        return fail(GB_INVALID_VALUE, "gb_bfs_noalloc: colidx and rowidx must be 16-byte aligned");
    if ((uintptr_t)status & 3) return fail(GB_INVALID_VALUE, "gb_bfs_noalloc: status must be 4-byte aligned");
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(GB_INVALID_VALUE, "gb_bfs_noalloc: device %d unsupported", dev);
    Device *D = &devices[dev];
    {
        // set-up on the first call for this device (with it current)
        std::lock_guard<std::mutex> g(mu);
        if (!D->ready) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_bfs_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_bfs_scratch)", __FILE__, __LINE__);
            int occ = 0, sms = 0;
            GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bfsk::bfs_kernel(0), bfsk::BLOCK, 0));
            GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            if (occ < 1) return fail(GB_PANIC, "gb_bfs_noalloc: BFS kernel cannot be resident");
            D->base = (unsigned char *)p;
            D->grid = occ * sms;
            D->ready = true;
        }
    }
    unsigned char *base = D->base;
    cudaStream_t s = (cudaStream_t)stream;
    BfsArgs a;
    a.n = n;
    a.nwords = (n + 31) / 32;
    a.m = nnz;
    a.src = src;
    a.rp_out = rowptr;
    a.ci_out = colidx;
    a.rp_in = colptr;
    a.ci_in = rowidx;
    a.csr_is_csc = colptr == rowptr && rowidx == colidx;
    a.levels = levels;
    a.parents = parents;
    a.visited = (uint32_t *)(base + OFF_VISITED);
    for (int k = 0; k < 3; ++k) a.front[k] = (uint32_t *)(base + OFF_FRONT) + (size_t)k * a.nwords;
    a.q[0] = (uint32_t *)(base + OFF_Q); a.q[1] = a.q[0] + n + 1;
    a.qp[0] = (uint32_t *)(base + OFF_QP); a.qp[1] = a.qp[0] + n + 1;
    a.qr[0] = (uint32_t *)(base + OFF_QR); a.qr[1] = a.qr[0] + n + 1;
    a.live_rec = nullptr;        // no live table here: the first pull takes every vertex
    a.live_count = nullptr;
    a.ul[0] = (uint32_t *)(base + OFF_UL); a.ul[1] = (uint32_t *)(base + OFF_UL) + n + 1;
    a.comp_size = nullptr;
    a.ebits = 64 - bits_for((uint64_t)n + 1);
    a.emask = (1ull << a.ebits) - 1;
    a.mode = GB_AUTO;
    a.beta = 10u;
    a.st = (BfsState *)(base + OFF_ST);
    a.timeout_ns = 4000000000ull;
    a.total_limit_ns = 120000000000ull;
    a.err_sticky = nullptr;
    a.status_out = status;   // the caller's word: 0 or GB_TIMEOUT once the kernel has finished
    a.withhold = false;
    if (const uint64_t t = test_withhold_ns()) {
        a.timeout_ns = t;
        a.withhold = true;
    }
    // the kernel needs a zeroed working state; the last call's contents may remain
    GB_CUDA(cudaMemsetAsync(a.st, 0, sizeof(BfsState), s));
    void *args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel(bfsk::bfs_kernel(0), dim3(D->grid), dim3(bfsk::BLOCK), args, 0, s));
    return GB_SUCCESS;
}

// Autotuner of the push/pull switch (Table 9's rule pull iff |E_f| > |E|/beta):
// times BFS from the given sources for each candidate beta with CUDA
// events on the context stream and keeps the fastest on the matrix.
extern "C" gb_info gb_bfs_autotune(gb_context *ctx, gb_matrix *A, const uint32_t *srcs, uint32_t k,
                                   uint32_t *best_beta, double *best_ms) {
    if (!ctx || !A || !srcs || !best_beta) return fail(GB_NULL_POINTER, "gb_bfs_autotune: NULL argument");
    if (!A->built || A->nrows != A->ncols) return fail(GB_INVALID_VALUE, "gb_bfs_autotune: needs a built square matrix");
    if (k == 0) return fail(GB_INVALID_VALUE, "gb_bfs_autotune: no sources");
    for (uint32_t q = 0; q < k; ++q)
        if (srcs[q] >= A->nrows) return fail(GB_INVALID_INDEX, "gb_bfs_autotune: source out of range");
    GB_CUDA(cudaSetDevice(ctx->device));
    BfsWorkspace *w = nullptr;
    GB_CHECK(bfs_workspace(ctx, A->nrows, &w));
    Scratch lv(ctx), pa(ctx);
    GB_CHECK(lv.alloc((size_t)A->nrows * 4 + 16));
    GB_CHECK(pa.alloc((size_t)A->nrows * 4 + 16));
    static const uint32_t cand[] = {4, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 96, 128, 192, 256};
    constexpr int NC = sizeof(cand) / sizeof(cand[0]);
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    gb_desc d;
    double tmin[NC];
    for (int c = 0; c < NC; ++c) tmin[c] = 1e30;
    // the threshold is tuned with the default tile shape, the shape at the
    // chosen threshold
    A->bfs_pull_width = 0;
    A->bfs_blocks_per_sm = 0;
    // two passes over the candidates, forward then backward, keeping each
    // candidate's faster pass (so a slow drift of the clock favours none)
    for (int pass = 0; pass < 2; ++pass) {
        for (int ci = 0; ci < NC; ++ci) {
            const int c = pass == 0 ? ci : NC - 1 - ci;
            d.beta = (int)cand[c];
            // one warm launch, then the timed set
            gb_info r = bfs_launch(ctx, A, srcs[0], lv.as<int32_t>(), pa.as<int32_t>(), &d, w, 0);
            if (r == GB_SUCCESS) r = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? GB_SUCCESS : GB_PANIC;
            for (uint32_t q = 0; q < k && r == GB_SUCCESS; ++q)
                r = bfs_launch(ctx, A, srcs[q], lv.as<int32_t>(), pa.as<int32_t>(), &d, w, 0);
            if (r == GB_SUCCESS && cudaEventRecord(e1, ctx->stream) != cudaSuccess) r = GB_PANIC;
            if (r == GB_SUCCESS && cudaEventSynchronize(e1) != cudaSuccess) r = GB_PANIC;
            if (r != GB_SUCCESS) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return r == GB_PANIC ? fail(GB_PANIC, "gb_bfs_autotune: CUDA error") : r;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < tmin[c]) tmin[c] = ms;
        }
    }
    double best = 1e30;
    uint32_t bb = 10;
    for (int c = 0; c < NC; ++c)
        if (tmin[c] < best) { best = tmin[c]; bb = cand[c]; }
    // tile shape at that threshold: pull candidates per lane in flight x
    // blocks per SM, timed the same way (two passes, the faster kept); the
    // default shape's time is the threshold pass's
    {
        static const uint32_t widths[] = {1, 2, 4};
        static const uint32_t per_sm[] = {1, 0};   // one block per SM, or as many as fit
        constexpr int NP = 2, NS = 3 * NP;
        double ts[NS];
        for (int c = 0; c < NS; ++c) ts[c] = 1e30;
        d.beta = (int)bb;
        for (int pass = 0; pass < 2; ++pass) {
            for (int ci = 0; ci < NS; ++ci) {
                const int c = pass == 0 ? ci : NS - 1 - ci;
                A->bfs_pull_width = widths[c / NP];
                A->bfs_blocks_per_sm = per_sm[c % NP];
                gb_info r = bfs_launch(ctx, A, srcs[0], lv.as<int32_t>(), pa.as<int32_t>(), &d, w, 0);
                if (r == GB_SUCCESS) r = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? GB_SUCCESS : GB_PANIC;
                for (uint32_t q = 0; q < k && r == GB_SUCCESS; ++q)
                    r = bfs_launch(ctx, A, srcs[q], lv.as<int32_t>(), pa.as<int32_t>(), &d, w, 0);
                if (r == GB_SUCCESS && cudaEventRecord(e1, ctx->stream) != cudaSuccess) r = GB_PANIC;
                if (r == GB_SUCCESS && cudaEventSynchronize(e1) != cudaSuccess) r = GB_PANIC;
                if (r != GB_SUCCESS) {
                    A->bfs_pull_width = 0;
                    A->bfs_blocks_per_sm = 0;
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return r == GB_PANIC ? fail(GB_PANIC, "gb_bfs_autotune: CUDA error") : r;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < ts[c]) ts[c] = ms;
            }
        }
        uint32_t bw = 0, bp = 0;
        for (int c = 0; c < NS; ++c)
            if (ts[c] < best) { best = ts[c]; bw = widths[c / NP]; bp = per_sm[c % NP]; }
        A->bfs_pull_width = bw;
        A->bfs_blocks_per_sm = bp;
    }
    // the single-cluster schedule, timed the same way (two passes)
    int sched = GB_SCHED_GRID;
    if (bfs_cluster_available(ctx)) {
        double tcl = 1e30;
        // one untimed and one timed launch first: a schedule four times slower
        // per BFS than the best grid one is not timed any further
        bool hopeless = false;
        {
            gb_info r = bfs_cluster_run(ctx, A, srcs[0], lv.as<int32_t>(), pa.as<int32_t>(), w);
            if (r == GB_SUCCESS) r = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? GB_SUCCESS : GB_PANIC;
            if (r == GB_SUCCESS) r = bfs_cluster_run(ctx, A, srcs[0], lv.as<int32_t>(), pa.as<int32_t>(), w);
            if (r == GB_SUCCESS && cudaEventRecord(e1, ctx->stream) != cudaSuccess) r = GB_PANIC;
            if (r == GB_SUCCESS && cudaEventSynchronize(e1) != cudaSuccess) r = GB_PANIC;
            if (r != GB_SUCCESS) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return r == GB_PANIC ? fail(GB_PANIC, "gb_bfs_autotune: CUDA error") : r;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            hopeless = (double)ms > 4.0 * best / k;
        }
        for (int pass = 0; pass < 2 && !hopeless; ++pass) {
            gb_info r = bfs_cluster_run(ctx, A, srcs[0], lv.as<int32_t>(), pa.as<int32_t>(), w);
            if (r == GB_SUCCESS) r = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? GB_SUCCESS : GB_PANIC;
            for (uint32_t q = 0; q < k && r == GB_SUCCESS; ++q)
                r = bfs_cluster_run(ctx, A, srcs[q], lv.as<int32_t>(), pa.as<int32_t>(), w);
            if (r == GB_SUCCESS && cudaEventRecord(e1, ctx->stream) != cudaSuccess) r = GB_PANIC;
            if (r == GB_SUCCESS && cudaEventSynchronize(e1) != cudaSuccess) r = GB_PANIC;
            if (r != GB_SUCCESS) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return r == GB_PANIC ? fail(GB_PANIC, "gb_bfs_autotune: CUDA error") : r;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < tcl) tcl = ms;
        }
        if (tcl < best) { best = tcl; sched = GB_SCHED_CLUSTER; }
    }
    // the barrier-free schedule (levels by unit-weight relaxation, then the
    // parents), timed the same way after one untimed run and a hopeless check
    {
        double ta = 1e30;
        bool hopeless = false;
        for (int pass = 0; pass < 3 && !hopeless; ++pass) {
            const uint32_t kk = pass == 0 ? 1u : k;
            gb_info r = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? GB_SUCCESS : GB_PANIC;
            for (uint32_t q = 0; q < kk && r == GB_SUCCESS; ++q)
                r = async_relax_run(ctx, A, 1, srcs[q], lv.as<uint32_t>(), pa.as<uint32_t>(), 0, nullptr,
                                    "gb_bfs_autotune");
            if (r == GB_SUCCESS && cudaEventRecord(e1, ctx->stream) != cudaSuccess) r = GB_PANIC;
            if (r == GB_SUCCESS && cudaEventSynchronize(e1) != cudaSuccess) r = GB_PANIC;
            if (r != GB_SUCCESS) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return r == GB_PANIC ? fail(GB_PANIC, "gb_bfs_autotune: CUDA error") : r;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass == 0) hopeless = (double)ms > 4.0 * best / k;   // the first run also warms the schedule up
            else if (ms < ta) ta = ms;
        }
        if (ta < best) { best = ta; sched = GB_SCHED_ASYNC; }
    }
    A->tuned_schedule = sched;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    A->tuned_beta = bb;
    *best_beta = bb;
    if (best_ms) *best_ms = best / k;
    return GB_SUCCESS;
}

extern "C" gb_info gb_bfs_set_shape(gb_matrix *A, uint32_t pull_width, uint32_t blocks_per_sm) {
    if (!A) return fail(GB_NULL_POINTER, "gb_bfs_set_shape: NULL matrix");
    if (pull_width != 0 && pull_width != 1 && pull_width != 2 && pull_width != 4)
        return fail(GB_INVALID_VALUE, "gb_bfs_set_shape: pull width %u is not 0, 1, 2 or 4", pull_width);
    if (blocks_per_sm > 4)
        return fail(GB_INVALID_VALUE, "gb_bfs_set_shape: %u blocks per SM (at most 4)", blocks_per_sm);
    A->bfs_pull_width = pull_width;
    A->bfs_blocks_per_sm = blocks_per_sm;
    return GB_SUCCESS;
}

extern "C" gb_info gb_bfs_get_shape(const gb_matrix *A, uint32_t *pull_width, uint32_t *blocks_per_sm) {
    if (!A || !pull_width || !blocks_per_sm) return fail(GB_NULL_POINTER, "gb_bfs_get_shape: NULL argument");
    *pull_width = A->bfs_pull_width ? A->bfs_pull_width : (uint32_t)bfsk::PULL_WPW;
    *blocks_per_sm = A->bfs_blocks_per_sm;
    return GB_SUCCESS;
}
