/*
 * ORACLE -- test infrastructure only. Plain, slow, single-threaded CPU
 * definitions of what the CUDA path computes. Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this library; the
 * product path never does. It shares no code with the CUDA library.
 *
 * Every function states the passage of the paper (Yang, Buluc, Owens,
 * "GraphBLAST", ACM TOMS 2021, arXiv 1908.01407) that it follows. Where the
 * method reaches an exact result with a plain definition (BFS depths,
 * shortest distances, components, triangle counts) the oracle is that
 * definition; PageRank is an iteration and is run in the paper's order, in
 * double precision.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* Matrix build (Section 4.3: CSR storage; Table 4 "build" with a dup  */
/* operator combining repeated (i, j) tuples).                          */
/* ------------------------------------------------------------------ */
enum { ORC_DUP_FIRST = 0, ORC_DUP_SECOND = 1, ORC_DUP_PLUS = 2, ORC_DUP_MIN = 3, ORC_DUP_MAX = 4 };

typedef struct { uint32_t col; uint64_t pos; } orc_entry;

static int cmp_entry(const void *a, const void *b) {
    const orc_entry *x = (const orc_entry *)a, *y = (const orc_entry *)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/*
 * Builds CSR (rowptr[n+1], colidx, optional vals) from ntup (row, col[, val])
 * tuples. Columns within a row are sorted ascending; tuples with equal
 * (row, col) are combined by `dup` in tuple order. Returns the number of
 * stored entries, or -1 on an out-of-range index / allocation failure.
 */
int64_t orc_csr_build(uint32_t nrows, uint32_t ncols, uint64_t ntup,
                      const uint32_t *rows, const uint32_t *cols, const uint32_t *vals,
                      int dup, uint64_t *rowptr, uint32_t *colidx, uint32_t *outvals) {
    uint64_t *cnt = (uint64_t *)calloc((size_t)nrows + 1, sizeof(uint64_t));
    orc_entry *ent = (orc_entry *)malloc(sizeof(orc_entry) * (ntup ? ntup : 1));
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)nrows + 1));
    if (!cnt || !ent || !fill) { free(cnt); free(ent); free(fill); return -1; }
    for (uint64_t t = 0; t < ntup; ++t) {
        if (rows[t] >= nrows || cols[t] >= ncols) { free(cnt); free(ent); free(fill); return -1; }
        cnt[rows[t] + 1]++;
    }
    for (uint32_t i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
    memcpy(fill, cnt, sizeof(uint64_t) * ((size_t)nrows + 1));
    for (uint64_t t = 0; t < ntup; ++t) {
        uint64_t p = fill[rows[t]]++;
        ent[p].col = cols[t];
        ent[p].pos = t;
    }
    uint64_t out = 0;
    rowptr[0] = 0;
    for (uint32_t i = 0; i < nrows; ++i) {
        uint64_t b = cnt[i], e = cnt[i + 1];
        qsort(ent + b, (size_t)(e - b), sizeof(orc_entry), cmp_entry);
        for (uint64_t p = b; p < e; ++p) {
            uint32_t v = vals ? vals[ent[p].pos] : 0;
            if (p > b && ent[p].col == ent[p - 1].col) {
                if (outvals) {
                    uint32_t *acc = &outvals[out - 1];
                    switch (dup) {
                    case ORC_DUP_FIRST: break;
                    case ORC_DUP_SECOND: *acc = v; break;
                    case ORC_DUP_PLUS: *acc = *acc + v; break;
                    case ORC_DUP_MIN: if (v < *acc) *acc = v; break;
                    case ORC_DUP_MAX: if (v > *acc) *acc = v; break;
                    }
                }
                continue;
            }
            colidx[out] = ent[p].col;
            if (outvals) outvals[out] = v;
            ++out;
        }
        rowptr[i + 1] = out;
    }
    free(cnt); free(ent); free(fill);
    return (int64_t)out;
}

/* ------------------------------------------------------------------ */
/* BFS (Algorithm 1; Section 7.1): depth of every vertex from s.        */
/* Plain FIFO-queue breadth-first search. level[s] = 0, unreachable -1  */
/* (the paper counts the source as depth 1 and unvisited as 0; this is  */
/* that value minus one).                                               */
/* ------------------------------------------------------------------ */
void orc_bfs(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx,
             uint32_t src, int32_t *level) {
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; ++i) level[i] = -1;
    if (src >= n) { free(queue); return; }
    uint64_t head = 0, tail = 0;
    level[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
            uint32_t v = colidx[p];
            if (level[v] < 0) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
}

static int has_edge(const uint64_t *rowptr, const uint32_t *colidx, uint32_t u, uint32_t v) {
    uint64_t lo = rowptr[u], hi = rowptr[u + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (colidx[mid] == v) return 1;
        if (colidx[mid] < v) lo = mid + 1; else hi = mid;
    }
    return 0;
}

/*
 * Checks a BFS parent array against exact levels (Section 7.1: BFS yields
 * a spanning tree of shortest paths). Valid iff parent[s] = s, every reached
 * v != s has an edge (parent[v], v) with level[parent[v]] = level[v] - 1,
 * and unreached vertices have parent -1. Needs sorted CSR rows.
 * Returns the number of violating vertices.
 */
uint64_t orc_bfs_parent_violations(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx,
                                   uint32_t src, const int32_t *level, const int32_t *parent) {
    uint64_t bad = 0;
    for (uint32_t v = 0; v < n; ++v) {
        if (level[v] < 0) { bad += parent[v] != -1; continue; }
        if (v == src) { bad += parent[v] != (int32_t)src; continue; }
        int32_t p = parent[v];
        if (p < 0 || (uint32_t)p >= n) { ++bad; continue; }
        if (level[p] != level[v] - 1) { ++bad; continue; }
        if (!has_edge(rowptr, colidx, (uint32_t)p, v)) { ++bad; continue; }
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* SSSP (Section 7.2): exact shortest distances. The paper's adaptive   */
/* Bellman-Ford converges to the shortest-path distances; the plain     */
/* definition is Dijkstra's algorithm with a binary heap. Distances are */
/* summed in 64 bits; unreachable = UINT32_MAX.                         */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t d; uint32_t v; } heap_item;

static void heap_push(heap_item *h, uint64_t *sz, heap_item x) {
    uint64_t i = (*sz)++;
    h[i] = x;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, uint64_t *sz) {
    heap_item top = h[0];
    h[0] = h[--(*sz)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *sz && h[l].d < h[m].d) m = l;
        if (r < *sz && h[r].d < h[m].d) m = r;
        if (m == i) break;
        heap_item t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

/* returns 0, or -1 if a finite distance does not fit below UINT32_MAX */
int orc_sssp(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx,
             const uint32_t *weight, uint32_t src, uint32_t *dist_out) {
    uint64_t *dist = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint64_t m = rowptr[n];
    heap_item *heap = (heap_item *)malloc(sizeof(heap_item) * (m + 2));
    uint64_t sz = 0;
    int rc = 0;
    for (uint32_t i = 0; i < n; ++i) dist[i] = UINT64_MAX;
    if (src < n) {
        dist[src] = 0;
        heap_item s = {0, src};
        heap_push(heap, &sz, s);
    }
    while (sz > 0) {
        heap_item it = heap_pop(heap, &sz);
        if (it.d != dist[it.v]) continue;   /* stale entry */
        uint32_t u = it.v;
        for (uint64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
            uint64_t nd = dist[u] + weight[p];
            uint32_t v = colidx[p];
            if (nd < dist[v]) {
                dist[v] = nd;
                heap_item x = {nd, v};
                heap_push(heap, &sz, x);
            }
        }
    }
    for (uint32_t i = 0; i < n; ++i) {
        if (dist[i] == UINT64_MAX) dist_out[i] = UINT32_MAX;
        else if (dist[i] >= UINT32_MAX) { dist_out[i] = UINT32_MAX; rc = -1; }
        else dist_out[i] = (uint32_t)dist[i];
    }
    free(dist); free(heap);
    return rc;
}

/* ------------------------------------------------------------------ */
/* PageRank (Section 7.3): pull formulation, p' = (1-a)/n + a * (A^T   */
/* scaled p). Each vertex j shares p(j) equally among its deg(j)        */
/* neighbours; the mass of vertices with no edges is spread uniformly   */
/* (the paper leaves dangling vertices unaddressed; this reading keeps  */
/* sum(p) = 1). p0 = 1/n, exactly `iters` iterations, FP64 throughout.  */
/* residual[k] = sum_i |p_k+1(i) - p_k(i)|.                             */
/* ------------------------------------------------------------------ */
/* rowptr/colidx list each vertex's in-neighbours; out_rowptr gives the  */
/* out-degrees (NULL: the same structure, a symmetric graph).           */
void orc_pagerank(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx, const uint64_t *out_rowptr,
                  double alpha, uint32_t iters, double *p, double *residual) {
    const uint64_t *od = out_rowptr ? out_rowptr : rowptr;
    double *q = (double *)malloc(sizeof(double) * (n ? n : 1));
    for (uint32_t i = 0; i < n; ++i) p[i] = 1.0 / n;
    for (uint32_t it = 0; it < iters; ++it) {
        double dangling = 0.0;
        for (uint32_t j = 0; j < n; ++j)
            if (od[j + 1] == od[j]) dangling += p[j];
        for (uint32_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (uint64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                uint32_t j = colidx[e];
                s += p[j] / (double)(od[j + 1] - od[j]);
            }
            q[i] = (1.0 - alpha) / n + alpha * (s + dangling / n);
        }
        double r = 0.0;
        for (uint32_t i = 0; i < n; ++i) { r += fabs(q[i] - p[i]); p[i] = q[i]; }
        if (residual) residual[it] = r;
    }
    free(q);
}

/* ------------------------------------------------------------------ */
/* Adaptive PageRank, also called PageRankDelta (Section 5.1 lists it   */
/* among the uses of the output mask; Section 7.3 names it and leaves it */
/* out). The recurrence of orc_pagerank, except that a vertex whose value */
/* moved by at most eps times its new value in an iteration has          */
/* converged: it is masked out of every later iteration (its value stays */
/* as it is, and other vertices keep reading it). The decision           */
/* |p'(i) - p(i)| <= eps * p'(i) is taken on the values rounded to FP32, */
/* in FP32 arithmetic, the precision of the GPU path; everything else is */
/* FP64. The dangling mass D = sum of p over vertices without edges is   */
/* taken over all of them, frozen or not. Stops when no vertex is active */
/* or after max_iters iterations; returns the iterations run.            */
/* active[k] = vertices updated in iteration k (may be NULL).            */
/* ------------------------------------------------------------------ */
uint32_t orc_pagerank_delta(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx, const uint64_t *out_rowptr,
                            double alpha, float eps, uint32_t max_iters, double *p, uint32_t *active) {
    const uint64_t *od = out_rowptr ? out_rowptr : rowptr;
    double *q = (double *)malloc(sizeof(double) * (n ? n : 1));
    unsigned char *on = (unsigned char *)malloc(n ? n : 1);
    uint32_t nact = n, it = 0;
    for (uint32_t i = 0; i < n; ++i) { p[i] = 1.0 / n; on[i] = 1; }
    while (it < max_iters && nact > 0) {
        if (active) active[it] = nact;
        double dangling = 0.0;
        for (uint32_t j = 0; j < n; ++j)
            if (od[j + 1] == od[j]) dangling += p[j];
        for (uint32_t i = 0; i < n; ++i) {
            if (!on[i]) { q[i] = p[i]; continue; }
            double s = 0.0;
            for (uint64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                uint32_t j = colidx[e];
                s += p[j] / (double)(od[j + 1] - od[j]);
            }
            q[i] = (1.0 - alpha) / n + alpha * (s + dangling / n);
        }
        uint32_t next = 0;
        for (uint32_t i = 0; i < n; ++i) {
            if (on[i]) {
                float a = (float)q[i], b = (float)p[i];
                if (fabsf(a - b) <= eps * a) on[i] = 0; else ++next;
            }
            p[i] = q[i];
        }
        nact = next;
        ++it;
    }
    free(q);
    free(on);
    return it;
}

/* Connected components (Section 7.4): label(v) = smallest vertex id in */
/* v's component. Union-find with path halving, union by smaller root.  */
/* ------------------------------------------------------------------ */
static uint32_t uf_find(uint32_t *par, uint32_t x) {
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

void orc_cc(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx, uint32_t *label) {
    for (uint32_t i = 0; i < n; ++i) label[i] = i;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
            uint32_t a = uf_find(label, u), b = uf_find(label, colidx[p]);
            if (a < b) label[b] = a; else if (b < a) label[a] = b;
        }
    for (uint32_t i = 0; i < n; ++i) label[i] = uf_find(label, i);
}

/* ------------------------------------------------------------------ */
/* Triangle counting (Section 7.5): the number of vertex triples        */
/* u < v < w with all three edges present. Node iterator over sorted    */
/* adjacency: for every edge u < v, count common neighbours w > v.      */
/* ------------------------------------------------------------------ */
uint64_t orc_tc(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx) {
    uint64_t total = 0;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
            uint32_t v = colidx[p];
            if (v <= u) continue;
            uint64_t a = rowptr[u], ae = rowptr[u + 1], b = rowptr[v], be = rowptr[v + 1];
            while (a < ae && b < be) {
                uint32_t x = colidx[a], y = colidx[b];
                if (x < y) ++a;
                else if (y < x) ++b;
                else { if (x > v) ++total; ++a; ++b; }
            }
        }
    }
    return total;
}

/*
 * Degree ordering for triangle counting (Section 7.5 sorts rows of L by
 * their number of nonzeros). Reading used here: new ids in order of
 * decreasing degree, ties broken by lower old id first. new_id[old] out.
 */
static const uint64_t *g_rp;
static int cmp_deg(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    uint64_t dx = g_rp[x + 1] - g_rp[x], dy = g_rp[y + 1] - g_rp[y];
    if (dx != dy) return dx > dy ? -1 : 1;
    return x < y ? -1 : (x > y);
}

void orc_degree_order(uint32_t n, const uint64_t *rowptr, uint32_t *new_id) {
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    g_rp = rowptr;
    qsort(order, n, sizeof(uint32_t), cmp_deg);
    for (uint32_t r = 0; r < n; ++r) new_id[order[r]] = r;
    free(order);
}

/*
 * Entries of the masked product C<L> = L * L over (plus, pair) for a
 * symmetric graph given by its full sorted adjacency (Section 6.3.4 masked
 * SpGEMM; Section 7.5). L is the strictly lower triangle. For the k-th
 * stored entry (i, j), j < i, of L in row-major order:
 *   C(i,j) = |{k : L(i,k) != 0 and L(k,j) != 0}| = |{k : j < k < i, (i,k), (k,j) in E}|.
 * Writes nnz(L) counts; returns their sum.
 */
uint64_t orc_masked_LL(uint32_t n, const uint64_t *rowptr, const uint32_t *colidx, uint32_t *cvals) {
    uint64_t out = 0, total = 0;
    for (uint32_t i = 0; i < n; ++i) {
        for (uint64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            uint32_t j = colidx[p];
            if (j >= i) continue;
            uint32_t c = 0;
            uint64_t a = rowptr[i], ae = rowptr[i + 1], b = rowptr[j], be = rowptr[j + 1];
            while (a < ae && b < be) {
                uint32_t x = colidx[a], y = colidx[b];
                if (x < y) ++a;
                else if (y < x) ++b;
                else { if (x > j && x < i) ++c; ++a; ++b; }
            }
            cvals[out++] = c;
            total += c;
        }
    }
    return total;
}
