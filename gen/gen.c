/*
 * Seeded synthetic graph inputs (R-MAT and 2-D grid), shared by the oracle
 * and the CUDA path. This file holds none of the method's arithmetic: it only
 * emits edge tuples (u, v, w) and picks source vertices. Matrix build
 * (sorting, duplicate removal, offsets) happens independently on each side.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: every draw is mix(mix(seed, stream) + counter), so any edge can
 * be generated independently and in parallel with the same result.
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with the paper's parameters
 * a=0.57 b=0.19 c=0.19 d=0.05 (Section 8, dataset paragraph). Quadrants are
 * chosen with integer thresholds floor(p * 2^32) so that no floating-point
 * rounding can make two machines disagree.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define STREAM_RMAT   0x524d4154ull   /* quadrant draws */
#define STREAM_PERM   0x5045524dull   /* vertex permutation */
#define STREAM_WEIGHT 0x57474854ull   /* edge weights */
#define STREAM_DEL    0x44454c45ull   /* grid edge deletion */
#define STREAM_SRC    0x53524320ull   /* source choice */

static inline uint64_t sm64_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One counter-based draw: 64 random bits for (seed, stream, counter). */
uint64_t gen_draw(uint64_t seed, uint64_t stream, uint64_t counter) {
    return sm64_mix(sm64_mix(seed ^ sm64_mix(stream)) + counter);
}

/* Symmetric edge weight in [1, wmax]: a function of the unordered pair only,
 * so (u,v) and (v,u) and every duplicate of {u,v} carry the same weight. */
uint32_t gen_edge_weight(uint64_t seed, uint32_t u, uint32_t v, uint32_t wmax) {
    uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
    if (wmax == 0) return 1u;
    return (uint32_t)(1u + gen_draw(seed, STREAM_WEIGHT, (hi << 32) | lo) % wmax);
}

/* Seeded random permutation of [0, n) by Fisher-Yates (Durstenfeld). */
void gen_permutation(uint64_t seed, uint32_t n, uint32_t *perm) {
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n; i > 1; --i) {
        uint32_t j = (uint32_t)(gen_draw(seed, STREAM_PERM, i) % i);
        uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
    }
}

/*
 * R-MAT edges. Generates nedges = edgefactor * 2^scale directed tuples, maps
 * both endpoints through a seeded vertex permutation, drops self-loops and
 * emits each remaining edge in both directions (the graph is undirected).
 * Duplicates are kept: removing them is the matrix build's job.
 * thr[0..2] are the cumulative quadrant thresholds floor(a*2^32),
 * floor((a+b)*2^32), floor((a+b+c)*2^32).
 * Output arrays must hold 2 * nedges entries; w may be NULL.
 * Returns the number of tuples written.
 */
uint64_t gen_rmat(uint32_t scale, uint32_t edgefactor, const uint32_t thr[3],
                  uint64_t seed, uint32_t wmax, int permute,
                  uint32_t *src, uint32_t *dst, uint32_t *w) {
    uint64_t n = 1ull << scale;
    uint64_t nedges = (uint64_t)edgefactor << scale;
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!perm) return 0;
    if (permute) gen_permutation(seed, (uint32_t)n, perm);
    else for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;

    /* each edge is independent: fill slot 2e and 2e+1, mark self-loops */
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)nedges; ++e) {
        uint64_t r = 0, c = 0;
        for (uint32_t l = 0; l < scale; ++l) {
            uint32_t x = (uint32_t)gen_draw(seed, STREAM_RMAT, (uint64_t)e * 64u + l);
            uint32_t rb, cb;
            if (x < thr[0])      { rb = 0; cb = 0; }
            else if (x < thr[1]) { rb = 0; cb = 1; }
            else if (x < thr[2]) { rb = 1; cb = 0; }
            else                 { rb = 1; cb = 1; }
            r = (r << 1) | rb;
            c = (c << 1) | cb;
        }
        uint32_t u = perm[r], v = perm[c];
        src[2 * e] = u; dst[2 * e] = v;
        src[2 * e + 1] = v; dst[2 * e + 1] = u;
        if (w) {
            uint32_t ww = gen_edge_weight(seed, u, v, wmax);
            w[2 * e] = ww; w[2 * e + 1] = ww;
        }
    }
    free(perm);
    /* compact away self-loops (stable, keeps tuple order) */
    uint64_t k = 0;
    for (uint64_t t = 0; t < 2 * nedges; ++t) {
        if (src[t] == dst[t]) continue;
        src[k] = src[t]; dst[k] = dst[t];
        if (w) w[k] = w[t];
        ++k;
    }
    return k;
}

/*
 * rows x cols 4-neighbour lattice, vertex id = r * cols + c. Each undirected
 * lattice edge is deleted independently with probability del_thr / 2^32.
 * Emits both directions of every kept edge; arrays must hold
 * 2 * (rows*(cols-1) + (rows-1)*cols) entries. Returns tuples written.
 */
uint64_t gen_grid(uint32_t rows, uint32_t cols, uint32_t del_thr, uint64_t seed,
                  uint32_t wmax, uint32_t *src, uint32_t *dst, uint32_t *w) {
    uint64_t k = 0;
    for (uint64_t r = 0; r < rows; ++r) {
        for (uint64_t c = 0; c < cols; ++c) {
            uint64_t id = r * cols + c;
            for (int dir = 0; dir < 2; ++dir) {
                uint64_t nb;
                if (dir == 0) { if (c + 1 >= cols) continue; nb = id + 1; }
                else          { if (r + 1 >= rows) continue; nb = id + cols; }
                uint32_t x = (uint32_t)gen_draw(seed, STREAM_DEL, 2 * id + dir);
                if (x < del_thr) continue;
                uint32_t ww = w ? gen_edge_weight(seed, (uint32_t)id, (uint32_t)nb, wmax) : 0;
                src[k] = (uint32_t)id; dst[k] = (uint32_t)nb; if (w) w[k] = ww; ++k;
                src[k] = (uint32_t)nb; dst[k] = (uint32_t)id; if (w) w[k] = ww; ++k;
            }
        }
    }
    return k;
}

/*
 * k distinct source vertices drawn uniformly from those that touch at least
 * one tuple (non-isolated), in draw order. has_edge is a byte per vertex.
 * Returns the number chosen (< k only if fewer candidates exist).
 */
uint32_t gen_sources(uint64_t seed, uint32_t n, const uint8_t *has_edge,
                     uint32_t k, uint32_t *out) {
    uint64_t cand = 0;
    for (uint32_t i = 0; i < n; ++i) cand += has_edge[i] != 0;
    if (cand < k) k = (uint32_t)cand;
    uint8_t *taken = (uint8_t *)calloc(n ? n : 1, 1);
    uint32_t got = 0;
    for (uint64_t t = 0; got < k; ++t) {
        uint32_t v = (uint32_t)(gen_draw(seed, STREAM_SRC, t) % n);
        if (!has_edge[v] || taken[v]) continue;
        taken[v] = 1;
        out[got++] = v;
    }
    free(taken);
    return got;
}

/* byte flag per vertex: 1 if the vertex appears in any tuple */
void gen_touched(uint32_t n, uint64_t ntuples, const uint32_t *src, uint8_t *has_edge) {
    memset(has_edge, 0, n);
    for (uint64_t t = 0; t < ntuples; ++t) has_edge[src[t]] = 1;
}
