/*
 * gbx.h -- C ABI of a GB300 (sm_103a) library for the masked
 * generalized-semiring graph operations of GraphBLAST (Yang, Buluc, Owens,
 * "GraphBLAST: A High-Performance Linear Algebra-based Graph Framework on
 * the GPU", ACM TOMS 2021, arXiv 1908.01407).
 *
 * Conventions (apply to every call):
 *  - Every call returns gb_info. No call aborts the process; on failure
 *    gb_last_error() gives a message (per host thread).
 *  - Objects (context, matrix, vector, descriptor, server) are opaque
 *    handles owned by the library until the matching *_free / destroy.
 *  - Input arrays are BORROWED: the call reads them before returning (or,
 *    for device pointers, in stream order before any later work on the
 *    context stream) and keeps no reference. A gb_mem argument says whether
 *    a pointer is host memory (GB_HOST) or device memory of the context's
 *    GPU (GB_DEVICE).
 *  - Outputs go into caller-provided buffers of the stated length.
 *  - All device work is ordered on the context stream (gb_context_set_stream).
 *    Calls that write to GB_HOST buffers synchronise that stream before
 *    returning; calls that write to GB_DEVICE buffers do not.
 *  - Indices are uint32: n, ncols and stored-entry counts must be < 2^32
 *    (GB_INVALID_VALUE otherwise).
 */
#ifndef GBX_H
#define GBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes, modelled on the GraphBLAS C API's GrB_Info (Section 3.3,
 * "Info is an error type ... according to the C API specification"). */
typedef enum {
    GB_SUCCESS = 0,
    GB_NO_VALUE = 1,            /* extract_element on a position with no value */
    GB_NULL_POINTER = 2,
    GB_INVALID_VALUE = 3,       /* bad enum, size >= 2^32, object not built */
    GB_INVALID_INDEX = 4,       /* an index outside the dimension */
    GB_DOMAIN_MISMATCH = 5,     /* unsupported (semiring, type) combination */
    GB_DIMENSION_MISMATCH = 6,
    GB_OUT_OF_MEMORY = 7,
    GB_NOT_IMPLEMENTED = 8,
    GB_TIMEOUT = 9,             /* a bounded device wait ran out, or server wait */
    GB_PANIC = 10,              /* a CUDA error; the message names it */
    GB_INSUFFICIENT_SPACE = 11  /* an output buffer is too small */
} gb_info;

typedef enum { GB_HOST = 0, GB_DEVICE = 1 } gb_mem;

/* Element types (the paper's Matrix<T>/Vector<T> template types, Section 3.6). */
typedef enum { GB_BOOL = 0, GB_INT32 = 1, GB_UINT32 = 2, GB_UINT64 = 3, GB_FP32 = 4, GB_FP64 = 5 } gb_type;

/* Binary operators: accumulators, dup operators and eWise operators. */
typedef enum {
    GB_NOP = 0,       /* "no accumulator" (accum argument only) */
    GB_PLUS = 1, GB_TIMES = 2, GB_MIN = 3, GB_MAX = 4, GB_LOR = 5, GB_LAND = 6,
    GB_FIRST = 7, GB_SECOND = 8, GB_PAIR = 9, GB_MINUS = 10
} gb_binop;

/* Monoids of Table 5 (operator and identity). */
typedef enum {
    GB_MONOID_PLUS = 0, GB_MONOID_TIMES = 1, GB_MONOID_MIN = 2, GB_MONOID_MAX = 3,
    GB_MONOID_LOR = 4, GB_MONOID_LAND = 5
} gb_monoid;

/* Semirings (add monoid, multiply operator): the five of Table 5, plus
 * min.second used by the connected-components listing (Appendix A.4) and
 * plus.pair used for triangle counting (Section 7.5). For integer types the
 * "plus" of MIN_PLUS/MAX_PLUS saturates at the type's max/min, so the
 * identity behaves as infinity. Supported (semiring, type) pairs:
 *   PLUS_TIMES, MIN_PLUS, MIN_TIMES: INT32 UINT32 FP32 FP64
 *   MAX_PLUS: INT32 FP32 FP64     LOR_LAND: BOOL
 *   MIN_SECOND: INT32 UINT32 FP32 FP64     PLUS_PAIR: INT32 UINT32 UINT64 FP32 */
typedef enum {
    GB_PLUS_TIMES = 0, GB_LOR_LAND = 1, GB_MIN_PLUS = 2, GB_MAX_PLUS = 3,
    GB_MIN_TIMES = 4, GB_MIN_SECOND = 5, GB_PLUS_PAIR = 6
} gb_semiring;

/* Descriptor fields and values (Table 6; Descriptor::toggle, Section 3.6). */
typedef enum {
    GB_MASK = 0,        /* value: GB_DEFAULT, or a bitwise OR of GB_SCMP and GB_STRUCTURE */
    GB_OUTP = 1,        /* GB_DEFAULT or GB_REPLACE */
    GB_INP0 = 2,        /* GB_DEFAULT or GB_TRAN */
    GB_INP1 = 3,        /* GB_DEFAULT or GB_TRAN */
    GB_DIRECTION = 4,   /* GB_AUTO (default), GB_PUSH or GB_PULL */
    GB_SWITCH_BETA = 5, /* integer beta of the push/pull rule |E_f| > |E| / beta; 0 = tuned default */
    GB_SCHEDULE = 6,    /* BFS, SSSP: GB_SCHED_AUTO (default), GB_SCHED_GRID, GB_SCHED_CLUSTER or GB_SCHED_ASYNC */
    GB_SSSP_DELTA = 7   /* SSSP: width of the distance buckets of the near-far frontier; 0 = automatic,
                           a width of at least 2^31 - 1 = no buckets (the plain changed-set iteration) */
} gb_field;

enum {
    GB_DEFAULT = 0,
    GB_SCMP = 1, GB_STRUCTURE = 2,   /* GB_MASK bits */
    GB_REPLACE = 1,                  /* GB_OUTP */
    GB_TRAN = 1,                     /* GB_INP0 / GB_INP1 */
    GB_AUTO = 0, GB_PUSH = 1, GB_PULL = 2,
    /* GB_SCHEDULE values. GRID: one persistent cooperative kernel over the
     * whole GPU, push or pull per level. CLUSTER: the whole traversal in one
     * thread-block cluster (push only, levels separated by the cluster
     * barrier; for graphs of high diameter). ASYNC: no level barriers at
     * all: one persistent launch relaxes (value, vertex) work items through a
     * ring that warps poll, until no item is in flight (the asynchronous
     * execution model of Section 9; for graphs of high diameter; gb_bfs,
     * gb_sssp; gb_cc_async is the components form). AUTO: what
     * gb_bfs_autotune chose for the matrix (BFS), GRID if it was not tuned. */
    GB_SCHED_AUTO = 0, GB_SCHED_GRID = 1, GB_SCHED_CLUSTER = 2, GB_SCHED_ASYNC = 3
};

/* Matrix build flags. */
enum {
    GB_BUILD_DEFAULT = 0,
    GB_SYMMETRIC = 1,   /* caller asserts A == A^T: the CSC copy aliases the CSR copy */
    GB_CSR_ONLY = 2     /* store CSR only (Section 4.3: users may drop one copy); push over columns is then unavailable */
};

typedef struct gb_context_t gb_context;
typedef struct gb_matrix_t gb_matrix;
typedef struct gb_vector_t gb_vector;
typedef struct gb_desc_t gb_desc;
typedef struct gb_server_t gb_server;

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`, owning a device memory pool
 * (Section 6.1 keeps a pool of device memory for temporaries) and a stream
 * (default: a new non-blocking stream). */
gb_info gb_init(int device, gb_context **ctx);
/* Orders all later work on `stream` (a cudaStream_t, e.g. torch's current
 * stream); NULL selects the legacy default stream. The stream is borrowed. */
gb_info gb_context_set_stream(gb_context *ctx, void *stream);
/* Waits for the context stream. Returns GB_TIMEOUT (once) if a BFS that
 * was launched without waiting for it (gb_bfs with GB_DEVICE outputs and no
 * stats) ran out of a bounded device wait since the last such report; its
 * outputs are then undefined. */
gb_info gb_context_synchronize(gb_context *ctx);
/* Bytes held by the context's pool and its high-water mark. */
gb_info gb_context_pool_stats(gb_context *ctx, uint64_t *held_bytes, uint64_t *peak_bytes);
/* Fault injection for tests: the next `count` pool allocations fail with
 * GB_OUT_OF_MEMORY (host-side; no GPU fault). */
gb_info gb_context_inject_alloc_failures(gb_context *ctx, uint32_t count);
/* Self-test of the bounded device waits that every persistent kernel uses
 * (their grid barriers): launches one block that waits at a barrier sized
 * for two blocks, so the wait can only run out. After limit_us (clamped to
 * 1..1,000,000) the block records GB_TIMEOUT in its status word and leaves;
 * *status receives that word (GB_TIMEOUT on a correct wait). Returns
 * GB_SUCCESS when the kernel finished and the context is still usable. The
 * paper has no counterpart: it is how failure handling is tested without a
 * GPU fault. */
gb_info gb_context_selftest_wait(gb_context *ctx, uint32_t limit_us, int32_t *status);
/* Kernel timing: while enabled, each operation records a pair of CUDA
 * events on the context stream around its main kernel launch. Enabling or
 * disabling clears earlier records. profile_get sums the recorded spans of
 * the kernel named `kernel` (e.g. "bfs", "bfs_multi", "sssp", "pagerank_spmv",
 * "cc", "tc") into *total_ms over *launches spans; it synchronises. */
gb_info gb_context_profile(gb_context *ctx, int enable);
gb_info gb_context_profile_get(gb_context *ctx, const char *kernel, double *total_ms, uint64_t *launches);
gb_info gb_finalize(gb_context *ctx);
/* Copies the calling thread's last error message (NUL-terminated). */
gb_info gb_last_error(char *buf, size_t len);
/* Library version string, e.g. "gbx 0.1 sm_103a". */
const char *gb_version(void);

/* ----------------------------------------------------------------- matrix */

/* Table 4 "Matrix": an nrows x ncols matrix of `type`, initially empty. */
gb_info gb_matrix_new(gb_matrix **A, gb_context *ctx, gb_type type, uint64_t nrows, uint64_t ncols);
/* Table 4 "build" (Section 4.3 storage): builds CSR and CSC from nvals
 * (row, col[, val]) tuples. vals == NULL builds a structural matrix whose
 * stored values are all 1 (Section 7.1 "structure-only"). Tuples with equal
 * (row, col) are combined with `dup` (PLUS/MIN/MAX/FIRST/SECOND/LOR/LAND;
 * FIRST/SECOND by tuple order). Columns within a row come out sorted.
 * rows/cols/vals live in `mem`. Index >= dimension: GB_INVALID_INDEX.
 * Rebuilding a built matrix replaces its contents. A square matrix with a
 * CSC also gets, on the device, the traversal tables of its pulls (the
 * vertices with in-edges and their heads) and the size of every vertex's
 * weakly connected component (FastSV; 4 bytes per vertex), with which a BFS
 * that has reached its source's whole component stops without expanding
 * its last frontier (the paper has neither; matrices that calls such as
 * gb_mxm or gb_matrix_tril build as results get the tables but not the
 * component sizes). */
gb_info gb_matrix_build(gb_matrix *A, const uint32_t *rows, const uint32_t *cols, const void *vals,
                        uint64_t nvals, gb_binop dup, gb_mem mem, uint32_t flags);
gb_info gb_matrix_nrows(const gb_matrix *A, uint64_t *n);
gb_info gb_matrix_ncols(const gb_matrix *A, uint64_t *n);
gb_info gb_matrix_nvals(const gb_matrix *A, uint64_t *n);
/* Table 4 "extractTuples": stored entries in CSR (row-major, sorted) order.
 * *n_inout: capacity in, count out. vals may be NULL. */
gb_info gb_matrix_extract_tuples(const gb_matrix *A, uint32_t *rows, uint32_t *cols, void *vals,
                                 uint64_t *n_inout, gb_mem mem);
/* Copies the CSR arrays: rowptr[nrows+1], colidx[nvals], vals[nvals] (may be NULL). */
gb_info gb_matrix_export_csr(const gb_matrix *A, uint32_t *rowptr, uint32_t *colidx, void *vals, gb_mem mem);
/* Copies the CSC arrays: colptr[ncols+1], rowidx[nvals], vals[nvals] (may be NULL). */
gb_info gb_matrix_export_csc(const gb_matrix *A, uint32_t *colptr, uint32_t *rowidx, void *vals, gb_mem mem);
/* L = strictly lower triangle of A (entries with col < row), CSR + CSC (Section 7.5). */
gb_info gb_matrix_tril(gb_matrix *L, const gb_matrix *A);
/* B = A with vertex v renamed new_id[v], where the order is decreasing
 * degree, ties by lower old id (Section 7.5 sorts rows by nonzero count).
 * A must be square; new_id (nrows entries, may be NULL) receives the map. */
gb_info gb_matrix_degree_order(gb_matrix *B, const gb_matrix *A, uint32_t *new_id, gb_mem mem);
gb_info gb_matrix_free(gb_matrix **A);

/* ----------------------------------------------------------------- vector */

/* Table 4 "Vector": size n, no stored values. Storage holds a dense value
 * array, a presence bitmap, and a sparse index list kept alongside
 * (Section 4.3: the backend switches dense/sparse; operand reuse). */
gb_info gb_vector_new(gb_vector **v, gb_context *ctx, gb_type type, uint64_t n);
/* Table 4 "build": stores vals[k] at idx[k] (vals == NULL stores 1);
 * duplicates combined with dup. Previous contents are cleared. */
gb_info gb_vector_build(gb_vector *v, const uint32_t *idx, const void *vals, uint64_t nvals,
                        gb_binop dup, gb_mem mem);
/* Table 4 "buildDense": every position present with vals[i] (n entries). */
gb_info gb_vector_build_dense(gb_vector *v, const void *vals, gb_mem mem);
/* Table 4 "fill": every position present with *scalar (host pointer). */
gb_info gb_vector_fill(gb_vector *v, const void *scalar);
gb_info gb_vector_set_element(gb_vector *v, uint32_t idx, const void *scalar);
/* GB_NO_VALUE if position idx holds no value. *out is a host pointer. */
gb_info gb_vector_extract_element(const gb_vector *v, uint32_t idx, void *out);
/* Stored (index, value) pairs in increasing index order; *n_inout capacity
 * in, count out; vals may be NULL. */
gb_info gb_vector_extract_tuples(const gb_vector *v, uint32_t *idx, void *vals, uint64_t *n_inout, gb_mem mem);
/* Dense view: vals[n] (absent positions get `absent_value`, host scalar)
 * and optionally present[n] bytes (1 = stored). */
gb_info gb_vector_extract_dense(const gb_vector *v, void *vals, uint8_t *present, const void *absent_value,
                                gb_mem mem);
gb_info gb_vector_size(const gb_vector *v, uint64_t *n);
gb_info gb_vector_nvals(const gb_vector *v, uint64_t *n);
/* Table 4 "dup": *out becomes a new vector equal to v. */
gb_info gb_vector_dup(gb_vector **out, const gb_vector *v);
/* Table 4 "clear": no stored values. */
gb_info gb_vector_clear(gb_vector *v);
gb_info gb_vector_free(gb_vector **v);

/* ------------------------------------------------------------- descriptor */

gb_info gb_desc_new(gb_desc **d);
gb_info gb_desc_set(gb_desc *d, gb_field field, int value);
gb_info gb_desc_get(const gb_desc *d, gb_field field, int *value);
/* Descriptor::toggle (Section 3.6): GB_MASK flips GB_SCMP, GB_OUTP flips
 * GB_REPLACE, GB_INP0/GB_INP1 flip GB_TRAN. */
gb_info gb_desc_toggle(gb_desc *d, gb_field field);
gb_info gb_desc_free(gb_desc **d);

/* ------------------------------------------------------------- operations */
/*
 * Table 7 operations with the semantics of Section 3.2 (mask), Table 6
 * (descriptor) and the GraphBLAS C API for accum/replace (Section 3.6 notes
 * the paper itself ignores accum and omits REPLACE; this library honours
 * both): with t the product,
 *   z = accum == GB_NOP ? t : accum(w, t)   (union of w and t)
 *   w(i) = z(i) where the mask allows i; elsewhere w(i) is kept, or
 *   removed under GB_REPLACE.
 * mask == NULL allows every position. A value mask allows i when it stores
 * a nonzero at i; GB_STRUCTURE allows stored positions; GB_SCMP inverts.
 * desc == NULL means all defaults. All operands of one call share a type,
 * except that a structural matrix (built without values) acts as all-ones.
 */

/* Table 7 mxv: w<mask> = accum(w, A (+).(x) u); GB_INP0 = GB_TRAN uses A^T.
 * Direction optimisation (Section 4): push = SpMSpV over the columns of A
 * (CSC) selected by u's stored entries; pull = SpMV over the rows of A
 * (CSR) the mask allows (Section 5: mask first). GB_AUTO picks push when
 * the frontier's edge count |E_f| <= |E| / beta (Table 9). */
gb_info gb_mxv(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_semiring s, const gb_matrix *A,
               const gb_vector *u, const gb_desc *desc);
/* Table 7 vxm: w<mask> = accum(w, u (+).(x) A), i.e. w(j) = (+)_i u(i) (x) A(i,j);
 * identical to mxv with A transposed (Figure 4 caption). */
gb_info gb_vxm(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_semiring s, const gb_vector *u,
               const gb_matrix *A, const gb_desc *desc);
/* Table 7 mxm (Section 6.3.4 masked SpGEMM, Section 7.5):
 * C<M> = accum(C, A (+).(x) B); GB_INP0/GB_INP1 = GB_TRAN transpose A/B.
 * With a mask M (not complemented) only the positions stored in M are
 * computed (mask first): for each M(i,j) the row A(i,:) is intersected with
 * the column B(:,j). Without a mask (M = NULL), or with GB_SCMP, the whole
 * product is formed by expanding every A(i,k) (x) B(k,j) into a tuple,
 * dropping the positions a complemented mask excludes, and sorting and
 * reducing equal positions with the semiring's add (as Section 6.3.1's
 * SpMSpV does with its expanded products); the products must number fewer
 * than 2^32 (GB_OUT_OF_MEMORY otherwise). Then accum, the mask and
 * GB_REPLACE act as for the other operations (C may be empty or hold any
 * entries). GB_SCMP with M = NULL allows no position. */
gb_info gb_mxm(gb_matrix *C, const gb_matrix *M, gb_binop accum, gb_semiring s, const gb_matrix *A,
               const gb_matrix *B, const gb_desc *desc);
/* Table 7 eWiseAdd (union) and eWiseMult (intersection) of vectors with a
 * binary operator. */
gb_info gb_ewise_add(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_binop op, const gb_vector *u,
                     const gb_vector *v, const gb_desc *desc);
gb_info gb_ewise_mult(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_binop op, const gb_vector *u,
                      const gb_vector *v, const gb_desc *desc);
/* Table 7 reduce to scalar: monoid over the stored values (identity if none).
 * *out (host) has the vector's type; accum combines with the prior *out. */
gb_info gb_reduce_vector(void *out, gb_binop accum, gb_monoid m, const gb_vector *u);
gb_info gb_reduce_matrix(void *out, gb_binop accum, gb_monoid m, const gb_matrix *A);
/* Table 7 reduce to vector: w(i) = (+)_j A(i,j) (GB_INP0 = GB_TRAN: over columns). */
gb_info gb_reduce_rows(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_monoid m, const gb_matrix *A,
                       const gb_desc *desc);

/* ------------------------------------------------------------- algorithms */

#define GB_TRACE_LEVELS 32

typedef struct {
    uint32_t depth;              /* 1 + the largest level; levels expanded = push_levels + pull_levels
                                    (one fewer when the source's whole component was reached first) */
    uint32_t push_levels;
    uint32_t pull_levels;
    uint32_t status;             /* 0, or GB_TIMEOUT if a bounded device wait ran out */
    uint64_t vertices_reached;
    uint64_t edges_examined;     /* adjacency entries read (push and pull) */
    uint64_t frontier_edges;     /* sum of degrees of all frontiers */
    uint64_t alg_bytes;          /* algorithmic bytes: 8 n (levels, parents) + per push level
                                    8 |V_f| + 4 |E_f| + 12 |V_next|, per pull level min(n/8, 4 |C|)
                                    + 8 (unvisited candidates of C) + 4 |E_examined| + 12 |V_next|,
                                    C = the candidates the pull walks (gb_bfs) */
    /* per-level trace of the first GB_TRACE_LEVELS levels (gb_bfs, gb_bfs_multi) */
    uint32_t trace_len;
    uint32_t trace_dir[GB_TRACE_LEVELS];        /* 1 = push, 2 = pull */
    uint32_t trace_vertices[GB_TRACE_LEVELS];   /* frontier size */
    uint64_t trace_edges[GB_TRACE_LEVELS];      /* frontier out-edges */
    float trace_us[GB_TRACE_LEVELS];            /* level duration (device clock) */
    float init_us;                              /* kernel entry to the start of level 0 */
    float final_us;                             /* end of the last level to the kernel's exit */
    uint32_t schedule;                          /* GB_SCHED_GRID, GB_SCHED_CLUSTER or GB_SCHED_ASYNC: the kernel
                                                   that ran. With GB_SCHED_ASYNC there are no levels:
                                                   push_levels = distance buckets (1 without buckets), depth =
                                                   the same for SSSP and components and 1 + the largest level
                                                   for BFS, vertices_reached = work items relaxed (stale ones
                                                   not counted) for SSSP and components and the vertices
                                                   reached for BFS, edges_examined = frontier_edges = out-edges
                                                   relaxed, alg_bytes = 4 n + 12 per item + 4 per edge (8 with
                                                   weights) + 4 per improvement + 8 per ring entry read,
                                                   final_us = device time of the traversal, no trace */
} gb_bfs_stats;

/* Direction-optimised BFS (Algorithm 1, Section 7.1): levels[v] = hop count
 * from src (src 0, unreachable -1; the paper's depth minus one), and, if
 * parents != NULL, a BFS-tree parent (parents[src] = src, unreachable -1).
 * A must be square and symmetric-or-CSC-built. levels/parents have nrows
 * entries in `mem`. stats may be NULL. desc: GB_DIRECTION, GB_SWITCH_BETA,
 * GB_SCHEDULE (a device that cannot co-schedule a cluster runs GB_SCHED_GRID;
 * GB_SCHED_ASYNC computes the levels without level barriers and then each
 * parent as the smallest in-neighbour one level up, and always waits).
 * With GB_HOST outputs or stats the call waits and returns GB_TIMEOUT if a
 * bounded device wait ran out; with GB_DEVICE outputs and no stats it
 * returns without waiting, and such a timeout is reported by the next
 * gb_context_synchronize (the outputs are then undefined). */
gb_info gb_bfs(gb_context *ctx, const gb_matrix *A, uint32_t src, int32_t *levels, int32_t *parents,
               gb_mem mem, const gb_desc *desc, gb_bfs_stats *stats);
/* k independent direction-optimised BFS runs (Algorithm 1, Section 7.1),
 * one per source srcs[q] (host array, k >= 1, every entry < nrows or
 * GB_INVALID_INDEX before anything runs): row q of levels and of parents
 * (each k x nrows, row-major, in `mem`; parents may be NULL) holds what
 * gb_bfs from srcs[q] would give. With GB_HOST outputs the runs write to two
 * alternating device buffers and the device-to-host copy of run q, on a
 * stream of the call's own, overlaps run q+1 (the paper has no counterpart:
 * it keeps the copy engines busy while the traversal kernels run; host
 * buffers should be pinned, pageable ones work but serialise the copies).
 * desc as for gb_bfs. The call synchronises and returns GB_TIMEOUT if a
 * bounded device wait ran out in any run. */
gb_info gb_bfs_batch(gb_context *ctx, const gb_matrix *A, const uint32_t *srcs, uint32_t k, int32_t *levels,
                     int32_t *parents, gb_mem mem, const gb_desc *desc);
/* Autotuner of the push/pull switch threshold (Table 9: pull iff
 * |E_f| > |E| / beta; Section 5.3 suggests Table 9 as a starting point for
 * finding the best threshold on given hardware). Runs gb_bfs from the k
 * given sources (host array) for each beta in {4, 6, 8, 10, 12, 16, 20, 24,
 * 32, 48, 64, 96, 128, 192, 256}, timed with CUDA events in two passes over
 * the candidates (forward, then backward; each keeps its faster pass), and
 * stores the fastest beta on the matrix; the single-cluster and the
 * barrier-free schedules are timed the same way and kept for the matrix when
 * faster still (graphs of high diameter). Later gb_bfs calls
 * whose descriptor leaves GB_SWITCH_BETA at 0 use it (untuned matrices use
 * the paper's beta = 10). *best_ms (may be NULL) = mean ms per BFS at it. */
gb_info gb_bfs_autotune(gb_context *ctx, gb_matrix *A, const uint32_t *srcs, uint32_t k, uint32_t *best_beta,
                        double *best_ms);
/* BFS tile shape of the persistent grid kernel (its pull walks candidates
 * in groups of 32 x pull_width, each lane pull_width of them with their
 * loads in flight together; its launch puts blocks_per_sm blocks of 512
 * threads on every SM, at most as many as fit: two for pull widths 1 and 2,
 * one for 4). gb_bfs_autotune times pull widths {1, 2, 4} x {1, all that
 * fit} blocks per SM at the threshold it chose and keeps the fastest on the
 * matrix; gb_bfs_set_shape sets them by hand (pull_width 0, 1, 2 or 4,
 * 0 = the default 2; blocks_per_sm 0..4, 0 = as many as fit, a larger
 * number than fit runs as many as fit; else GB_INVALID_VALUE). The outputs of a BFS do not depend on the shape. The
 * paper fixes its kernels' launch shapes (Section 6); tuning them per graph
 * is this library's. gb_bfs_get_shape reports the pull width in effect and
 * the blocks per SM (0 = as many as fit). */
gb_info gb_bfs_set_shape(gb_matrix *A, uint32_t pull_width, uint32_t blocks_per_sm);
gb_info gb_bfs_get_shape(const gb_matrix *A, uint32_t *pull_width, uint32_t *blocks_per_sm);
/* BFS that allocates no device memory (the paper has no counterpart; it is
 * an extra for callers that cannot allocate on the call path: a process
 * whose device memory belongs to another allocator such as a framework's
 * caching allocator or a fixed arena, a latency-critical loop that cannot
 * absorb the device-wide synchronisation of cudaFree, or a deployment that
 * forbids dynamic allocation after start-up). Same traversal and outputs as
 * gb_bfs with the default descriptor, but no gb_context or gb_matrix: the
 * caller passes device pointers to CSR (rowptr[n+1], colidx[nnz]; out-edges)
 * and optionally CSC (colptr[n+1], rowidx[nnz]; in-edges; pass the CSR
 * pointers again for a symmetric graph, or NULL for push-only), and the
 * outputs levels[n] and parents[n] (parents may be NULL). colidx and rowidx
 * must start on a 16-byte boundary and stay readable for 16 bytes past
 * their last entry. status (a device int32, 4-byte aligned, may be NULL)
 * receives the kernel's exit status when it finishes: 0, or GB_TIMEOUT if a
 * bounded device wait ran out, in which case levels and parents are
 * undefined; with status NULL such a timeout cannot be observed. All
 * scratch lives in one array built into the library (about 8.5 MB, enough
 * for n <= GB_NOALLOC_MAX_VERTICES); each GPU that loads the library holds
 * it until the process exits. n above that limit: GB_INVALID_VALUE. The
 * first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture. Work is
 * enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream)
 * and the call returns without waiting. Every call shares the one array and
 * the array keeps the last call's contents: calls whose work overlaps on
 * the GPU (e.g. on different streams) race, so order them on one stream or
 * with events. */
#define GB_NOALLOC_MAX_VERTICES 262144u
gb_info gb_bfs_noalloc(const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *colptr, const uint32_t *rowidx,
                       uint32_t n, uint64_t nnz, uint32_t src, int32_t *levels, int32_t *parents, int32_t *status,
                       void *stream);
/* Multi-source BFS as Boolean SpMM over 64-bit bit-packed frontiers
 * (Section 3.3 multi-nodeset traversal; Section 9 matrix direction
 * optimisation): k >= 1 sources, levels is k x nrows (row q = source q).
 * One launch serves up to 256 sources: each vertex carries one 64-bit word
 * of frontier bits per 64 sources (1, 2 or 4 words for up to 64, 128 or 256
 * sources), and every level chooses push (SpMM from the frontier rows) or
 * pull (the masked product over the rows some search has not reached, with
 * the early exit once all searches are covered) for all of them at once.
 * More than 256 sources are served by consecutive launches of 256 (the
 * statistics then sum or maximise over them, the trace is the first
 * launch's). */
gb_info gb_bfs_multi(gb_context *ctx, const gb_matrix *A, const uint32_t *srcs, uint32_t k, int32_t *levels,
                     gb_mem mem, const gb_desc *desc, gb_bfs_stats *stats);
/* SSSP (Section 7.2): adaptive Bellman-Ford by min.plus mxv restricted to
 * the vertices whose distance changed. A holds uint32 weights. dist[v] =
 * shortest distance (UINT32_MAX unreachable). iterations may be NULL.
 * desc: GB_DIRECTION, GB_SWITCH_BETA, GB_SCHEDULE (GB_SCHED_CLUSTER relaxes
 * by push inside one thread-block cluster; GB_SCHED_ASYNC relaxes without
 * any barrier inside a distance bucket (GB_SSSP_DELTA wide, the automatic
 * width when 0, one bucket for a width >= 2^31 - 1), one grid barrier pair
 * per bucket, the fastest on graphs of high diameter such as the weighted
 * 4096^2 grid; GB_SCHED_AUTO and GB_SCHED_GRID use the persistent grid
 * kernel with one barrier per iteration). stats (may
 * be NULL) receives, as for gb_bfs, the iterations (depth), push and pull
 * iterations, frontier out-edges, the per-iteration trace and alg_bytes:
 * 4 n value writes, per push iteration 8 per frontier vertex and 8 per
 * frontier out-edge (index and weight), per pull iteration 4 (n + 1) row
 * offsets + n / 8 frontier bits + 4 per stored entry (indices) + 4 per
 * frontier out-edge (weights), and 4 per improved value. */
gb_info gb_sssp(gb_context *ctx, const gb_matrix *A, uint32_t src, uint32_t *dist, gb_mem mem,
                const gb_desc *desc, uint32_t *iterations, gb_bfs_stats *stats);
/* PageRank (Section 7.3), pull SpMV in FP32 with FP32 accumulation:
 * p0 = 1/n; p' = (1-damping)/n + damping * (sum_{j in N(i)} p(j)/deg(j)
 * + dangling/n), exactly `iters` iterations; the per-iteration L1 residual
 * sum|p'-p| and the dangling mass are reduced in FP64 over FP32 sums of 4
 * consecutive vertices, the final normalisation in FP64. The result is
 * bit-reproducible run to run (fixed summation orders, no float atomics).
 * rank[n] in `mem`; residuals[iters] (host, may be NULL). The call waits for
 * the result; GB_TIMEOUT if a bounded device wait ran out (the staging copy
 * of the most-referenced ranks into shared memory). */
gb_info gb_pagerank(gb_context *ctx, const gb_matrix *A, float damping, uint32_t iters, float *rank,
                    double *residuals, gb_mem mem);
/* Autotuner of the PageRank SpMV layout (the paper has no counterpart; its
 * merge-path SpMV of Section 6.3.2 has a fixed work per thread): times
 * gb_pagerank on A with warp tiles of 256, 512 and 1,024 nonzeros (8, 16 or
 * 32 gathers in flight per lane; the larger tiles use more registers, so
 * fewer warps) on A as stored, and with tiles of 256 and 512 on a copy of A
 * whose vertices are renamed by decreasing out-degree, where every block
 * stages the ranks of the first 16,384 or 32,768 vertices (the most
 * referenced ones) in shared memory; two passes over the candidates. The
 * fastest is kept on A for later gb_pagerank calls (untuned: 512 as
 * stored); the copy stays on A while it is chosen (nnz + 2n words more).
 * *tile_nnz receives the tile, *degree_order (may be NULL) 1 if the copy
 * won, *staged_ranks (may be NULL) the staged count (0 as stored),
 * *ms_per_iteration (may be NULL) the time per iteration. The result is
 * the same PageRank either way, up to the order of the FP32 row sums. */
gb_info gb_pagerank_autotune(gb_context *ctx, gb_matrix *A, uint32_t *tile_nnz, int32_t *degree_order,
                             uint32_t *staged_ranks, double *ms_per_iteration);
/* Sets the PageRank tile of A by hand: 256, 512 or 1,024 nonzeros, or 0 for
 * the default (GB_INVALID_VALUE otherwise). */
gb_info gb_pagerank_set_tile(gb_matrix *A, uint32_t tile_nnz);
/* Sets the PageRank vertex order of A by hand: 0 = as stored, 1 = the
 * degree-ordered copy (built at the next gb_pagerank; a 1,024-nonzero tile
 * runs as 512 there) with staged_ranks ranks in shared memory (a multiple
 * of 1,024 up to 57,344; 0 = 32,768). GB_INVALID_VALUE otherwise. */
gb_info gb_pagerank_set_order(gb_matrix *A, int32_t degree_order, uint32_t staged_ranks);
/* Adaptive PageRank, also called PageRankDelta (Section 5.1: converged
 * vertices as the output mask; Section 7.3 names the variant): the
 * gb_pagerank recurrence, where a vertex whose value moved by at most eps
 * times its new value (tested in FP32) is masked out of every later
 * iteration, its value kept and still read by the others. Stops when no
 * vertex is active or after max_iters iterations. rank[nrows] in `mem`;
 * iterations, residuals[max_iters] (L1 change per iteration, FP64) and
 * active[max_iters] (vertices updated per iteration) are host pointers and
 * may be NULL. Results are bit-reproducible. eps must be at least
 * GB_PAGERANK_DELTA_MIN_EPS (GB_INVALID_VALUE below it, and for NaN): the
 * FP32 values carry rounding of about 1e-6 relative after the summation of
 * long rows, so a smaller threshold would be decided by that rounding
 * rather than by eps. A negative eps never freezes a vertex (max_iters
 * plain iterations). */
#define GB_PAGERANK_DELTA_MIN_EPS 1e-5f
gb_info gb_pagerank_delta(gb_context *ctx, const gb_matrix *A, float damping, float eps, uint32_t max_iters,
                          float *rank, gb_mem mem, uint32_t *iterations, double *residuals, uint32_t *active);
/* Connected components (Section 7.4) by min-label propagation
 * (min.second mxv to a fixed point): labels[v] = smallest vertex id in v's
 * component. iterations and stats (as for gb_sssp, without weights) may be
 * NULL. */
gb_info gb_cc(gb_context *ctx, const gb_matrix *A, uint32_t *labels, gb_mem mem, uint32_t *iterations,
              gb_bfs_stats *stats);
/* Connected components by min-label propagation without level barriers
 * (the asynchronous execution model of Section 9; the fixed point of
 * gb_cc, so labels[v] = smallest vertex id in v's component, bit-identical
 * to gb_cc): every vertex starts as a work item (label, vertex), and a
 * persistent launch relaxes items through a ring that warps poll until none
 * is in flight. Labels are taken in buckets of label_bucket values (the
 * near-far discipline of SSSP applied to label values: labels below the
 * bound spread first, larger ones wait, one grid-barrier triple per bucket),
 * so a vertex is relabelled fewer times; 0 = automatic (n / 1024, at
 * least 1,024), nrows or more = one bucket. Uses the out-edges (CSR): for a
 * symmetric A these are the components. stats (may be NULL) as for gb_sssp
 * with GB_SCHED_ASYNC. */
gb_info gb_cc_async(gb_context *ctx, const gb_matrix *A, uint32_t *labels, gb_mem mem, uint32_t label_bucket,
                    gb_bfs_stats *stats);
/* Connected components by FastSV (Section 7.4: the paper's CC algorithm):
 * per iteration mngf = A min.second gf, stochastic hooking
 * f(f(u)) = min(f(f(u)), mngf(u)), aggressive hooking and shortcut
 * f(u) = min(f(u), mngf(u), gf(u)), grandparents gf = f(f), until gf stops
 * changing. labels[v] = smallest vertex id in v's component (the same
 * result as gb_cc). A must be square and built symmetric or with its CSC;
 * for a non-symmetric A the components are the weak ones (both edge
 * directions). labels[nrows] in `mem`; *iterations (may be NULL) = FastSV
 * iterations. GB_TIMEOUT if a bounded device wait or the iteration budget
 * ran out; GB_INVALID_VALUE for a CSR-only matrix. */
gb_info gb_cc_fastsv(gb_context *ctx, const gb_matrix *A, uint32_t *labels, gb_mem mem, uint32_t *iterations);
/* Triangle counting (Section 7.5) as the masked SpGEMM C<L> = L (+).(x) L
 * over plus.pair, reduced on the fly: L is a strictly lower-triangular
 * matrix with CSR and CSC (gb_matrix_tril). *count (host) = number of
 * triangles. If C != NULL it also receives C's values in L's structure
 * (C(i,j) = the k with L(i,k) and L(k,j); GB_UINT32). */
gb_info gb_tc(gb_context *ctx, const gb_matrix *L, uint64_t *count, gb_matrix *C);

/* ---------------------------------------------------------------- serving */

typedef enum { GB_REQ_BFS = 0, GB_REQ_SSSP = 1, GB_REQ_PAGERANK = 2 } gb_request_kind;

typedef struct {
    uint32_t max_inflight;       /* requests running at once (default 8) */
    uint32_t batch_window_us;    /* how long a BFS waits for batch partners (default 200) */
    uint64_t hbm_budget_bytes;   /* admission limit on working memory (0 = 80% of free) */
    uint32_t pagerank_iters;     /* default 50 */
    float pagerank_damping;      /* default 0.85 */
} gb_server_cfg;

typedef struct {
    gb_request_kind kind;
    uint32_t graph_id;
    uint32_t src;                /* BFS/SSSP source */
} gb_request;

typedef struct {
    gb_info status;
    uint32_t n;                  /* result length (vertices) */
    double latency_us;           /* submit -> completion visible on the host */
    uint32_t batch_size;         /* BFS requests served by the same launch */
} gb_result;

typedef struct {
    uint64_t submitted, completed, batches, batched_bfs;
    double p50_us, p99_us, mean_us, qps;
    uint64_t hbm_in_use, hbm_peak;
} gb_server_stats;

/* A request loop on the context's GPU: graphs stay resident; requests are
 * admitted while slots (max_inflight) and memory (HBM budget) are free;
 * concurrent BFS requests on one graph are packed (up to 64) into one
 * multi-source bit-frontier BFS; running requests overlap on separate
 * streams, each slot's persistent kernels sized so all slots fit on the GPU
 * at once. Results stay on the device until fetched and count against the
 * budget until then; a job that cannot fit even with nothing running or
 * held fails with GB_OUT_OF_MEMORY. Latency is from submit to completion. */
gb_info gb_server_create(gb_server **s, gb_context *ctx, const gb_server_cfg *cfg);
/* The graph must outlive the server; it needs uint32 weights for SSSP. */
gb_info gb_server_add_graph(gb_server *s, const gb_matrix *A, uint32_t *graph_id);
gb_info gb_server_submit(gb_server *s, const gb_request *req, uint64_t *ticket);
/* Waits up to timeout_ms for the ticket (GB_TIMEOUT if not done). */
gb_info gb_server_wait(gb_server *s, uint64_t ticket, uint32_t timeout_ms, gb_result *res);
/* Copies a finished ticket's result (int32 levels, uint32 distances or
 * float ranks; res.n entries) into out and releases it. */
gb_info gb_server_fetch(gb_server *s, uint64_t ticket, void *out, gb_mem mem);
gb_info gb_server_stats_get(gb_server *s, gb_server_stats *st);
gb_info gb_server_destroy(gb_server **s);

#ifdef __cplusplus
}
#endif
#endif /* GBX_H */
