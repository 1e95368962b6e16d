// Matrix objects: CSR + CSC storage built on the device from tuples
// (Section 4.3: both CSR for row access / pull and CSC for column access /
// push are stored; either copy may be dropped to save memory).
#include "common.cuh"
#include "types.cuh"

using namespace gbx;

namespace gbx {
namespace {
inline unsigned nblk(uint64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

__global__ void k_expand_rows(const uint32_t *rowptr, uint32_t nrows, uint32_t *rows) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nrows)
        for (uint32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) rows[p] = i;
}

__global__ void k_tril_flags(const uint32_t *rows, const uint32_t *cols, uint64_t n, uint32_t *flag) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cols[i] < rows[i] ? 1u : 0u;
}

template <typename T>
__global__ void k_compact(const uint32_t *flag, const uint32_t *pos, uint64_t n, const uint32_t *rows,
                          const uint32_t *cols, const T *vals, uint32_t *orows, uint32_t *ocols, T *ovals) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        uint32_t p = pos[i];
        orows[p] = rows[i];
        ocols[p] = cols[i];
        if (vals) ovals[p] = vals[i];
    }
}

__global__ void k_degree_keys(const uint32_t *rowptr, uint32_t n, uint32_t dmax, int vbits, uint64_t *keys) {
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        uint32_t d = rowptr[v + 1] - rowptr[v];
        keys[v] = ((uint64_t)(dmax - d) << vbits) | v;
    }
}

__global__ void k_rank_to_newid(const uint64_t *keys, uint32_t n, int vbits, uint32_t *new_id) {
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) new_id[(uint32_t)(keys[r] & ((1ull << vbits) - 1))] = r;
}

__global__ void k_map_ids(const uint32_t *in, uint64_t n, const uint32_t *map, uint32_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = map[in[i]];
}

void release(gb_matrix *A) {
    gb_context *ctx = A->ctx;
    if (A->csc_alias) { A->colptr = nullptr; A->rowidx = nullptr; A->cvals = nullptr; }
    dfree(ctx, A->rowptr); dfree(ctx, A->colidx); dfree(ctx, A->vals);
    dfree(ctx, A->colptr); dfree(ctx, A->rowidx); dfree(ctx, A->cvals);
    dfree(ctx, A->hub_list); dfree(ctx, A->hub_pre);
    dfree(ctx, A->live_list);
    dfree(ctx, A->live_rec);
    dfree(ctx, A->comp_size);
    A->comp_size = nullptr;
    if (A->pr_view) gb_matrix_free(&A->pr_view);
    dfree(ctx, A->pr_new_id);
    A->pr_new_id = nullptr;
    A->live_list = A->live_count = nullptr;
    A->live_rec = nullptr;
    A->hub_list = A->hub_pre = nullptr;
    A->nhub = 0; A->hub_edges = 0; A->hub_ready = false;
    A->rowptr = A->colidx = A->colptr = A->rowidx = nullptr;
    A->vals = A->cvals = nullptr;
    A->built = false; A->has_csc = false; A->csc_alias = false; A->nvals = 0;
}
}  // namespace

gb_info matrix_expand_rows(const gb_matrix *A, uint32_t *rows) {
    if (A->nrows)
        k_expand_rows<<<nblk(A->nrows), 256, 0, A->ctx->stream>>>(A->rowptr, A->nrows, rows);
    GB_LAUNCH_CHECK();
    return GB_SUCCESS;
}

namespace {
__global__ void k_live_flags(const uint32_t *ptr, uint32_t n, uint32_t *flag) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = ptr[i + 1] > ptr[i] ? 1u : 0u;
}
__global__ void k_live_emit(const uint32_t *flag, const uint32_t *pos, uint32_t n, uint32_t *list) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) list[pos[i]] = i;
}
// The head of a live vertex: its four in-neighbours of largest out-degree
// (ties: earlier in the row), taken from the first LIVE_HEAD_SCAN entries of
// its row; a pull finds a frontier vertex among them far more often than
// among the first four in row order, since large-degree vertices join the
// frontier early.
constexpr uint32_t LIVE_HEAD_SCAN = 256;
__global__ void k_live_table(const uint32_t *list, const uint32_t *count, const uint32_t *colptr,
                             const uint32_t *rowidx, const uint32_t *rowptr, PullRec *rec) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const uint32_t v = list[i];
    const uint32_t b = colptr[v], l = colptr[v + 1] - b;
    uint32_t best[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
    uint32_t bd[4] = {0, 0, 0, 0};
    const uint32_t lim = l < LIVE_HEAD_SCAN ? l : LIVE_HEAD_SCAN;
    for (uint32_t k = 0; k < lim; ++k) {
        const uint32_t u = rowidx[b + k];
        const uint32_t du = rowptr[u + 1] - rowptr[u] + 1;   // +1: a neighbour always beats an empty slot
        if (du <= bd[3]) continue;
        int p = 3;
        while (p > 0 && du > bd[p - 1]) {
            best[p] = best[p - 1];
            bd[p] = bd[p - 1];
            --p;
        }
        best[p] = u;
        bd[p] = du;
    }
    PullRec r;
    r.v = v;
    r.len = l;
    r.b = b;
    r.deg = rowptr[v + 1] - rowptr[v];
    r.head = make_uint4(best[0], best[1], best[2], best[3]);
    rec[i] = r;
}
}  // namespace

// The ascending list of vertices with a nonempty CSC row (an in-edge): the
// only vertices a pull step can ever reach, with, in list order, each one's
// pull record (its CSC row, out-degree and four in-neighbours of largest
// out-degree; 32 bytes, so a pull reads a candidate with one sector and
// needs the row itself only when the head has no frontier vertex). The list
// length stays on the device.
gb_info matrix_live(gb_matrix *A) {
    gb_context *ctx = A->ctx;
    const uint32_t n = A->ncols;
    GB_CHECK(dalloc_t(ctx, &A->live_list, (size_t)n + 1));
    A->live_count = A->live_list + n;
    Scratch flag(ctx), pos(ctx);
    GB_CHECK(flag.alloc(((size_t)n + 1) * 4));
    GB_CHECK(pos.alloc(((size_t)n + 1) * 4));
    if (n) k_live_flags<<<nblk(n), 256, 0, ctx->stream>>>(A->colptr, n, flag.as<uint32_t>());
    GB_CHECK(scan_exclusive_u32(ctx, flag.as<uint32_t>(), pos.as<uint32_t>(), n, A->live_count));
    if (n) k_live_emit<<<nblk(n), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), n, A->live_list);
    GB_CHECK(dalloc_t(ctx, &A->live_rec, (size_t)n + 1));
    if (n)
        k_live_table<<<nblk(n), 256, 0, ctx->stream>>>(A->live_list, A->live_count, A->colptr, A->rowidx, A->rowptr,
                                                       A->live_rec);
    GB_LAUNCH_CHECK();
    return GB_SUCCESS;
}

// Builds A (CSR, and CSC per flags) from device tuples; replaces contents.
gb_info matrix_build_device(gb_matrix *A, const uint32_t *rows, const uint32_t *cols, const void *vals, uint64_t ntup,
                            gb_binop dup, uint32_t flags) {
    gb_context *ctx = A->ctx;
    release(A);
    uint64_t nnz = 0;
    void *ov = nullptr;
    GB_CHECK(build_csr_from_device_tuples(ctx, A->nrows, A->ncols, ntup, rows, cols, vals, A->type, dup, &A->rowptr,
                                          &A->colidx, vals ? &ov : nullptr, &nnz));
    A->vals = ov;
    A->has_vals = vals != nullptr;
    A->nvals = nnz;
    A->built = true;
    if (flags & GB_SYMMETRIC) {
        if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "GB_SYMMETRIC needs a square matrix");
        A->colptr = A->rowptr; A->rowidx = A->colidx; A->cvals = A->vals;
        A->csc_alias = true; A->has_csc = true;
    } else if (!(flags & GB_CSR_ONLY)) {
        // CSC = CSR of the transpose: sort the (col, row) pairs
        Scratch r(ctx);
        GB_CHECK(r.alloc((nnz + 1) * sizeof(uint32_t)));
        GB_CHECK(matrix_expand_rows(A, r.as<uint32_t>()));
        uint64_t nnz2 = 0;
        void *cv = nullptr;
        GB_CHECK(build_csr_from_device_tuples(ctx, A->ncols, A->nrows, nnz, A->colidx, r.as<uint32_t>(), A->vals,
                                              A->type, GB_FIRST, &A->colptr, &A->rowidx, A->vals ? &cv : nullptr,
                                              &nnz2));
        A->cvals = cv;
        A->has_csc = true;
    }
    if (A->has_csc && A->nrows == A->ncols) GB_CHECK(matrix_live(A));
    return GB_SUCCESS;
}

namespace {
__global__ void k_hub_flags(const uint32_t *ptr, uint32_t n, uint32_t min_len, uint32_t *flag, uint32_t *len) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint32_t l = ptr[i + 1] - ptr[i];
        flag[i] = l > min_len ? 1u : 0u;
        len[i] = l > min_len ? l : 0u;
    }
}
__global__ void k_hub_emit(const uint32_t *flag, const uint32_t *pos, const uint32_t *lpre, uint32_t n, uint32_t *list,
                           uint32_t *pre) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        list[pos[i]] = i;
        pre[pos[i]] = lpre[i];
    }
}
}  // namespace

// Columns of A (rows of its CSC copy) with more than min_len entries, and
// the exclusive prefix of their lengths; computed once and cached.
gb_info matrix_hubs(const gb_matrix *Ac, uint32_t min_len) {
    gb_matrix *A = const_cast<gb_matrix *>(Ac);
    std::lock_guard<std::mutex> lock(A->cache_mu);
    if (A->hub_ready) return GB_SUCCESS;
    gb_context *ctx = A->ctx;
    const uint32_t *ptr = A->has_csc ? A->colptr : A->rowptr;
    uint32_t n = A->has_csc ? A->ncols : A->nrows;
    Scratch flag(ctx), len(ctx), pos(ctx), lpre(ctx), cnt(ctx), tot(ctx);
    GB_CHECK(flag.alloc(((size_t)n + 1) * 4));
    GB_CHECK(len.alloc(((size_t)n + 1) * 4));
    GB_CHECK(pos.alloc(((size_t)n + 1) * 4));
    GB_CHECK(lpre.alloc(((size_t)n + 1) * 4));
    GB_CHECK(cnt.alloc(4));
    GB_CHECK(tot.alloc(4));
    if (n) k_hub_flags<<<nblk(n), 256, 0, ctx->stream>>>(ptr, n, min_len, flag.as<uint32_t>(), len.as<uint32_t>());
    GB_CHECK(scan_exclusive_u32(ctx, flag.as<uint32_t>(), pos.as<uint32_t>(), n, cnt.as<uint32_t>()));
    GB_CHECK(scan_exclusive_u32(ctx, len.as<uint32_t>(), lpre.as<uint32_t>(), n, tot.as<uint32_t>()));
    uint32_t h[2] = {0, 0};
    GB_CUDA(cudaMemcpyAsync(&h[0], cnt.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(&h[1], tot.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    GB_CHECK(dalloc_t(ctx, &A->hub_list, (size_t)h[0] + 1));
    GB_CHECK(dalloc_t(ctx, &A->hub_pre, (size_t)h[0] + 1));
    if (n) k_hub_emit<<<nblk(n), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), lpre.as<uint32_t>(), n,
                                                        A->hub_list, A->hub_pre);
    GB_LAUNCH_CHECK();
    GB_CHECK(sync(ctx));
    A->nhub = h[0];
    A->hub_edges = h[1];
    A->hub_ready = true;
    return GB_SUCCESS;
}

}  // namespace gbx

extern "C" {

gb_info gb_matrix_new(gb_matrix **A, gb_context *ctx, gb_type type, uint64_t nrows, uint64_t ncols) {
    if (!A || !ctx) return fail(GB_NULL_POINTER, "gb_matrix_new: NULL argument");
    if (!valid_type(type)) return fail(GB_INVALID_VALUE, "gb_matrix_new: bad type %d", (int)type);
    if (nrows >= (1ull << 32) || ncols >= (1ull << 32))
        return fail(GB_INVALID_VALUE, "gb_matrix_new: dimensions must be < 2^32");
    gb_matrix *m = new gb_matrix();
    m->ctx = ctx; m->type = type; m->nrows = (uint32_t)nrows; m->ncols = (uint32_t)ncols;
    *A = m;
    return GB_SUCCESS;
}

gb_info gb_matrix_build(gb_matrix *A, const uint32_t *rows, const uint32_t *cols, const void *vals, uint64_t nvals,
                        gb_binop dup, gb_mem mem, uint32_t flags) {
    if (!A) return fail(GB_NULL_POINTER, "gb_matrix_build: A is NULL");
    if (nvals && (!rows || !cols)) return fail(GB_NULL_POINTER, "gb_matrix_build: rows/cols NULL");
    if (nvals >= (1ull << 32)) return fail(GB_INVALID_VALUE, "gb_matrix_build: nvals must be < 2^32");
    if (dup < GB_PLUS || dup > GB_MINUS) return fail(GB_INVALID_VALUE, "gb_matrix_build: bad dup operator");
    if (flags & ~(uint32_t)(GB_SYMMETRIC | GB_CSR_ONLY)) return fail(GB_INVALID_VALUE, "gb_matrix_build: bad flags");
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch r(ctx), c(ctx), v(ctx);
    const uint32_t *dr = rows, *dc = cols;
    const void *dv = vals;
    size_t vs = type_size(A->type);
    if (mem == GB_HOST) {
        GB_CHECK(r.alloc(nvals * 4 + 16));
        GB_CHECK(c.alloc(nvals * 4 + 16));
        GB_CHECK(copy_in(ctx, r.p, rows, nvals * 4, GB_HOST));
        GB_CHECK(copy_in(ctx, c.p, cols, nvals * 4, GB_HOST));
        dr = r.as<uint32_t>(); dc = c.as<uint32_t>();
        if (vals) {
            GB_CHECK(v.alloc(nvals * vs + 16));
            GB_CHECK(copy_in(ctx, v.p, vals, nvals * vs, GB_HOST));
            dv = v.p;
        }
    }
    GB_CHECK(matrix_build_device(A, dr, dc, dv, nvals, dup, flags));
    // a user's square matrix with a CSC also gets its component sizes, for
    // the early stop of BFS (matrices the library builds as results do not)
    if (A->has_csc && A->nrows == A->ncols) GB_CHECK(matrix_components(ctx, A));
    GB_CHECK(sync(ctx));
    return GB_SUCCESS;
}

gb_info gb_matrix_nrows(const gb_matrix *A, uint64_t *n) {
    if (!A || !n) return fail(GB_NULL_POINTER, "gb_matrix_nrows: NULL");
    *n = A->nrows;
    return GB_SUCCESS;
}
gb_info gb_matrix_ncols(const gb_matrix *A, uint64_t *n) {
    if (!A || !n) return fail(GB_NULL_POINTER, "gb_matrix_ncols: NULL");
    *n = A->ncols;
    return GB_SUCCESS;
}
gb_info gb_matrix_nvals(const gb_matrix *A, uint64_t *n) {
    if (!A || !n) return fail(GB_NULL_POINTER, "gb_matrix_nvals: NULL");
    *n = A->nvals;
    return GB_SUCCESS;
}

gb_info gb_matrix_extract_tuples(const gb_matrix *A, uint32_t *rows, uint32_t *cols, void *vals, uint64_t *n_inout,
                                 gb_mem mem) {
    if (!A || !n_inout) return fail(GB_NULL_POINTER, "gb_matrix_extract_tuples: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_matrix_extract_tuples: matrix not built");
    if (*n_inout < A->nvals) { *n_inout = A->nvals; return fail(GB_INSUFFICIENT_SPACE, "extract_tuples: buffer too small"); }
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    uint64_t m = A->nvals;
    if (rows) {
        Scratch r(ctx);
        GB_CHECK(r.alloc((m + 1) * 4));
        GB_CHECK(matrix_expand_rows(A, r.as<uint32_t>()));
        GB_CHECK(copy_out(ctx, rows, r.p, m * 4, mem));
    }
    if (cols) GB_CHECK(copy_out(ctx, cols, A->colidx, m * 4, mem));
    if (vals) {
        size_t vs = type_size(A->type);
        if (A->has_vals) GB_CHECK(copy_out(ctx, vals, A->vals, m * vs, mem));
        else return fail(GB_NO_VALUE, "extract_tuples: structural matrix has no value array");
    }
    GB_CHECK(sync(ctx));
    *n_inout = m;
    return GB_SUCCESS;
}

gb_info gb_matrix_export_csr(const gb_matrix *A, uint32_t *rowptr, uint32_t *colidx, void *vals, gb_mem mem) {
    if (!A) return fail(GB_NULL_POINTER, "gb_matrix_export_csr: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_matrix_export_csr: matrix not built");
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    if (rowptr) GB_CHECK(copy_out(ctx, rowptr, A->rowptr, ((size_t)A->nrows + 1) * 4, mem));
    if (colidx) GB_CHECK(copy_out(ctx, colidx, A->colidx, A->nvals * 4, mem));
    if (vals) {
        if (!A->has_vals) return fail(GB_NO_VALUE, "export_csr: structural matrix");
        GB_CHECK(copy_out(ctx, vals, A->vals, A->nvals * type_size(A->type), mem));
    }
    return sync(ctx);
}

gb_info gb_matrix_export_csc(const gb_matrix *A, uint32_t *colptr, uint32_t *rowidx, void *vals, gb_mem mem) {
    if (!A) return fail(GB_NULL_POINTER, "gb_matrix_export_csc: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_matrix_export_csc: matrix not built");
    if (!A->has_csc) return fail(GB_INVALID_VALUE, "gb_matrix_export_csc: built with GB_CSR_ONLY");
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    if (colptr) GB_CHECK(copy_out(ctx, colptr, A->colptr, ((size_t)A->ncols + 1) * 4, mem));
    if (rowidx) GB_CHECK(copy_out(ctx, rowidx, A->rowidx, A->nvals * 4, mem));
    if (vals) {
        if (!A->has_vals) return fail(GB_NO_VALUE, "export_csc: structural matrix");
        GB_CHECK(copy_out(ctx, vals, A->cvals, A->nvals * type_size(A->type), mem));
    }
    return sync(ctx);
}

gb_info gb_matrix_tril(gb_matrix *L, const gb_matrix *A) {
    if (!L || !A) return fail(GB_NULL_POINTER, "gb_matrix_tril: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_matrix_tril: A not built");
    if (L == A) return fail(GB_INVALID_VALUE, "gb_matrix_tril: L must differ from A");
    if (L->nrows != A->nrows || L->ncols != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_matrix_tril: dims");
    if (A->has_vals && L->type != A->type) return fail(GB_DOMAIN_MISMATCH, "gb_matrix_tril: type");
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    uint64_t m = A->nvals;
    Scratch rows(ctx), flag(ctx), pos(ctx), tot(ctx), orow(ctx), ocol(ctx), oval(ctx);
    size_t vs = type_size(A->type);
    GB_CHECK(rows.alloc((m + 1) * 4));
    GB_CHECK(flag.alloc((m + 1) * 4));
    GB_CHECK(pos.alloc((m + 1) * 4));
    GB_CHECK(tot.alloc(4));
    GB_CHECK(orow.alloc((m + 1) * 4));
    GB_CHECK(ocol.alloc((m + 1) * 4));
    if (A->has_vals) GB_CHECK(oval.alloc((m + 1) * vs));
    GB_CHECK(matrix_expand_rows(A, rows.as<uint32_t>()));
    if (m) k_tril_flags<<<nblk(m), 256, 0, ctx->stream>>>(rows.as<uint32_t>(), A->colidx, m, flag.as<uint32_t>());
    GB_CHECK(scan_exclusive_u32(ctx, flag.as<uint32_t>(), pos.as<uint32_t>(), m, tot.as<uint32_t>()));
    if (m) {
        if (A->has_vals) {
            switch (vs) {
            case 1: k_compact<uint8_t><<<nblk(m), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), m, rows.as<uint32_t>(), A->colidx, (const uint8_t *)A->vals, orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.as<uint8_t>()); break;
            case 4: k_compact<uint32_t><<<nblk(m), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), m, rows.as<uint32_t>(), A->colidx, (const uint32_t *)A->vals, orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.as<uint32_t>()); break;
            default: k_compact<uint64_t><<<nblk(m), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), m, rows.as<uint32_t>(), A->colidx, (const uint64_t *)A->vals, orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.as<uint64_t>()); break;
            }
        } else {
            k_compact<uint32_t><<<nblk(m), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), m, rows.as<uint32_t>(), A->colidx, (const uint32_t *)nullptr, orow.as<uint32_t>(), ocol.as<uint32_t>(), (uint32_t *)nullptr);
        }
        GB_LAUNCH_CHECK();
    }
    uint32_t nl = 0;
    GB_CUDA(cudaMemcpyAsync(&nl, tot.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    gb_type keep = L->type;
    if (A->has_vals) L->type = A->type;
    GB_CHECK(matrix_build_device(L, orow.as<uint32_t>(), ocol.as<uint32_t>(), A->has_vals ? oval.p : nullptr, nl,
                                 GB_FIRST, GB_BUILD_DEFAULT));
    if (!A->has_vals) L->type = keep;
    return sync(ctx);
}

gb_info gb_matrix_degree_order(gb_matrix *B, const gb_matrix *A, uint32_t *new_id, gb_mem mem) {
    if (!B || !A) return fail(GB_NULL_POINTER, "gb_matrix_degree_order: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_matrix_degree_order: A not built");
    if (A->nrows != A->ncols || B->nrows != A->nrows || B->ncols != A->ncols)
        return fail(GB_DIMENSION_MISMATCH, "gb_matrix_degree_order: needs square matrices of equal size");
    if (B == A) return fail(GB_INVALID_VALUE, "gb_matrix_degree_order: B must differ from A");
    if (A->has_vals && B->type != A->type) return fail(GB_DOMAIN_MISMATCH, "gb_matrix_degree_order: type");
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    uint32_t n = A->nrows;
    uint64_t m = A->nvals;
    int vbits = bits_for(n), dbits = bits_for((uint64_t)A->ncols + 1);
    Scratch keys(ctx), nid(ctx), rows(ctx), r2(ctx), c2(ctx);
    GB_CHECK(keys.alloc(((size_t)n + 1) * 8));
    GB_CHECK(nid.alloc(((size_t)n + 1) * 4));
    GB_CHECK(rows.alloc((m + 1) * 4));
    GB_CHECK(r2.alloc((m + 1) * 4));
    GB_CHECK(c2.alloc((m + 1) * 4));
    if (n) {
        k_degree_keys<<<nblk(n), 256, 0, ctx->stream>>>(A->rowptr, n, A->ncols, vbits, keys.as<uint64_t>());
        GB_CHECK(radix_sort_pairs(ctx, keys.as<uint64_t>(), nullptr, n, vbits + dbits));
        k_rank_to_newid<<<nblk(n), 256, 0, ctx->stream>>>(keys.as<uint64_t>(), n, vbits, nid.as<uint32_t>());
        GB_LAUNCH_CHECK();
    }
    GB_CHECK(matrix_expand_rows(A, rows.as<uint32_t>()));
    if (m) {
        k_map_ids<<<nblk(m), 256, 0, ctx->stream>>>(rows.as<uint32_t>(), m, nid.as<uint32_t>(), r2.as<uint32_t>());
        k_map_ids<<<nblk(m), 256, 0, ctx->stream>>>(A->colidx, m, nid.as<uint32_t>(), c2.as<uint32_t>());
        GB_LAUNCH_CHECK();
    }
    if (new_id) GB_CHECK(copy_out(ctx, new_id, nid.p, (size_t)n * 4, mem));
    gb_type keep = B->type;
    if (A->has_vals) B->type = A->type;
    GB_CHECK(matrix_build_device(B, r2.as<uint32_t>(), c2.as<uint32_t>(), A->has_vals ? A->vals : nullptr, m, GB_FIRST,
                                 A->csc_alias ? GB_SYMMETRIC : (A->has_csc ? GB_BUILD_DEFAULT : GB_CSR_ONLY)));
    if (!A->has_vals) B->type = keep;
    return sync(ctx);
}

gb_info gb_matrix_free(gb_matrix **A) {
    if (!A) return fail(GB_NULL_POINTER, "gb_matrix_free: NULL");
    if (*A) {
        cudaSetDevice((*A)->ctx->device);
        release(*A);
        delete *A;
        *A = nullptr;
    }
    return GB_SUCCESS;
}

}  // extern "C"
