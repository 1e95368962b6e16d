// Table 7 operations at the C ABI: mxv, vxm, mxm, eWiseAdd, eWiseMult and
// reduce, with the mask / accumulator / REPLACE semantics of Section 3.2
// and the GraphBLAS C API (see gbx.h), and the direction choice of
// Section 4 (Table 9) for mxv/vxm.
#include "ops_impl.cuh"
#include "vector_impl.cuh"

using namespace gbx;

namespace gbx {

gb_info matrix_build_device(gb_matrix *A, const uint32_t *rows, const uint32_t *cols, const void *vals, uint64_t ntup,
                            gb_binop dup, uint32_t flags);
gb_info matrix_expand_rows(const gb_matrix *A, uint32_t *rows);

namespace {
inline unsigned nblk(uint64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

#define DISPATCH_T(type, ...)                                   \
    switch (type) {                                             \
    case GB_BOOL: { typedef uint8_t T; __VA_ARGS__; } break;    \
    case GB_INT32: { typedef int32_t T; __VA_ARGS__; } break;   \
    case GB_UINT32: { typedef uint32_t T; __VA_ARGS__; } break; \
    case GB_UINT64: { typedef uint64_t T; __VA_ARGS__; } break; \
    case GB_FP32: { typedef float T; __VA_ARGS__; } break;      \
    case GB_FP64: { typedef double T; __VA_ARGS__; } break;     \
    }

// allowed(i) from a mask vector (Section 3.2.1): a stored nonzero (or,
// with GB_STRUCTURE, any stored entry) lets i through; GB_SCMP inverts.
// Without a mask every position is allowed, and GB_SCMP allows none.
template <typename T>
__global__ void k_mask_bits(const T *mvals, const uint32_t *mbits, uint32_t n, uint32_t nwords, bool structural,
                            bool scmp, uint32_t *allowed) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool m = false;
    if (i < n) {
        if (mbits) {
            bool pres = (mbits[i >> 5] >> (i & 31)) & 1u;
            m = structural ? pres : (pres && mvals[i] != (T)0);
        } else {
            m = true;
        }
        if (scmp) m = !m;
    }
    uint32_t word = __ballot_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < nwords) allowed[i >> 5] = word;
}

// w = mask ? (accum ? union-accum(w, t) : t) : (replace ? nothing : w)
template <typename T>
__global__ void k_finish(T *wv, uint32_t *wb, const T *tv, const uint32_t *tb, const uint32_t *allowed, uint32_t n,
                         gb_binop accum, bool replace) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool pres = false;
    if (i < n) {
        bool wp = (wb[i >> 5] >> (i & 31)) & 1u;
        bool tp = (tb[i >> 5] >> (i & 31)) & 1u;
        bool al = allowed ? ((allowed[i >> 5] >> (i & 31)) & 1u) : true;
        if (al) {
            if (accum == GB_NOP) {
                pres = tp;
                if (tp) wv[i] = tv[i];
            } else {
                pres = wp || tp;
                if (wp && tp) wv[i] = apply_binop<T>(accum, wv[i], tv[i]);
                else if (tp) wv[i] = tv[i];
            }
        } else {
            pres = replace ? false : wp;
        }
    }
    uint32_t word = __ballot_sync(0xffffffffu, pres);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < ((n + 31) / 32)) wb[i >> 5] = word;
}

template <typename T>
__global__ void k_ewise(const T *uv, const uint32_t *ub, const T *vv, const uint32_t *vb, uint32_t n, gb_binop op,
                        bool uni, T *tv, uint32_t *tb) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool pres = false;
    if (i < n) {
        bool up = (ub[i >> 5] >> (i & 31)) & 1u;
        bool vp = (vb[i >> 5] >> (i & 31)) & 1u;
        if (up && vp) { tv[i] = apply_binop<T>(op, uv[i], vv[i]); pres = true; }
        else if (uni && up) { tv[i] = uv[i]; pres = true; }
        else if (uni && vp) { tv[i] = vv[i]; pres = true; }
    }
    uint32_t word = __ballot_sync(0xffffffffu, pres);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < ((n + 31) / 32)) tb[i >> 5] = word;
}

template <typename T>
__host__ __device__ __forceinline__ T monoid_identity(gb_monoid m) {
    switch (m) {
    case GB_MONOID_PLUS: return (T)0;
    case GB_MONOID_TIMES: return (T)1;
    case GB_MONOID_MIN: return Lim<T>::max();
    case GB_MONOID_MAX: return Lim<T>::min();
    case GB_MONOID_LOR: return (T)0;
    case GB_MONOID_LAND: return (T)1;
    }
    return (T)0;
}

template <typename T>
__host__ __device__ __forceinline__ T monoid_op(gb_monoid m, T a, T b) {
    switch (m) {
    case GB_MONOID_PLUS: return wrap_add<T>(a, b);
    case GB_MONOID_TIMES: return wrap_mul<T>(a, b);
    case GB_MONOID_MIN: return b < a ? b : a;
    case GB_MONOID_MAX: return a < b ? b : a;
    case GB_MONOID_LOR: return (T)((a != (T)0) || (b != (T)0));
    case GB_MONOID_LAND: return (T)((a != (T)0) && (b != (T)0));
    }
    return a;
}

// deterministic reduction: fixed per-block order, then one block over partials
constexpr int RBLOCK = 256;
template <typename T>
__global__ void k_reduce_partial(const T *vals, const uint32_t *bits, uint64_t n, gb_monoid m, T *part) {
    __shared__ T sh[RBLOCK];
    T acc = monoid_identity<T>(m);
    uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    uint64_t b0 = per * blockIdx.x, b1 = b0 + per < n ? b0 + per : n;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += RBLOCK)
        if (!bits || ((bits[i >> 5] >> (i & 31)) & 1u)) acc = monoid_op<T>(m, acc, vals ? vals[i] : (T)1);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RBLOCK / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = monoid_op<T>(m, sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename T>
gb_info reduce_dense(gb_context *ctx, const T *vals, const uint32_t *bits, uint64_t n, gb_monoid m, T *out_host) {
    unsigned blocks = (unsigned)(n / (RBLOCK * 16) + 1);
    if (blocks > 1024) blocks = 1024;
    Scratch part(ctx), fin(ctx);
    GB_CHECK(part.alloc((size_t)blocks * sizeof(T) + 16));
    GB_CHECK(fin.alloc(sizeof(T) + 16));
    k_reduce_partial<T><<<blocks, RBLOCK, 0, ctx->stream>>>(vals, bits, n, m, part.as<T>());
    k_reduce_partial<T><<<1, RBLOCK, 0, ctx->stream>>>(part.as<T>(), nullptr, blocks, m, fin.as<T>());
    GB_LAUNCH_CHECK();
    GB_CUDA(cudaMemcpyAsync(out_host, fin.p, sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    return sync(ctx);
}

// reduce each row of a CSR-like structure (warp per row, fixed order)
template <typename T>
__global__ void k_reduce_rows(const uint32_t *ptr, const void *vals, uint32_t n, gb_monoid m, T *tv, uint32_t *tb) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < n; i += nwarps) {
        uint32_t b = ptr[i], e = ptr[i + 1];
        if (b == e) continue;
        T acc = monoid_identity<T>(m);
        for (uint32_t q = b + lane; q < e; q += 32) acc = monoid_op<T>(m, acc, load_val<T>(vals, q));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = monoid_op<T>(m, acc, shfl_xor_t<T>(acc, o));
        if (lane == 0) {
            tv[i] = acc;
            atomicOr(&tb[i >> 5], 1u << (i & 31));
        }
    }
}

// masked mxm assembly: position q of M kept if allowed (value mask) and the
// product exists; the previous C is merged for accum / kept outside M
template <typename T>
__global__ void k_mxm_flags(const uint8_t *cpres, const T *mvals, bool structural, uint64_t nm, uint32_t *flag) {
    uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nm) flag[q] = (cpres[q] && (structural || !mvals || mvals[q] != (T)0)) ? 1u : 0u;
}

template <typename T>
__global__ void k_mxm_emit(const uint32_t *flag, const uint32_t *pos, uint64_t nm, const uint32_t *mrows,
                           const uint32_t *midx, const T *cv, uint32_t *orow, uint32_t *ocol, T *oval) {
    uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nm && flag[q]) {
        uint32_t p = pos[q];
        orow[p] = mrows[q];
        ocol[p] = midx[q];
        oval[p] = cv[q];
    }
}

// entries of the old C: inside M (accumulated into the new value) or outside
template <typename T, typename MT>
__global__ void k_old_c(const uint32_t *crows, const uint32_t *cidx, const T *cvals, uint64_t nc, const uint32_t *m_ptr,
                        const uint32_t *m_idx, const MT *mvals, bool structural, const uint32_t *newflag, T *newval,
                        gb_binop accum, bool replace, uint32_t *keep_old, uint32_t *newpresent_from_old) {
    uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    uint32_t i = crows[q], j = cidx[q];
    uint32_t lo = m_ptr[i], hi = m_ptr[i + 1], pos = 0;
    bool inm = bsearch_u32(m_idx, lo, hi, j, &pos);
    if (inm && !structural && mvals && mvals[pos] == (MT)0) inm = false;   // a stored zero does not allow
    keep_old[q] = 0;
    if (inm) {
        if (accum != GB_NOP) {
            if (newflag[pos]) newval[pos] = apply_binop<T>(accum, cvals ? cvals[q] : (T)1, newval[pos]);
            else { newval[pos] = cvals ? cvals[q] : (T)1; newpresent_from_old[pos] = 1; }
        }
    } else if (!replace) {
        keep_old[q] = 1;
    }
}

__global__ void k_or_flags(uint32_t *a, const uint32_t *b, uint64_t n) {
    uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n && b[q]) a[q] = 1;
}

template <typename T>
__global__ void k_emit_old(const uint32_t *keep, const uint32_t *pos, uint64_t nc, uint32_t base, const uint32_t *crows,
                           const uint32_t *cidx, const T *cvals, uint32_t *orow, uint32_t *ocol, T *oval) {
    uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nc && keep[q]) {
        uint32_t p = base + pos[q];
        orow[p] = crows[q];
        ocol[p] = cidx[q];
        oval[p] = cvals ? cvals[q] : (T)1;
    }
}

// ---- mxm without a mask or with a complemented mask: expand, sort, compress.
// Every product A(i,k) (x) B(k,j) becomes a tuple (i, j, value); the device
// build then sorts the tuples and reduces equal positions with the
// semiring's add, as the paper's SpMSpV reduces its expanded products by
// radix sort (Section 6.3.1).

// rows[q] = the row of stored entry q of a compressed structure (ptr, n rows)
__global__ void k_expand_ptr(const uint32_t *ptr, uint32_t n, uint32_t *rows) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (uint32_t q = ptr[i]; q < ptr[i + 1]; ++q) rows[q] = i;
}

// products of entry q of op(A): the length of op(B)'s row a_idx[q]
__global__ void k_product_counts(const uint32_t *a_idx, uint64_t na, const uint32_t *b_ptr, uint32_t *cnt) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < na) cnt[q] = b_ptr[a_idx[q] + 1] - b_ptr[a_idx[q]];
}

template <typename T, Mul MU>
__global__ void k_products(const uint32_t *arows, const uint32_t *a_idx, const T *a_vals, uint64_t na,
                           const uint32_t *b_ptr, const uint32_t *b_idx, const T *b_vals, const uint32_t *off,
                           uint32_t *orow, uint32_t *ocol, T *oval) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= na) return;
    const uint32_t i = arows[q], k = a_idx[q];
    const T a = a_vals ? a_vals[q] : (T)1;
    uint32_t o = off[q];
    for (uint32_t p = b_ptr[k]; p < b_ptr[k + 1]; ++p, ++o) {
        orow[o] = i;
        ocol[o] = b_idx[p];
        oval[o] = mul_op<T, MU>(a, b_vals ? b_vals[p] : (T)1);
    }
}

// is (i, j) allowed by the mask M (a stored nonzero, or any stored entry
// when structural)? The complement inverts it.
template <typename MT>
__device__ __forceinline__ bool mask_has(const uint32_t *m_ptr, const uint32_t *m_idx, const MT *m_vals,
                                         bool structural, uint32_t i, uint32_t j) {
    uint32_t pos = 0;
    bool in = bsearch_u32(m_idx, m_ptr[i], m_ptr[i + 1], j, &pos);
    if (in && !structural && m_vals && m_vals[pos] == (MT)0) in = false;
    return in;
}

template <typename MT>
__global__ void k_product_allowed(const uint32_t *orow, const uint32_t *ocol, uint64_t np, const uint32_t *m_ptr,
                                  const uint32_t *m_idx, const MT *m_vals, bool structural, uint32_t *flag) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < np) flag[t] = mask_has<MT>(m_ptr, m_idx, m_vals, structural, orow[t], ocol[t]) ? 0u : 1u;
}

template <typename T>
__global__ void k_compact_products(const uint32_t *flag, const uint32_t *pos, uint64_t np, const uint32_t *orow,
                                   const uint32_t *ocol, const T *oval, uint32_t *r2, uint32_t *c2, T *v2) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < np && flag[t]) {
        r2[pos[t]] = orow[t];
        c2[pos[t]] = ocol[t];
        v2[pos[t]] = oval[t];
    }
}

// entries of the old C against the product T (sorted rows): an entry at a
// position of T is accumulated into T's value (accum) or replaced by it; one
// elsewhere stays when the mask allows it and there is an accumulator, or
// when the mask does not allow it and there is no REPLACE
template <typename T, typename MT>
__global__ void k_merge_old_c(const uint32_t *crows, const uint32_t *cidx, const T *cvals, uint64_t nc,
                              const uint32_t *t_ptr, const uint32_t *t_idx, T *t_vals, const uint32_t *m_ptr,
                              const uint32_t *m_idx, const MT *m_vals, bool has_mask, bool structural, bool scmp,
                              gb_binop accum, bool replace, uint32_t *keep) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    const uint32_t i = crows[q], j = cidx[q];
    const T c = cvals ? cvals[q] : (T)1;
    uint32_t pos = 0;
    keep[q] = 0;
    if (bsearch_u32(t_idx, t_ptr[i], t_ptr[i + 1], j, &pos)) {
        if (accum != GB_NOP) t_vals[pos] = apply_binop<T>(accum, c, t_vals[pos]);
        return;
    }
    const bool allowed = has_mask ? (mask_has<MT>(m_ptr, m_idx, m_vals, structural, i, j) != scmp) : !scmp;
    keep[q] = (allowed ? accum != GB_NOP : !replace) ? 1u : 0u;
}

template <typename T>
gb_info mxm_expand(gb_context *ctx, gb_semiring s, const uint32_t *arows, const uint32_t *a_idx, const void *a_vals,
                   uint64_t na, const uint32_t *b_ptr, const uint32_t *b_idx, const void *b_vals, const uint32_t *off,
                   uint32_t *orow, uint32_t *ocol, void *oval) {
    const T *av = (const T *)a_vals, *bv = (const T *)b_vals;
    T *ov = (T *)oval;
    const unsigned g = nblk(na);
    if (!na) return GB_SUCCESS;
    switch (s) {
    case GB_PLUS_TIMES: case GB_MIN_TIMES:
        k_products<T, Mul::TIMES><<<g, 256, 0, ctx->stream>>>(arows, a_idx, av, na, b_ptr, b_idx, bv, off, orow, ocol, ov); break;
    case GB_MIN_PLUS: case GB_MAX_PLUS:
        k_products<T, Mul::SATPLUS><<<g, 256, 0, ctx->stream>>>(arows, a_idx, av, na, b_ptr, b_idx, bv, off, orow, ocol, ov); break;
    case GB_MIN_SECOND:
        k_products<T, Mul::SECOND><<<g, 256, 0, ctx->stream>>>(arows, a_idx, av, na, b_ptr, b_idx, bv, off, orow, ocol, ov); break;
    case GB_PLUS_PAIR:
        k_products<T, Mul::PAIR><<<g, 256, 0, ctx->stream>>>(arows, a_idx, av, na, b_ptr, b_idx, bv, off, orow, ocol, ov); break;
    case GB_LOR_LAND:
        k_products<T, Mul::LAND><<<g, 256, 0, ctx->stream>>>(arows, a_idx, av, na, b_ptr, b_idx, bv, off, orow, ocol, ov); break;
    }
    GB_LAUNCH_CHECK();
    return GB_SUCCESS;
}

// the build's duplicate operator that is the semiring's add monoid
gb_binop semiring_add_op(gb_semiring s) {
    switch (s) {
    case GB_PLUS_TIMES: case GB_PLUS_PAIR: return GB_PLUS;
    case GB_LOR_LAND: return GB_LOR;
    case GB_MAX_PLUS: return GB_MAX;
    default: return GB_MIN;
    }
}

struct Desc {
    bool scmp = false, structure = false, replace = false, tran0 = false, tran1 = false;
    int direction = GB_AUTO;
    int beta = 10;
};

Desc read_desc(const gb_desc *d) {
    Desc r;
    if (d) {
        r.scmp = d->mask & GB_SCMP;
        r.structure = d->mask & GB_STRUCTURE;
        r.replace = d->outp == GB_REPLACE;
        r.tran0 = d->inp0 == GB_TRAN;
        r.tran1 = d->inp1 == GB_TRAN;
        r.direction = d->direction;
        r.beta = d->beta > 0 ? d->beta : 10;
    }
    return r;
}

bool valid_accum(gb_binop a) { return a >= GB_NOP && a <= GB_MINUS; }

gb_info make_allowed(gb_context *ctx, const gb_vector *mask, const Desc &d, uint32_t n, Scratch &buf,
                     const uint32_t **allowed) {
    *allowed = nullptr;
    if (!mask && !d.scmp) return GB_SUCCESS;
    if (mask && mask->n != n) return fail(GB_DIMENSION_MISMATCH, "mask size %u != output size %u", mask->n, n);
    uint32_t nw = (n + 31) / 32;
    GB_CHECK(buf.alloc(((size_t)nw + 1) * 4));
    if (n) {
        if (mask) {
            DISPATCH_T(mask->type, k_mask_bits<T><<<nblk(n), 256, 0, ctx->stream>>>(
                                       (const T *)mask->vals, mask->bitmap, n, nw, d.structure, d.scmp,
                                       buf.as<uint32_t>()))
        } else {
            k_mask_bits<uint8_t><<<nblk(n), 256, 0, ctx->stream>>>(nullptr, nullptr, n, nw, true, true,
                                                                  buf.as<uint32_t>());
        }
        GB_LAUNCH_CHECK();
    }
    *allowed = buf.as<uint32_t>();
    return GB_SUCCESS;
}

gb_info finish_vector(gb_context *ctx, gb_vector *w, const void *tv, const uint32_t *tb, const uint32_t *allowed,
                      gb_binop accum, bool replace) {
    if (w->n) {
        DISPATCH_T(w->type, k_finish<T><<<nblk(w->n), 256, 0, ctx->stream>>>((T *)w->vals, w->bitmap, (const T *)tv,
                                                                             tb, allowed, w->n, accum, replace))
        GB_LAUNCH_CHECK();
    }
    w->list_valid = false;
    return GB_SUCCESS;
}

// mxv (vec_first = false) or vxm (vec_first = true) with the matrix possibly transposed
gb_info mxv_common(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_semiring s, const gb_matrix *A,
                   const gb_vector *u, const gb_desc *desc, bool vec_first, const char *who) {
    if (!w || !A || !u) return fail(GB_NULL_POINTER, "%s: NULL argument", who);
    if (!A->built) return fail(GB_INVALID_VALUE, "%s: matrix not built", who);
    if (!valid_accum(accum)) return fail(GB_INVALID_VALUE, "%s: bad accumulator", who);
    if (s < GB_PLUS_TIMES || s > GB_PLUS_PAIR) return fail(GB_INVALID_VALUE, "%s: bad semiring", who);
    Desc d = read_desc(desc);
    const bool tran = vec_first ? d.tran1 : d.tran0;
    // rows of P are indexed by the output, rows of S by the input
    bool out_is_row = vec_first ? tran : !tran;
    uint32_t nout = out_is_row ? A->nrows : A->ncols;
    uint32_t nin = out_is_row ? A->ncols : A->nrows;
    if (w->n != nout || u->n != nin)
        return fail(GB_DIMENSION_MISMATCH, "%s: sizes w=%u u=%u do not match the matrix", who, w->n, u->n);
    if (u->type != w->type) return fail(GB_DOMAIN_MISMATCH, "%s: u and w types differ", who);
    if (A->has_vals && A->type != w->type) return fail(GB_DOMAIN_MISMATCH, "%s: matrix and vector types differ", who);
    if (!semiring_supported(s, w->type)) return fail(GB_DOMAIN_MISMATCH, "%s: semiring not available for this type", who);
    gb_context *ctx = w->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    MxvPlan p;
    p.ctx = ctx;
    if (out_is_row) {
        p.p_ptr = A->rowptr; p.p_idx = A->colidx; p.p_vals = A->has_vals ? A->vals : nullptr;
        p.s_ptr = A->colptr; p.s_idx = A->rowidx; p.s_vals = A->has_vals ? A->cvals : nullptr;
    } else {
        p.p_ptr = A->colptr; p.p_idx = A->rowidx; p.p_vals = A->has_vals ? A->cvals : nullptr;
        p.s_ptr = A->rowptr; p.s_idx = A->colidx; p.s_vals = A->has_vals ? A->vals : nullptr;
    }
    p.has_vals = A->has_vals;
    p.vec_first = vec_first;
    p.nout = nout;
    p.nin = nin;
    p.uvals = u->vals;
    p.ubits = u->bitmap;
    bool can_pull = p.p_ptr != nullptr, can_push = p.s_ptr != nullptr;
    // direction (Table 9): push iff |E_f| ~ d * nnz(u) <= |E| / beta
    uint64_t ulen = 0;
    GB_CHECK(vector_list(const_cast<gb_vector *>(u), &ulen));
    bool push;
    if (d.direction == GB_PUSH) push = can_push;
    else if (d.direction == GB_PULL) push = !can_pull;
    else push = can_push && (!can_pull || ulen * (uint64_t)d.beta <= (uint64_t)nin);
    p.push = push;
    p.ulist = u->list;
    p.ulen = ulen;
    Scratch mb(ctx), tv(ctx), tb(ctx);
    GB_CHECK(make_allowed(ctx, mask, d, nout, mb, &p.allowed));
    uint32_t nw = (nout + 31) / 32;
    GB_CHECK(tv.alloc((size_t)nout * type_size(w->type) + 16));
    GB_CHECK(tb.alloc(((size_t)nw + 1) * 4));
    GB_CHECK(memset_async(ctx, tb.p, 0, ((size_t)nw + 1) * 4));
    p.tvals = tv.p;
    p.tbits = tb.as<uint32_t>();
    bool handled = false;
    GB_CHECK(mxv_dispatch_plus(s, w->type, p, &handled));
    if (!handled) GB_CHECK(mxv_dispatch_min(s, w->type, p, &handled));
    if (!handled) GB_CHECK(mxv_dispatch_other(s, w->type, p, &handled));
    if (!handled) return fail(GB_DOMAIN_MISMATCH, "%s: semiring not available for this type", who);
    return finish_vector(ctx, w, tv.p, tb.as<uint32_t>(), p.allowed, accum, d.replace);
}

gb_info ewise_common(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_binop op, const gb_vector *u,
                     const gb_vector *v, const gb_desc *desc, bool uni, const char *who) {
    if (!w || !u || !v) return fail(GB_NULL_POINTER, "%s: NULL argument", who);
    if (!valid_accum(accum) || op < GB_PLUS || op > GB_MINUS) return fail(GB_INVALID_VALUE, "%s: bad operator", who);
    if (u->n != w->n || v->n != w->n) return fail(GB_DIMENSION_MISMATCH, "%s: sizes differ", who);
    if (u->type != w->type || v->type != w->type) return fail(GB_DOMAIN_MISMATCH, "%s: types differ", who);
    gb_context *ctx = w->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    Desc d = read_desc(desc);
    Scratch mb(ctx), tv(ctx), tb(ctx);
    const uint32_t *allowed = nullptr;
    GB_CHECK(make_allowed(ctx, mask, d, w->n, mb, &allowed));
    uint32_t nw = (w->n + 31) / 32;
    GB_CHECK(tv.alloc((size_t)w->n * type_size(w->type) + 16));
    GB_CHECK(tb.alloc(((size_t)nw + 1) * 4));
    if (w->n) {
        DISPATCH_T(w->type, k_ewise<T><<<nblk(w->n), 256, 0, ctx->stream>>>(
                                (const T *)u->vals, u->bitmap, (const T *)v->vals, v->bitmap, w->n, op, uni,
                                tv.as<T>(), tb.as<uint32_t>()))
        GB_LAUNCH_CHECK();
    }
    return finish_vector(ctx, w, tv.p, tb.as<uint32_t>(), allowed, accum, d.replace);
}

template <typename T>
void host_accum(void *out, gb_binop accum, T r) {
    T *o = (T *)out;
    *o = accum == GB_NOP ? r : apply_binop<T>(accum, *o, r);
}

__global__ void k_sum_u32(const uint32_t *x, uint64_t n, unsigned long long *total) {
    unsigned long long acc = 0;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x)
        acc += x[q];
    acc = dev::warp_sum<unsigned long long>(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// C<M> = accum(C, A (+).(x) B) where M is absent or complemented (the
// masked product of the same call computes only M's positions instead).
gb_info mxm_general(gb_matrix *C, const gb_matrix *M, gb_binop accum, gb_semiring s, const gb_matrix *A,
                    const gb_matrix *B, const Desc &d) {
    gb_context *ctx = C->ctx;
    const gb_type t = C->type;
    const size_t vs = type_size(t);
    // rows of op(A) and of op(B)
    const uint32_t *a_ptr = d.tran0 ? A->colptr : A->rowptr, *a_idx = d.tran0 ? A->rowidx : A->colidx;
    const void *a_vals = A->has_vals ? (d.tran0 ? A->cvals : A->vals) : nullptr;
    const uint32_t *b_ptr = d.tran1 ? B->colptr : B->rowptr, *b_idx = d.tran1 ? B->rowidx : B->colidx;
    const void *b_vals = B->has_vals ? (d.tran1 ? B->cvals : B->vals) : nullptr;
    if (!a_ptr || !b_ptr) return fail(GB_INVALID_VALUE, "gb_mxm: a needed CSC copy is missing");
    const uint32_t ar = C->nrows;
    const uint64_t na = A->nvals;
    // ---- expand: one tuple per product
    Scratch arows(ctx), cnt(ctx), off(ctx), tot(ctx);
    GB_CHECK(arows.alloc((na + 1) * 4));
    GB_CHECK(cnt.alloc((na + 1) * 4));
    GB_CHECK(off.alloc((na + 1) * 4));
    GB_CHECK(tot.alloc(16));
    GB_CHECK(memset_async(ctx, tot.p, 0, 16));
    if (ar) k_expand_ptr<<<nblk(ar) < 4096 ? nblk(ar) : 4096, 256, 0, ctx->stream>>>(a_ptr, ar, arows.as<uint32_t>());
    if (na) {
        k_product_counts<<<nblk(na), 256, 0, ctx->stream>>>(a_idx, na, b_ptr, cnt.as<uint32_t>());
        k_sum_u32<<<1024, 256, 0, ctx->stream>>>(cnt.as<uint32_t>(), na, tot.as<unsigned long long>());
    }
    GB_LAUNCH_CHECK();
    unsigned long long np = 0;
    GB_CUDA(cudaMemcpyAsync(&np, tot.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (np >= 0xffffffffull) return fail(GB_OUT_OF_MEMORY, "gb_mxm: %llu products exceed the 2^32 limit", np);
    GB_CHECK(scan_exclusive_u32(ctx, cnt.as<uint32_t>(), off.as<uint32_t>(), na, nullptr));
    Scratch orow(ctx), ocol(ctx), oval(ctx);
    GB_CHECK(orow.alloc((np + 1) * 4));
    GB_CHECK(ocol.alloc((np + 1) * 4));
    GB_CHECK(oval.alloc((np + 1) * vs + 16));
    DISPATCH_T(t, GB_CHECK(mxm_expand<T>(ctx, s, arows.as<uint32_t>(), a_idx, a_vals, na, b_ptr, b_idx, b_vals,
                                         off.as<uint32_t>(), orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.p)))
    // ---- a complemented mask drops the products at positions M allows; the
    // complement of an absent mask allows nothing
    const bool structural = d.structure || (M && !M->has_vals);
    uint64_t nkeep = np;
    Scratch flag(ctx), pos(ctx), ktot(ctx), r2(ctx), c2(ctx), v2(ctx);
    const uint32_t *trow = orow.as<uint32_t>(), *tcol = ocol.as<uint32_t>();
    const void *tval = oval.p;
    if (d.scmp && !M) nkeep = 0;
    if (d.scmp && M && np) {
        GB_CHECK(flag.alloc((np + 1) * 4));
        GB_CHECK(pos.alloc((np + 1) * 4));
        GB_CHECK(ktot.alloc(8));
        DISPATCH_T(M->has_vals ? M->type : GB_UINT32,
                   k_product_allowed<T><<<nblk(np), 256, 0, ctx->stream>>>(
                       orow.as<uint32_t>(), ocol.as<uint32_t>(), np, M->rowptr, M->colidx,
                       M->has_vals ? (const T *)M->vals : nullptr, structural, flag.as<uint32_t>()))
        GB_LAUNCH_CHECK();
        GB_CHECK(scan_exclusive_u32(ctx, flag.as<uint32_t>(), pos.as<uint32_t>(), np, ktot.as<uint32_t>()));
        uint32_t k32 = 0;
        GB_CUDA(cudaMemcpyAsync(&k32, ktot.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CHECK(sync(ctx));
        nkeep = k32;
        GB_CHECK(r2.alloc((nkeep + 1) * 4));
        GB_CHECK(c2.alloc((nkeep + 1) * 4));
        GB_CHECK(v2.alloc((nkeep + 1) * vs + 16));
        DISPATCH_T(t, k_compact_products<T><<<nblk(np), 256, 0, ctx->stream>>>(
                          flag.as<uint32_t>(), pos.as<uint32_t>(), np, orow.as<uint32_t>(), ocol.as<uint32_t>(),
                          (const T *)oval.p, r2.as<uint32_t>(), c2.as<uint32_t>(), (T *)v2.p))
        GB_LAUNCH_CHECK();
        trow = r2.as<uint32_t>();
        tcol = c2.as<uint32_t>();
        tval = v2.p;
    }
    // ---- sort and compress: P = the product, equal positions reduced by the semiring's add
    gb_matrix *P = nullptr;
    GB_CHECK(gb_matrix_new(&P, ctx, t, C->nrows, C->ncols));
    struct Freer { gb_matrix **m; ~Freer() { gb_matrix_free(m); } } freer{&P};
    GB_CHECK(matrix_build_device(P, trow, tcol, tval, nkeep, semiring_add_op(s), GB_CSR_ONLY));
    // ---- merge with the old C (accum, mask, REPLACE)
    const uint64_t nc = C->built ? C->nvals : 0;
    const uint64_t nt = P->nvals;
    Scratch crows(ctx), keep(ctx), kpos(ctx), kt(ctx);
    uint32_t nold = 0;
    if (nc) {
        GB_CHECK(crows.alloc((nc + 1) * 4));
        GB_CHECK(keep.alloc((nc + 1) * 4));
        GB_CHECK(kpos.alloc((nc + 1) * 4));
        GB_CHECK(kt.alloc(8));
        GB_CHECK(matrix_expand_rows(C, crows.as<uint32_t>()));
        // the mask's values are read as raw bits of their width (as for the masked product)
        const void *mv = M && M->has_vals ? M->vals : nullptr;
        const size_t ms = M && M->has_vals ? type_size(M->type) : 4;
        const uint32_t *mp = M ? M->rowptr : nullptr, *mi = M ? M->colidx : nullptr;
        DISPATCH_T(t, {
            const T *cvals = C->has_vals ? (const T *)C->vals : nullptr;
            T *tv = (T *)P->vals;
            if (ms == 1)
                k_merge_old_c<T, uint8_t><<<nblk(nc), 256, 0, ctx->stream>>>(
                    crows.as<uint32_t>(), C->colidx, cvals, nc, P->rowptr, P->colidx, tv, mp, mi, (const uint8_t *)mv,
                    M != nullptr, structural, d.scmp, accum, d.replace, keep.as<uint32_t>());
            else if (ms == 4)
                k_merge_old_c<T, uint32_t><<<nblk(nc), 256, 0, ctx->stream>>>(
                    crows.as<uint32_t>(), C->colidx, cvals, nc, P->rowptr, P->colidx, tv, mp, mi,
                    (const uint32_t *)mv, M != nullptr, structural, d.scmp, accum, d.replace, keep.as<uint32_t>());
            else
                k_merge_old_c<T, uint64_t><<<nblk(nc), 256, 0, ctx->stream>>>(
                    crows.as<uint32_t>(), C->colidx, cvals, nc, P->rowptr, P->colidx, tv, mp, mi,
                    (const uint64_t *)mv, M != nullptr, structural, d.scmp, accum, d.replace, keep.as<uint32_t>());
        })
        GB_LAUNCH_CHECK();
        GB_CHECK(scan_exclusive_u32(ctx, keep.as<uint32_t>(), kpos.as<uint32_t>(), nc, kt.as<uint32_t>()));
        GB_CUDA(cudaMemcpyAsync(&nold, kt.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CHECK(sync(ctx));
    }
    // ---- the result: T's entries and the kept old ones (distinct positions)
    const uint64_t nr = nt + nold;
    Scratch frow(ctx), fcol(ctx), fval(ctx);
    GB_CHECK(frow.alloc((nr + 1) * 4));
    GB_CHECK(fcol.alloc((nr + 1) * 4));
    GB_CHECK(fval.alloc((nr + 1) * vs + 16));
    if (nt) {
        GB_CHECK(matrix_expand_rows(P, frow.as<uint32_t>()));
        GB_CUDA(cudaMemcpyAsync(fcol.p, P->colidx, nt * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(fval.p, P->vals, nt * vs, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (nold) {
        DISPATCH_T(t, k_emit_old<T><<<nblk(nc), 256, 0, ctx->stream>>>(
                          keep.as<uint32_t>(), kpos.as<uint32_t>(), nc, (uint32_t)nt, crows.as<uint32_t>(), C->colidx,
                          C->has_vals ? (const T *)C->vals : nullptr, frow.as<uint32_t>(), fcol.as<uint32_t>(),
                          (T *)fval.p))
        GB_LAUNCH_CHECK();
    }
    GB_CHECK(matrix_build_device(C, frow.as<uint32_t>(), fcol.as<uint32_t>(), fval.p, nr, GB_FIRST, GB_BUILD_DEFAULT));
    return sync(ctx);
}

}  // namespace
}  // namespace gbx

extern "C" {

gb_info gb_mxv(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_semiring s, const gb_matrix *A,
               const gb_vector *u, const gb_desc *desc) {
    return mxv_common(w, mask, accum, s, A, u, desc, false, "gb_mxv");
}

gb_info gb_vxm(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_semiring s, const gb_vector *u,
               const gb_matrix *A, const gb_desc *desc) {
    return mxv_common(w, mask, accum, s, A, u, desc, true, "gb_vxm");
}

gb_info gb_ewise_add(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_binop op, const gb_vector *u,
                     const gb_vector *v, const gb_desc *desc) {
    return ewise_common(w, mask, accum, op, u, v, desc, true, "gb_ewise_add");
}

gb_info gb_ewise_mult(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_binop op, const gb_vector *u,
                      const gb_vector *v, const gb_desc *desc) {
    return ewise_common(w, mask, accum, op, u, v, desc, false, "gb_ewise_mult");
}

gb_info gb_reduce_vector(void *out, gb_binop accum, gb_monoid m, const gb_vector *u) {
    if (!out || !u) return fail(GB_NULL_POINTER, "gb_reduce_vector: NULL");
    if (m < GB_MONOID_PLUS || m > GB_MONOID_LAND || !valid_accum(accum))
        return fail(GB_INVALID_VALUE, "gb_reduce_vector: bad monoid or accumulator");
    gb_context *ctx = u->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    DISPATCH_T(u->type, {
        T r;
        GB_CHECK(reduce_dense<T>(ctx, (const T *)u->vals, u->bitmap, u->n, m, &r));
        host_accum<T>(out, accum, r);
    })
    return GB_SUCCESS;
}

gb_info gb_reduce_matrix(void *out, gb_binop accum, gb_monoid m, const gb_matrix *A) {
    if (!out || !A) return fail(GB_NULL_POINTER, "gb_reduce_matrix: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_reduce_matrix: matrix not built");
    if (m < GB_MONOID_PLUS || m > GB_MONOID_LAND || !valid_accum(accum))
        return fail(GB_INVALID_VALUE, "gb_reduce_matrix: bad monoid or accumulator");
    gb_context *ctx = A->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    DISPATCH_T(A->type, {
        T r;
        GB_CHECK(reduce_dense<T>(ctx, A->has_vals ? (const T *)A->vals : nullptr, nullptr, A->nvals, m, &r));
        host_accum<T>(out, accum, r);
    })
    return GB_SUCCESS;
}

gb_info gb_reduce_rows(gb_vector *w, const gb_vector *mask, gb_binop accum, gb_monoid m, const gb_matrix *A,
                       const gb_desc *desc) {
    if (!w || !A) return fail(GB_NULL_POINTER, "gb_reduce_rows: NULL");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_reduce_rows: matrix not built");
    if (m < GB_MONOID_PLUS || m > GB_MONOID_LAND || !valid_accum(accum))
        return fail(GB_INVALID_VALUE, "gb_reduce_rows: bad monoid or accumulator");
    Desc d = read_desc(desc);
    const uint32_t *ptr = d.tran0 ? A->colptr : A->rowptr;
    const void *vals = A->has_vals ? (d.tran0 ? A->cvals : A->vals) : nullptr;
    uint32_t n = d.tran0 ? A->ncols : A->nrows;
    if (!ptr) return fail(GB_INVALID_VALUE, "gb_reduce_rows: the matrix has no CSC copy");
    if (w->n != n) return fail(GB_DIMENSION_MISMATCH, "gb_reduce_rows: size mismatch");
    if (A->has_vals && A->type != w->type) return fail(GB_DOMAIN_MISMATCH, "gb_reduce_rows: types differ");
    gb_context *ctx = w->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    Scratch mb(ctx), tv(ctx), tb(ctx);
    const uint32_t *allowed = nullptr;
    GB_CHECK(make_allowed(ctx, mask, d, n, mb, &allowed));
    uint32_t nw = (n + 31) / 32;
    GB_CHECK(tv.alloc((size_t)n * type_size(w->type) + 16));
    GB_CHECK(tb.alloc(((size_t)nw + 1) * 4));
    GB_CHECK(memset_async(ctx, tb.p, 0, ((size_t)nw + 1) * 4));
    if (n) {
        unsigned blocks = (unsigned)((n + 7) / 8 < 65535 * 16 ? (n + 7) / 8 : 65535 * 16);
        DISPATCH_T(w->type, k_reduce_rows<T><<<blocks, 256, 0, ctx->stream>>>(ptr, vals, n, m, tv.as<T>(),
                                                                              tb.as<uint32_t>()))
        GB_LAUNCH_CHECK();
    }
    return finish_vector(ctx, w, tv.p, tb.as<uint32_t>(), allowed, accum, d.replace);
}

gb_info gb_mxm(gb_matrix *C, const gb_matrix *M, gb_binop accum, gb_semiring s, const gb_matrix *A,
               const gb_matrix *B, const gb_desc *desc) {
    if (!C || !A || !B) return fail(GB_NULL_POINTER, "gb_mxm: NULL argument");
    if (!A->built || !B->built || (M && !M->built)) return fail(GB_INVALID_VALUE, "gb_mxm: an input is not built");
    if (!valid_accum(accum)) return fail(GB_INVALID_VALUE, "gb_mxm: bad accumulator");
    if (s < GB_PLUS_TIMES || s > GB_PLUS_PAIR) return fail(GB_INVALID_VALUE, "gb_mxm: bad semiring");
    Desc d = read_desc(desc);
    uint32_t ar = d.tran0 ? A->ncols : A->nrows, ak = d.tran0 ? A->nrows : A->ncols;
    uint32_t bk = d.tran1 ? B->ncols : B->nrows, bc = d.tran1 ? B->nrows : B->ncols;
    if (ak != bk || C->nrows != ar || C->ncols != bc || (M && (M->nrows != ar || M->ncols != bc)))
        return fail(GB_DIMENSION_MISMATCH, "gb_mxm: dimensions do not match");
    gb_type t = C->type;
    if ((A->has_vals && A->type != t) || (B->has_vals && B->type != t))
        return fail(GB_DOMAIN_MISMATCH, "gb_mxm: input and output types differ");
    if (!semiring_supported(s, t)) return fail(GB_DOMAIN_MISMATCH, "gb_mxm: semiring not available for this type");
    if (!M || d.scmp) {
        // no mask or a complemented one: the whole product (expand, sort, compress)
        GB_CUDA(cudaSetDevice(C->ctx->device));
        return mxm_general(C, M, accum, s, A, B, d);
    }
    MxmPlan p;
    p.ctx = C->ctx;
    gb_context *ctx = C->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    p.nrows = ar;
    p.m_ptr = M->rowptr; p.m_idx = M->colidx;
    p.a_ptr = d.tran0 ? A->colptr : A->rowptr;
    p.a_idx = d.tran0 ? A->rowidx : A->colidx;
    p.a_vals = A->has_vals ? (d.tran0 ? A->cvals : A->vals) : nullptr;
    p.b_ptr = d.tran1 ? B->rowptr : B->colptr;
    p.b_idx = d.tran1 ? B->colidx : B->rowidx;
    p.b_vals = B->has_vals ? (d.tran1 ? B->vals : B->cvals) : nullptr;
    if (!p.a_ptr || !p.b_ptr) return fail(GB_INVALID_VALUE, "gb_mxm: a needed CSC copy is missing");
    uint64_t nm = M->nvals;
    size_t vs = type_size(t);
    Scratch cv(ctx), cp(ctx), flag(ctx), pos(ctx), tot(ctx), mrows(ctx);
    GB_CHECK(cv.alloc(nm * vs + 16));
    GB_CHECK(cp.alloc(nm + 16));
    GB_CHECK(flag.alloc((nm + 1) * 4));
    GB_CHECK(pos.alloc((nm + 1) * 4));
    GB_CHECK(tot.alloc(8));
    GB_CHECK(mrows.alloc((nm + 1) * 4));
    p.cvals = cv.p;
    p.cpresent = cp.as<uint8_t>();
    bool handled = false;
    GB_CHECK(mxm_dispatch(s, t, p, &handled));
    if (!handled) return fail(GB_DOMAIN_MISMATCH, "gb_mxm: semiring not available for this type");
    GB_CHECK(matrix_expand_rows(M, mrows.as<uint32_t>()));
    const bool structural = d.structure || !M->has_vals;
    if (nm) {
        DISPATCH_T(M->has_vals ? M->type : GB_UINT32,
                   k_mxm_flags<T><<<nblk(nm), 256, 0, ctx->stream>>>(cp.as<uint8_t>(),
                                                                     M->has_vals ? (const T *)M->vals : nullptr,
                                                                     structural, nm, flag.as<uint32_t>()))
        GB_LAUNCH_CHECK();
    }
    // merge with the old C: accumulate inside M, keep outside M unless REPLACE
    uint64_t nc = C->built ? C->nvals : 0;
    Scratch crows(ctx), keep(ctx), kpos(ctx), ktot(ctx), fromold(ctx);
    if (nc) {
        GB_CHECK(crows.alloc((nc + 1) * 4));
        GB_CHECK(keep.alloc((nc + 1) * 4));
        GB_CHECK(kpos.alloc((nc + 1) * 4));
        GB_CHECK(ktot.alloc(8));
        GB_CHECK(fromold.alloc((nm + 1) * 4));
        GB_CHECK(memset_async(ctx, fromold.p, 0, (nm + 1) * 4));
        GB_CHECK(matrix_expand_rows(C, crows.as<uint32_t>()));
        // the mask's values are reinterpreted as raw bits of their width: "== 0" on the bits
        // equals "== 0" on the value for every supported type except -0.0
        const void *mv = M->has_vals ? M->vals : nullptr;
        size_t ms = M->has_vals ? type_size(M->type) : 4;
        DISPATCH_T(t, {
            if (ms == 1)
                k_old_c<T, uint8_t><<<nblk(nc), 256, 0, ctx->stream>>>(
                    crows.as<uint32_t>(), C->colidx, C->has_vals ? (const T *)C->vals : nullptr, nc, M->rowptr,
                    M->colidx, (const uint8_t *)mv, structural, flag.as<uint32_t>(), cv.as<T>(), accum, d.replace,
                    keep.as<uint32_t>(), fromold.as<uint32_t>());
            else if (ms == 4)
                k_old_c<T, uint32_t><<<nblk(nc), 256, 0, ctx->stream>>>(
                    crows.as<uint32_t>(), C->colidx, C->has_vals ? (const T *)C->vals : nullptr, nc, M->rowptr,
                    M->colidx, (const uint32_t *)mv, structural, flag.as<uint32_t>(), cv.as<T>(), accum, d.replace,
                    keep.as<uint32_t>(), fromold.as<uint32_t>());
            else
                k_old_c<T, uint64_t><<<nblk(nc), 256, 0, ctx->stream>>>(
                    crows.as<uint32_t>(), C->colidx, C->has_vals ? (const T *)C->vals : nullptr, nc, M->rowptr,
                    M->colidx, (const uint64_t *)mv, structural, flag.as<uint32_t>(), cv.as<T>(), accum, d.replace,
                    keep.as<uint32_t>(), fromold.as<uint32_t>());
        })
        if (nm) k_or_flags<<<nblk(nm), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), fromold.as<uint32_t>(), nm);
        GB_LAUNCH_CHECK();
        GB_CHECK(scan_exclusive_u32(ctx, keep.as<uint32_t>(), kpos.as<uint32_t>(), nc, ktot.as<uint32_t>()));
    }
    GB_CHECK(scan_exclusive_u32(ctx, flag.as<uint32_t>(), pos.as<uint32_t>(), nm, tot.as<uint32_t>()));
    uint32_t nnew = 0, nkeep = 0;
    GB_CUDA(cudaMemcpyAsync(&nnew, tot.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (nc) GB_CUDA(cudaMemcpyAsync(&nkeep, ktot.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    uint64_t nt = (uint64_t)nnew + nkeep;
    Scratch orow(ctx), ocol(ctx), oval(ctx);
    GB_CHECK(orow.alloc((nt + 1) * 4));
    GB_CHECK(ocol.alloc((nt + 1) * 4));
    GB_CHECK(oval.alloc((nt + 1) * vs + 16));
    DISPATCH_T(t, {
        if (nm)
            k_mxm_emit<T><<<nblk(nm), 256, 0, ctx->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), nm,
                                                             mrows.as<uint32_t>(), M->colidx, cv.as<T>(),
                                                             orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.as<T>());
        if (nc)
            k_emit_old<T><<<nblk(nc), 256, 0, ctx->stream>>>(keep.as<uint32_t>(), kpos.as<uint32_t>(), nc, nnew,
                                                             crows.as<uint32_t>(), C->colidx,
                                                             C->has_vals ? (const T *)C->vals : nullptr,
                                                             orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.as<T>());
    })
    GB_LAUNCH_CHECK();
    GB_CHECK(matrix_build_device(C, orow.as<uint32_t>(), ocol.as<uint32_t>(), oval.p, nt, GB_FIRST, GB_BUILD_DEFAULT));
    return sync(ctx);
}

}  // extern "C"
