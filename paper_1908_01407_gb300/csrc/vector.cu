// Vector objects (Table 4): a dense value array plus a presence bitmap,
// with a sorted index list built on demand (Section 4.3: the backend keeps
// both dense and sparse forms and switches between them).
#include "common.cuh"
#include "types.cuh"
#include "vector_impl.cuh"

using namespace gbx;

namespace gbx {
namespace {
inline unsigned nblk(uint64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

template <typename T>
__global__ void k_fill(T *vals, uint32_t n, T x) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) vals[i] = x;
}

__global__ void k_bits_all(uint32_t *bits, uint32_t nwords, uint32_t n) {
    uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nwords) {
        uint32_t v = ~0u;
        if (w == nwords - 1 && (n & 31)) v = (1u << (n & 31)) - 1u;
        bits[w] = v;
    }
}

__global__ void k_check_idx(const uint32_t *idx, uint64_t k, uint32_t n, uint32_t *bad) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k && idx[i] >= n) atomicOr(bad, 1u);
}

__global__ void k_iota(uint32_t *p, uint64_t k) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) p[i] = (uint32_t)i;
}

__global__ void k_idx_keys(const uint32_t *idx, uint64_t k, uint64_t *keys) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) keys[i] = idx[i];
}

// one thread per run head of the sorted (index, tuple order) pairs
template <typename T>
__global__ void k_vec_emit(const uint64_t *keys, const uint32_t *order, uint64_t k, const T *src, gb_binop dup,
                           T *vals, uint32_t *bits) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    if (i > 0 && keys[i] == keys[i - 1]) return;
    uint32_t v = (uint32_t)keys[i];
    T acc = src ? src[order[i]] : (T)1;
    for (uint64_t j = i + 1; j < k && keys[j] == keys[i]; ++j) acc = apply_binop<T>(dup, acc, src ? src[order[j]] : (T)1);
    vals[v] = acc;
    atomicOr(&bits[v >> 5], 1u << (v & 31));
}

template <typename T>
__global__ void k_set1(T *vals, uint32_t *bits, uint32_t i, T x) {
    vals[i] = x;
    atomicOr(&bits[i >> 5], 1u << (i & 31));
}

__global__ void k_popc_words(const uint32_t *bits, uint32_t nwords, uint32_t *cnt) {
    uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nwords) cnt[w] = __popc(bits[w]);
}

__global__ void k_list_from_bits(const uint32_t *bits, const uint32_t *pos, uint32_t nwords, uint32_t *list) {
    uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    uint32_t b = bits[w], p = pos[w];
    while (b) {
        list[p++] = w * 32 + (__ffs(b) - 1);
        b &= b - 1;
    }
}

template <typename T>
__global__ void k_gather(const uint32_t *list, uint64_t k, const T *vals, T *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) out[i] = vals[list[i]];
}

template <typename T>
__global__ void k_dense_out(const T *vals, const uint32_t *bits, uint32_t n, T absent, T *out, uint8_t *present) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool p = (bits[i >> 5] >> (i & 31)) & 1u;
    out[i] = p ? vals[i] : absent;
    if (present) present[i] = p ? 1 : 0;
}
}  // namespace

gb_info vector_alloc(gb_vector *v) {
    size_t vs = type_size(v->type);
    GB_CHECK(dalloc(v->ctx, &v->vals, (size_t)v->n * vs + 16));
    GB_CHECK(dalloc_t(v->ctx, &v->bitmap, (size_t)v->nwords + 1));
    GB_CHECK(memset_async(v->ctx, v->bitmap, 0, ((size_t)v->nwords + 1) * 4));
    v->list_valid = false;
    return GB_SUCCESS;
}

gb_info vector_invalidate(gb_vector *v) {
    v->list_valid = false;
    return GB_SUCCESS;
}

// Builds the sorted index list of the stored entries (cached until the
// vector changes); *len receives its length.
gb_info vector_list(gb_vector *v, uint64_t *len) {
    gb_context *ctx = v->ctx;
    if (v->list_valid) { *len = v->list_len; return GB_SUCCESS; }
    if (!v->list) GB_CHECK(dalloc_t(ctx, &v->list, (size_t)v->n + 1));
    Scratch cnt(ctx), pos(ctx), tot(ctx);
    GB_CHECK(cnt.alloc(((size_t)v->nwords + 1) * 4));
    GB_CHECK(pos.alloc(((size_t)v->nwords + 1) * 4));
    GB_CHECK(tot.alloc(4));
    if (v->nwords) {
        k_popc_words<<<nblk(v->nwords), 256, 0, ctx->stream>>>(v->bitmap, v->nwords, cnt.as<uint32_t>());
        GB_CHECK(scan_exclusive_u32(ctx, cnt.as<uint32_t>(), pos.as<uint32_t>(), v->nwords, tot.as<uint32_t>()));
        k_list_from_bits<<<nblk(v->nwords), 256, 0, ctx->stream>>>(v->bitmap, pos.as<uint32_t>(), v->nwords, v->list);
        GB_LAUNCH_CHECK();
        uint32_t h = 0;
        GB_CUDA(cudaMemcpyAsync(&h, tot.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CHECK(sync(ctx));
        v->list_len = h;
    } else {
        v->list_len = 0;
    }
    v->list_valid = true;
    *len = v->list_len;
    return GB_SUCCESS;
}

gb_info vector_nvals(const gb_vector *v, uint64_t *n) {
    // the list holds exactly the stored entries
    return vector_list(const_cast<gb_vector *>(v), n);
}

}  // namespace gbx

#define DISPATCH_T(type, ...)                                  \
    switch (type) {                                            \
    case GB_BOOL: { typedef uint8_t T; __VA_ARGS__; } break;   \
    case GB_INT32: { typedef int32_t T; __VA_ARGS__; } break;  \
    case GB_UINT32: { typedef uint32_t T; __VA_ARGS__; } break; \
    case GB_UINT64: { typedef uint64_t T; __VA_ARGS__; } break; \
    case GB_FP32: { typedef float T; __VA_ARGS__; } break;     \
    case GB_FP64: { typedef double T; __VA_ARGS__; } break;    \
    }

extern "C" {

gb_info gb_vector_new(gb_vector **v, gb_context *ctx, gb_type type, uint64_t n) {
    if (!v || !ctx) return fail(GB_NULL_POINTER, "gb_vector_new: NULL argument");
    if (!valid_type(type)) return fail(GB_INVALID_VALUE, "gb_vector_new: bad type %d", (int)type);
    if (n >= (1ull << 32)) return fail(GB_INVALID_VALUE, "gb_vector_new: size must be < 2^32");
    GB_CUDA(cudaSetDevice(ctx->device));
    gb_vector *x = new gb_vector();
    x->ctx = ctx; x->type = type; x->n = (uint32_t)n; x->nwords = (uint32_t)((n + 31) / 32);
    gb_info r = vector_alloc(x);
    if (r != GB_SUCCESS) { dfree(ctx, x->vals); dfree(ctx, x->bitmap); delete x; return r; }
    *v = x;
    return GB_SUCCESS;
}

gb_info gb_vector_build(gb_vector *v, const uint32_t *idx, const void *vals, uint64_t nvals, gb_binop dup, gb_mem mem) {
    if (!v) return fail(GB_NULL_POINTER, "gb_vector_build: v is NULL");
    if (nvals && !idx) return fail(GB_NULL_POINTER, "gb_vector_build: idx is NULL");
    if (dup < GB_PLUS || dup > GB_MINUS) return fail(GB_INVALID_VALUE, "gb_vector_build: bad dup operator");
    if (nvals >= (1ull << 32)) return fail(GB_INVALID_VALUE, "gb_vector_build: nvals must be < 2^32");
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    size_t vs = type_size(v->type);
    Scratch di(ctx), dv(ctx), keys(ctx), order(ctx), bad(ctx);
    const uint32_t *pi = idx;
    const void *pv = vals;
    if (mem == GB_HOST && nvals) {
        GB_CHECK(di.alloc(nvals * 4 + 16));
        GB_CHECK(copy_in(ctx, di.p, idx, nvals * 4, GB_HOST));
        pi = di.as<uint32_t>();
        if (vals) {
            GB_CHECK(dv.alloc(nvals * vs + 16));
            GB_CHECK(copy_in(ctx, dv.p, vals, nvals * vs, GB_HOST));
            pv = dv.p;
        }
    }
    GB_CHECK(memset_async(ctx, v->bitmap, 0, ((size_t)v->nwords + 1) * 4));
    v->list_valid = false;
    if (!nvals) return sync(ctx);
    GB_CHECK(bad.alloc(4));
    GB_CHECK(memset_async(ctx, bad.p, 0, 4));
    k_check_idx<<<nblk(nvals), 256, 0, ctx->stream>>>(pi, nvals, v->n, bad.as<uint32_t>());
    uint32_t hb = 0;
    GB_CUDA(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (hb) return fail(GB_INVALID_INDEX, "gb_vector_build: an index is >= the vector size");
    GB_CHECK(keys.alloc(nvals * 8));
    GB_CHECK(order.alloc(nvals * 4 + 16));
    k_idx_keys<<<nblk(nvals), 256, 0, ctx->stream>>>(pi, nvals, keys.as<uint64_t>());
    k_iota<<<nblk(nvals), 256, 0, ctx->stream>>>(order.as<uint32_t>(), nvals);
    GB_CHECK(radix_sort_pairs(ctx, keys.as<uint64_t>(), order.as<uint32_t>(), nvals, bits_for(v->n)));
    DISPATCH_T(v->type, k_vec_emit<T><<<nblk(nvals), 256, 0, ctx->stream>>>(
                            keys.as<uint64_t>(), order.as<uint32_t>(), nvals, (const T *)pv, dup, (T *)v->vals,
                            v->bitmap))
    GB_LAUNCH_CHECK();
    return sync(ctx);
}

gb_info gb_vector_build_dense(gb_vector *v, const void *vals, gb_mem mem) {
    if (!v || !vals) return fail(GB_NULL_POINTER, "gb_vector_build_dense: NULL");
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    GB_CHECK(copy_in(ctx, v->vals, vals, (size_t)v->n * type_size(v->type), mem));
    if (v->nwords) k_bits_all<<<nblk(v->nwords), 256, 0, ctx->stream>>>(v->bitmap, v->nwords, v->n);
    GB_LAUNCH_CHECK();
    v->list_valid = false;
    return sync(ctx);
}

gb_info gb_vector_fill(gb_vector *v, const void *scalar) {
    if (!v || !scalar) return fail(GB_NULL_POINTER, "gb_vector_fill: NULL");
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    if (v->n) {
        DISPATCH_T(v->type, k_fill<T><<<nblk(v->n), 256, 0, ctx->stream>>>((T *)v->vals, v->n, *(const T *)scalar))
        k_bits_all<<<nblk(v->nwords), 256, 0, ctx->stream>>>(v->bitmap, v->nwords, v->n);
        GB_LAUNCH_CHECK();
    }
    v->list_valid = false;
    return GB_SUCCESS;
}

gb_info gb_vector_set_element(gb_vector *v, uint32_t idx, const void *scalar) {
    if (!v || !scalar) return fail(GB_NULL_POINTER, "gb_vector_set_element: NULL");
    if (idx >= v->n) return fail(GB_INVALID_INDEX, "gb_vector_set_element: index %u >= size %u", idx, v->n);
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    DISPATCH_T(v->type, k_set1<T><<<1, 1, 0, ctx->stream>>>((T *)v->vals, v->bitmap, idx, *(const T *)scalar))
    GB_LAUNCH_CHECK();
    v->list_valid = false;
    return GB_SUCCESS;
}

gb_info gb_vector_extract_element(const gb_vector *v, uint32_t idx, void *out) {
    if (!v || !out) return fail(GB_NULL_POINTER, "gb_vector_extract_element: NULL");
    if (idx >= v->n) return fail(GB_INVALID_INDEX, "gb_vector_extract_element: index %u >= size %u", idx, v->n);
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    uint32_t word = 0;
    size_t vs = type_size(v->type);
    GB_CUDA(cudaMemcpyAsync(&word, v->bitmap + (idx >> 5), 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(out, (const char *)v->vals + (size_t)idx * vs, vs, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CHECK(sync(ctx));
    if (!((word >> (idx & 31)) & 1u)) return GB_NO_VALUE;
    return GB_SUCCESS;
}

gb_info gb_vector_extract_tuples(const gb_vector *v, uint32_t *idx, void *vals, uint64_t *n_inout, gb_mem mem) {
    if (!v || !n_inout) return fail(GB_NULL_POINTER, "gb_vector_extract_tuples: NULL");
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    uint64_t k = 0;
    GB_CHECK(vector_list(const_cast<gb_vector *>(v), &k));
    if (*n_inout < k) { *n_inout = k; return fail(GB_INSUFFICIENT_SPACE, "extract_tuples: buffer too small"); }
    if (idx) GB_CHECK(copy_out(ctx, idx, v->list, k * 4, mem));
    if (vals && k) {
        Scratch g(ctx);
        size_t vs = type_size(v->type);
        GB_CHECK(g.alloc(k * vs + 16));
        DISPATCH_T(v->type, k_gather<T><<<nblk(k), 256, 0, ctx->stream>>>(v->list, k, (const T *)v->vals, g.as<T>()))
        GB_LAUNCH_CHECK();
        GB_CHECK(copy_out(ctx, vals, g.p, k * vs, mem));
    }
    GB_CHECK(sync(ctx));
    *n_inout = k;
    return GB_SUCCESS;
}

gb_info gb_vector_extract_dense(const gb_vector *v, void *vals, uint8_t *present, const void *absent_value, gb_mem mem) {
    if (!v || !vals || !absent_value) return fail(GB_NULL_POINTER, "gb_vector_extract_dense: NULL");
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaSetDevice(ctx->device));
    size_t vs = type_size(v->type);
    Scratch o(ctx), p(ctx);
    void *dv = vals;
    uint8_t *dp = present;
    if (mem == GB_HOST) {
        GB_CHECK(o.alloc((size_t)v->n * vs + 16));
        dv = o.p;
        if (present) { GB_CHECK(p.alloc((size_t)v->n + 16)); dp = p.as<uint8_t>(); }
    }
    if (v->n) {
        DISPATCH_T(v->type, k_dense_out<T><<<nblk(v->n), 256, 0, ctx->stream>>>(
                                (const T *)v->vals, v->bitmap, v->n, *(const T *)absent_value, (T *)dv, dp))
        GB_LAUNCH_CHECK();
    }
    if (mem == GB_HOST) {
        GB_CHECK(copy_out(ctx, vals, dv, (size_t)v->n * vs, GB_HOST));
        if (present) GB_CHECK(copy_out(ctx, present, dp, v->n, GB_HOST));
    }
    return sync(ctx);
}

gb_info gb_vector_size(const gb_vector *v, uint64_t *n) {
    if (!v || !n) return fail(GB_NULL_POINTER, "gb_vector_size: NULL");
    *n = v->n;
    return GB_SUCCESS;
}

gb_info gb_vector_nvals(const gb_vector *v, uint64_t *n) {
    if (!v || !n) return fail(GB_NULL_POINTER, "gb_vector_nvals: NULL");
    GB_CUDA(cudaSetDevice(v->ctx->device));
    return vector_nvals(v, n);
}

gb_info gb_vector_dup(gb_vector **out, const gb_vector *v) {
    if (!out || !v) return fail(GB_NULL_POINTER, "gb_vector_dup: NULL");
    gb_vector *w = nullptr;
    GB_CHECK(gb_vector_new(&w, v->ctx, v->type, v->n));
    gb_context *ctx = v->ctx;
    GB_CUDA(cudaMemcpyAsync(w->vals, v->vals, (size_t)v->n * type_size(v->type), cudaMemcpyDeviceToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(w->bitmap, v->bitmap, (size_t)v->nwords * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    *out = w;
    return GB_SUCCESS;
}

gb_info gb_vector_clear(gb_vector *v) {
    if (!v) return fail(GB_NULL_POINTER, "gb_vector_clear: NULL");
    GB_CUDA(cudaSetDevice(v->ctx->device));
    GB_CHECK(memset_async(v->ctx, v->bitmap, 0, ((size_t)v->nwords + 1) * 4));
    v->list_valid = false;
    return GB_SUCCESS;
}

gb_info gb_vector_free(gb_vector **v) {
    if (!v) return fail(GB_NULL_POINTER, "gb_vector_free: NULL");
    if (*v) {
        gb_context *ctx = (*v)->ctx;
        cudaSetDevice(ctx->device);
        dfree(ctx, (*v)->vals);
        dfree(ctx, (*v)->bitmap);
        dfree(ctx, (*v)->list);
        delete *v;
        *v = nullptr;
    }
    return GB_SUCCESS;
}

}  // extern "C"
