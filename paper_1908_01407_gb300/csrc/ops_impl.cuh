// Generic masked semiring matrix-vector and matrix-matrix kernels
// (Sections 4-5): mxv/vxm as pull (masked SpMV, mask first, Boolean early
// exit) or push (SpMSpV over the stored entries of u, the mask tested
// before the atomic write), and the masked SpGEMM of Section 6.3.4.
#pragma once

#include "common.cuh"
#include "types.cuh"

namespace gbx {

// One mxv/vxm, already resolved to "rows of P are the outputs" (pull) and
// "rows of S are the inputs" (push). For mxv, P = CSR(A) and S = CSC(A);
// for vxm, P = CSC(A) and S = CSR(A); a transposed input swaps them.
struct MxvPlan {
    gb_context *ctx;
    const uint32_t *p_ptr, *p_idx;
    const void *p_vals;
    const uint32_t *s_ptr, *s_idx;
    const void *s_vals;
    bool has_vals;            // false: every stored matrix value is 1
    bool vec_first;           // vxm: u(i) (x) A(i,j); mxv: A(i,j) (x) u(j)
    uint32_t nout, nin;
    const void *uvals;
    const uint32_t *ubits;
    const uint32_t *ulist;
    uint64_t ulen;
    const uint32_t *allowed;  // output positions the mask lets through (nullptr: all)
    void *tvals;              // product t: values ...
    uint32_t *tbits;          // ... and presence (zeroed by the caller)
    bool push;
};

// Masked matrix-matrix product C<M> = A (+).(x) B over M's stored
// positions: the row A(i,:) is given by (a_ptr, a_idx, a_vals), the column
// B(:,j) by (b_ptr, b_idx, b_vals) (CSR of A or A^T, CSC of B or B^T).
struct MxmPlan {
    gb_context *ctx;
    uint32_t nrows;
    const uint32_t *m_ptr, *m_idx;
    const uint32_t *a_ptr, *a_idx;
    const void *a_vals;
    const uint32_t *b_ptr, *b_idx;
    const void *b_vals;
    void *cvals;               // [nnz(M)] result values in M's order
    uint8_t *cpresent;         // [nnz(M)] 1 where the intersection was not empty
};

template <typename T>
__device__ __forceinline__ T shfl_xor_t(T v, int o) {
    return __shfl_xor_sync(0xffffffffu, v, o);
}
template <>
__device__ __forceinline__ uint8_t shfl_xor_t<uint8_t>(uint8_t v, int o) {
    return (uint8_t)__shfl_xor_sync(0xffffffffu, (unsigned)v, o);
}

template <typename T>
__device__ __forceinline__ T load_val(const void *vals, uint32_t k) {
    return vals ? reinterpret_cast<const T *>(vals)[k] : (T)1;
}

__device__ __forceinline__ bool bit_of(const uint32_t *bits, uint32_t i) {
    return (bits[i >> 5] >> (i & 31)) & 1u;
}

// pull: a warp per output row; the mask is tested first (only allowed rows
// are computed); under the LOR monoid the row stops at its first true term
template <typename T, Add A, Mul M, bool VF>
__global__ void k_mxv_pull(MxvPlan p) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const T *u = reinterpret_cast<const T *>(p.uvals);
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < p.nout; i += nwarps) {
        if (p.allowed && !bit_of(p.allowed, (uint32_t)i)) continue;
        uint32_t b = p.p_ptr[i], e = p.p_ptr[i + 1];
        T acc = Monoid<T, A>::identity();
        bool any = false;
        for (uint32_t q0 = b; q0 < e; q0 += 32) {
            uint32_t q = q0 + lane;
            if (q < e) {
                uint32_t k = p.p_idx[q];
                if (bit_of(p.ubits, k)) {
                    T a = load_val<T>(p.p_vals, q);
                    T term = VF ? mul_op<T, M>(u[k], a) : mul_op<T, M>(a, u[k]);
                    acc = any ? Monoid<T, A>::op(acc, term) : term;
                    any = true;
                }
            }
            if (A == Add::LOR && __any_sync(0xffffffffu, any && acc != (T)0)) break;
        }
        // warp reduction in a fixed order (deterministic for a given row)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T oa = shfl_xor_t<T>(acc, o);
            int on = __shfl_xor_sync(0xffffffffu, (int)any, o);
            if (on) acc = any ? Monoid<T, A>::op(acc, oa) : oa;
            any = any || on;
        }
        if (lane == 0 && any) {
            reinterpret_cast<T *>(p.tvals)[i] = acc;
            atomicOr(&p.tbits[i >> 5], 1u << (i & 31));
        }
    }
}

// push: a warp per stored entry j of u; each entry of row j of S updates
// t(i) with an atomic monoid operation if the mask allows i
template <typename T, Add A, Mul M, bool VF>
__global__ void k_mxv_push(MxvPlan p) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const T *u = reinterpret_cast<const T *>(p.uvals);
    T *t = reinterpret_cast<T *>(p.tvals);
    for (uint64_t x = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); x < p.ulen; x += nwarps) {
        uint32_t j = p.ulist[x];
        T uj = u[j];
        uint32_t b = p.s_ptr[j], e = p.s_ptr[j + 1];
        for (uint32_t q = b + lane; q < e; q += 32) {
            uint32_t i = p.s_idx[q];
            if (p.allowed && !bit_of(p.allowed, i)) continue;
            T a = load_val<T>(p.s_vals, q);
            T term = VF ? mul_op<T, M>(uj, a) : mul_op<T, M>(a, uj);
            atomic_monoid<T, A>(&t[i], term);
            uint32_t bit = 1u << (i & 31);
            if (!(__ldcg(&p.tbits[i >> 5]) & bit)) atomicOr(&p.tbits[i >> 5], bit);
        }
    }
}

template <typename T>
__global__ void k_fill_identity(T *t, uint32_t n, T x) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) t[i] = x;
}

template <typename T, Add A, Mul M, bool VF>
gb_info mxv_run(const MxvPlan &p) {
    cudaStream_t s = p.ctx->stream;
    int span = prof_begin(p.ctx, p.push ? "mxv_push" : "mxv_pull");
    if (p.push) {
        if (p.nout) k_fill_identity<T><<<(p.nout + 255) / 256, 256, 0, s>>>((T *)p.tvals, p.nout, Monoid<T, A>::identity());
        uint64_t warps = p.ulen ? p.ulen : 1;
        unsigned blocks = (unsigned)((warps + 7) / 8 < 65535 * 16 ? (warps + 7) / 8 : 65535 * 16);
        k_mxv_push<T, A, M, VF><<<blocks, 256, 0, s>>>(p);
    } else {
        uint64_t warps = p.nout ? p.nout : 1;
        unsigned blocks = (unsigned)((warps + 7) / 8 < 65535 * 16 ? (warps + 7) / 8 : 65535 * 16);
        k_mxv_pull<T, A, M, VF><<<blocks, 256, 0, s>>>(p);
    }
    prof_end(p.ctx, span);
    GB_LAUNCH_CHECK();
    return GB_SUCCESS;
}

// masked SpGEMM: a warp per row i of M; for each M(i,j) the lanes take the
// entries of the shorter of A(i,:), B(:,j) and binary-search them in the
// longer (Section 7.5: repeated binary search from the shorter list)
__device__ __forceinline__ bool bsearch_u32(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t x, uint32_t *pos) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint32_t v = a[mid];
        if (v == x) { *pos = mid; return true; }
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

template <typename T, Add A, Mul M>
__global__ void k_mxm_masked(MxmPlan p) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < p.nrows; i += nwarps) {
        uint32_t ab = p.a_ptr[i], ae = p.a_ptr[i + 1];
        for (uint32_t mq = p.m_ptr[i]; mq < p.m_ptr[i + 1]; ++mq) {
            uint32_t j = p.m_idx[mq];
            uint32_t bb = p.b_ptr[j], be = p.b_ptr[j + 1];
            bool a_short = (ae - ab) <= (be - bb);
            uint32_t sb = a_short ? ab : bb, se = a_short ? ae : be;
            uint32_t lb = a_short ? bb : ab, le = a_short ? be : ae;
            const uint32_t *sidx = a_short ? p.a_idx : p.b_idx;
            const uint32_t *lidx = a_short ? p.b_idx : p.a_idx;
            T acc = Monoid<T, A>::identity();
            bool any = false;
            for (uint32_t q = sb + lane; q < se; q += 32) {
                uint32_t k = sidx[q], pos;
                if (bsearch_u32(lidx, lb, le, k, &pos)) {
                    uint32_t qa = a_short ? q : pos, qb = a_short ? pos : q;
                    T term = mul_op<T, M>(load_val<T>(p.a_vals, qa), load_val<T>(p.b_vals, qb));
                    acc = any ? Monoid<T, A>::op(acc, term) : term;
                    any = true;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T oa = shfl_xor_t<T>(acc, o);
                int on = __shfl_xor_sync(0xffffffffu, (int)any, o);
                if (on) acc = any ? Monoid<T, A>::op(acc, oa) : oa;
                any = any || on;
            }
            if (lane == 0) {
                reinterpret_cast<T *>(p.cvals)[mq] = any ? acc : Monoid<T, A>::identity();
                p.cpresent[mq] = any ? 1 : 0;
            }
        }
    }
}

template <typename T, Add A, Mul M>
gb_info mxm_run(const MxmPlan &p) {
    uint64_t warps = p.nrows ? p.nrows : 1;
    unsigned blocks = (unsigned)((warps + 7) / 8 < 65535 * 16 ? (warps + 7) / 8 : 65535 * 16);
    int span = prof_begin(p.ctx, "mxm");
    k_mxm_masked<T, A, M><<<blocks, 256, 0, p.ctx->stream>>>(p);
    prof_end(p.ctx, span);
    GB_LAUNCH_CHECK();
    return GB_SUCCESS;
}

// per-family dispatchers (one translation unit each)
gb_info mxv_dispatch_plus(gb_semiring s, gb_type t, const MxvPlan &p, bool *handled);
gb_info mxv_dispatch_min(gb_semiring s, gb_type t, const MxvPlan &p, bool *handled);
gb_info mxv_dispatch_other(gb_semiring s, gb_type t, const MxvPlan &p, bool *handled);
gb_info mxm_dispatch(gb_semiring s, gb_type t, const MxmPlan &p, bool *handled);
bool semiring_supported(gb_semiring s, gb_type t);

}  // namespace gbx
