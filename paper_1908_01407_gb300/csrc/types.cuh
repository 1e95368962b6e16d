// Element types, binary operators, monoids and semirings as __device__
// functors (Section 6.2: semirings and monoids are __host__ __device__
// functors carrying an identity; here they are compile-time template
// parameters of the kernels and selected at the C ABI by enum).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <float.h>
#include <math.h>

#include "../../include/gbx.h"

namespace gbx {

template <typename T> struct Lim;
template <> struct Lim<uint8_t>  { __host__ __device__ static uint8_t  max() { return 1; }          __host__ __device__ static uint8_t  min() { return 0; } };
template <> struct Lim<int32_t>  { __host__ __device__ static int32_t  max() { return INT32_MAX; }  __host__ __device__ static int32_t  min() { return INT32_MIN; } };
template <> struct Lim<uint32_t> { __host__ __device__ static uint32_t max() { return UINT32_MAX; } __host__ __device__ static uint32_t min() { return 0; } };
template <> struct Lim<uint64_t> { __host__ __device__ static uint64_t max() { return UINT64_MAX; } __host__ __device__ static uint64_t min() { return 0; } };
template <> struct Lim<float>    { __host__ __device__ static float    max() { return INFINITY; }   __host__ __device__ static float    min() { return -INFINITY; } };
template <> struct Lim<double>   { __host__ __device__ static double   max() { return INFINITY; }   __host__ __device__ static double   min() { return -INFINITY; } };

template <typename T> struct IsFloat { static constexpr bool value = false; };
template <> struct IsFloat<float> { static constexpr bool value = true; };
template <> struct IsFloat<double> { static constexpr bool value = true; };

// wrap-around integer arithmetic without signed-overflow UB
template <typename T> __host__ __device__ __forceinline__ T wrap_add(T a, T b) { return a + b; }
template <> __host__ __device__ __forceinline__ int32_t wrap_add<int32_t>(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a + (uint32_t)b);
}
template <typename T> __host__ __device__ __forceinline__ T wrap_mul(T a, T b) { return a * b; }
template <> __host__ __device__ __forceinline__ int32_t wrap_mul<int32_t>(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a * (uint32_t)b);
}
template <> __host__ __device__ __forceinline__ uint8_t wrap_mul<uint8_t>(uint8_t a, uint8_t b) { return (a && b) ? 1 : 0; }
template <> __host__ __device__ __forceinline__ uint8_t wrap_add<uint8_t>(uint8_t a, uint8_t b) { return (a || b) ? 1 : 0; }
template <typename T> __host__ __device__ __forceinline__ T wrap_sub(T a, T b) { return a - b; }
template <> __host__ __device__ __forceinline__ int32_t wrap_sub<int32_t>(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a - (uint32_t)b);
}
template <> __host__ __device__ __forceinline__ uint8_t wrap_sub<uint8_t>(uint8_t a, uint8_t b) { return (a != 0) != (b != 0); }

// saturating add: the identities of min.plus / max.plus absorb
template <typename T> __host__ __device__ __forceinline__ T sat_add(T a, T b) { return a + b; }
template <> __host__ __device__ __forceinline__ uint32_t sat_add<uint32_t>(uint32_t a, uint32_t b) {
    uint32_t s = a + b;
    return s < a ? UINT32_MAX : s;
}
template <> __host__ __device__ __forceinline__ uint64_t sat_add<uint64_t>(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    return s < a ? UINT64_MAX : s;
}
template <> __host__ __device__ __forceinline__ int32_t sat_add<int32_t>(int32_t a, int32_t b) {
    int64_t s = (int64_t)a + (int64_t)b;
    return s > INT32_MAX ? INT32_MAX : (s < INT32_MIN ? INT32_MIN : (int32_t)s);
}
template <> __host__ __device__ __forceinline__ uint8_t sat_add<uint8_t>(uint8_t a, uint8_t b) { return (a || b) ? 1 : 0; }

template <typename T>
__host__ __device__ __forceinline__ T apply_binop(gb_binop op, T a, T b) {
    switch (op) {
    case GB_PLUS: return wrap_add<T>(a, b);
    case GB_TIMES: return wrap_mul<T>(a, b);
    case GB_MIN: return b < a ? b : a;
    case GB_MAX: return a < b ? b : a;
    case GB_LOR: return (T)((a != (T)0) || (b != (T)0));
    case GB_LAND: return (T)((a != (T)0) && (b != (T)0));
    case GB_FIRST: return a;
    case GB_SECOND: return b;
    case GB_PAIR: return (T)1;
    case GB_MINUS: return wrap_sub<T>(a, b);
    default: return a;
    }
}

enum class Add { PLUS, LOR, MIN, MAX };
enum class Mul { TIMES, LAND, SATPLUS, SECOND, PAIR };

template <typename T, Add A>
struct Monoid {
    __host__ __device__ __forceinline__ static T identity() {
        if (A == Add::PLUS || A == Add::LOR) return (T)0;
        if (A == Add::MIN) return Lim<T>::max();
        return Lim<T>::min();
    }
    __host__ __device__ __forceinline__ static T op(T a, T b) {
        if (A == Add::PLUS) return wrap_add<T>(a, b);
        if (A == Add::LOR) return (T)((a != (T)0) || (b != (T)0));
        if (A == Add::MIN) return b < a ? b : a;
        return a < b ? b : a;
    }
};

template <typename T, Mul M>
__host__ __device__ __forceinline__ T mul_op(T a, T b) {
    if (M == Mul::TIMES) return wrap_mul<T>(a, b);
    if (M == Mul::LAND) return (T)((a != (T)0) && (b != (T)0));
    if (M == Mul::SATPLUS) return sat_add<T>(a, b);
    if (M == Mul::SECOND) return b;
    return (T)1;
}

// ---------------------------------------------------------------- atomics
__device__ __forceinline__ void atomic_or_byte(uint8_t *p, uint8_t v) {
    if (!v) return;
    uintptr_t a = (uintptr_t)p;
    unsigned int *w = (unsigned int *)(a & ~(uintptr_t)3);
    atomicOr(w, 1u << (8 * (a & 3)));
}

template <typename T> __device__ __forceinline__ void atomic_plus(T *p, T v);
template <> __device__ __forceinline__ void atomic_plus<int32_t>(int32_t *p, int32_t v) { atomicAdd((int *)p, (int)v); }
template <> __device__ __forceinline__ void atomic_plus<uint32_t>(uint32_t *p, uint32_t v) { atomicAdd((unsigned *)p, v); }
template <> __device__ __forceinline__ void atomic_plus<uint64_t>(uint64_t *p, uint64_t v) {
    atomicAdd((unsigned long long *)p, (unsigned long long)v);
}
template <> __device__ __forceinline__ void atomic_plus<float>(float *p, float v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void atomic_plus<double>(double *p, double v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void atomic_plus<uint8_t>(uint8_t *p, uint8_t v) { atomic_or_byte(p, v); }

template <typename T> __device__ __forceinline__ void atomic_min(T *p, T v);
template <> __device__ __forceinline__ void atomic_min<int32_t>(int32_t *p, int32_t v) { atomicMin((int *)p, (int)v); }
template <> __device__ __forceinline__ void atomic_min<uint32_t>(uint32_t *p, uint32_t v) { atomicMin((unsigned *)p, v); }
template <> __device__ __forceinline__ void atomic_min<uint64_t>(uint64_t *p, uint64_t v) {
    atomicMin((unsigned long long *)p, (unsigned long long)v);
}
template <> __device__ __forceinline__ void atomic_min<float>(float *p, float v) {
    int *ip = (int *)p;
    int old = *ip;
    while (v < __int_as_float(old)) {
        int prev = atomicCAS(ip, old, __float_as_int(v));
        if (prev == old) break;
        old = prev;
    }
}
template <> __device__ __forceinline__ void atomic_min<double>(double *p, double v) {
    unsigned long long *ip = (unsigned long long *)p;
    unsigned long long old = *ip;
    while (v < __longlong_as_double((long long)old)) {
        unsigned long long prev = atomicCAS(ip, old, (unsigned long long)__double_as_longlong(v));
        if (prev == old) break;
        old = prev;
    }
}
template <> __device__ __forceinline__ void atomic_min<uint8_t>(uint8_t *p, uint8_t v) {
    if (v) return;
    uintptr_t a = (uintptr_t)p;
    atomicAnd((unsigned int *)(a & ~(uintptr_t)3), ~(0xffu << (8 * (a & 3))));
}

template <typename T> __device__ __forceinline__ void atomic_max(T *p, T v);
template <> __device__ __forceinline__ void atomic_max<int32_t>(int32_t *p, int32_t v) { atomicMax((int *)p, (int)v); }
template <> __device__ __forceinline__ void atomic_max<uint32_t>(uint32_t *p, uint32_t v) { atomicMax((unsigned *)p, v); }
template <> __device__ __forceinline__ void atomic_max<uint64_t>(uint64_t *p, uint64_t v) {
    atomicMax((unsigned long long *)p, (unsigned long long)v);
}
template <> __device__ __forceinline__ void atomic_max<float>(float *p, float v) {
    int *ip = (int *)p;
    int old = *ip;
    while (__int_as_float(old) < v) {
        int prev = atomicCAS(ip, old, __float_as_int(v));
        if (prev == old) break;
        old = prev;
    }
}
template <> __device__ __forceinline__ void atomic_max<double>(double *p, double v) {
    unsigned long long *ip = (unsigned long long *)p;
    unsigned long long old = *ip;
    while (__longlong_as_double((long long)old) < v) {
        unsigned long long prev = atomicCAS(ip, old, (unsigned long long)__double_as_longlong(v));
        if (prev == old) break;
        old = prev;
    }
}
template <> __device__ __forceinline__ void atomic_max<uint8_t>(uint8_t *p, uint8_t v) { atomic_or_byte(p, v); }

template <typename T, Add A>
__device__ __forceinline__ void atomic_monoid(T *p, T v) {
    if (A == Add::PLUS) atomic_plus<T>(p, v);
    else if (A == Add::LOR) {
        if (sizeof(T) == 1) atomic_or_byte((uint8_t *)p, (uint8_t)(v != (T)0));
        else if (v != (T)0) atomic_max<T>(p, (T)1);
    } else if (A == Add::MIN) atomic_min<T>(p, v);
    else atomic_max<T>(p, v);
}

}  // namespace gbx
