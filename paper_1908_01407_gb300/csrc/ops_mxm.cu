// masked SpGEMM instantiations and the (semiring, type) support table.
#include "ops_impl.cuh"

namespace gbx {

bool semiring_supported(gb_semiring s, gb_type t) {
    if (s == GB_PLUS_TIMES) return t == GB_INT32 || t == GB_UINT32 || t == GB_FP32 || t == GB_FP64;
    if (s == GB_PLUS_PAIR) return t == GB_INT32 || t == GB_UINT32 || t == GB_UINT64 || t == GB_FP32;
    if (s == GB_MIN_PLUS) return t == GB_INT32 || t == GB_UINT32 || t == GB_FP32 || t == GB_FP64;
    if (s == GB_MIN_TIMES) return t == GB_INT32 || t == GB_UINT32 || t == GB_FP32 || t == GB_FP64;
    if (s == GB_MIN_SECOND) return t == GB_INT32 || t == GB_UINT32 || t == GB_FP32 || t == GB_FP64;
    if (s == GB_MAX_PLUS) return t == GB_INT32 || t == GB_FP32 || t == GB_FP64;
    if (s == GB_LOR_LAND) return t == GB_BOOL;
    return false;
}

gb_info mxm_dispatch(gb_semiring s, gb_type t, const MxmPlan &p, bool *handled) {
    *handled = true;
    if (s == GB_PLUS_TIMES && t == GB_INT32) return mxm_run<int32_t, Add::PLUS, Mul::TIMES>(p);
    if (s == GB_PLUS_TIMES && t == GB_UINT32) return mxm_run<uint32_t, Add::PLUS, Mul::TIMES>(p);
    if (s == GB_PLUS_TIMES && t == GB_FP32) return mxm_run<float, Add::PLUS, Mul::TIMES>(p);
    if (s == GB_PLUS_TIMES && t == GB_FP64) return mxm_run<double, Add::PLUS, Mul::TIMES>(p);
    if (s == GB_PLUS_PAIR && t == GB_INT32) return mxm_run<int32_t, Add::PLUS, Mul::PAIR>(p);
    if (s == GB_PLUS_PAIR && t == GB_UINT32) return mxm_run<uint32_t, Add::PLUS, Mul::PAIR>(p);
    if (s == GB_PLUS_PAIR && t == GB_UINT64) return mxm_run<uint64_t, Add::PLUS, Mul::PAIR>(p);
    if (s == GB_PLUS_PAIR && t == GB_FP32) return mxm_run<float, Add::PLUS, Mul::PAIR>(p);
    if (s == GB_MIN_PLUS && t == GB_INT32) return mxm_run<int32_t, Add::MIN, Mul::SATPLUS>(p);
    if (s == GB_MIN_PLUS && t == GB_UINT32) return mxm_run<uint32_t, Add::MIN, Mul::SATPLUS>(p);
    if (s == GB_MIN_PLUS && t == GB_FP32) return mxm_run<float, Add::MIN, Mul::SATPLUS>(p);
    if (s == GB_MIN_PLUS && t == GB_FP64) return mxm_run<double, Add::MIN, Mul::SATPLUS>(p);
    if (s == GB_MIN_TIMES && t == GB_INT32) return mxm_run<int32_t, Add::MIN, Mul::TIMES>(p);
    if (s == GB_MIN_TIMES && t == GB_UINT32) return mxm_run<uint32_t, Add::MIN, Mul::TIMES>(p);
    if (s == GB_MIN_TIMES && t == GB_FP32) return mxm_run<float, Add::MIN, Mul::TIMES>(p);
    if (s == GB_MIN_TIMES && t == GB_FP64) return mxm_run<double, Add::MIN, Mul::TIMES>(p);
    if (s == GB_MIN_SECOND && t == GB_INT32) return mxm_run<int32_t, Add::MIN, Mul::SECOND>(p);
    if (s == GB_MIN_SECOND && t == GB_UINT32) return mxm_run<uint32_t, Add::MIN, Mul::SECOND>(p);
    if (s == GB_MIN_SECOND && t == GB_FP32) return mxm_run<float, Add::MIN, Mul::SECOND>(p);
    if (s == GB_MIN_SECOND && t == GB_FP64) return mxm_run<double, Add::MIN, Mul::SECOND>(p);
    if (s == GB_MAX_PLUS && t == GB_INT32) return mxm_run<int32_t, Add::MAX, Mul::SATPLUS>(p);
    if (s == GB_MAX_PLUS && t == GB_FP32) return mxm_run<float, Add::MAX, Mul::SATPLUS>(p);
    if (s == GB_MAX_PLUS && t == GB_FP64) return mxm_run<double, Add::MAX, Mul::SATPLUS>(p);
    if (s == GB_LOR_LAND && t == GB_BOOL) return mxm_run<uint8_t, Add::LOR, Mul::LAND>(p);
    *handled = false;
    return GB_SUCCESS;
}

}  // namespace gbx
