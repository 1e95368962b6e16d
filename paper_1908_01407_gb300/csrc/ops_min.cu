// mxv/vxm instantiations for the semiring family "min" (one translation
// unit per family keeps the build parallel).
#include "ops_impl.cuh"

namespace gbx {

gb_info mxv_dispatch_min(gb_semiring s, gb_type t, const MxvPlan &p, bool *handled) {
    *handled = true;
    if (s == GB_MIN_PLUS && t == GB_INT32) return p.vec_first ? mxv_run<int32_t, Add::MIN, Mul::SATPLUS, true>(p) : mxv_run<int32_t, Add::MIN, Mul::SATPLUS, false>(p);
    if (s == GB_MIN_PLUS && t == GB_UINT32) return p.vec_first ? mxv_run<uint32_t, Add::MIN, Mul::SATPLUS, true>(p) : mxv_run<uint32_t, Add::MIN, Mul::SATPLUS, false>(p);
    if (s == GB_MIN_PLUS && t == GB_FP32) return p.vec_first ? mxv_run<float, Add::MIN, Mul::SATPLUS, true>(p) : mxv_run<float, Add::MIN, Mul::SATPLUS, false>(p);
    if (s == GB_MIN_PLUS && t == GB_FP64) return p.vec_first ? mxv_run<double, Add::MIN, Mul::SATPLUS, true>(p) : mxv_run<double, Add::MIN, Mul::SATPLUS, false>(p);
    if (s == GB_MIN_TIMES && t == GB_INT32) return p.vec_first ? mxv_run<int32_t, Add::MIN, Mul::TIMES, true>(p) : mxv_run<int32_t, Add::MIN, Mul::TIMES, false>(p);
    if (s == GB_MIN_TIMES && t == GB_UINT32) return p.vec_first ? mxv_run<uint32_t, Add::MIN, Mul::TIMES, true>(p) : mxv_run<uint32_t, Add::MIN, Mul::TIMES, false>(p);
    if (s == GB_MIN_TIMES && t == GB_FP32) return p.vec_first ? mxv_run<float, Add::MIN, Mul::TIMES, true>(p) : mxv_run<float, Add::MIN, Mul::TIMES, false>(p);
    if (s == GB_MIN_TIMES && t == GB_FP64) return p.vec_first ? mxv_run<double, Add::MIN, Mul::TIMES, true>(p) : mxv_run<double, Add::MIN, Mul::TIMES, false>(p);
    if (s == GB_MIN_SECOND && t == GB_INT32) return p.vec_first ? mxv_run<int32_t, Add::MIN, Mul::SECOND, true>(p) : mxv_run<int32_t, Add::MIN, Mul::SECOND, false>(p);
    if (s == GB_MIN_SECOND && t == GB_UINT32) return p.vec_first ? mxv_run<uint32_t, Add::MIN, Mul::SECOND, true>(p) : mxv_run<uint32_t, Add::MIN, Mul::SECOND, false>(p);
    if (s == GB_MIN_SECOND && t == GB_FP32) return p.vec_first ? mxv_run<float, Add::MIN, Mul::SECOND, true>(p) : mxv_run<float, Add::MIN, Mul::SECOND, false>(p);
    if (s == GB_MIN_SECOND && t == GB_FP64) return p.vec_first ? mxv_run<double, Add::MIN, Mul::SECOND, true>(p) : mxv_run<double, Add::MIN, Mul::SECOND, false>(p);
    *handled = false;
    return GB_SUCCESS;
}

}  // namespace gbx
