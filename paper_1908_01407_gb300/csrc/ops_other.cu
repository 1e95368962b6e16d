// mxv/vxm instantiations for the semiring family "other" (one translation
// unit per family keeps the build parallel).
#include "ops_impl.cuh"

namespace gbx {

gb_info mxv_dispatch_other(gb_semiring s, gb_type t, const MxvPlan &p, bool *handled) {
    *handled = true;
    if (s == GB_MAX_PLUS && t == GB_INT32) return p.vec_first ? mxv_run<int32_t, Add::MAX, Mul::SATPLUS, true>(p) : mxv_run<int32_t, Add::MAX, Mul::SATPLUS, false>(p);
    if (s == GB_MAX_PLUS && t == GB_FP32) return p.vec_first ? mxv_run<float, Add::MAX, Mul::SATPLUS, true>(p) : mxv_run<float, Add::MAX, Mul::SATPLUS, false>(p);
    if (s == GB_MAX_PLUS && t == GB_FP64) return p.vec_first ? mxv_run<double, Add::MAX, Mul::SATPLUS, true>(p) : mxv_run<double, Add::MAX, Mul::SATPLUS, false>(p);
    if (s == GB_LOR_LAND && t == GB_BOOL) return p.vec_first ? mxv_run<uint8_t, Add::LOR, Mul::LAND, true>(p) : mxv_run<uint8_t, Add::LOR, Mul::LAND, false>(p);
    *handled = false;
    return GB_SUCCESS;
}

}  // namespace gbx
