// mxv/vxm instantiations for the semiring family "plus" (one translation
// unit per family keeps the build parallel).
#include "ops_impl.cuh"

namespace gbx {

gb_info mxv_dispatch_plus(gb_semiring s, gb_type t, const MxvPlan &p, bool *handled) {
    *handled = true;
    if (s == GB_PLUS_TIMES && t == GB_INT32) return p.vec_first ? mxv_run<int32_t, Add::PLUS, Mul::TIMES, true>(p) : mxv_run<int32_t, Add::PLUS, Mul::TIMES, false>(p);
    if (s == GB_PLUS_TIMES && t == GB_UINT32) return p.vec_first ? mxv_run<uint32_t, Add::PLUS, Mul::TIMES, true>(p) : mxv_run<uint32_t, Add::PLUS, Mul::TIMES, false>(p);
    if (s == GB_PLUS_TIMES && t == GB_FP32) return p.vec_first ? mxv_run<float, Add::PLUS, Mul::TIMES, true>(p) : mxv_run<float, Add::PLUS, Mul::TIMES, false>(p);
    if (s == GB_PLUS_TIMES && t == GB_FP64) return p.vec_first ? mxv_run<double, Add::PLUS, Mul::TIMES, true>(p) : mxv_run<double, Add::PLUS, Mul::TIMES, false>(p);
    if (s == GB_PLUS_PAIR && t == GB_INT32) return p.vec_first ? mxv_run<int32_t, Add::PLUS, Mul::PAIR, true>(p) : mxv_run<int32_t, Add::PLUS, Mul::PAIR, false>(p);
    if (s == GB_PLUS_PAIR && t == GB_UINT32) return p.vec_first ? mxv_run<uint32_t, Add::PLUS, Mul::PAIR, true>(p) : mxv_run<uint32_t, Add::PLUS, Mul::PAIR, false>(p);
    if (s == GB_PLUS_PAIR && t == GB_UINT64) return p.vec_first ? mxv_run<uint64_t, Add::PLUS, Mul::PAIR, true>(p) : mxv_run<uint64_t, Add::PLUS, Mul::PAIR, false>(p);
    if (s == GB_PLUS_PAIR && t == GB_FP32) return p.vec_first ? mxv_run<float, Add::PLUS, Mul::PAIR, true>(p) : mxv_run<float, Add::PLUS, Mul::PAIR, false>(p);
    *handled = false;
    return GB_SUCCESS;
}

}  // namespace gbx
