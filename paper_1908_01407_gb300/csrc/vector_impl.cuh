// Internal vector helpers shared by the operation translation units.
#pragma once
#include "common.cuh"

namespace gbx {
gb_info vector_alloc(gb_vector *v);
gb_info vector_list(gb_vector *v, uint64_t *len);
gb_info vector_nvals(const gb_vector *v, uint64_t *n);
gb_info vector_invalidate(gb_vector *v);
}  // namespace gbx
