// Field kernels instantiated for __nv_bfloat16 tables.
#include "nh_field.cuh"

namespace nh {
NH_INSTANTIATE_FIELD(__nv_bfloat16)
}  // namespace nh
