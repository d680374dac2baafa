// Fused training kernel instantiated for bf16 tables.
#include "nh_field.cuh"

namespace nh {
NH_INSTANTIATE_TRAIN(__nv_bfloat16)
}  // namespace nh
