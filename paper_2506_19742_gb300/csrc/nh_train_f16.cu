// Fused training kernel instantiated for f16 tables.
#include "nh_field.cuh"

namespace nh {
NH_INSTANTIATE_TRAIN(__half)
}  // namespace nh
