// Fused training kernel instantiated for float tables.
#include "nh_field.cuh"

namespace nh {
NH_INSTANTIATE_TRAIN(float)
}  // namespace nh
