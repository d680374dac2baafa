// Field kernels instantiated for float tables.
#include "nh_field.cuh"

namespace nh {
NH_INSTANTIATE_FIELD(float)
}  // namespace nh
