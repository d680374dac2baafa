// Field kernels instantiated for __half tables.
#include "nh_field.cuh"

namespace nh {
NH_INSTANTIATE_FIELD(__half)
}  // namespace nh
