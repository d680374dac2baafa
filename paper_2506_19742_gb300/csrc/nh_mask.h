// Launcher of the FFT channel-mask selection (Sec. 2.3), outside the training
// translation units.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "nh_internal.h"

namespace nh {

constexpr int kMaskMaxG = 128;

// Device workspace bytes of one selection on a G^3 grid with D channels.
size_t mask_workspace_bytes(int G, int D);
// Fields the selection kernels are compiled for (F = 2, L = 8 or 16).
bool mask_supported(const FieldArgs& fa);
// frac: double[D]; mask_out: float[D] or null; apply != 0 also installs the mask in
// the field's device state. ws: mask_workspace_bytes(G, D) bytes, 256-byte aligned.
cudaError_t launch_select_mask(const FieldArgs& fa, int G, double cutoff, double threshold, int apply, double* frac,
                               float* mask_out, void* ws, cudaStream_t st);

}  // namespace nh
