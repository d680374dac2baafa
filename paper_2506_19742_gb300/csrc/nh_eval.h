// Launchers of the evaluation kernels that live outside the training translation
// units (3-D SSIM, the image-quality score reported beside PSNR in Sec. 3.2).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace nh {

constexpr int kSsimRadius = 5;       // 11-voxel Gaussian window per axis
constexpr int kSsimMaxD = 1024;

// Device workspace bytes of one 3-D SSIM evaluation of D^3 volumes (D >= 11).
size_t ssim_workspace_bytes(int D);

// x, y float[D^3] ([z][y][x]); mean: double[1]; map: double[M^3] or null,
// M = D - 10. ws: ssim_workspace_bytes(D) bytes, 8-byte aligned.
cudaError_t launch_ssim3d(const float* x, const float* y, int D, double data_range, double* mean,
                          double* map, void* ws, cudaStream_t st);

}  // namespace nh
