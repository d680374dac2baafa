// Cone-beam forward projector, the stand-in for the TIGRE projections of Sec. 3.1:
// A = sum_i vol(x_i) Delta over n = ceil((far - near) D oversample) midpoint steps of
// the clipped ray, vol trilinearly interpolated between voxel centres (k + 1/2) / D
// with zero outside the volume (the Beer-Lambert integral of Eq. 1 for a voxel field).
// One thread per detector pixel; the ray prefix is the training sampler's.
#include <cuda_runtime.h>

#include "nh_device.cuh"
#include "nh_internal.h"

namespace nh {

__device__ __forceinline__ float voxel(const float* __restrict__ vol, int D, int x, int y, int z) {
    if ((unsigned)x >= (unsigned)D || (unsigned)y >= (unsigned)D || (unsigned)z >= (unsigned)D) return 0.f;
    return __ldg(vol + ((size_t)z * D + y) * D + x);
}

__global__ void __launch_bounds__(256) k_project(ViewArgs va, const float* __restrict__ vol, int D,
                                                 int oversample, float* __restrict__ proj) {
    const int npix = va.nu * va.nv;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    RayGeo g = ray_setup(va, p, 1);                  // delta = far - near
    float A = 0.f;
    if (g.hit) {
        const float chord = g.delta;
        const int n = (int)ceilf(__fmul_rn(chord, (float)(D * oversample)));
        g.delta = __fdiv_rn(chord, (float)n);
        const float fD = (float)D;
        float acc = 0.f;
        for (int i = 0; i < n; i++) {
            float x[3];
            sample_position(g, i, 0.5f, x);
            int i0[3];
            float f[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float pc = __fsub_rn(__fmul_rn(x[k], fD), 0.5f);
                const float fl = floorf(pc);
                i0[k] = (int)fl;
                f[k] = __fsub_rn(pc, fl);
            }
            float val = 0.f;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
                const float w = (bx ? f[0] : 1.f - f[0]) * (by ? f[1] : 1.f - f[1]) * (bz ? f[2] : 1.f - f[2]);
                val = fmaf(w, voxel(vol, D, i0[0] + bx, i0[1] + by, i0[2] + bz), val);
            }
            acc += val;
        }
        A = acc * g.delta;
    }
    proj[p] = A;
}

cudaError_t launch_project(const ViewArgs& va, int view, const float* vol, int D, int oversample,
                           float* proj, cudaStream_t st) {
    const int npix = va.nu * va.nv;
    if (npix == 0) return cudaSuccess;
    k_project<<<(npix + 255) / 256, 256, 0, st>>>(va, vol, D, oversample, proj + (size_t)view * npix);
    return cudaGetLastError();
}

}  // namespace nh

namespace nh {

// Sum of squared differences in double: fixed grid of partials, then one block
// sums them in order (deterministic for a given n).
constexpr int kMseBlocks = 1024;

__global__ void __launch_bounds__(256) k_sq_diff(const float* __restrict__ a, const float* __restrict__ b,
                                                 int64_t n, double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_sum_parts(const double* __restrict__ part, int np, int64_t n,
                                                   double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] / (double)n;
}

size_t mse_workspace_bytes() { return sizeof(double) * kMseBlocks; }

cudaError_t launch_mse(const float* a, const float* b, int64_t n, double* out, void* ws, cudaStream_t st) {
    k_sq_diff<<<kMseBlocks, 256, 0, st>>>(a, b, n, (double*)ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_parts<<<1, 256, 0, st>>>((const double*)ws, kMseBlocks, n, out);
    return cudaGetLastError();
}

}  // namespace nh
