// 3-D structural similarity of two voxel volumes: the image-quality score the
// paper reports beside PSNR (Sec. 3.2, Fig. 7 and 8), with the settings of the
// SSIM paper it cites (Wang, Bovik, Sheikh and Simoncelli, IEEE TIP 2004): a
// Gaussian window of standard deviation 1.5 voxels and width 11 per axis,
// normalised to sum 1, K1 = 0.01, K2 = 0.03, and the mean of the local index over
// the window positions that lie wholly inside the volume.
//
// The 3-D window is the product of three 1-D Gaussians, so its weighted sums of
// x, y, x^2, y^2 and xy are taken one axis at a time: along x, then y, then z.
// The last pass forms the local index from those five moments
// (sigma^2 = E[x^2] - E[x]^2, sigma_xy = E[xy] - E[x] E[y]) and sums it. All
// arithmetic is FP64: the variances are differences of nearly equal moments in
// flat regions, where only C2 = 9e-4 separates the index from 0 / 0. The sum runs
// over a fixed grid of partials, then in one block in a fixed order, so the score
// is deterministic.
//
// Layout (doubles): pass x writes 5 planes of [D][D][M], pass y 5 planes of
// [D][M][M], M = D - 10; the local index is written [M][M][M] when asked for.
#include <cmath>

#include "nh_eval.h"

namespace nh {
namespace {

constexpr int kW = 2 * kSsimRadius + 1;
constexpr int kSsimBlocks = 1024;
constexpr int kThreads = 256;

struct Window {
    double g[kW];
};

__global__ void __launch_bounds__(kThreads) k_ssim_window_x(const float* __restrict__ x, const float* __restrict__ y,
                                                            int D, int64_t plane, Window w,
                                                            double* __restrict__ out) {
    const int M = D - 2 * kSsimRadius;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= plane) return;                                  // plane = D * D * M
    const int64_t m = t % M, row = t / M;                    // row = z * D + y
    const float* px = x + row * D + m;
    const float* py = y + row * D + m;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
#pragma unroll
    for (int k = 0; k < kW; ++k) {
        const double a = (double)__ldg(px + k), b = (double)__ldg(py + k), g = w.g[k];
        s0 += g * a;
        s1 += g * b;
        s2 += g * a * a;
        s3 += g * b * b;
        s4 += g * a * b;
    }
    out[t] = s0;
    out[plane + t] = s1;
    out[2 * plane + t] = s2;
    out[3 * plane + t] = s3;
    out[4 * plane + t] = s4;
}

// in: 5 planes of [D][D][M] (stride in_plane); out: 5 planes of [D][M][M].
__global__ void __launch_bounds__(kThreads) k_ssim_window_y(const double* __restrict__ in, int D, int64_t in_plane,
                                                            int64_t plane, Window w, double* __restrict__ out) {
    const int M = D - 2 * kSsimRadius;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= plane) return;                                  // plane = D * M * M
    const int64_t mx = t % M, my = (t / M) % M, z = t / ((int64_t)M * M);
    const int64_t base = (z * D + my) * M + mx;
#pragma unroll 1
    for (int s = 0; s < 5; ++s) {
        const double* p = in + s * in_plane + base;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < kW; ++k) acc += w.g[k] * __ldg(p + (int64_t)k * M);
        out[s * plane + t] = acc;
    }
}

// in: 5 planes of [D][M][M] (stride in_plane); the local index over [M][M][M],
// optionally stored, and summed per block into part[blockIdx.x].
__global__ void __launch_bounds__(kThreads) k_ssim_index(const double* __restrict__ in, int D, int64_t in_plane,
                                                         Window w, double c1, double c2,
                                                         double* __restrict__ map, double* __restrict__ part) {
    __shared__ double red[kThreads];
    const int M = D - 2 * kSsimRadius;
    const int64_t n = (int64_t)M * M * M, mm = (int64_t)M * M;
    double local = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t % mm, mz = t / mm;               // r = my * M + mx
        double e[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const double* p = in + s * in_plane + mz * mm + r;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < kW; ++k) acc += w.g[k] * __ldg(p + (int64_t)k * mm);
            e[s] = acc;
        }
        const double mx = e[0], my = e[1];
        const double vx = e[2] - mx * mx, vy = e[3] - my * my, cxy = e[4] - mx * my;
        const double v = ((2.0 * mx * my + c1) * (2.0 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
        if (map) map[t] = v;
        local += v;
    }
    red[threadIdx.x] = local;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kThreads) k_ssim_mean(const double* __restrict__ part, int np, int64_t n,
                                                        double* __restrict__ out) {
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] / (double)n;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

size_t ssim_workspace_bytes(int D) {
    const int64_t M = D - 2 * kSsimRadius;
    return sizeof(double) * (size_t)(5 * (int64_t)D * D * M + 5 * (int64_t)D * M * M + kSsimBlocks);
}

cudaError_t launch_ssim3d(const float* x, const float* y, int D, double data_range, double* mean, double* map,
                          void* ws, cudaStream_t st) {
    const int64_t M = D - 2 * kSsimRadius;
    Window w;
    double sum = 0.0;
    for (int k = 0; k < kW; ++k) {
        const double t = (double)(k - kSsimRadius);
        w.g[k] = std::exp(-(t * t) / (2.0 * 1.5 * 1.5));
        sum += w.g[k];
    }
    for (int k = 0; k < kW; ++k) w.g[k] /= sum;
    const double c1 = (0.01 * data_range) * (0.01 * data_range);
    const double c2 = (0.03 * data_range) * (0.03 * data_range);
    const int64_t px = (int64_t)D * D * M, py = (int64_t)D * M * M;
    double* sx = (double*)ws;
    double* sy = sx + 5 * px;
    double* part = sy + 5 * py;
    k_ssim_window_x<<<blocks_for(px), kThreads, 0, st>>>(x, y, D, px, w, sx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ssim_window_y<<<blocks_for(py), kThreads, 0, st>>>(sx, D, px, py, w, sy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ssim_index<<<kSsimBlocks, kThreads, 0, st>>>(sy, D, py, w, c1, c2, map, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ssim_mean<<<1, kThreads, 0, st>>>(part, kSsimBlocks, M * M * M, mean);
    return cudaGetLastError();
}

}  // namespace nh
