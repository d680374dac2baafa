// FFT channel-mask selection (Sec. 2.3): some channels of the hash features carry
// noise rather than structure, a Fourier transform tells them apart, and they are
// masked during training. The paper gives no grid, statistic or threshold; the
// reading computed here:
//
//  1. every channel c of the hash features h (the gather's output, before the
//     normalization) is sampled at the voxel centres (k + 1/2) / G of a G^3 grid
//     over the volume, the grid the reconstruction is read out on;
//  2. the channel's mean over the grid is removed;
//  3. its 3-D discrete Fourier transform X_c(kz, ky, kx) is taken, one axis at a
//     time (x, then y, then z; a direct DFT of length G per line, FP64);
//  4. its high-frequency fraction is the share of the power |X_c|^2 at radial
//     frequencies |k| > cutoff, in cycles per voxel (|k| in [0, sqrt(3) / 2]);
//     a channel without variance has fraction 0;
//  5. a channel whose fraction exceeds the threshold gets mask 0, every other 1.
//
// Bin frequencies follow the usual FFT ordering: index i < (G + 1) / 2 is i / G
// cycles per voxel, larger indices (i - G) / G; each is formed as the integer
// times 1 / G in FP64, and the radius as sqrt((kx^2 + ky^2) + kz^2) with every
// operation rounded once, so the |k| > cutoff decision is that of any IEEE FP64
// evaluation in that order.
//
// Sums over the grid (the means, the power sums) are block reductions in a fixed
// order, so the fractions are the same on every run. This is an occasional step
// between training steps, not part of the step.
//
// Workspace (caller-owned): two complex FP64 planes of G^3 x D values (the real
// samples of step 1 reuse the second), the D means; 268 MB at G = 64, D = 32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "nh_device.cuh"
#include "nh_mask.h"

namespace nh {
namespace {

constexpr int kThreads = 256;

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Step 1: the L * F features of every voxel centre of the G^3 grid, channel-major
// (h[c][z][y][x]) in FP64. Coordinates are (k + 1/2) / G, each a rounded float32
// op, the same points the read-out grid uses.
template <int L, typename TT>
__global__ void __launch_bounds__(kThreads) k_mask_gather(FieldArgs fa, const void* tables, int G,
                                                          double* __restrict__ h) {
    const long long n = (long long)G * G * G;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int ix = (int)(t % G), iy = (int)((t / G) % G), iz = (int)(t / ((long long)G * G));
    const float fG = (float)G;
    const float x[3] = {__fdiv_rn(__fadd_rn((float)ix, 0.5f), fG), __fdiv_rn(__fadd_rn((float)iy, 0.5f), fG),
                        __fdiv_rn(__fadd_rn((float)iz, 0.5f), fG)};
    float f[2 * L];
    encode_point<L, TT>(fa, tables, x, f);
#pragma unroll
    for (int c = 0; c < 2 * L; c++) h[(long long)c * n + t] = (double)f[c];
}

// Fixed-order sum of one block: each thread adds its strided elements in turn,
// then a tree over the block's threads.
__device__ __forceinline__ double block_sum(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Step 2: mean of each channel (one block per channel).
__global__ void __launch_bounds__(kThreads) k_mask_mean(const double* __restrict__ h, long long n,
                                                        double* __restrict__ mean) {
    __shared__ double red[kThreads];
    const double* p = h + (long long)blockIdx.x * n;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += kThreads) s += p[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) mean[blockIdx.x] = s / (double)n;
}

// exp(-2 pi i m / G) for m = 0 .. G-1, in shared memory.
__device__ __forceinline__ void twiddles(int G, double2* tw) {
    for (int m = threadIdx.x; m < G; m += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)G, &s, &c);
        tw[m] = make_double2(c, -s);
    }
    __syncthreads();
}

// Step 3, first axis (x): X[c][z][y][kx] = sum_x (h[c][z][y][x] - mean_c) w^(x kx).
// One thread per output bin; the threads of a line read the same G inputs.
__global__ void __launch_bounds__(kThreads) k_dft_x(const double* __restrict__ h, const double* __restrict__ mean,
                                                    int G, long long total, double2* __restrict__ out) {
    extern __shared__ double2 tw[];
    twiddles(G, tw);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const long long n3 = (long long)G * G * G;
    const int k = (int)(t % G);
    const long long line = t - k;
    const double m = mean[t / n3];
    double re = 0.0, im = 0.0;
    int e = 0;                                   // (x k) mod G
    for (int x = 0; x < G; x++) {
        const double v = h[line + x] - m;
        re = fma(v, tw[e].x, re);
        im = fma(v, tw[e].y, im);
        e += k;
        if (e >= G) e -= G;
    }
    out[t] = make_double2(re, im);
}

// Step 3, a strided axis (y: stride G, z: stride G^2): one thread per output bin,
// consecutive threads along x, so every read of a line is coalesced across the warp.
__global__ void __launch_bounds__(kThreads) k_dft_strided(const double2* __restrict__ in, int G, long long stride,
                                                          long long total, double2* __restrict__ out) {
    extern __shared__ double2 tw[];
    twiddles(G, tw);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int k = (int)((t / stride) % G);
    const long long base = t - (long long)k * stride;
    double re = 0.0, im = 0.0;
    int e = 0;
    for (int j = 0; j < G; j++) {
        const double2 v = in[base + (long long)j * stride];
        const double2 w = tw[e];
        re = fma(v.x, w.x, fma(-v.y, w.y, re));
        im = fma(v.x, w.y, fma(v.y, w.x, im));
        e += k;
        if (e >= G) e -= G;
    }
    out[t] = make_double2(re, im);
}

// Frequency of bin i in cycles per voxel: the integer (i or i - G) times 1 / G.
__device__ __forceinline__ double bin_freq(int i, int G) {
    const int q = i < (G + 1) / 2 ? i : i - G;
    return __dmul_rn((double)q, 1.0 / (double)G);
}

// Steps 4 and 5 (one block per channel): total and high-band power, fraction, mask.
__global__ void __launch_bounds__(kThreads) k_mask_power(const double2* __restrict__ X, int G, double cutoff,
                                                         double threshold, int apply, double* __restrict__ frac,
                                                         float* __restrict__ mask_out, DeviceState* state) {
    __shared__ double red[kThreads];
    const long long n3 = (long long)G * G * G;
    const double2* p = X + (long long)blockIdx.x * n3;
    double tot = 0.0, hi = 0.0;
    for (long long i = threadIdx.x; i < n3; i += kThreads) {
        const int ix = (int)(i % G), iy = (int)((i / G) % G), iz = (int)(i / ((long long)G * G));
        const double fx = bin_freq(ix, G), fy = bin_freq(iy, G), fz = bin_freq(iz, G);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz));
        const double2 v = p[i];
        const double pw = __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
        tot += pw;
        if (__dsqrt_rn(r2) > cutoff) hi += pw;
    }
    tot = block_sum(tot, red);
    hi = block_sum(hi, red);
    if (threadIdx.x == 0) {
        const double f = tot > 0.0 ? hi / tot : 0.0;
        const float m = f > threshold ? 0.f : 1.f;
        frac[blockIdx.x] = f;
        if (mask_out) mask_out[blockIdx.x] = m;
        if (apply) state->mask[blockIdx.x] = m;
    }
}

template <typename TT>
cudaError_t gather_tt(const FieldArgs& fa, int G, double* h, cudaStream_t st) {
    const long long n = (long long)G * G * G;
    const unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
    const void* tables = sizeof(TT) == 4 ? (const void*)fa.params : fa.tables_lp;
    if (fa.L == 8) k_mask_gather<8, TT><<<blocks, kThreads, 0, st>>>(fa, tables, G, h);
    else if (fa.L == 16) k_mask_gather<16, TT><<<blocks, kThreads, 0, st>>>(fa, tables, G, h);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace

size_t mask_workspace_bytes(int G, int D) {
    const size_t n = (size_t)G * G * G * (size_t)D;
    return 2 * align256(n * sizeof(double2)) + align256((size_t)D * sizeof(double));
}

bool mask_supported(const FieldArgs& fa) { return fa.F == 2 && (fa.L == 8 || fa.L == 16); }

cudaError_t launch_select_mask(const FieldArgs& fa, int G, double cutoff, double threshold, int apply, double* frac,
                               float* mask_out, void* ws, cudaStream_t st) {
    const long long n3 = (long long)G * G * G;
    const long long total = n3 * fa.D;
    const size_t plane = align256((size_t)total * sizeof(double2));
    double2* A = (double2*)ws;
    double2* B = (double2*)((char*)ws + plane);
    double* h = (double*)B;                       // real samples; B is next written by the y pass
    double* mean = (double*)((char*)ws + 2 * plane);
    cudaError_t e;
    switch (fa.precision) {
        case NH_PREC_F32: e = gather_tt<float>(fa, G, h, st); break;
        case NH_PREC_BF16: e = gather_tt<__nv_bfloat16>(fa, G, h, st); break;
        case NH_PREC_F16: e = gather_tt<__half>(fa, G, h, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_mask_mean<<<fa.D, kThreads, 0, st>>>(h, n3, mean);
    const unsigned blocks = (unsigned)((total + kThreads - 1) / kThreads);
    const size_t sm = (size_t)G * sizeof(double2);
    k_dft_x<<<blocks, kThreads, sm, st>>>(h, mean, G, total, A);
    k_dft_strided<<<blocks, kThreads, sm, st>>>(A, G, G, total, B);
    k_dft_strided<<<blocks, kThreads, sm, st>>>(B, G, (long long)G * G, total, A);
    k_mask_power<<<fa.D, kThreads, 0, st>>>(A, G, cutoff, threshold, apply, frac, mask_out, fa.state);
    return cudaGetLastError();
}

}  // namespace nh
