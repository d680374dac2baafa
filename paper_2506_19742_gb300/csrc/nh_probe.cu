// Roofline probes: the chip's own capacity for the access patterns of the gather
// and scatter stages, timed by the caller with CUDA events. They have no
// counterpart in the paper; they give the denominators of the gather / scatter
// roofline fractions.
//
//  k_l2_read        streaming 16-byte reads of a buffer, `reps` sweeps (L2 bandwidth
//                   when the buffer fits in L2)
//  k_random_gather  independent random 4- or 8-byte loads from a table (the hashed
//                   levels' corner loads), eight in flight per thread
//  k_random_red     random red.global.add.v2.f32 into a float2 table (the scatter)
//  k_random_red16   random packed 16-bit reductions (bf16x2 or f16x2, 4 bytes) into a
//                   table of 4-byte entries: the scatter a 16-bit gradient table
//                   would issue
//
// Random indices come from a multiply-xorshift integer mix (the lowbias32 constants
// published by C. Wellons) of a per-thread counter.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "nh_internal.h"

namespace nh {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// A value no finite sum of the probes' loads reaches in practice; the store keeps
// the loads live.
constexpr float kNever = 1.2345e-37f;

__global__ void __launch_bounds__(256) k_l2_read(const float4* __restrict__ buf, size_t n4, int reps,
                                                 float* sink) {
    const size_t T = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int r = 0; r < reps; r++) {
        size_t i = t0;
        for (; i + 3 * T < n4; i += 4 * T) {
            const float4 v0 = __ldcg(buf + i), v1 = __ldcg(buf + i + T);
            const float4 v2 = __ldcg(buf + i + 2 * T), v3 = __ldcg(buf + i + 3 * T);
            a0 += v0.x + v0.w;
            a1 += v1.x + v1.w;
            a2 += v2.x + v2.w;
            a3 += v3.x + v3.w;
        }
        for (; i < n4; i += T) {
            const float4 v = __ldcg(buf + i);
            a0 += v.x + v.w;
        }
    }
    const float acc = (a0 + a1) + (a2 + a3);
    if (acc == kNever) *sink = acc;
}

template <int EB>
__global__ void __launch_bounds__(256) k_random_gather(const void* __restrict__ table, uint32_t mask,
                                                       int64_t per_thread, float* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t seed = mix32(t * 2u + 1u);
    float acc = 0.f;
    for (int64_t j = 0; j < per_thread; j += 8) {
        uint32_t idx[8];
#pragma unroll
        for (int k = 0; k < 8; k++) idx[k] = mix32(seed ^ (uint32_t)(j + k) * 0x9e3779b9u) & mask;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if constexpr (EB == 8) {
                const float2 v = __ldg(reinterpret_cast<const float2*>(table) + idx[k]);
                acc += v.x + v.y;
            } else {
                const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(table) + idx[k]);
                acc += __uint_as_float(u & 0x3fffffffu);
            }
        }
    }
    if (acc == kNever) *sink = acc;
}

__global__ void __launch_bounds__(256) k_random_red(float* __restrict__ table, uint32_t mask, int64_t per_thread) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t seed = mix32(t * 2u + 1u);
    for (int64_t j = 0; j < per_thread; j += 8) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t idx = mix32(seed ^ (uint32_t)(j + k) * 0x9e3779b9u) & mask;
            atomicAdd(reinterpret_cast<float2*>(table) + idx, make_float2(1e-30f, 1e-30f));
        }
    }
}

template <int FMT>
__global__ void __launch_bounds__(256) k_random_red16(void* __restrict__ table, uint32_t mask, int64_t per_thread) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t seed = mix32(t * 2u + 1u);
    for (int64_t j = 0; j < per_thread; j += 8) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t idx = mix32(seed ^ (uint32_t)(j + k) * 0x9e3779b9u) & mask;
            if constexpr (FMT == 1)
                atomicAdd(reinterpret_cast<__nv_bfloat162*>(table) + idx, __floats2bfloat162_rn(1e-30f, 1e-30f));
            else
                atomicAdd(reinterpret_cast<__half2*>(table) + idx, __floats2half2_rn(1e-7f, 1e-7f));
        }
    }
}

static int probe_blocks() {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 8;   // eight 256-thread CTAs per SM: 64 resident warps
}

cudaError_t launch_probe_l2_read(const void* buf, size_t bytes, int reps, float* sink, cudaStream_t st) {
    if (bytes == 0 || reps == 0) return cudaSuccess;
    k_l2_read<<<probe_blocks(), 256, 0, st>>>(reinterpret_cast<const float4*>(buf), bytes / 16, reps, sink);
    return cudaGetLastError();
}

static int64_t per_thread_of(int64_t n, int threads) {
    int64_t p = (n + threads - 1) / threads;
    return (p + 7) & ~int64_t(7);
}

cudaError_t launch_probe_random_gather(const void* table, size_t n_entries, int entry_bytes, int64_t n_loads,
                                       float* sink, int64_t* n_done, cudaStream_t st) {
    *n_done = 0;
    if (n_loads == 0) return cudaSuccess;
    const int blocks = probe_blocks();
    const int64_t pt = per_thread_of(n_loads, blocks * 256);
    *n_done = pt * blocks * 256;
    const uint32_t mask = (uint32_t)(n_entries - 1);
    if (entry_bytes == 8)
        k_random_gather<8><<<blocks, 256, 0, st>>>(table, mask, pt, sink);
    else
        k_random_gather<4><<<blocks, 256, 0, st>>>(table, mask, pt, sink);
    return cudaGetLastError();
}

cudaError_t launch_probe_random_red(float* table, size_t n_entries, int64_t n_ops, int64_t* n_done,
                                    cudaStream_t st) {
    *n_done = 0;
    if (n_ops == 0) return cudaSuccess;
    const int blocks = probe_blocks();
    const int64_t pt = per_thread_of(n_ops, blocks * 256);
    *n_done = pt * blocks * 256;
    k_random_red<<<blocks, 256, 0, st>>>(table, (uint32_t)(n_entries - 1), pt);
    return cudaGetLastError();
}

cudaError_t launch_probe_random_red16(void* table, size_t n_entries, int fmt, int64_t n_ops, int64_t* n_done,
                                      cudaStream_t st) {
    *n_done = 0;
    if (n_ops == 0) return cudaSuccess;
    const int blocks = probe_blocks();
    const int64_t pt = per_thread_of(n_ops, blocks * 256);
    *n_done = pt * blocks * 256;
    if (fmt == 1)
        k_random_red16<1><<<blocks, 256, 0, st>>>(table, (uint32_t)(n_entries - 1), pt);
    else
        k_random_red16<2><<<blocks, 256, 0, st>>>(table, (uint32_t)(n_entries - 1), pt);
    return cudaGetLastError();
}

}  // namespace nh
