// Device building blocks of the field kernels: cone-beam ray setup and
// midpoint sampling (Sec. 2.2 / 2.5), hash-grid corner indexing and the
// trilinear gather (hash encoding, Sec. 1), the Normalized Hash Encoder
// (Sec. 2.3) and the FFMA MLP.
//
// The ray-setup / sample / cell prefix is a fixed sequence of explicitly
// rounded float32 operations (__fadd_rn & co. are never contracted into FMA),
// so positions and corner indices are reproducible bit for bit by any IEEE
// float32 implementation that follows the same sequence.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nh_internal.h"

namespace nh {

constexpr uint32_t kPrimeY = 2654435761u;   // Instant-NGP spatial-hash primes
constexpr uint32_t kPrimeZ = 805459861u;

// ----------------------------------------------------------------------------- rays
struct RayGeo {
    float o[3], d[3];
    float near, delta;
    bool hit;
};

// Source-to-pixel ray, unit direction, slab clip to [0,1]^3, midpoint step.
__device__ __forceinline__ RayGeo ray_setup(const ViewArgs& V, int pix, int N) {
    RayGeo g;
    const int i = pix % V.nu, j = pix / V.nu;
    const float half_nu = __fmul_rn((float)V.nu, 0.5f);
    const float half_nv = __fmul_rn((float)V.nv, 0.5f);
    const float ou = __fmul_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), half_nu), V.du);
    const float ov = __fmul_rn(__fsub_rn(__fadd_rn((float)j, 0.5f), half_nv), V.dv);
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float P = __fadd_rn(__fadd_rn(V.c[k], __fmul_rn(ou, V.u[k])), __fmul_rn(ov, V.v[k]));
        d[k] = __fsub_rn(P, V.s[k]);
    }
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])),
                                 __fmul_rn(d[2], d[2]));
    const float len = __fsqrt_rn(len2);
    float near = 0.f, far = __int_as_float(0x7f800000);
    bool hit = true;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        g.o[k] = V.s[k];
        g.d[k] = __fdiv_rn(d[k], len);
        if (g.d[k] != 0.f) {
            const float ta = __fdiv_rn(__fsub_rn(0.f, V.s[k]), g.d[k]);
            const float tb = __fdiv_rn(__fsub_rn(1.f, V.s[k]), g.d[k]);
            near = fmaxf(near, fminf(ta, tb));
            far = fminf(far, fmaxf(ta, tb));
        } else if (V.s[k] < 0.f || V.s[k] > 1.f) {
            hit = false;
        }
    }
    hit = hit && (near < far);
    if (!hit) { near = 0.f; far = 0.f; }
    g.hit = hit;
    g.near = near;
    g.delta = __fdiv_rn(__fsub_rn(far, near), (float)N);
    return g;
}

// Offset u of sample i inside its stratum [i, i + 1) of the ray of pixel `pix`: 1/2
// (the midpoint rule) when seed is 0, else stratified jitter: the top 24 bits of
// output number pix * N + i + 1 of the SplitMix64 generator started at `seed`
// (Steele, Lea and Flood, 2014), times 2^-24, exact in float32.
__device__ __forceinline__ float stratum_offset(unsigned long long seed, int32_t pix, int N, int i) {
    if (seed == 0ull) return 0.5f;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull *
                                      ((unsigned long long)(uint32_t)pix * (unsigned long long)N +
                                       (unsigned long long)i + 1ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)(uint32_t)(z >> 40) * 0x1p-24f;
}

// x_i = o + (near + (i + u) delta) d
__device__ __forceinline__ void sample_position(const RayGeo& g, int i, float u, float x[3]) {
    const float t = __fadd_rn(g.near, __fmul_rn(__fadd_rn((float)i, u), g.delta));
#pragma unroll
    for (int k = 0; k < 3; k++) x[k] = __fadd_rn(g.o[k], __fmul_rn(t, g.d[k]));
}

// ----------------------------------------------------------------------------- hashing
// Cell corner c = min(floor(clamp(x) * N), N - 1) and fraction w = x * N - c (exact).
__device__ __forceinline__ void level_cell(const float x[3], int res, uint32_t c[3], float w[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float xc = fminf(fmaxf(x[k], 0.f), 1.f);
        const float p = __fmul_rn(xc, (float)res);
        int ci = (int)floorf(p);
        ci = min(ci, res - 1);
        c[k] = (uint32_t)ci;
        w[k] = __fsub_rn(p, (float)ci);
    }
}

__device__ __forceinline__ uint32_t corner_index(uint32_t cx, uint32_t cy, uint32_t cz,
                                                 uint32_t stride, bool dense, uint32_t Tmask) {
    if (dense) return cx + cy * stride + cz * stride * stride;
    return (cx ^ (cy * kPrimeY) ^ (cz * kPrimeZ)) & Tmask;
}

// Corner k (bit 0: +x, bit 1: +y, bit 2: +z): index and trilinear weight.
__device__ __forceinline__ void corner(const uint32_t c[3], const float w[3], int k, uint32_t stride,
                                       bool dense, uint32_t Tmask, uint32_t& idx, float& wk) {
    const uint32_t bx = k & 1, by = (k >> 1) & 1, bz = (k >> 2) & 1;
    idx = corner_index(c[0] + bx, c[1] + by, c[2] + bz, stride, dense, Tmask);
    const float wx = bx ? w[0] : 1.f - w[0];
    const float wy = by ? w[1] : 1.f - w[1];
    const float wz = bz ? w[2] : 1.f - w[2];
    wk = (wx * wy) * wz;
}

// ----------------------------------------------------------------------------- tables
// F = 2 features per entry: one 8-byte (f32) or 4-byte (bf16x2 / f16x2) load.
template <typename TT> struct Table;
template <> struct Table<float> {
    static __device__ __forceinline__ float2 load(const void* base, size_t entry) {
        return __ldg(reinterpret_cast<const float2*>(base) + entry);
    }
};
template <> struct Table<__nv_bfloat16> {
    static __device__ __forceinline__ float2 load(const void* base, size_t entry) {
        const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(base) + entry);
        __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&u);
        return __bfloat1622float2(v);
    }
};
template <> struct Table<__half> {
    static __device__ __forceinline__ float2 load(const void* base, size_t entry) {
        const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(base) + entry);
        __half2 v = *reinterpret_cast<const __half2*>(&u);
        return __half22float2(v);
    }
};

// h[2l + f] = sum_k w_k T_l[idx_k][f] for every level (F = 2).
template <int L, typename TT>
__device__ __forceinline__ void encode_point(const FieldArgs& fa, const void* tables, const float x[3],
                                             float (&h)[2 * L]) {
    const size_t T = (size_t)fa.Tmask + 1;
#pragma unroll
    for (int l = 0; l < L; l++) {
        uint32_t c[3];
        float w[3];
        const int res = fa.res[l];
        level_cell(x, res, c, w);
        const bool dense = (fa.dense_mask >> l) & 1u;
        const uint32_t stride = (uint32_t)res + 1u;
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            uint32_t idx;
            float wk;
            corner(c, w, k, stride, dense, fa.Tmask, idx, wk);
            const float2 t = Table<TT>::load(tables, (size_t)l * T + idx);
            a0 = fmaf(wk, t.x, a0);
            a1 = fmaf(wk, t.y, a1);
        }
        h[2 * l] = a0;
        h[2 * l + 1] = a1;
    }
}

// Scatter-add of dL/dh into the float32 gradient tables (one 8-byte vector red per corner).
__device__ __forceinline__ void red_add_f2(float* addr, float a, float b) {
    atomicAdd(reinterpret_cast<float2*>(addr), make_float2(a, b));
}

// Scatter of one sample per lane; all 32 lanes of the warp call it together, and
// lanes whose sample must not contribute pass zeros in dh. Consecutive lanes hold
// consecutive samples of one ray, so lanes in the same cell of a level form one
// contiguous run: where a level has such runs, each run is summed with a segmented
// shuffle reduction (per corner and feature; as many doubling steps as the longest
// run needs) and only its first lane issues the 8 vector atomics. Levels whose
// cells are all distinct scatter directly.
// dhrow: this lane's dL/dh in shared memory, element k at dhrow[k ^ lane] (2 L <= 32).
template <int L>
__device__ __forceinline__ void scatter_point(const FieldArgs& fa, const float x[3], const float* dhrow, int lane) {
    const size_t T = (size_t)fa.Tmask + 1;
#pragma unroll 1
    for (int l = 0; l < L; l++) {
        uint32_t c[3];
        float w[3];
        const int res = fa.res[l];
        level_cell(x, res, c, w);
        const bool dense = (fa.dense_mask >> l) & 1u;
        const uint32_t stride = (uint32_t)res + 1u;
        const float d0 = dhrow[(2 * l) ^ lane], d1 = dhrow[(2 * l + 1) ^ lane];
        const uint32_t px = __shfl_up_sync(0xffffffffu, c[0], 1);
        const uint32_t py = __shfl_up_sync(0xffffffffu, c[1], 1);
        const uint32_t pz = __shfl_up_sync(0xffffffffu, c[2], 1);
        const bool head = lane == 0 || px != c[0] || py != c[1] || pz != c[2];
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        float v[16];
        uint32_t idx[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            float wk;
            corner(c, w, k, stride, dense, fa.Tmask, idx[k], wk);
            v[2 * k] = wk * d0;
            v[2 * k + 1] = wk * d1;
        }
        if (heads != 0xffffffffu) {
            const uint32_t after = lane == 31 ? 0u : (heads & (0xffffffffu << (lane + 1)));
            const int seg_end = after ? (__ffs(after) - 2) : 31;
            // after the steps of offsets 1 .. off, every lane holds the sum over the
            // next 2 off lanes of its run, so the longest run sets the step count
            const int longest = (int)__reduce_max_sync(0xffffffffu, (unsigned)(seg_end - lane + 1));
#pragma unroll 1
            for (int off = 1; off < longest; off <<= 1) {
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    const float t = __shfl_down_sync(0xffffffffu, v[e], off);
                    if (lane + off <= seg_end) v[e] += t;
                }
            }
        }
        if (head) {
            float* gl = fa.grads + (size_t)l * T * 2;
#pragma unroll
            for (int k = 0; k < 8; k++) red_add_f2(gl + (size_t)idx[k] * 2, v[2 * k], v[2 * k + 1]);
        }
    }
}

// ----------------------------------------------------------------------------- normalization
// Per-point LayerNorm over groups of GS features: hhat = (h - mean) / sqrt(var + eps).
template <int D, int GS>
__device__ __forceinline__ void ln_stats(const float (&h)[D], float eps, float (&hhat)[D],
                                         float (&rstd)[D / GS]) {
#pragma unroll
    for (int g = 0; g < D / GS; g++) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < GS; k++) s += h[g * GS + k];
        const float mean = s * (1.f / GS);
        float q = 0.f;
#pragma unroll
        for (int k = 0; k < GS; k++) {
            const float c = h[g * GS + k] - mean;
            q = fmaf(c, c, q);
        }
        const float r = 1.f / sqrtf(q * (1.f / GS) + eps);
        rstd[g] = r;
#pragma unroll
        for (int k = 0; k < GS; k++) hhat[g * GS + k] = (h[g * GS + k] - mean) * r;
    }
}

// dh = rstd (dhhat - mean(dhhat) - hhat mean(dhhat hhat)) per group.
template <int D, int GS>
__device__ __forceinline__ void ln_backward(const float (&hhat)[D], const float (&rstd)[D / GS],
                                            float (&dx)[D]) {
#pragma unroll
    for (int g = 0; g < D / GS; g++) {
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int k = 0; k < GS; k++) {
            s1 += dx[g * GS + k];
            s2 = fmaf(dx[g * GS + k], hhat[g * GS + k], s2);
        }
        s1 *= (1.f / GS);
        s2 *= (1.f / GS);
#pragma unroll
        for (int k = 0; k < GS; k++)
            dx[g * GS + k] = rstd[g] * (dx[g * GS + k] - s1 - hhat[g * GS + k] * s2);
    }
}

// ----------------------------------------------------------------------------- MLP (FFMA)
// out[j] = b[j] + sum_i W[j][i] in[i]; W row-major [OUT][IN] in shared memory.
// Paired FMAs (two per instruction): one half of the pair sums the bias and the
// even-indexed terms, the other the odd-indexed terms, in increasing i; the halves
// are added at the end. The training kernels' rolled layer products use the same
// order, so the forward-only kernels give the same bits.
template <int IN, int OUT>
__device__ __forceinline__ void linear_fwd(const float* __restrict__ sW, const float* __restrict__ sb,
                                           const float (&in)[IN], float (&out)[OUT]) {
#pragma unroll
    for (int j = 0; j < OUT; j++) {
        float2 acc = make_float2(sb[j], 0.f);
#pragma unroll
        for (int i = 0; i < IN; i += 4) {
            const float4 w = *reinterpret_cast<const float4*>(sW + j * IN + i);
            acc = __ffma2_rn(make_float2(w.x, w.y), make_float2(in[i], in[i + 1]), acc);
            acc = __ffma2_rn(make_float2(w.z, w.w), make_float2(in[i + 2], in[i + 3]), acc);
        }
        out[j] = acc.x + acc.y;
    }
}

// ----------------------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace nh
