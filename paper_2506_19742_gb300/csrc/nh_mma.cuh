// Tensor-core MLP for the BF16 / FP16 precision modes: warp-level
// mma.sync.m16n8k16 with float32 accumulation on 32-sample warp tiles.
//
// Fragment layouts (lane = 4 g + t):
//   A 16x16 (row): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]
//   B 16x8  (col): b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C 16x8  (f32): c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
// A warp tile is 32 samples (m-tiles mt = 0, 1) by 32 features (n-tiles nt = 0..3,
// k-steps ks = 0, 1). The C fragments of one layer, after ReLU and packing, are the
// A fragments of the next: A[mt][ks] = {C[mt][2ks].c01, C[mt][2ks].c23,
// C[mt][2ks+1].c01, C[mt][2ks+1].c23}.
//
// Weights live in shared memory as 16-bit copies of W [out][in] and of W^T
// [in][out], rows padded to 40 elements (80 bytes: conflict-free fragment loads
// and 16-byte aligned ldmatrix rows).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace nh {

constexpr int kWS = 40;   // padded row stride (elements) of 16-bit tiles

template <typename T> struct Mma;

template <> struct Mma<__nv_bfloat16> {
    static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    static __device__ __forceinline__ uint16_t one(float x) {
        __nv_bfloat16 v = __float2bfloat16_rn(x);
        return *reinterpret_cast<uint16_t*>(&v);
    }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

template <> struct Mma<__half> {
    static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
        __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    static __device__ __forceinline__ uint16_t one(float x) {
        __half v = __float2half_rn(x);
        return *reinterpret_cast<uint16_t*>(&v);
    }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* row_addr) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(row_addr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ bool pos_lo(uint32_t u) { return (u & 0x8000u) == 0u && (u & 0x7fffu) != 0u; }
__device__ __forceinline__ bool pos_hi(uint32_t u) { return (u & 0x80000000u) == 0u && (u & 0x7fff0000u) != 0u; }

// A fragments [mt][ks] of a [32][kWS] 16-bit tile (row = sample).
template <int KS>
__device__ __forceinline__ void load_afrag(const uint16_t* tile, int lane, uint32_t (&A)[2][KS][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < KS; ks++) {
            const uint16_t* r0 = tile + (16 * mt + g) * kWS + 16 * ks + 2 * t;
            const uint16_t* r1 = r0 + 8 * kWS;
            A[mt][ks][0] = *reinterpret_cast<const uint32_t*>(r0);
            A[mt][ks][1] = *reinterpret_cast<const uint32_t*>(r1);
            A[mt][ks][2] = *reinterpret_cast<const uint32_t*>(r0 + 8);
            A[mt][ks][3] = *reinterpret_cast<const uint32_t*>(r1 + 8);
        }
}

// Writes A fragments back to a [32][kWS] tile (inverse of load_afrag).
template <int KS>
__device__ __forceinline__ void store_afrag(uint16_t* tile, int lane, const uint32_t (&A)[2][KS][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < KS; ks++) {
            uint16_t* r0 = tile + (16 * mt + g) * kWS + 16 * ks + 2 * t;
            uint16_t* r1 = r0 + 8 * kWS;
            *reinterpret_cast<uint32_t*>(r0) = A[mt][ks][0];
            *reinterpret_cast<uint32_t*>(r1) = A[mt][ks][1];
            *reinterpret_cast<uint32_t*>(r0 + 8) = A[mt][ks][2];
            *reinterpret_cast<uint32_t*>(r1 + 8) = A[mt][ks][3];
        }
}

// C[mt][nt] = bias + sum_ks A[mt][ks] B[ks][nt], B from a 16-bit [NOUT][kWS] matrix
// (row n holds the K inputs of output n), NOUT = 8 NT.
template <typename T, int KS, int NT>
__device__ __forceinline__ void mma_layer(const uint16_t* Wn, const float* bias, const uint32_t (&A)[2][KS][4],
                                          int lane, float (&Cf)[2][NT][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const float b0 = bias ? bias[8 * nt + 2 * t] : 0.f;
        const float b1 = bias ? bias[8 * nt + 2 * t + 1] : 0.f;
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            Cf[mt][nt][0] = b0;
            Cf[mt][nt][1] = b1;
            Cf[mt][nt][2] = b0;
            Cf[mt][nt][3] = b1;
        }
    }
#pragma unroll
    for (int ks = 0; ks < KS; ks++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const uint16_t* w = Wn + (8 * nt + g) * kWS + 16 * ks + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(w);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(w + 8);
#pragma unroll
            for (int mt = 0; mt < 2; mt++) Mma<T>::mma(Cf[mt][nt], A[mt][ks], b0, b1);
        }
}

// C[mt][nt] += sum_ks A[mt][ks] B[ks][nt] (no bias, accumulate).
template <typename T, int KS, int NT>
__device__ __forceinline__ void mma_accumulate(const uint16_t* Wn, const uint32_t (&A)[2][KS][4], int lane,
                                               float (&Cf)[2][NT][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < KS; ks++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const uint16_t* w = Wn + (8 * nt + g) * kWS + 16 * ks + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(w);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(w + 8);
#pragma unroll
            for (int mt = 0; mt < 2; mt++) Mma<T>::mma(Cf[mt][nt], A[mt][ks], b0, b1);
        }
}

// 16-bit value of x and the 16-bit rounding of its remainder: x ~ hi + lo with
// about twice the mantissa bits of one 16-bit value.
template <typename T>
__device__ __forceinline__ void split16(float x, uint16_t& hi, uint16_t& lo);
template <>
__device__ __forceinline__ void split16<__nv_bfloat16>(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = *reinterpret_cast<const uint16_t*>(&h);
    lo = *reinterpret_cast<const uint16_t*>(&l);
}
template <>
__device__ __forceinline__ void split16<__half>(float x, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    hi = *reinterpret_cast<const uint16_t*>(&h);
    lo = *reinterpret_cast<const uint16_t*>(&l);
}

// Pack C fragments into hi and lo A fragments (x ~ hi + lo).
template <typename T>
__device__ __forceinline__ void pack_afrag_split(const float (&Cf)[2][4][4], uint32_t (&Ah)[2][2][4],
                                                 uint32_t (&Al)[2][2][4]) {
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < 2; ks++)
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const float* src = Cf[mt][2 * ks + (r >> 1)];
                const int e = (r & 1) * 2;
                uint16_t h0, l0, h1, l1;
                split16<T>(src[e], h0, l0);
                split16<T>(src[e + 1], h1, l1);
                Ah[mt][ks][r] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                Al[mt][ks][r] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
}

// ReLU and pack C fragments (32 outputs) into next-layer A fragments (K = 32).
template <typename T>
__device__ __forceinline__ void relu_pack(const float (&Cf)[2][4][4], uint32_t (&A)[2][2][4]) {
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const float* lo = Cf[mt][2 * ks];
            const float* hi = Cf[mt][2 * ks + 1];
            A[mt][ks][0] = Mma<T>::pack(fmaxf(lo[0], 0.f), fmaxf(lo[1], 0.f));
            A[mt][ks][1] = Mma<T>::pack(fmaxf(lo[2], 0.f), fmaxf(lo[3], 0.f));
            A[mt][ks][2] = Mma<T>::pack(fmaxf(hi[0], 0.f), fmaxf(hi[1], 0.f));
            A[mt][ks][3] = Mma<T>::pack(fmaxf(hi[2], 0.f), fmaxf(hi[3], 0.f));
        }
}

// Pack C fragments (no activation) into A fragments.
template <typename T>
__device__ __forceinline__ void pack_afrag(const float (&Cf)[2][4][4], uint32_t (&A)[2][2][4]) {
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const float* lo = Cf[mt][2 * ks];
            const float* hi = Cf[mt][2 * ks + 1];
            A[mt][ks][0] = Mma<T>::pack(lo[0], lo[1]);
            A[mt][ks][1] = Mma<T>::pack(lo[2], lo[3]);
            A[mt][ks][2] = Mma<T>::pack(hi[0], hi[1]);
            A[mt][ks][3] = Mma<T>::pack(hi[2], hi[3]);
        }
}

}  // namespace nh
