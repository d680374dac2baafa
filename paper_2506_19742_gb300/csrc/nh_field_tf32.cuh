// FP32 MLP of the training kernels on tensor cores. One warp runs the MLP of its 32
// samples as 32 x 32 tiles with mma.sync.m16n8k8 on TF32 operands and float32
// accumulation. A TF32 value keeps 10 of float32's 23 stored mantissa bits, so every
// operand is split in two, x = hi + lo with hi = tf32(x) and lo = tf32(x - hi)
// (x - hi is exact in float32), and each product takes three tensor-core products,
// lo_a hi_b + hi_a lo_b + hi_a hi_b (the small ones first); the dropped lo_a lo_b
// and the rounding of lo leave about 2^-21 of |a| |b| per product, so a 32-term
// dot product stays within about 1e-6 of the magnitudes it sums, against the
// 1e-5 relative bound of the FP32 forward.
//
// Fragment layouts of m16n8k8 (lane = 4 g + t):
//   A 16x8 (row): a0 = A[g][t], a1 = A[g+8][t], a2 = A[g][t+4], a3 = A[g+8][t+4]
//   B 8x8  (col): b0 = B[t][g], b1 = B[t+4][g]
//   C 16x8 (f32): c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
// A warp tile is 32 samples (m-tiles mt = 0, 1) by 32 features (n-tiles nt = 0..3).
// Inside each 8-wide k-step the contraction index is permuted, logical t <-> 2t
// and logical t + 4 <-> 2t + 1, so the C fragments of one layer are the A fragments
// of the next without leaving registers: a = {c0, c2, c1, c3}; B fragments follow
// the same permutation (b0 = B[8 ks + 2t][g], b1 = B[8 ks + 2t + 1][g]).
//
// Shared memory: per CTA the float32 W_l^T ([IN][32], l < H) in tiles whose
// columns are XOR-swizzled by wtsw, in place of W_l in the CTA's copy of the dense
// parameters; per warp two 32 x 32 float tiles (tsw swizzle), one for a layer's
// input rows (or C fragments) and one for dz. The swizzles make fragment-pattern
// loads and stores conflict-free. The weights are constant within a launch, so
// where shared memory allows (PS), the CTA splits each of them once at staging:
// the W^T tile then holds hi and a second tile of the same layout holds lo, and
// the products read both halves instead of splitting the weight at every use
// (the same bits either way).
#pragma once
#include <stdint.h>

namespace nh {

// Element (row, col) of a 32-column weight tile: the column's bits 3-4 are XORed
// with a 2-bit hash of the row, so that the forward's column reads (rows 8 ks + 2t
// and 8 ks + 2t + 1, columns 8 nt + g) and the data gradient's row reads (row
// 8 nt + g, columns 8 ks + 2t and + 1) hit 32 different banks.
__device__ __forceinline__ int wtsw(int row, int col) {
    return row * 32 + (col ^ ((((row >> 1) ^ row) & 3) << 3));
}
// Element (row, col) of a warp's 32 x 32 tile (row = sample): column bits 3-4 XOR
// row bits 0-1, so that C-fragment stores, A-fragment row loads and the weight
// gradient's column loads are conflict-free, and float2 / float4 groups stay whole.
__device__ __forceinline__ int tsw(int row, int col) { return row * 32 + (col ^ ((row & 3) << 3)); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(__fsub_rn(x, __uint_as_float(hi)));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c += a b with both operands split: lo_a hi_b + hi_a lo_b + hi_a hi_b.
__device__ __forceinline__ void mma3s(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                      uint32_t bh0, uint32_t bl0, uint32_t bh1, uint32_t bl1) {
    mma_tf32(c, al, bh0, bh1);
    mma_tf32(c, ah, bl0, bl1);
    mma_tf32(c, ah, bh0, bh1);
}

// B operand pair (b0, b1) of a weight tile at elements e0, e1: split here, or
// (PS) read as hi from the W^T tile and lo from the lo tile.
template <bool PS>
__device__ __forceinline__ void wt_operand(const float* Wt, const float* Wlo, int e0, int e1, uint32_t& bh0,
                                           uint32_t& bl0, uint32_t& bh1, uint32_t& bl1) {
    if constexpr (PS) {
        bh0 = __float_as_uint(Wt[e0]);
        bh1 = __float_as_uint(Wt[e1]);
        bl0 = __float_as_uint(Wlo[e0]);
        bl1 = __float_as_uint(Wlo[e1]);
    } else {
        split_tf32(Wt[e0], bh0, bl0);
        split_tf32(Wt[e1], bh1, bl1);
    }
}

// Split A fragment of k-step ks taken from C fragments (permuted contraction index).
__device__ __forceinline__ void afrag_from_c(const float (&c)[4], uint32_t (&ah)[4], uint32_t (&al)[4]) {
    split_tf32(c[0], ah[0], al[0]);
    split_tf32(c[2], ah[1], al[1]);
    split_tf32(c[1], ah[2], al[2]);
    split_tf32(c[3], ah[3], al[3]);
}

// CTA staging of the float32 W_l^T tiles (l < H): the tile of layer l takes the
// place of W_l ([32][IN], 32 IN floats) in the CTA's copy of the dense parameters
// (sp + lay.W(l)), read again from global memory (gdense: the dense block), so the
// tiles cost no shared memory of their own. Only the training kernels' tensor-core
// MLP reads sp's W_l (l < H), and only as these tiles. With wlo (kW x kW floats
// per layer, layer l at wlo + l kW kW) the weights are split here: the tile gets
// hi = tf32(w) and wlo's tile lo = tf32(w - hi).
__device__ __forceinline__ void stage_wt_tf32(const float* __restrict__ gdense, const DenseLayout& lay, int D,
                                              float* sp, float* wlo) {
    for (int l = 0; l < lay.H; l++) {
        const int IN = l == 0 ? D : kW;
        const float* W = gdense + lay.W(l);
        float* Wt = sp + lay.W(l);
        for (int e = threadIdx.x; e < 32 * IN; e += blockDim.x) {
            const int j = e / IN, i = e - j * IN;
            if (wlo) {
                uint32_t hi, lo;
                split_tf32(W[e], hi, lo);
                Wt[wtsw(i, j)] = __uint_as_float(hi);
                wlo[l * kW * kW + wtsw(i, j)] = __uint_as_float(lo);
            } else {
                Wt[wtsw(i, j)] = W[e];
            }
        }
    }
}

// C fragments (rows = samples, NT n-tiles of columns) <-> a warp tile.
template <int NT>
__device__ __forceinline__ void frag_to_tile(float* tile, int lane, const float (&c)[2][NT][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int r = 16 * mt + g, col = 8 * nt + 2 * t;
            *reinterpret_cast<float2*>(tile + tsw(r, col)) = make_float2(c[mt][nt][0], c[mt][nt][1]);
            *reinterpret_cast<float2*>(tile + tsw(r + 8, col)) = make_float2(c[mt][nt][2], c[mt][nt][3]);
        }
}
template <int NT>
__device__ __forceinline__ void tile_to_frag(const float* tile, int lane, float (&c)[2][NT][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int r = 16 * mt + g, col = 8 * nt + 2 * t;
            const float2 u = *reinterpret_cast<const float2*>(tile + tsw(r, col));
            const float2 v = *reinterpret_cast<const float2*>(tile + tsw(r + 8, col));
            c[mt][nt][0] = u.x;
            c[mt][nt][1] = u.y;
            c[mt][nt][2] = v.x;
            c[mt][nt][3] = v.y;
        }
}

// This lane's row (N floats, N a multiple of 4) <-> a warp tile.
template <int N>
__device__ __forceinline__ void row_to_tile(float* tile, int lane, const float (&v)[N]) {
#pragma unroll
    for (int q = 0; q < N / 4; q++)
        *reinterpret_cast<float4*>(tile + tsw(lane, 4 * q)) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                                          v[4 * q + 3]);
}
template <int N>
__device__ __forceinline__ void tile_to_row(const float* tile, int lane, float (&v)[N]) {
#pragma unroll
    for (int q = 0; q < N / 4; q++) {
        const float4 u = *reinterpret_cast<const float4*>(tile + tsw(lane, 4 * q));
        v[4 * q] = u.x;
        v[4 * q + 1] = u.y;
        v[4 * q + 2] = u.z;
        v[4 * q + 3] = u.w;
    }
}

// z[s][j] = b[j] + sum_i in[s][i] W[j][i] for the warp's 32 samples, 32 outputs.
// Input rows from a warp tile (KS = IN / 8 k-steps). Wlo: the lo tile (PS only).
template <int KS, bool PS>
__device__ __forceinline__ void tf32_layer_tile(const float* tile, const float* Wt, const float* Wlo,
                                                const float* bias, int lane, float (&z)[2][4][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            z[mt][nt][0] = b0;
            z[mt][nt][1] = b1;
            z[mt][nt][2] = b0;
            z[mt][nt][3] = b1;
        }
    }
#pragma unroll
    for (int ks = 0; ks < KS; ks++) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            const float2 u = *reinterpret_cast<const float2*>(tile + tsw(16 * mt + g, 8 * ks + 2 * t));
            const float2 v = *reinterpret_cast<const float2*>(tile + tsw(16 * mt + g + 8, 8 * ks + 2 * t));
            const float c[4] = {u.x, u.y, v.x, v.y};
            afrag_from_c(c, ah[mt], al[mt]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            uint32_t bh0, bl0, bh1, bl1;
            wt_operand<PS>(Wt, Wlo, wtsw(8 * ks + 2 * t, 8 * nt + g), wtsw(8 * ks + 2 * t + 1, 8 * nt + g), bh0, bl0,
                           bh1, bl1);
#pragma unroll
            for (int mt = 0; mt < 2; mt++) mma3s(z[mt][nt], ah[mt], al[mt], bh0, bl0, bh1, bl1);
        }
    }
}

// The same with the input in C fragments (32 features, the previous layer's output).
template <bool PS>
__device__ __forceinline__ void tf32_layer_frag(const float (&a)[2][4][4], const float* Wt, const float* Wlo,
                                                const float* bias, int lane, float (&z)[2][4][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            z[mt][nt][0] = b0;
            z[mt][nt][1] = b1;
            z[mt][nt][2] = b0;
            z[mt][nt][3] = b1;
        }
    }
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) afrag_from_c(a[mt][ks], ah[mt], al[mt]);
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            uint32_t bh0, bl0, bh1, bl1;
            wt_operand<PS>(Wt, Wlo, wtsw(8 * ks + 2 * t, 8 * nt + g), wtsw(8 * ks + 2 * t + 1, 8 * nt + g), bh0, bl0,
                           bh1, bl1);
#pragma unroll
            for (int mt = 0; mt < 2; mt++) mma3s(z[mt][nt], ah[mt], al[mt], bh0, bl0, bh1, bl1);
        }
    }
}

// Data gradient din[s][i] = sum_j dz[s][j] W[j][i], NT = IN / 8 output n-tiles; dz in
// C fragments (32 columns j), B[j][i] = W^T[i][j] read as pairs from the W^T tile.
template <int NT, bool PS>
__device__ __forceinline__ void tf32_dgrad(const float (&dz)[2][4][4], const float* Wt, const float* Wlo, int lane,
                                           float (&din)[2][NT][4]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int c = 0; c < 4; c++) din[mt][nt][c] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) afrag_from_c(dz[mt][ks], ah[mt], al[mt]);
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int e = wtsw(8 * nt + g, 8 * ks + 2 * t);
            const float2 b = *reinterpret_cast<const float2*>(Wt + e);
            uint32_t bh0, bl0, bh1, bl1;
            if constexpr (PS) {
                const float2 bl = *reinterpret_cast<const float2*>(Wlo + e);
                bh0 = __float_as_uint(b.x);
                bh1 = __float_as_uint(b.y);
                bl0 = __float_as_uint(bl.x);
                bl1 = __float_as_uint(bl.y);
            } else {
                split_tf32(b.x, bh0, bl0);
                split_tf32(b.y, bh1, bl1);
            }
#pragma unroll
            for (int mt = 0; mt < 2; mt++) mma3s(din[mt][nt], ah[mt], al[mt], bh0, bl0, bh1, bl1);
        }
    }
}

// Weight gradient dW[j][i] = sum_s dz[s][j] act[s][i] of the warp's 32 samples,
// added to the CTA accumulator gW (element (j, i) at j IN + wswz(i, j, IN)).
// M = j (two 16-row halves), N = i (IN / 8 n-tiles), K = s (four k-steps); A and B
// come from the dz and input tiles. Each k-step splits its B values once for both
// halves of j.
template <int IN>
__device__ __forceinline__ void tf32_wgrad(const float* dzt, const float* act, float* gW, int lane) {
    constexpr int NT = IN / 8;
    const int g = lane >> 2, t = lane & 3;
    float dw[2][NT][4];
#pragma unroll
    for (int mj = 0; mj < 2; mj++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int c = 0; c < 4; c++) dw[mj][nt][c] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        const int s0 = 8 * ks + t, s1 = s0 + 4;
        uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            split_tf32(act[tsw(s0, 8 * nt + g)], bh[nt][0], bl[nt][0]);
            split_tf32(act[tsw(s1, 8 * nt + g)], bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int mj = 0; mj < 2; mj++) {
            const int j0 = 16 * mj + g;
            uint32_t ah[4], al[4];
            split_tf32(dzt[tsw(s0, j0)], ah[0], al[0]);
            split_tf32(dzt[tsw(s0, j0 + 8)], ah[1], al[1]);
            split_tf32(dzt[tsw(s1, j0)], ah[2], al[2]);
            split_tf32(dzt[tsw(s1, j0 + 8)], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
                mma_tf32(dw[mj][nt], al, bh[nt][0], bh[nt][1]);
                mma_tf32(dw[mj][nt], ah, bl[nt][0], bl[nt][1]);
                mma_tf32(dw[mj][nt], ah, bh[nt][0], bh[nt][1]);
            }
        }
    }
#pragma unroll
    for (int mj = 0; mj < 2; mj++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int j = 16 * mj + g + 8 * (c >> 1), i = 8 * nt + 2 * t + (c & 1);
                atomicAdd(gW + j * IN + wswz(i, j, IN), dw[mj][nt][c]);
            }
}

// mu = sigmoid(b_o + sum_j w_o[j] a[s][j]) of the warp's samples from the last
// hidden layer's C fragments; this lane's sample's mu is returned (rowbuf: 32 floats).
__device__ __forceinline__ float tf32_out_forward(const float* wo, float bo, const float (&a)[2][4][4],
                                                  float* rowbuf, int lane) {
    const int g = lane >> 2, t = lane & 3;
    float zr[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            float s = 0.f;
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                s = fmaf(wo[8 * nt + 2 * t], a[mt][nt][2 * h], s);
                s = fmaf(wo[8 * nt + 2 * t + 1], a[mt][nt][2 * h + 1], s);
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            zr[mt][h] = s;
        }
    __syncwarp();
    if (t == 0) {
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
            for (int h = 0; h < 2; h++) rowbuf[16 * mt + 8 * h + g] = zr[mt][h];
    }
    __syncwarp();
    const float zo = rowbuf[lane] + bo;
    __syncwarp();
    return 1.f / (1.f + expf(-zo));
}

}  // namespace nh
