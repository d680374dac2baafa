// Mixed-precision (BF16 / FP16) MLP of the field kernels on tensor cores: one warp
// runs the MLP of its 32 samples as 32 x 32 tiles with mma.sync.m16n8k16 and
// float32 accumulation (layers chained in registers, see nh_mma.cuh). Included by
// nh_field.cuh after DenseLayout / nhe_forward.
//
// Tensor-memory layout of one thread (row = sample) in the training kernels:
//   columns [0, 32)        hhat (float, D values)
//   columns 32 + 16 l ...  A fragments (16 x 32-bit) of layer l's input, l < H
//   columns 32 + 16 H ...  the last hidden layer's pre-activations (32 floats)
// Per-warp shared scratch: a 16-bit [32][kWS] activation tile, a 16-bit [32][kWS]
// dz tile (aliased by a float [32][D+2] dy tile and the LN-gradient transpose),
// and a 32-float row buffer.
#pragma once
#include "nh_mma.cuh"
#include "nh_tmem.cuh"

namespace nh {

constexpr int kTile16 = 32 * kWS;                 // elements of one 16-bit tile
constexpr int kMmaWarpFloats = kTile16 + 32;      // two 16-bit tiles + a 32-float row
constexpr int kMmaLayerElems = 2 * 32 * kWS;      // W and W^T of one layer (16-bit)

__host__ __device__ constexpr int mma_tmem_cols_per_thread(int H) { return 32 + 16 * H; }

// 16-bit copies of W_l [32][IN] and W_l^T [IN][32] for l < H, from the float copy.
template <typename T>
__device__ __forceinline__ void stage_weights16(const float* sp, const DenseLayout& lay, int D, uint16_t* sw) {
    for (int l = 0; l < lay.H; l++) {
        const int IN = l == 0 ? D : kW;
        const float* W = sp + lay.W(l);
        uint16_t* Wn = sw + l * kMmaLayerElems;
        uint16_t* Wt = Wn + 32 * kWS;
        for (int e = threadIdx.x; e < 32 * IN; e += blockDim.x) {
            const int j = e / IN, i = e - j * IN;
            const uint16_t u = Mma<T>::one(W[e]);
            Wn[j * kWS + i] = u;
            Wt[i * kWS + j] = u;
        }
    }
}

template <int N>
__device__ __forceinline__ void tm_st_u32(uint32_t taddr, const uint32_t* u) {
    float v[N];
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = __uint_as_float(u[i]);
    tmem_st(taddr, v);
}
template <int N>
__device__ __forceinline__ void tm_ld_u32(uint32_t taddr, uint32_t* u) {
    float v[N];
    tmem_ld(taddr, v);
#pragma unroll
    for (int i = 0; i < N; i++) u[i] = __float_as_uint(v[i]);
}
template <int N>
__device__ __forceinline__ void tmem_st_frag16(uint32_t taddr, const uint32_t* u);

// Writes this lane's row of D floats as 16-bit values into the activation tile.
template <typename T, int D>
__device__ __forceinline__ void put_row16(uint16_t* tile, int lane, const float (&y)[D]) {
    uint16_t* row = tile + lane * kWS;
#pragma unroll
    for (int q = 0; q < D / 8; q++) {
        uint4 u;
        u.x = Mma<T>::pack(y[8 * q], y[8 * q + 1]);
        u.y = Mma<T>::pack(y[8 * q + 2], y[8 * q + 3]);
        u.z = Mma<T>::pack(y[8 * q + 4], y[8 * q + 5]);
        u.w = Mma<T>::pack(y[8 * q + 6], y[8 * q + 7]);
        *reinterpret_cast<uint4*>(row + 8 * q) = u;
    }
}

// Forward MLP of the warp's 32 samples. Each lane passes its sample's y and gets
// its mu; C returns the last hidden layer's pre-activations (f32 fragments). With
// STORE, the A fragments of every layer input go to tensor memory at col0 + 16 l.
template <typename T, int D, bool STORE>
__device__ __forceinline__ float mlp_mu_mma(const DenseLayout& lay, const float* sp, const uint16_t* sw,
                                            const float (&y)[D], uint16_t* tile, float* rowbuf, int lane,
                                            uint32_t tcol0, float (&C)[2][4][4]) {
    constexpr int KS0 = D / 16;
    const int g = lane >> 2, t = lane & 3;
    __syncwarp();
    put_row16<T, D>(tile, lane, y);
    __syncwarp();
    {
        uint32_t A0[2][KS0][4];
        load_afrag<KS0>(tile, lane, A0);
        if constexpr (STORE) {
            uint32_t u[16];
#pragma unroll
            for (int i = 0; i < 16; i++) u[i] = 0u;
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int ks = 0; ks < KS0; ks++)
#pragma unroll
                    for (int r = 0; r < 4; r++) u[(mt * 2 + ks) * 4 + r] = A0[mt][ks][r];
            tm_st_u32<16>(tcol0, u);
        }
        mma_layer<T, KS0, 4>(sw, sp + lay.b(0), A0, lane, C);
    }
#pragma unroll 1
    for (int l = 1; l < lay.H; l++) {
        uint32_t A[2][2][4];
        relu_pack<T>(C, A);
        if constexpr (STORE) tm_st_u32<16>(tcol0 + 16 * l, &A[0][0][0]);
        mma_layer<T, 2, 4>(sw + l * kMmaLayerElems, sp + lay.b(l), A, lane, C);
    }
    // output layer 32 -> 1 on the float activations
    const float* wo = sp + lay.W(lay.H);
    float zr[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            float s = 0.f;
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                s = fmaf(wo[8 * nt + 2 * t], fmaxf(C[mt][nt][2 * h], 0.f), s);
                s = fmaf(wo[8 * nt + 2 * t + 1], fmaxf(C[mt][nt][2 * h + 1], 0.f), s);
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            zr[mt][h] = s;
        }
    if (t == 0) {
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
            for (int h = 0; h < 2; h++) rowbuf[16 * mt + 8 * h + g] = zr[mt][h];
    }
    __syncwarp();
    const float zo = rowbuf[lane] + sp[lay.b(lay.H)];
    __syncwarp();
    return 1.f / (1.f + expf(-zo));
}

// Column sums over the warp's 32 rows of a C-fragment tile, accumulated into sdst[col]
// (lanes with g == 0 add; the 8-row groups are reduced with shuffles).
template <int NT>
__device__ __forceinline__ void add_colsum(const float (&Cf)[2][NT][4], float* sdst, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
            float s = Cf[0][nt][e] + Cf[0][nt][2 + e] + Cf[1][nt][e] + Cf[1][nt][2 + e];
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            s += __shfl_xor_sync(0xffffffffu, s, 8);
            s += __shfl_xor_sync(0xffffffffu, s, 16);
            if (g == 0) atomicAdd(sdst + 8 * nt + 2 * t + e, s);
        }
}

// CTA-cooperative weight gradient of the fused training kernel: instead of every
// warp adding its 32-sample partial of dW_l to the CTA accumulator with shared
// atomics, the CTA's warps first write their dz and input tiles, meet at a named
// barrier, and warp u computes output unit u = (16-row half mj of j, 16-column
// group np of i) over all the CTA's samples (K = 32 nw), adding it to the
// accumulator with plain read-modify-writes: every accumulator element has one
// owner. Every warp of the CTA takes part in every barrier, including warps whose
// ray misses the volume (`live` false), which write zero tiles.
struct CoopArgs {
    const float* wbuf0;   // warp 0's scratch; warp v's is wbuf0 + v * wf
    int wf;               // scratch floats per warp
    int nw;               // warps in the CTA (>= 4 units of work; the kernels launch >= 5)
    int warp;
    bool live;            // this warp holds samples of a ray that meets the volume
};

__device__ __forceinline__ void coop_barrier() {
    asm volatile("bar.sync 1, %0;\n" :: "r"((int)blockDim.x) : "memory");
}

template <typename T, int IN>
__device__ __forceinline__ void coop_wgrad(const CoopArgs& co, float* gW, int lane) {
    constexpr int NP = IN / 16;
    const int u = co.warp;
    if (u >= 2 * NP) return;
    const int mj = u / NP, np = u - mj * NP;
    const int g = lane >> 2, t = lane & 3;
    const int q = lane >> 3, r8 = lane & 7;
    float dW[2][4];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int c = 0; c < 4; c++) dW[h][c] = 0.f;
#pragma unroll 1
    for (int v = 0; v < co.nw; v++) {
        const uint16_t* vt = reinterpret_cast<const uint16_t*>(co.wbuf0 + v * co.wf);
        const uint16_t* vdz = vt + kTile16;
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            uint32_t AdT[4], Bq[4];
            ldsm_x4_trans(AdT, vdz + (16 * ks + (q >> 1) * 8 + r8) * kWS + 16 * mj + (q & 1) * 8);
            ldsm_x4_trans(Bq, vt + (16 * ks + (q & 1) * 8 + r8) * kWS + 16 * np + (q >> 1) * 8);
            Mma<T>::mma(dW[0], AdT, Bq[0], Bq[1]);
            Mma<T>::mma(dW[1], AdT, Bq[2], Bq[3]);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int j = 16 * mj + g + 8 * (c >> 1), i = 8 * (2 * np + h) + 2 * t + (c & 1);
            gW[j * IN + wswz(i, j, IN)] += dW[h][c];
        }
}

// Backward of the mixed-precision MLP for the warp's 32 samples. dz enters as the
// gradient at the last hidden layer's pre-activation (f32 fragments); dy leaves as
// this lane's row of dL/dy (the LN output), D floats.
// With COOP (the fused training kernel only) the weight gradient is the
// CTA-cooperative one above and every warp of the CTA must call this function in
// every round; a warp with live == false passes dz = 0 and contributes zero tiles.
template <typename T, int D, bool COOP = false>
__device__ __forceinline__ void mlp_backward_mma(const DenseLayout& lay, const uint16_t* sw, float* sg,
                                                 uint16_t* tile, uint16_t* dztile, int lane, uint32_t tcol0,
                                                 float (&dz)[2][4][4], float (&dy)[D],
                                                 const CoopArgs& co = CoopArgs{nullptr, 0, 0, 0, true}) {
    const bool live = !COOP || co.live;
    const int g = lane >> 2, t = lane & 3;
    const int q = lane >> 3, r8 = lane & 7;
#pragma unroll 1
    for (int l = lay.H - 1; l >= 0; l--) {
        const uint16_t* Wn = sw + l * kMmaLayerElems;
        const uint16_t* Wt = Wn + 32 * kWS;
        const bool first = (l == 0);
        const int IN = first ? D : kW;
        // db_l; dz as hi + lo 16-bit fragments: the data gradient uses both (so the
        // rounding does not compound along the chain), the dz tile holds hi
        if (live) add_colsum<4>(dz, sg + lay.b(l), lane);
        uint32_t Adz[2][2][4], Adl[2][2][4];
        pack_afrag_split<T>(dz, Adz, Adl);
        {
            // layer input fragments from tensor memory into the activation tile
            uint32_t Aact[2][2][4];
            if (live) {
                tm_ld_u32<16>(tcol0 + 16 * l, &Aact[0][0][0]);
            } else {
#pragma unroll
                for (int mt = 0; mt < 2; mt++)
#pragma unroll
                    for (int ks = 0; ks < 2; ks++)
#pragma unroll
                        for (int r = 0; r < 4; r++) Aact[mt][ks][r] = 0u;
            }
            if constexpr (COOP) {
                if (l < lay.H - 1) coop_barrier();   // every warp's reads of layer l + 1's tiles are done
            }
            __syncwarp();
            store_afrag<2>(dztile, lane, Adz);
            if (first && D == 16) {
                uint32_t A1[2][1][4];
#pragma unroll
                for (int mt = 0; mt < 2; mt++)
#pragma unroll
                    for (int rr = 0; rr < 4; rr++) A1[mt][0][rr] = Aact[mt][0][rr];
                store_afrag<1>(tile, lane, A1);
            } else {
                store_afrag<2>(tile, lane, Aact);
            }
            __syncwarp();
        }
        if constexpr (COOP) {
            coop_barrier();   // every warp's tiles of layer l are written
            if (first) coop_wgrad<T, D>(co, sg + lay.W(l), lane);
            else coop_wgrad<T, kW>(co, sg + lay.W(l), lane);
        } else {
        // dW_l[j][i] = sum_s dz[s][j] act[s][i]: A = dz^T (m = j, k = s), B = act (k = s, n = i),
        // one 16-row half of j at a time
        {
            float* gW = sg + lay.W(l);
            const int NP = IN / 16;
#pragma unroll 1
            for (int mj = 0; mj < 2; mj++) {
                uint32_t AdT[2][4];
#pragma unroll
                for (int ks = 0; ks < 2; ks++) {
                    const int s_off = (q >> 1) * 8, j_off = (q & 1) * 8;
                    ldsm_x4_trans(AdT[ks], dztile + (16 * ks + s_off + r8) * kWS + 16 * mj + j_off);
                }
                float dW[4][4];
#pragma unroll
                for (int nt = 0; nt < 4; nt++)
#pragma unroll
                    for (int c = 0; c < 4; c++) dW[nt][c] = 0.f;
#pragma unroll
                for (int ks = 0; ks < 2; ks++)
#pragma unroll
                    for (int np = 0; np < 2; np++) {
                        if (np < NP) {
                            uint32_t Bq[4];
                            const int s_off = (q & 1) * 8, i_off = (q >> 1) * 8;
                            ldsm_x4_trans(Bq, tile + (16 * ks + s_off + r8) * kWS + 16 * np + i_off);
                            Mma<T>::mma(dW[2 * np], AdT[ks], Bq[0], Bq[1]);
                            Mma<T>::mma(dW[2 * np + 1], AdT[ks], Bq[2], Bq[3]);
                        }
                    }
#pragma unroll
                for (int nt = 0; nt < 4; nt++) {
                    if (nt < IN / 8) {
#pragma unroll
                        for (int c = 0; c < 4; c++) {
                            const int j = 16 * mj + g + 8 * (c >> 1), i = 8 * nt + 2 * t + (c & 1);
                            atomicAdd(gW + j * IN + wswz(i, j, IN), dW[nt][c]);
                        }
                    }
                }
            }
        }
        }
        if (!live) {
            if constexpr (COOP) {
                if (first) coop_barrier();   // matches the barrier before the dy rows below
            }
            continue;
        }
        // data gradient din[s][i] = sum_j dz[s][j] W[j][i] (B = W^T rows), from the
        // hi and lo parts of dz so that the rounding does not compound along the chain
        float din[2][4][4];
        if (first && D == 16) {
            float d2[2][2][4];
            mma_layer<T, 2, 2>(Wt, nullptr, Adz, lane, d2);
            mma_accumulate<T, 2, 2>(Wt, Adl, lane, d2);
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 4; nt++)
#pragma unroll
                    for (int c = 0; c < 4; c++) din[mt][nt][c] = nt < 2 ? d2[mt][nt][c] : 0.f;
        } else {
            mma_layer<T, 2, 4>(Wt, nullptr, Adz, lane, din);
            mma_accumulate<T, 2, 4>(Wt, Adl, lane, din);
        }
        if (!first) {
            // ReLU mask of layer l's input, read again from its A fragments
            uint32_t Aact[2][2][4];
            tm_ld_u32<16>(tcol0 + 16 * l, &Aact[0][0][0]);
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 4; nt++) {
                    const uint32_t lo = Aact[mt][nt >> 1][(nt & 1) * 2];
                    const uint32_t hi = Aact[mt][nt >> 1][(nt & 1) * 2 + 1];
                    dz[mt][nt][0] = pos_lo(lo) ? din[mt][nt][0] : 0.f;
                    dz[mt][nt][1] = pos_hi(lo) ? din[mt][nt][1] : 0.f;
                    dz[mt][nt][2] = pos_lo(hi) ? din[mt][nt][2] : 0.f;
                    dz[mt][nt][3] = pos_hi(hi) ? din[mt][nt][3] : 0.f;
                }
        } else {
            // dy rows: fragments -> float tile [32][D + 2] -> this lane's row
            if constexpr (COOP) coop_barrier();   // every warp's reads of layer 0's tiles are done
            __syncwarp();
            float* ft = reinterpret_cast<float*>(tile);
            constexpr int SF = D + 2;
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < D / 8; nt++) {
                    const int c0 = 8 * nt + 2 * t;
                    *reinterpret_cast<float2*>(ft + (16 * mt + g) * SF + c0) = make_float2(din[mt][nt][0], din[mt][nt][1]);
                    *reinterpret_cast<float2*>(ft + (16 * mt + g + 8) * SF + c0) = make_float2(din[mt][nt][2], din[mt][nt][3]);
                }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < D; k += 2) {
                const float2 v = *reinterpret_cast<const float2*>(ft + lane * SF + k);
                dy[k] = v.x;
                dy[k + 1] = v.y;
            }
            __syncwarp();
        }
    }
}

// Output-layer gradients and the entry dz of the mixed-precision backward.
template <int NT>
__device__ __forceinline__ void out_layer_backward_mma(const DenseLayout& lay, const float* sp, float* sg,
                                                       float* rowbuf, int lane, float dzo,
                                                       const float (&C)[2][NT][4], float (&dz)[2][NT][4]) {
    const int g = lane >> 2, t = lane & 3;
    __syncwarp();
    rowbuf[lane] = dzo;
    __syncwarp();
    float dr[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int h = 0; h < 2; h++) dr[mt][h] = rowbuf[16 * mt + 8 * h + g];
    __syncwarp();
    const float* wo = sp + lay.W(lay.H);
    float* gwo = sg + lay.W(lay.H);
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int col = 8 * nt + 2 * t + e;
            float s = 0.f;
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const float a = C[mt][nt][2 * h + e];
                    s = fmaf(dr[mt][h], fmaxf(a, 0.f), s);
                    dz[mt][nt][2 * h + e] = a > 0.f ? wo[col] * dr[mt][h] : 0.f;
                }
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            s += __shfl_xor_sync(0xffffffffu, s, 8);
            s += __shfl_xor_sync(0xffffffffu, s, 16);
            if (g == 0) atomicAdd(gwo + col, s);
        }
    const float bs = warp_sum(dzo);
    if (lane == 0) atomicAdd(sg + lay.b(lay.H), bs);
}

}  // namespace nh
