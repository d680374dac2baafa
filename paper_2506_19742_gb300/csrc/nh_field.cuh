// Field kernels of the NeRF-CBCT training step, templated on the table type (float,
// or bf16 / f16 with the tensor-core MLP of nh_field_mma.cuh); nh_field_*.cu and
// nh_train_*.cu instantiate them, nh_field.cu dispatches.
//
//  k_ray_train     the fused training step: a CTA holds whole rays; each warp runs
//                  sample -> hash gather -> Normalized Hash Encoder -> MLP -> mu
//                  for 32 samples with activations in tensor memory, the CTA forms
//                  the Beer-Lambert sums A = sum_i mu_i delta_i (Eq. 1), the loss
//                  (Eq. 3) and dL/dA, and the same warps run the MLP backward, the
//                  LN backward and the hash scatter-add (red.global.add.v2.f32).
//                  MLP / LN weight gradients are reduced per warp and per CTA in
//                  shared memory and flushed once per CTA.
//  k_ray_forward,  the split path for rays of more than 16 chunks: forward sums,
//  k_ray_loss,     loss, and a backward that recomputes the forward of each sample
//  k_ray_backward  (features are never stored in HBM).
//  k_points,       the same field at explicit points: query (forward) and the MCI
//  k_points_fit    voxel-loss step (Eq. 2, forward + backward in one pass).
#pragma once
#include <cuda_runtime.h>

#include "nh_adam_prep.cuh"
#include "nh_device.cuh"
#include "nh_internal.h"
#include "nh_tmem.cuh"

namespace nh {

constexpr int kW = 32;   // MLP width compiled in

// Offsets inside the dense parameter block (gamma at 0, beta at D, then W_k, b_k).
struct DenseLayout {
    int D, H;
    __device__ __forceinline__ int W(int k) const {   // start of W_k
        // W_0: [kW][D]; W_1..W_{H-1}: [kW][kW]; W_H: [1][kW]
        if (k == 0) return 2 * D;
        return 2 * D + (kW * D + kW) + (k - 1) * (kW * kW + kW);
    }
    __device__ __forceinline__ int b(int k) const {
        if (k == 0) return 2 * D + kW * D;
        if (k < H) return W(k) + kW * kW;
        return W(k) + kW;
    }
};

// Column permutation of the shared-memory weight-gradient accumulators of W_l
// (l < H, 32 rows of IN = 16 or 32 columns): element (j, i) lives at
// j IN + wswz(i, j, IN). It spreads every warp-wide accumulation of tensor-core
// gradient fragments (8 rows x 4 column pairs) over 32 banks and keeps whole-row
// accumulations conflict-free.
__host__ __device__ __forceinline__ int wswz(int i, int j, int IN) {
    return IN == 32 ? (i ^ ((j & 1) | ((j & 6) << 2))) : (i ^ (((j >> 1) & 1) | (((j >> 2) & 1) << 3)));
}

__device__ __forceinline__ void load_dense(const FieldArgs& fa, float* sp, float* smask) {
    const float* src = fa.params + fa.n_table;
    for (int k = threadIdx.x; k < fa.n_dense; k += blockDim.x) sp[k] = src[k];
    for (int k = threadIdx.x; k < fa.D; k += blockDim.x) smask[k] = fa.state->mask[k];
}

template <typename TT>
__device__ __forceinline__ const void* table_base(const FieldArgs& fa) {
    return sizeof(TT) == 4 ? (const void*)fa.params : fa.tables_lp;
}

// Normalized Hash Encoder forward: hhat (or h when norm = none), per-group rstd, y.
// G = number of normalization groups held: 1 (one group or none) or D / 2 (per level);
// kernels instantiated with G = 1 are only launched for the one-group modes.
template <int D, int G = D / 2>
__device__ __forceinline__ void nhe_forward(const FieldArgs& fa, const float* sp, const float* smask,
                                            const float (&h)[D], float (&hhat)[D],
                                            float (&rstd)[G], float (&y)[D]) {
    static_assert(G == 1 || G == D / 2, "normalization groups");
    if (fa.norm == NH_NORM_LN) {
        float r1[1];
        ln_stats<D, D>(h, fa.eps, hhat, r1);
#pragma unroll
        for (int g = 0; g < G; g++) rstd[g] = r1[0];
    } else if (G == D / 2 && fa.norm == NH_NORM_LN_PER_LEVEL) {
        if constexpr (G == D / 2) ln_stats<D, 2>(h, fa.eps, hhat, rstd);
    } else {
#pragma unroll
        for (int k = 0; k < D; k++) hhat[k] = h[k];
#pragma unroll
        for (int g = 0; g < G; g++) rstd[g] = 1.f;
    }
    const bool affine = fa.norm != NH_NORM_NONE;
#pragma unroll
    for (int k = 0; k < D; k++) {
        const float gk = affine ? sp[k] : 1.f;
        const float bk = affine ? sp[D + k] : 0.f;
        y[k] = fmaf(gk, hhat[k], bk) * smask[k];
    }
}

// mu = sigmoid(MLP(y)) without storing activations.
template <int D>
__device__ __forceinline__ float mlp_mu(const DenseLayout& lay, const float* sp, const float (&y)[D]) {
    float a[kW], z[kW];
    linear_fwd<D, kW>(sp + lay.W(0), sp + lay.b(0), y, z);
#pragma unroll
    for (int j = 0; j < kW; j++) a[j] = fmaxf(z[j], 0.f);
#pragma unroll 1
    for (int k = 1; k < lay.H; k++) {
        linear_fwd<kW, kW>(sp + lay.W(k), sp + lay.b(k), a, z);
#pragma unroll
        for (int j = 0; j < kW; j++) a[j] = fmaxf(z[j], 0.f);
    }
    const float* wo = sp + lay.W(lay.H);
    float zo = sp[lay.b(lay.H)];
#pragma unroll
    for (int j = 0; j < kW; j++) zo = fmaf(wo[j], a[j], zo);
    return 1.f / (1.f + expf(-zo));
}

template <int D, typename TT>
__device__ __forceinline__ float field_mu(const FieldArgs& fa, const float* sp, const float* smask,
                                          const float x[3]) {
    float h[D], hhat[D], rstd[D / 2], y[D];
    encode_point<D / 2, TT>(fa, table_base<TT>(fa), x, h);
    nhe_forward<D>(fa, sp, smask, h, hhat, rstd, y);
    const DenseLayout lay{D, fa.H};
    return mlp_mu<D>(lay, sp, y);
}

}  // namespace nh

#include "nh_field_mma.cuh"
#include "nh_field_tf32.cuh"

namespace nh {

// Low-precision tables run the MLP on 16-bit tensor cores (warp-collective). Float
// tables run the per-thread FFMA MLP in the forward-only kernels and the TF32 x 3
// tensor-core MLP (nh_field_tf32.cuh) in the training kernels.
template <typename TT>
constexpr bool kMmaPath = sizeof(TT) == 2;

// Shared-memory carve-up of the forward / query kernels: float dense params, mask,
// 16-bit weights (tensor-core path) and per-warp tile + row buffer.
template <typename TT>
__host__ __device__ inline int fwd_warp_floats() { return kMmaPath<TT> ? kTile16 / 2 + 32 : 0; }

template <typename TT>
static size_t fwd_smem_bytes(const FieldArgs& fa, int warps) {
    size_t b = (size_t)(((fa.n_dense + 3) & ~3) + kMaxD) * sizeof(float);
    if (kMmaPath<TT>) b += (size_t)fa.H * kMmaLayerElems * 2 + (size_t)warps * fwd_warp_floats<TT>() * 4;
    return b;
}

struct FwdCta {
    float *sp, *smask, *wbuf;
    const uint16_t* sw;
};

template <typename TT>
__device__ __forceinline__ FwdCta fwd_begin(const FieldArgs& fa, float* smem) {
    FwdCta c;
    const int ndp = (fa.n_dense + 3) & ~3;
    c.sp = smem;
    c.smask = c.sp + ndp;
    uint16_t* sw = reinterpret_cast<uint16_t*>(c.smask + kMaxD);
    c.sw = sw;
    c.wbuf = reinterpret_cast<float*>(sw + fa.H * kMmaLayerElems) + (threadIdx.x >> 5) * fwd_warp_floats<TT>();
    load_dense(fa, c.sp, c.smask);
    if constexpr (kMmaPath<TT>) {
        __syncthreads();
        stage_weights16<TT>(c.sp, DenseLayout{fa.D, fa.H}, fa.D, sw);
    }
    __syncthreads();
    return c;
}

// mu of this lane's point. On the tensor-core path all 32 lanes must call together.
template <int D, typename TT>
__device__ __forceinline__ float point_mu(const FieldArgs& fa, const FwdCta& c, const float x[3], int lane) {
    if constexpr (kMmaPath<TT>) {
        float h[D], hhat[D], rstd[D / 2], y[D], C[2][4][4];
        encode_point<D / 2, TT>(fa, table_base<TT>(fa), x, h);
        nhe_forward<D>(fa, c.sp, c.smask, h, hhat, rstd, y);
        uint16_t* tile = reinterpret_cast<uint16_t*>(c.wbuf);
        float* rowbuf = c.wbuf + kTile16 / 2;
        return mlp_mu_mma<TT, D, false>(DenseLayout{D, fa.H}, c.sp, c.sw, y, tile, rowbuf, lane, 0u, C);
    } else {
        return field_mu<D, TT>(fa, c.sp, c.smask, x);
    }
}

// ============================================================================ forward
template <int D, typename TT>
__global__ void __launch_bounds__(256) k_ray_forward(FieldArgs fa, ViewArgs va,
                                                     const int32_t* __restrict__ pix, int R, int N,
                                                     int C, float* __restrict__ ray_part) {
    extern __shared__ __align__(16) float smem[];
    const FwdCta cta = fwd_begin<TT>(fa, smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long task = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (task >= (long long)R * C) return;
    const int r = (int)(task / C), c = (int)(task - (long long)r * C);
    const RayGeo g = ray_setup(va, pix[r], N);
    if (!g.hit) {
        if (lane == 0) ray_part[task] = 0.f;
        return;
    }
    const int i = c * 32 + lane;
    float mu = 0.f;
    if (kMmaPath<TT> || i < N) {
        float x[3];
        {
            const int ic = i < N ? i : N - 1;
            sample_position(g, ic, stratum_offset(va.jitter, pix[r], N, ic), x);
        }
        mu = point_mu<D, TT>(fa, cta, x, lane);
        if (i >= N) mu = 0.f;
    }
    const float s = warp_sum(mu);
    if (lane == 0) ray_part[task] = s * g.delta;
}

// ============================================================================ loss
// One CTA: A_r = sum over chunks in order, loss = mean over rays, dL/dA_r.
static __global__ void __launch_bounds__(1024) k_ray_loss(const float* __restrict__ ray_part, int R, int C,
                                                   const float* __restrict__ a_meas, int loss_kind,
                                                   float* __restrict__ a_pred, float* __restrict__ dLdA,
                                                   float* __restrict__ loss_out, DeviceState* state) {
    __shared__ float red[32];
    float acc = 0.f;
    const float invR = 1.f / (float)R;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        float A = 0.f;
        for (int c = 0; c < C; c++) A += ray_part[(size_t)r * C + c];
        if (a_pred) a_pred[r] = A;
        if (a_meas) {
            const float res = A - a_meas[r];
            float l, gr;
            if (loss_kind == NH_LOSS_MSE) {
                l = res * res;
                gr = 2.f * res * invR;
            } else {
                l = fabsf(res);
                gr = (res > 0.f ? 1.f : (res < 0.f ? -1.f : 0.f)) * invR;
            }
            acc += l;
            if (dLdA) dLdA[r] = gr;
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        v = warp_sum(v);
        if (threadIdx.x == 0 && a_meas) {
            const float loss = v * invR;
            if (loss_out) *loss_out = loss;
            if (!isfinite(loss)) atomicOr(&state->flags, NH_FLAG_NONFINITE);
        }
    }
}

// ============================================================================ backward
// Per-warp shared scratch (floats) of the FP32 path: an input tile [32][kW] (the
// gather's level rows, then a layer's input rows or C fragments) and a dz tile
// [32][kW]. The gather addresses the input tile with swz (XOR-swizzled float4
// groups, element j of row s at swz(s, j)); the tensor-core MLP with tsw. Each
// sample's activations live in TMEM: slot 0 holds hhat (or h without
// normalization), slot k (1 <= k < H) holds a_k, the ReLU output of layer k-1; a_H
// waits in the input tile.
constexpr int kStage = 32 * kW;
__host__ __device__ constexpr int warp_scratch_floats() { return kStage + 32 * kW; }
constexpr int kBwdWarps = 8;
constexpr int kMidTrainWarps = 12;   // rays of 9..12 chunks: 168 registers a thread
constexpr int kMaxTrainWarps = kMaxFusedChunks;

__device__ __forceinline__ int swz(int s, int j) {   // column j of dz row s
    return s * kW + ((((j >> 2) ^ (s & 7)) << 2) | (j & 3));
}

// Normalized Hash Encoder backward and the hash scatter of one sample per lane.
// dh enters as dL/dy and leaves as dL/dh; gamma / beta gradients are reduced across
// the warp through `col` (32 x 32 floats of per-warp scratch): lane s stores element
// k of its row at column k ^ s, conflict-free for both the writes and the column sums.
template <int D, int G>
__device__ __forceinline__ void nhe_backward_scatter(const FieldArgs& fa, const float* sp, const float* smask,
                                                     float* sg, float* col, const float (&hhat)[D],
                                                     const float (&rstd)[G], float (&dh)[D], const float x[3],
                                                     bool active, int lane) {
#pragma unroll
    for (int k = 0; k < D; k++) dh[k] *= smask[k];     // dL/d(gamma hhat + beta)
    if (fa.norm != NH_NORM_NONE) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < D; k++) col[lane * kW + (k ^ lane)] = dh[k] * hhat[k];
        __syncwarp();
        if (lane < D) {
            float s = 0.f;
#pragma unroll 8
            for (int t = 0; t < 32; t++) s += col[t * kW + (lane ^ t)];
            atomicAdd(sg + lane, s);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < D; k++) col[lane * kW + (k ^ lane)] = dh[k];
        __syncwarp();
        if (lane < D) {
            float s = 0.f;
#pragma unroll 8
            for (int t = 0; t < 32; t++) s += col[t * kW + (lane ^ t)];
            atomicAdd(sg + D + lane, s);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < D; k++) dh[k] *= sp[k];   // dL/dhhat
        if (fa.norm == NH_NORM_LN) {
            float r1[1] = {rstd[0]};
            ln_backward<D, D>(hhat, r1, dh);
        } else {
            if constexpr (G == D / 2) ln_backward<D, 2>(hhat, rstd, dh);
        }
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < D; k++) bad |= !isfinite(dh[k]);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&fa.state->flags, NH_FLAG_NONFINITE);
    // the scatter is warp-collective: lanes without a sample contribute zeros; the
    // row (32 floats of the 32 x 32 scratch) holds element k at column k ^ lane
    float* row = col + lane * kW;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < D; k++) row[k ^ lane] = active ? dh[k] : 0.f;
    scatter_point<D / 2>(fa, x, row, lane);
}

// Gather of one sample per lane for the training kernels, with the level loop kept
// rolled (the 8 corner loads of a level in flight together): each level's two
// features go to the lane's row of a 32 x 32 float tile of the warp's scratch
// (swizzled float4 groups, as the stage tile) and the whole row is read back at the
// end. Rolled, the gather is a fraction of the fully unrolled code with fewer
// registers live, which made the fused training kernels 10-15 % faster.
template <int L, typename TT>
__device__ __forceinline__ void encode_point_rolled(const FieldArgs& fa, const void* tables, const float x[3],
                                                    float* stage, int lane, float (&h)[2 * L]) {
    const size_t T = (size_t)fa.Tmask + 1;
#pragma unroll 1
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
        *reinterpret_cast<float2*>(stage + swz(lane, 2 * l)) = make_float2(a0, a1);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < L / 2; q++) {
        const float4 v = *reinterpret_cast<const float4*>(stage + swz(lane, 4 * q));
        h[4 * q] = v.x;
        h[4 * q + 1] = v.y;
        h[4 * q + 2] = v.z;
        h[4 * q + 3] = v.w;
    }
}

// State of one training sample carried from the forward half to the backward half
// (FP32 path). Everything else waits in tensor memory (slot 0: hhat, the lane's
// row; slot k, 1 <= k < H: a_k as the lane's 32 C-fragment values) or, for a_H, in
// the warp's input tile (C-fragment layout).
template <int D, int G>
struct F32Carry {
    float rstd[G];     // normalization groups: 1 (one LayerNorm / none) or L (per level)
    float mu;
};

template <int NT>
__device__ __forceinline__ void relu_frag(const float (&z)[2][NT][4], float (&a)[2][NT][4]) {
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int c = 0; c < 4; c++) a[mt][nt][c] = fmaxf(z[mt][nt][c], 0.f);
}
__device__ __forceinline__ void frag_tmem_st(uint32_t taddr, const float (&a)[2][4][4]) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = a[i >> 4][(i >> 2) & 3][i & 3];
    tmem_st(taddr, v);
}
__device__ __forceinline__ void frag_tmem_ld(uint32_t taddr, float (&a)[2][4][4]) {
    float v[32];
    tmem_ld(taddr, v);
#pragma unroll
    for (int i = 0; i < 32; i++) a[i >> 4][(i >> 2) & 3][i & 3] = v[i];
}

// Layer-0 input y = (gamma hhat + beta) m of this lane's sample (hhat = h without
// normalization).
template <int D>
__device__ __forceinline__ void affine_row(const FieldArgs& fa, const float* sp, const float* smask,
                                           const float (&hhat)[D], float (&y)[D]) {
    const bool affine = fa.norm != NH_NORM_NONE;
#pragma unroll
    for (int k = 0; k < D; k++) y[k] = (affine ? fmaf(sp[k], hhat[k], sp[D + k]) : hhat[k]) * smask[k];
}

// Forward of one sample per lane, the MLP on tensor cores (nh_field_tf32.cuh). All 32
// lanes must call it together. Warp scratch: the input tile (wbuf) and the dz tile
// (wbuf + 32 x 32), the latter also the output layer's row buffer.
template <int D, int G, typename TT, bool PS = false>
__device__ __forceinline__ void f32_forward(const FieldArgs& fa, const float* sp, const float* wlo, const float* smask,
                                            float* wbuf, uint32_t tslot0, const float x[3], int lane,
                                            F32Carry<D, G>& s) {
    constexpr int L = D / 2;
    const DenseLayout lay{D, fa.H};
    const int H = fa.H;
    float* act = wbuf;
    float* dzt = wbuf + kStage;
    float z[2][4][4];
    {
        float h[D], hhat[D], y[D];
        __syncwarp();   // the previous sample's readers of the tiles are done
        encode_point_rolled<L, TT>(fa, table_base<TT>(fa), x, act, lane, h);
        nhe_forward<D, G>(fa, sp, smask, h, hhat, s.rstd, y);
        tmem_st(tslot0, hhat);
        __syncwarp();   // the gather's reads of the tile are done
        row_to_tile<D>(act, lane, y);
        __syncwarp();
        tf32_layer_tile<D / 8, PS>(act, sp + lay.W(0), wlo, sp + lay.b(0), lane, z);
    }
    float a[2][4][4];
#pragma unroll 1
    for (int k = 1; k < H; k++) {
        relu_frag<4>(z, a);
        frag_tmem_st(tslot0 + 32 * k, a);
        tf32_layer_frag<PS>(a, sp + lay.W(k), wlo + k * kW * kW, sp + lay.b(k), lane, z);
    }
    relu_frag<4>(z, a);
    s.mu = tf32_out_forward(sp + lay.W(H), sp[lay.b(H)], a, dzt, lane);
    __syncwarp();   // every lane's layer-0 reads of the input tile are done
    frag_to_tile<4>(act, lane, a);   // a_H waits here for the backward
}

// Backward of one sample per lane given dL/dmu (already multiplied by the loss
// scale; 0 for lanes without a sample). All 32 lanes must call it together.
template <int D, int G, typename TT, bool PS = false>
__device__ __forceinline__ void f32_backward(const FieldArgs& fa, const float* sp, const float* wlo,
                                             const float* smask, float* sg, float* wbuf, uint32_t tslot0,
                                             const float x[3], bool active, int lane, const F32Carry<D, G>& s,
                                             float dmu) {
    const DenseLayout lay{D, fa.H};
    const int H = fa.H;
    float* act = wbuf;
    float* dzt = wbuf + kStage;
    const float dzo = dmu * s.mu * (1.f - s.mu);
    float dz[2][4][4];
    {
        float a[2][4][4];
        __syncwarp();
        tile_to_frag<4>(act, lane, a);   // a_H
        out_layer_backward_mma<4>(lay, sp, sg, dzt, lane, dzo, a, dz);
    }
    // hidden layers k = H-1 .. 1: input a_k from TMEM
#pragma unroll 1
    for (int k = H - 1; k >= 1; k--) {
        add_colsum<4>(dz, sg + lay.b(k), lane);
        {
            float a[2][4][4];
            frag_tmem_ld(tslot0 + 32 * k, a);
            __syncwarp();   // the previous readers of both tiles are done
            frag_to_tile<4>(dzt, lane, dz);
            frag_to_tile<4>(act, lane, a);
            __syncwarp();
        }
        tf32_wgrad<kW>(dzt, act, sg + lay.W(k), lane);
        float din[2][4][4];
        tf32_dgrad<4, PS>(dz, sp + lay.W(k), wlo + k * kW * kW, lane, din);
        float a[2][4][4];
        frag_tmem_ld(tslot0 + 32 * k, a);
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
            for (int nt = 0; nt < 4; nt++)
#pragma unroll
                for (int c = 0; c < 4; c++) dz[mt][nt][c] = a[mt][nt][c] > 0.f ? din[mt][nt][c] : 0.f;
    }
    // layer 0: input y = (gamma hhat + beta) m
    add_colsum<4>(dz, sg + lay.b(0), lane);
    float hhat[D];
    tmem_ld(tslot0, hhat);
    {
        float y[D];
        affine_row<D>(fa, sp, smask, hhat, y);
        __syncwarp();
        frag_to_tile<4>(dzt, lane, dz);
        row_to_tile<D>(act, lane, y);
        __syncwarp();
    }
    tf32_wgrad<D>(dzt, act, sg + lay.W(0), lane);
    float dh[D];
    {
        float din[2][D / 8][4];
        tf32_dgrad<D / 8, PS>(dz, sp + lay.W(0), wlo, lane, din);
        __syncwarp();   // the weight gradient's reads of the input tile are done
        frag_to_tile<D / 8>(act, lane, din);
        __syncwarp();
        tile_to_row<D>(act, lane, dh);   // dh <- dL/dy
    }
    nhe_backward_scatter<D, G>(fa, sp, smask, sg, dzt, hhat, s.rstd, dh, x, active, lane);
}

// Forward then backward of one sample per lane; dmu_of(mu) gives dL/dmu.
template <int D, int G, typename TT, class DmuFn>
__device__ __forceinline__ float sample_fwd_bwd(const FieldArgs& fa, const float* sp, const float* smask, float* sg,
                                                float* wbuf, uint32_t tslot0, const float x[3], bool active,
                                                int lane, DmuFn dmu_of) {
    F32Carry<D, G> s;
    f32_forward<D, G, TT>(fa, sp, nullptr, smask, wbuf, tslot0, x, lane, s);
    f32_backward<D, G, TT>(fa, sp, nullptr, smask, sg, wbuf, tslot0, x, active, lane, s,
                           active ? dmu_of(s.mu) : 0.f);
    return s.mu;
}

// Tensor-core path: the MLP of the warp's 32 samples runs on tensor cores
// (nh_field_mma.cuh); encoding, normalization, LN backward and the scatter are the
// per-sample float32 code. All 32 lanes must call these together. The last hidden
// layer's pre-activation fragments are parked in tensor memory after the layer
// inputs (column 32 + 16 H), so that only mu and the normalization statistics stay
// in registers between the forward and the backward.
template <int D, int G>
struct MmaCarry {
    float rstd[G];
    float mu;
};

__device__ __forceinline__ void frag_st(uint32_t taddr, const float (&C)[2][4][4]) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = C[i >> 4][(i >> 2) & 3][i & 3];
    tmem_st(taddr, v);
}
__device__ __forceinline__ void frag_ld(uint32_t taddr, float (&C)[2][4][4]) {
    float v[32];
    tmem_ld(taddr, v);
#pragma unroll
    for (int i = 0; i < 32; i++) C[i >> 4][(i >> 2) & 3][i & 3] = v[i];
}

template <int D, int G, typename TT>
__device__ __forceinline__ void mma_forward(const FieldArgs& fa, const float* sp, const uint16_t* sw,
                                            const float* smask, float* wbuf, uint32_t tslot0, const float x[3],
                                            int lane, MmaCarry<D, G>& s) {
    constexpr int L = D / 2;
    const DenseLayout lay{D, fa.H};
    uint16_t* tile = reinterpret_cast<uint16_t*>(wbuf);
    float* rowbuf = reinterpret_cast<float*>(tile + 2 * kTile16);
    float h[D], hhat[D], y[D];
    __syncwarp();   // the previous sample's readers of the warp's tiles are done
    encode_point_rolled<L, TT>(fa, table_base<TT>(fa), x, wbuf, lane, h);
    nhe_forward<D, G>(fa, sp, smask, h, hhat, s.rstd, y);
    tmem_st(tslot0, hhat);
    float C[2][4][4];
    s.mu = mlp_mu_mma<TT, D, true>(lay, sp, sw, y, tile, rowbuf, lane, tslot0 + 32, C);
    frag_st(tslot0 + 32 + 16 * fa.H, C);
}

// With COOP (the fused training kernel) every warp of the CTA calls this in every
// round and the MLP weight gradient is the CTA-cooperative one (nh_field_mma.cuh); a
// warp whose ray misses the volume (co.live false) only takes part in it.
template <int D, int G, typename TT, bool COOP = false>
__device__ __forceinline__ void mma_backward(const FieldArgs& fa, const float* sp, const uint16_t* sw,
                                             const float* smask, float* sg, float* wbuf, uint32_t tslot0,
                                             const float x[3], bool active, int lane, const MmaCarry<D, G>& s,
                                             float dmu, const CoopArgs& co = CoopArgs{nullptr, 0, 0, 0, true}) {
    const DenseLayout lay{D, fa.H};
    uint16_t* tile = reinterpret_cast<uint16_t*>(wbuf);
    uint16_t* dztile = tile + kTile16;
    float* rowbuf = reinterpret_cast<float*>(dztile + kTile16);
    const bool live = !COOP || co.live;
    const float dzo = dmu * s.mu * (1.f - s.mu);
    float dz[2][4][4];
    if (live) {
        float C[2][4][4];
        frag_ld(tslot0 + 32 + 16 * fa.H, C);
        out_layer_backward_mma<4>(lay, sp, sg, rowbuf, lane, dzo, C, dz);
    } else {
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
            for (int nt = 0; nt < 4; nt++)
#pragma unroll
                for (int c = 0; c < 4; c++) dz[mt][nt][c] = 0.f;
    }
    float dh[D];
    mlp_backward_mma<TT, D, COOP>(lay, sw, sg, tile, dztile, lane, tslot0 + 32, dz, dh, co);
    if (!live) return;
    float hhat[D];
    tmem_ld(tslot0, hhat);
    nhe_backward_scatter<D, G>(fa, sp, smask, sg, wbuf, hhat, s.rstd, dh, x, active, lane);
}

template <int D, int G, typename TT, class DmuFn>
__device__ __forceinline__ float sample_fwd_bwd_mma(const FieldArgs& fa, const float* sp, const uint16_t* sw,
                                                    const float* smask, float* sg, float* wbuf, uint32_t tslot0,
                                                    const float x[3], bool active, int lane, DmuFn dmu_of) {
    MmaCarry<D, G> s;
    mma_forward<D, G, TT>(fa, sp, sw, smask, wbuf, tslot0, x, lane, s);
    mma_backward<D, G, TT>(fa, sp, sw, smask, sg, wbuf, tslot0, x, active, lane, s, active ? dmu_of(s.mu) : 0.f);
    return s.mu;
}

// TMEM columns of one thread: FP32 path 32 H (hhat, a_1 .. a_{H-1}); 16-bit path
// 64 + 16 H (hhat, the A fragments of every layer input, the last hidden layer's
// pre-activations).
__host__ __device__ inline int bwd_cols_per_thread(int precision, int H) {
    return precision == NH_PREC_F32 ? 32 * H : mma_tmem_cols_per_thread(H) + 32;
}
// TMEM columns per CTA: two lane-quarter groups of warps, rounded to a power of two.
static uint32_t bwd_tmem_cols(const FieldArgs& fa, int nwarps = kBwdWarps) {
    uint32_t need = (uint32_t)((nwarps + 3) / 4) * (uint32_t)bwd_cols_per_thread(fa.precision, fa.H), c = 32;
    while (c < need) c <<= 1;
    return c;
}
// Shared memory of the backward kernels (bytes): float dense params (on the FP32
// path with W_l^T tiles in place of W_l, l < H), mask, gradient accumulators, 16-bit
// weights (16-bit path) and 8 warps of scratch. Registers
// cap residency at two CTAs per SM; when one CTA takes all 512 TMEM columns the
// request is padded so that only one CTA fits, and no tcgen05.alloc waits on a
// resident CTA.
// Per-warp scratch floats of the training kernels: the FP32 path's input + dz tiles,
// or the 16-bit path's two 16-bit tiles and row buffer.
__host__ __device__ inline int bwd_warp_floats(int precision) {
    return precision == NH_PREC_F32 ? warp_scratch_floats() : kMmaWarpFloats;
}

// FP32 fused training CTAs that split the MLP weights once at staging add the lo
// tiles (H kW kW floats) to their shared memory: CTAs of at most six warps always
// (two still fit per SM), CTAs of 9..12 warps (one per SM in any case) when the
// total stays within the opt-in limit. Eight-warp CTAs would lose their second CTA
// per SM to the 16 KB, and 16-warp CTAs, compiled for 128 registers, spill more
// with the split operands, so both split on load.
static size_t bwd_smem_bytes(const FieldArgs& fa, int nwarps = kBwdWarps, bool presplit = false) {
    const int ndp = (fa.n_dense + 3) & ~3;
    size_t b = (size_t)(2 * ndp + kMaxD + nwarps * bwd_warp_floats(fa.precision)) * sizeof(float);
    if (fa.precision != NH_PREC_F32) b += (size_t)fa.H * kMmaLayerElems * 2;
    else if (presplit) b += (size_t)fa.H * kW * kW * sizeof(float);
    if (512u / bwd_tmem_cols(fa, nwarps) < 2u && b < 120 * 1024) b = 120 * 1024;
    return b;
}

// CTA prologue / epilogue shared by the training kernels.
struct BwdCta {
    float *sp, *smask, *sg, *wbuf;
    const uint16_t* sw;   // 16-bit path: W and W^T per layer
    float* wlo;           // FP32 path with split weights: the lo tiles, else null
    uint32_t tbase, tslot0;
};

// PS: stage the FP32 weights split (the CTA was sized for the lo tiles).
template <typename TT, bool PS = false>
__device__ __forceinline__ BwdCta bwd_begin(const FieldArgs& fa, float* smem, uint32_t* s_tmem, uint32_t tcols) {
    BwdCta c;
    const int ndp = (fa.n_dense + 3) & ~3;
    const int warp = threadIdx.x >> 5;
    c.sp = smem;
    c.smask = c.sp + ndp;
    c.sg = c.smask + kMaxD;
    const int wf = bwd_warp_floats(fa.precision);
    c.wbuf = c.sg + ndp + warp * wf;
    uint16_t* sw = reinterpret_cast<uint16_t*>(c.sg + ndp + (int)(blockDim.x >> 5) * wf);
    c.sw = sw;
    c.wlo = (!kMmaPath<TT> && PS) ? reinterpret_cast<float*>(sw) : nullptr;
    if (warp == 0) tmem_alloc(s_tmem, tcols);
    load_dense(fa, c.sp, c.smask);
    for (int k = threadIdx.x; k < ndp; k += blockDim.x) c.sg[k] = 0.f;
    __syncthreads();
    if constexpr (kMmaPath<TT>)
        stage_weights16<TT>(c.sp, DenseLayout{fa.D, fa.H}, fa.D, sw);
    else
        stage_wt_tf32(fa.params + fa.n_table, DenseLayout{fa.D, fa.H}, fa.D, c.sp, c.wlo);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    c.tbase = *s_tmem;
    c.tslot0 = tmem_lane_addr(c.tbase, warp, (warp >> 2) * bwd_cols_per_thread(fa.precision, fa.H));
    return c;
}

// One training sample per lane through the FP32 (TF32 x 3) or the 16-bit tensor-core MLP.
template <int D, int G, typename TT, class DmuFn>
__device__ __forceinline__ float train_sample(const FieldArgs& fa, const BwdCta& c, const float x[3], bool active,
                                              int lane, DmuFn dmu_of) {
    if constexpr (kMmaPath<TT>)
        return sample_fwd_bwd_mma<D, G, TT>(fa, c.sp, c.sw, c.smask, c.sg, c.wbuf, c.tslot0, x, active, lane, dmu_of);
    else
        return sample_fwd_bwd<D, G, TT>(fa, c.sp, c.smask, c.sg, c.wbuf, c.tslot0, x, active, lane, dmu_of);
}

__device__ __forceinline__ void bwd_end(const FieldArgs& fa, const BwdCta& c, uint32_t tcols) {
    tmem_fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tmem_fence_after_sync();
        tmem_dealloc(c.tbase, tcols);
    }
    // flush: logical dense index k <- accumulator slot (W_l blocks are column-permuted)
    const DenseLayout lay{fa.D, fa.H};
    float* gd = fa.grads + fa.n_table;
    for (int k = threadIdx.x; k < fa.n_dense; k += blockDim.x) {
        int p = k;
        for (int l = 0; l < fa.H; l++) {
            const int IN = l == 0 ? fa.D : kW, o = k - lay.W(l);
            if (o >= 0 && o < kW * IN) {
                const int j = o / IN, i = o - j * IN;
                p = lay.W(l) + j * IN + wswz(i, j, IN);
            }
        }
        const float v = c.sg[p];
        if (v != 0.f) atomicAdd(gd + k, v);
    }
}

template <int D, int G, typename TT>
__global__ void __launch_bounds__(kBwdWarps * 32, 2)
k_ray_backward(FieldArgs fa, ViewArgs va, const int32_t* __restrict__ pix, int R, int N, int C,
               const float* __restrict__ dLdA, uint32_t tcols) {
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t s_tmem;
    const BwdCta cta = bwd_begin<TT>(fa, smem, &s_tmem, tcols);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float scale = fa.state->loss_scale;
    const long long ntask = (long long)R * C;
    for (long long task = (long long)blockIdx.x * kBwdWarps + warp; task < ntask;
         task += (long long)gridDim.x * kBwdWarps) {
        const int r = (int)(task / C), c = (int)(task - (long long)r * C);
        const RayGeo g = ray_setup(va, pix[r], N);
        if (!g.hit) continue;
        const int i = c * 32 + lane;
        const bool active = i < N;
        float x[3];
        const int ic = active ? i : N - 1;
        sample_position(g, ic, stratum_offset(va.jitter, pix[r], N, ic), x);
        const float gr = dLdA[r] * g.delta * scale;
        train_sample<D, G, TT>(fa, cta, x, active, lane, [gr](float) { return gr; });
    }
    bwd_end(fa, cta, tcols);
}

// ============================================================================ fused step
// One training step for batches whose rays fit a CTA (at most kMaxFusedChunks chunks
// of 32 samples per ray): a CTA takes rpr whole rays at a time, warp w computing
// chunk w % C of ray w / C. Each warp runs the forward of its samples with activations in
// tensor memory; the CTA sums each ray's chunks in order into A_r (Eq. 1), forms the
// loss term and dL/dA_r (MSE or L1, Eq. 3) in shared memory, and every warp carries
// on with the backward of the same samples. Ray-tile losses are accumulated in ray
// order per CTA; k_train_loss adds the CTA partials in a fixed order.
template <int D, int G, typename TT>
struct TrainCarry {
    using type = F32Carry<D, G>;
};

template <int D, int G>
struct TrainCarry<D, G, __nv_bfloat16> {
    using type = MmaCarry<D, G>;
};

template <int D, int G>
struct TrainCarry<D, G, __half> {
    using type = MmaCarry<D, G>;
};

// NW: most warps a CTA launches with. CTAs of at most six warps (rays of three,
// five or six chunks) are compiled with the register budget of two six-warp CTAs
// per SM instead of two eight-warp ones; CTAs of 9..16 warps (one long ray each)
// run one per SM, with the register budget of 12 warps (168 a thread) up to 12
// warps and of 16 warps (128) above. On the 16-bit path the six-warp CTAs (5 or 6 warps launched)
// take the CTA-cooperative MLP weight gradient; the larger CTAs, compiled for 128
// registers, keep the per-warp shared atomics, which need fewer registers.
// PS (FP32 path only): the CTA splits the MLP weights once at staging; its shared
// memory holds the lo tiles (bwd_smem_bytes with presplit).
template <int D, int G, typename TT, int NW, bool PS>
__global__ void __launch_bounds__(NW * 32, NW > 8 ? 1 : 2)
k_ray_train(FieldArgs fa, ViewArgs va, const int32_t* __restrict__ pix, const float* __restrict__ a_meas, int R,
            int N, int C, int rpr, int loss_kind, float* __restrict__ loss_part, uint32_t tcols) {
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t s_tmem;
    __shared__ float s_part[kMaxTrainWarps];
    __shared__ float s_g[kMaxTrainWarps];
    __shared__ float s_lr[kMaxTrainWarps];
    __shared__ float s_loss;
    const BwdCta cta = bwd_begin<TT, PS>(fa, smem, &s_tmem, tcols);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rl = warp / C, c = warp - rl * C;
    const float scale = fa.state->loss_scale;
    const float invR = 1.f / (float)R;
    if (threadIdx.x == 0) s_loss = 0.f;
    const int ngroups = (R + rpr - 1) / rpr;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int r = grp * rpr + rl;
        RayGeo g{};
        g.hit = false;
        if (r < R) g = ray_setup(va, pix[r], N);
        const bool work = g.hit;                       // uniform over the warp
        const int i = c * 32 + lane;
        const bool active = work && i < N;
        float x[3] = {0.f, 0.f, 0.f};
        typename TrainCarry<D, G, TT>::type st;
        st.mu = 0.f;
        if (work) {
            const int ic = i < N ? i : N - 1;
            sample_position(g, ic, stratum_offset(va.jitter, pix[r], N, ic), x);
            if constexpr (kMmaPath<TT>)
                mma_forward<D, G, TT>(fa, cta.sp, cta.sw, cta.smask, cta.wbuf, cta.tslot0, x, lane, st);
            else
                f32_forward<D, G, TT, PS>(fa, cta.sp, cta.wlo, cta.smask, cta.wbuf, cta.tslot0, x, lane, st);
        }
        const float part = warp_sum(active ? st.mu : 0.f) * (work ? g.delta : 0.f);
        if (lane == 0) s_part[warp] = part;
        __syncthreads();
        if ((int)threadIdx.x < rpr) {
            const int rr = grp * rpr + threadIdx.x;
            float gr = 0.f, l = 0.f;
            if (rr < R) {
                float A = 0.f;
                for (int cc = 0; cc < C; cc++) A += s_part[threadIdx.x * C + cc];
                const float res = A - a_meas[rr];
                if (loss_kind == NH_LOSS_MSE) {
                    l = res * res;
                    gr = 2.f * res * invR;
                } else {
                    l = fabsf(res);
                    gr = (res > 0.f ? 1.f : (res < 0.f ? -1.f : 0.f)) * invR;
                }
            }
            s_g[threadIdx.x] = gr * scale;
            s_lr[threadIdx.x] = l;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int t = 0; t < rpr && grp * rpr + t < R; t++) s_loss += s_lr[t];
        const float dmu = active ? s_g[rl] * g.delta : 0.f;
        if constexpr (kMmaPath<TT>) {
            if constexpr (NW <= 6) {
                // every warp takes part in the cooperative weight gradient, work or not
                const int wf = bwd_warp_floats(fa.precision);
                const CoopArgs co{cta.wbuf - warp * wf, wf, (int)(blockDim.x >> 5), warp, work};
                mma_backward<D, G, TT, true>(fa, cta.sp, cta.sw, cta.smask, cta.sg, cta.wbuf, cta.tslot0, x, active,
                                             lane, st, dmu, co);
            } else if (work) {
                mma_backward<D, G, TT>(fa, cta.sp, cta.sw, cta.smask, cta.sg, cta.wbuf, cta.tslot0, x, active, lane,
                                       st, dmu);
            }
        } else if (work) {
            f32_backward<D, G, TT, PS>(fa, cta.sp, cta.wlo, cta.smask, cta.sg, cta.wbuf, cta.tslot0, x, active, lane,
                                       st, dmu);
        }
    }
    bwd_end(fa, cta, tcols);
    if (threadIdx.x == 0) loss_part[blockIdx.x] = s_loss;
}

// Sum of n CTA partials in a fixed order with one warp: lane t adds partials
// t, t + 32, ... in turn, then a fixed butterfly combines the lane sums (lane 0's
// result is used), so the loss is the same on every run.
__device__ __forceinline__ float ordered_partial_sum(const float* __restrict__ part, int n, int lane) {
    float s = 0.f;
    for (int k = lane; k < n; k += 32) s += part[k];
    return warp_sum(s);
}

// loss = (ordered sum of the CTA partials) / R. With prologue set (an optimizer
// step follows) the same thread then runs Adam's prologue, after the loss's own
// non-finite check, so the step's launch count drops by one.
static __global__ void k_train_loss(const float* __restrict__ part, int n_part, int R, float* loss_out,
                                    DeviceState* state, AdamHyper hyper, int prologue) {
    const float s = ordered_partial_sum(part, n_part, threadIdx.x);
    if (threadIdx.x != 0) return;
    const float loss = s / (float)R;
    if (loss_out) *loss_out = loss;
    if (!isfinite(loss)) atomicOr(&state->flags, NH_FLAG_NONFINITE);
    if (prologue) adam_prologue(state, hyper);
}

// ============================================================================ points
// query: mu_out[p] = M(x_p), forward only.
// Warps take 32 consecutive points; lanes past the end evaluate the last point and
// discard it (the tensor-core MLP needs every lane).
template <int D, typename TT>
__global__ void __launch_bounds__(128) k_points(FieldArgs fa, int n, const float* __restrict__ xyz,
                                                float* __restrict__ mu_out) {
    extern __shared__ __align__(16) float smem[];
    const FwdCta cta = fwd_begin<TT>(fa, smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntask = ((long long)n + 31) / 32;
    for (long long task = (long long)blockIdx.x * (blockDim.x >> 5) + warp; task < ntask;
         task += (long long)gridDim.x * (blockDim.x >> 5)) {
        const long long p = task * 32 + lane;
        const long long pc = p < n ? p : (long long)n - 1;
        const float x[3] = {xyz[3 * pc], xyz[3 * pc + 1], xyz[3 * pc + 2]};
        const float mu = point_mu<D, TT>(fa, cta, x, lane);
        if (p < n) mu_out[p] = mu;
    }
}

// MCI fit: forward + backward of the voxel L1 loss (Eq. 2) in one pass, one CTA
// partial of sum |mu - mu_gt| per block.
template <int D, int G, typename TT>
__global__ void __launch_bounds__(kBwdWarps * 32, 2)
k_points_fit(FieldArgs fa, int n, const float* __restrict__ xyz, const float* __restrict__ mu_gt,
             float* __restrict__ loss_part, uint32_t tcols) {
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t s_tmem;
    __shared__ float red[kBwdWarps];
    const BwdCta cta = bwd_begin<TT>(fa, smem, &s_tmem, tcols);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float lsum = 0.f;
    const float scale = fa.state->loss_scale / (float)n;
    const long long ntask = ((long long)n + 31) / 32;
    for (long long task = (long long)blockIdx.x * kBwdWarps + warp; task < ntask;
         task += (long long)gridDim.x * kBwdWarps) {
        const long long p = task * 32 + lane;
        const bool active = p < n;
        const long long pc = active ? p : (long long)n - 1;
        const float x[3] = {xyz[3 * pc], xyz[3 * pc + 1], xyz[3 * pc + 2]};
        const float gt = mu_gt[pc];
        const float mu = train_sample<D, G, TT>(fa, cta, x, active, lane, [gt, scale](float m) {
            const float r = m - gt;
            return (r > 0.f ? scale : (r < 0.f ? -scale : 0.f));
        });
        if (active) lsum += fabsf(mu - gt);
    }
    bwd_end(fa, cta, tcols);
    lsum = warp_sum(lsum);
    if (lane == 0) red[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kBwdWarps; w++) s += red[w];
        loss_part[blockIdx.x] = s;
    }
}

static __global__ void k_points_loss(const float* __restrict__ part, int n_part, int n, float* loss_out,
                                     DeviceState* state) {
    const float s = ordered_partial_sum(part, n_part, threadIdx.x);
    if (threadIdx.x != 0) return;
    const float loss = s / (float)n;
    if (loss_out) *loss_out = loss;
    if (!isfinite(loss)) atomicOr(&state->flags, NH_FLAG_NONFINITE);
}

// ============================================================================ probes
static __global__ void k_sample_rays(ViewArgs va, const int32_t* __restrict__ pix, int R, int N,
                              float* __restrict__ xyz, float* __restrict__ delta) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)R * N) return;
    const int r = (int)(t / N), i = (int)(t - (long long)r * N);
    const RayGeo g = ray_setup(va, pix[r], N);
    float x[3];
    sample_position(g, i, stratum_offset(va.jitter, pix[r], N, i), x);
    xyz[3 * t] = x[0];
    xyz[3 * t + 1] = x[1];
    xyz[3 * t + 2] = x[2];
    if (i == 0) delta[r] = g.delta;
}

static __global__ void k_hash_corners(FieldArgs fa, int n, const float* __restrict__ xyz,
                               uint32_t* __restrict__ idx, float* __restrict__ wout) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float x[3] = {xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2]};
    for (int l = 0; l < fa.L; l++) {
        uint32_t c[3];
        float w[3];
        level_cell(x, fa.res[l], c, w);
        const bool dense = (fa.dense_mask >> l) & 1u;
        for (int k = 0; k < 8; k++) {
            uint32_t id;
            float wk;
            corner(c, w, k, (uint32_t)fa.res[l] + 1u, dense, fa.Tmask, id, wk);
            idx[(p * fa.L + l) * 8 + k] = id;
            wout[(p * fa.L + l) * 8 + k] = wk;
        }
    }
}

template <int D, typename TT>
__global__ void k_encode_points(FieldArgs fa, int n, const float* __restrict__ xyz, float* __restrict__ hout) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float x[3] = {xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2]};
    float h[D];
    encode_point<D / 2, TT>(fa, table_base<TT>(fa), x, h);
#pragma unroll
    for (int k = 0; k < D; k++) hout[p * D + k] = h[k];
}

static __global__ void k_voxel_centres(int D, float* __restrict__ xyz) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)D * D * D;
    if (t >= n) return;
    const int x = (int)(t % D), y = (int)((t / D) % D), z = (int)(t / ((long long)D * D));
    const float fD = (float)D;
    xyz[3 * t] = __fdiv_rn(__fadd_rn((float)x, 0.5f), fD);
    xyz[3 * t + 1] = __fdiv_rn(__fadd_rn((float)y, 0.5f), fD);
    xyz[3 * t + 2] = __fdiv_rn(__fadd_rn((float)z, 0.5f), fD);
}

// Query at voxel centres without materialising the coordinates.
template <int D_, typename TT>
__global__ void __launch_bounds__(256) k_query_volume(FieldArgs fa, int D, float* __restrict__ out) {
    extern __shared__ __align__(16) float smem[];
    const FwdCta cta = fwd_begin<TT>(fa, smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n = (long long)D * D * D;
    const long long ntask = (n + 31) / 32;
    const float fD = (float)D;
    for (long long task = (long long)blockIdx.x * (blockDim.x >> 5) + warp; task < ntask;
         task += (long long)gridDim.x * (blockDim.x >> 5)) {
        const long long t = task * 32 + lane;
        const long long tc = t < n ? t : n - 1;
        const int xi = (int)(tc % D), yi = (int)((tc / D) % D), zi = (int)(tc / ((long long)D * D));
        const float x[3] = {__fdiv_rn(__fadd_rn((float)xi, 0.5f), fD),
                            __fdiv_rn(__fadd_rn((float)yi, 0.5f), fD),
                            __fdiv_rn(__fadd_rn((float)zi, 0.5f), fD)};
        const float mu = point_mu<D_, TT>(fa, cta, x, lane);
        if (t < n) out[t] = mu;
    }
}

// ============================================================================ launchers
int num_sms();

static size_t dense_smem(const FieldArgs& fa) {
    return (size_t)(((fa.n_dense + 3) & ~3) + kMaxD) * sizeof(float);
}

// Persistent grid of the training kernels: CTAs resident per SM by registers and
// shared memory, and never more than TMEM holds (512 columns per SM), so every
// CTA's tcgen05.alloc is satisfied without waiting for another CTA to finish.
template <typename K>
static long long train_grid(K kernel, size_t smem, uint32_t tcols, long long need, int threads = kBwdWarps * 32);

// Opts the kernel into `bytes` of dynamic shared memory and the largest shared
// memory carveout, so that occupancy queries and launches see the same capacity.
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    cudaError_t e = cudaSuccess;
    if (bytes > 48 * 1024) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    }
    return e;
}

// Last persistent-grid decision of the training kernels (read by launch_info).
struct GridInfo {
    int sms, occupancy, by_tmem, blocks;
    uint32_t tmem_cols;
    size_t smem;
};
GridInfo& last_grid();

// CTAs of `threads` threads that fit on one SM by registers, shared memory and
// threads, from the compiled kernel's attributes and the device limits.
template <typename K>
static int resident_ctas(K kernel, size_t dyn_smem, int threads) {
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, kernel) != cudaSuccess) return 1;
    int dev = 0, regs_sm = 0, smem_sm = 0, reserved = 0, thr_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((at.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : 1;
    const size_t per_cta = dyn_smem + at.sharedSizeBytes + (size_t)reserved;
    const int by_smem = (int)((size_t)smem_sm / per_cta);
    const int by_thr = thr_sm / threads;
    int n = by_regs < by_smem ? by_regs : by_smem;
    return n < by_thr ? n : by_thr;
}

template <typename K>
static long long train_grid(K kernel, size_t smem, uint32_t tcols, long long need, int threads) {
    const int occ = resident_ctas(kernel, smem, threads);
    const int by_tmem = (int)(512u / tcols);
    int per_sm = occ < by_tmem ? occ : by_tmem;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)num_sms() * per_sm;
    if (blocks > need) blocks = need;
    GridInfo& g = last_grid();
    g.sms = num_sms();
    g.occupancy = occ;
    g.by_tmem = by_tmem;
    g.blocks = (int)blocks;
    g.tmem_cols = tcols;
    g.smem = smem;
    return blocks;
}

// Dispatch on the feature width D = L * F for a given table type TT.
#define NH_DISPATCH_D(fa, ...)                                      \
    do {                                                            \
        if ((fa).D == 16) { constexpr int D_ = 16; __VA_ARGS__; }   \
        else if ((fa).D == 32) { constexpr int D_ = 32; __VA_ARGS__; } \
        else return cudaErrorInvalidValue;                          \
    } while (0)

// Training kernels are also specialised on the number of normalization groups G
// (one statistic per level for the per-level LayerNorm, else one), which sets how
// many registers carry the statistics from the forward to the backward.
#define NH_DISPATCH_DG(fa, ...)                                                          \
    do {                                                                                 \
        const bool per_level_ = (fa).norm == NH_NORM_LN_PER_LEVEL;                       \
        if ((fa).D == 16 && per_level_) { constexpr int D_ = 16, G_ = 8; __VA_ARGS__; }  \
        else if ((fa).D == 16) { constexpr int D_ = 16, G_ = 1; __VA_ARGS__; }           \
        else if ((fa).D == 32 && per_level_) { constexpr int D_ = 32, G_ = 16; __VA_ARGS__; } \
        else if ((fa).D == 32) { constexpr int D_ = 32, G_ = 1; __VA_ARGS__; }           \
        else return cudaErrorInvalidValue;                                               \
    } while (0)

template <typename TT>
cudaError_t launch_ray_forward_tt(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, int R, int N,
                                  float* ray_part, cudaStream_t st) {
    const int C = (N + 31) / 32;
    const long long tasks = (long long)R * C;
    if (tasks == 0) return cudaSuccess;
    const long long blocks = (tasks + 7) / 8;
    const size_t sm = fwd_smem_bytes<TT>(fa, 8);
    NH_DISPATCH_D(fa, {
        auto k = k_ray_forward<D_, TT>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)blocks, 256, sm, st>>>(fa, va, pix, R, N, C, ray_part);
    });
    return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_ray_backward_tt(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, int R, int N,
                                   const float* dLdA, cudaStream_t st) {
    const int C = (N + 31) / 32;
    const long long tasks = (long long)R * C;
    if (tasks == 0) return cudaSuccess;
    const size_t sm = bwd_smem_bytes(fa);
    const uint32_t tcols = bwd_tmem_cols(fa);
    NH_DISPATCH_DG(fa, {
        auto k = k_ray_backward<D_, G_, TT>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        const long long blocks = train_grid(k, sm, tcols, (tasks + kBwdWarps - 1) / kBwdWarps);
        k<<<(unsigned)blocks, kBwdWarps * 32, sm, st>>>(fa, va, pix, R, N, C, dLdA, tcols);
    });
    return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_points_tt(const FieldArgs& fa, int n, const float* xyz, const float* mu_gt, float* mu_out,
                             float* loss_part, int n_part, float* loss_out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (mu_gt == nullptr) {
        const size_t sm = fwd_smem_bytes<TT>(fa, 4);
        NH_DISPATCH_D(fa, {
            auto k = k_points<D_, TT>;
            cudaError_t e = set_smem(k, sm);
            if (e != cudaSuccess) return e;
            long long blocks = ((long long)n + 127) / 128;
            if (blocks > (long long)num_sms() * 64) blocks = (long long)num_sms() * 64;
            k<<<(unsigned)blocks, 128, sm, st>>>(fa, n, xyz, mu_out);
        });
        return cudaGetLastError();
    }
    const size_t sm = bwd_smem_bytes(fa);
    const uint32_t tcols = bwd_tmem_cols(fa);
    NH_DISPATCH_DG(fa, {
        auto k = k_points_fit<D_, G_, TT>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        long long blocks = train_grid(k, sm, tcols, ((long long)n + 32 * kBwdWarps - 1) / (32 * kBwdWarps));
        if (blocks > n_part) blocks = n_part;
        k<<<(unsigned)blocks, kBwdWarps * 32, sm, st>>>(fa, n, xyz, mu_gt, loss_part, tcols);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_points_loss<<<1, 32, 0, st>>>(loss_part, (int)blocks, n, loss_out, fa.state);
    });
    return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_encode_points_tt(const FieldArgs& fa, int n, const float* xyz, float* h, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    NH_DISPATCH_D(fa, { k_encode_points<D_, TT><<<(n + 127) / 128, 128, 0, st>>>(fa, n, xyz, h); });
    return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_query_volume_tt(const FieldArgs& fa, int D, float* out, cudaStream_t st) {
    const long long n = (long long)D * D * D;
    if (n == 0) return cudaSuccess;
    const size_t sm = fwd_smem_bytes<TT>(fa, 8);
    NH_DISPATCH_D(fa, {
        auto k = k_query_volume<D_, TT>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        long long blocks = (n + 255) / 256;
        if (blocks > (long long)num_sms() * 32) blocks = (long long)num_sms() * 32;
        k<<<(unsigned)blocks, 256, sm, st>>>(fa, D, out);
    });
    return cudaGetLastError();
}

// Fused training step (k_ray_train) when a ray has at most kMaxFusedChunks chunks of
// 32 samples and the CTA's activations fit the SM's 512 TMEM columns; returns
// cudaErrorNotSupported otherwise, before launching anything (the caller then runs
// forward, loss and backward as separate kernels). Rays of up to 8 chunks are
// packed 8 / C to a CTA of C * (8 / C) warps, two CTAs per SM; longer rays take one
// CTA of C warps each, one CTA per SM (its TMEM groups fill the SM's 512 columns).
// loss_part: >= kTrainParts floats of workspace.
template <typename TT>
cudaError_t launch_ray_train_tt(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, const float* a_meas,
                                int R, int N, int loss_kind, float* loss_part, float* loss_out,
                                const AdamHyper* hyper, cudaStream_t st) {
    const int C = (N + 31) / 32;
    if (C > kMaxFusedChunks || R <= 0) return cudaErrorNotSupported;
    const int rpr = C <= kBwdWarps ? kBwdWarps / C : 1;
    const int nw = rpr * C;
    const int threads = nw * 32;
    const long long ngroups = ((long long)R + rpr - 1) / rpr;
    constexpr bool kF32 = !kMmaPath<TT>;
    const uint32_t tcols = bwd_tmem_cols(fa, nw);
    if (tcols > 512u) return cudaErrorNotSupported;   // deep MLPs with long rays: split path
    const bool ps = kF32 && (nw <= 6 || (nw > kBwdWarps && nw <= kMidTrainWarps &&
                                         bwd_smem_bytes(fa, nw, true) + 1024 <= 227 * 1024));
    const size_t sm = bwd_smem_bytes(fa, nw, ps);
    NH_DISPATCH_DG(fa, {
        auto k = nw <= 6 ? k_ray_train<D_, G_, TT, 6, kF32>
                 : nw <= kBwdWarps ? k_ray_train<D_, G_, TT, kBwdWarps, false>
                 : nw <= kMidTrainWarps
                       ? (ps ? k_ray_train<D_, G_, TT, kMidTrainWarps, kF32> : k_ray_train<D_, G_, TT, kMidTrainWarps, false>)
                       : k_ray_train<D_, G_, TT, kMaxTrainWarps, false>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        long long blocks = train_grid(k, sm, tcols, ngroups, threads);
        if (blocks > kTrainParts) blocks = kTrainParts;
        k<<<(unsigned)blocks, threads, sm, st>>>(fa, va, pix, a_meas, R, N, C, rpr, loss_kind, loss_part, tcols);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_train_loss<<<1, 32, 0, st>>>(loss_part, (int)blocks, R, loss_out, fa.state,
                                       hyper ? *hyper : AdamHyper{0.f, 0.f, 0.f, 0}, hyper ? 1 : 0);
    });
    return cudaGetLastError();
}

// The fused training launcher is instantiated in its own translation units
// (nh_train_*.cu) and the rest in nh_field_*.cu, so the build compiles them in
// parallel.
#define NH_INSTANTIATE_TRAIN(TT)                                                                            \
    template cudaError_t launch_ray_train_tt<TT>(const FieldArgs&, const ViewArgs&, const int32_t*, const float*, \
                                                 int, int, int, float*, float*, const AdamHyper*, cudaStream_t);

#define NH_INSTANTIATE_FIELD(TT)                                                                            \
    template cudaError_t launch_ray_forward_tt<TT>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, \
                                                   float*, cudaStream_t);                                   \
    template cudaError_t launch_ray_backward_tt<TT>(const FieldArgs&, const ViewArgs&, const int32_t*, int,   \
                                                    int, const float*, cudaStream_t);                        \
    template cudaError_t launch_points_tt<TT>(const FieldArgs&, int, const float*, const float*, float*,      \
                                              float*, int, float*, cudaStream_t);                            \
    template cudaError_t launch_encode_points_tt<TT>(const FieldArgs&, int, const float*, float*, cudaStream_t); \
    template cudaError_t launch_query_volume_tt<TT>(const FieldArgs&, int, float*, cudaStream_t);

}  // namespace nh
