// Adam over the whole flat parameter vector (Sec. 3.1: Adam, lr 1e-3) with the
// float32 master copy, the bf16 / f16 working copy of the tables, dynamic loss
// scaling and the non-finite step skip.
//
//  k_adam_prep  one thread: reads the step's flags, decides skip / apply, updates
//               the loss scale and step count, computes the bias corrections
//               (adam_prologue; a training step whose loss kernel already ran it
//               launches k_adam alone).
//  k_adam       float4 pass over the live ranges of the vector: m, v, p updated
//               in place (torch.optim.Adam semantics: bias-corrected, eps outside
//               the square root), grads zeroed, low-precision table copy
//               refreshed. A skipped step only zeroes the grads. Each range gets
//               its own share of the blocks, in proportion to its length, and
//               those blocks sweep it grid-stride, so the inner loop indexes one
//               contiguous range.
//
// Live ranges: a dense level l ((N_l + 1)^3 <= T) indexes only the first
// (N_l + 1)^3 of its T entries, since a corner's index there is at most
// (N_l + 1)^3 - 1. No gather or scatter reaches the others, so their gradients and
// moments stay zero and the update leaves them unchanged bit for bit (m = v = 0
// gives a zero step). The pass visits the reachable table entries and the dense
// MLP / LN block only; at T = 2^19, 16 levels from 16 to 2048, that skips 27 % of
// the vector, at T = 2^21 37 %.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "nh_adam_prep.cuh"
#include "nh_internal.h"

namespace nh {

__global__ void k_adam_prep(DeviceState* st, AdamHyper h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    adam_prologue(st, h);
}

template <typename LP>
__device__ __forceinline__ void store_lp(LP* lp, int64_t i, float4 p);
template <>
__device__ __forceinline__ void store_lp<__nv_bfloat16>(__nv_bfloat16* lp, int64_t i, float4 p) {
    __nv_bfloat162 a = __floats2bfloat162_rn(p.x, p.y), b = __floats2bfloat162_rn(p.z, p.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned int*>(&a);
    u.y = *reinterpret_cast<unsigned int*>(&b);
    *reinterpret_cast<uint2*>(lp + i) = u;
}
template <>
__device__ __forceinline__ void store_lp<__half>(__half* lp, int64_t i, float4 p) {
    __half2 a = __floats2half2_rn(p.x, p.y), b = __floats2half2_rn(p.z, p.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned int*>(&a);
    u.y = *reinterpret_cast<unsigned int*>(&b);
    *reinterpret_cast<uint2*>(lp + i) = u;
}
template <>
__device__ __forceinline__ void store_lp<float>(float*, int64_t, float4) {}

// The update needs a square root and a reciprocal per parameter; the IEEE-rounded
// forms are multi-instruction sequences that would make this HBM-bound pass
// instruction-bound, so it uses the single-instruction PTX approximations (a few
// ulp of relative error in the step, far below the step's own float32 rounding
// of p).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float adam1(float& p, float& m, float& v, float g, float b1, float b2,
                                       float eps, float step_size, float inv_bc2_sqrt) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p = fmaf(-step_size * m, rcp_approx(fmaf(sqrt_approx(v), inv_bc2_sqrt, eps)), p);
    return p;
}

// Float4 ranges of the flat vector that the pass visits, in order; range r starts
// at float4 start4[r], has cum4[r + 1] - cum4[r] float4s and is swept by blocks
// block0[r] .. block0[r + 1] - 1.
struct AdamRanges {
    int n;
    int64_t start4[kMaxLevels + 1];
    int64_t cum4[kMaxLevels + 2];
    int block0[kMaxLevels + 2];
};

// n_lp (a multiple of 4) leading entries of the vector refresh lp.
// Each thread owns kU float4 groups per sweep (strided by its range's blocks so
// every instruction is coalesced) and issues all of their loads before the first
// use, so one resident wave keeps enough bytes in flight to stream at HBM speed
// (120 registers, two blocks per SM; held to three blocks per SM the kernel
// spills and streams slower).
// Moments and zeroed gradients are written evict-first: only the next optimizer
// pass reads them. The parameters the next gather reads stay cacheable: the
// float32 vector on the FP32 path; on the 16-bit paths the low-precision copy,
// while the float32 master copy, read only by the optimizer, streams
// evict-first so that it does not displace the copy from L2.
constexpr int kU = 4;
// 16-bit paths: the float32 vector is a master copy that no gather reads.
template <typename LP> constexpr bool kMasterOnly = true;
template <> constexpr bool kMasterOnly<float> = false;

template <typename LP>
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v,
                                              const AdamRanges rg, LP* __restrict__ lp, int64_t n_lp,
                                              const DeviceState* st, float b1, float b2, float eps) {
    // this block's range, read with constant indices (no local copy of the table)
    int64_t n4 = 0, off = 0;
    int bb = 0, be = 1;
#pragma unroll
    for (int k = 0; k < kMaxLevels + 1; k++) {
        if (k < rg.n && (int)blockIdx.x >= rg.block0[k] && (int)blockIdx.x < rg.block0[k + 1]) {
            n4 = rg.cum4[k + 1] - rg.cum4[k];
            off = rg.start4[k];
            bb = rg.block0[k];
            be = rg.block0[k + 1];
        }
    }
    const int64_t T = (int64_t)(be - bb) * blockDim.x;
    const int64_t t0 = (int64_t)(blockIdx.x - bb) * blockDim.x + threadIdx.x;
    float4* g4 = reinterpret_cast<float4*>(g) + off;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (st->skip != 0u) {   // skipped step: only the gradients are cleared
        for (int64_t q = t0; q < n4; q += T) __stcs(g4 + q, z4);
        return;
    }
    const float inv_scale = st->inv_scale, step_size = st->step_size, ib2 = st->inv_bc2_sqrt;
    float4* p4 = reinterpret_cast<float4*>(p) + off;
    float4* m4 = reinterpret_cast<float4*>(m) + off;
    float4* v4 = reinterpret_cast<float4*>(v) + off;
    for (int64_t base = t0; base < n4; base += T * kU) {
        float4 gg[kU], pp[kU], mm[kU], vv[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const int64_t q = base + u * T;
            if (q < n4) {
                gg[u] = __ldcs(g4 + q);
                pp[u] = kMasterOnly<LP> ? __ldcs(p4 + q) : p4[q];
                mm[u] = __ldcs(m4 + q);
                vv[u] = __ldcs(v4 + q);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const int64_t q = base + u * T;
            if (q < n4) {
                adam1(pp[u].x, mm[u].x, vv[u].x, gg[u].x * inv_scale, b1, b2, eps, step_size, ib2);
                adam1(pp[u].y, mm[u].y, vv[u].y, gg[u].y * inv_scale, b1, b2, eps, step_size, ib2);
                adam1(pp[u].z, mm[u].z, vv[u].z, gg[u].z * inv_scale, b1, b2, eps, step_size, ib2);
                adam1(pp[u].w, mm[u].w, vv[u].w, gg[u].w * inv_scale, b1, b2, eps, step_size, ib2);
                if constexpr (kMasterOnly<LP>)
                    __stcs(p4 + q, pp[u]);
                else
                    p4[q] = pp[u];
                __stcs(m4 + q, mm[u]);
                __stcs(v4 + q, vv[u]);
                __stcs(g4 + q, z4);
                if (((off + q) << 2) < n_lp) store_lp<LP>(lp, (off + q) << 2, pp[u]);
            }
        }
    }
}

template <typename LP>
__global__ void k_refresh(const float* __restrict__ p, LP* __restrict__ lp, int64_t n) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (n >> 2);
         q += (int64_t)gridDim.x * blockDim.x)
        store_lp<LP>(lp, q << 2, reinterpret_cast<const float4*>(p)[q]);
}

__global__ void k_init_state(DeviceState* st, float loss_scale) {
    const int t = threadIdx.x;
    if (t == 0) {
        st->step = 0;
        st->loss_scale = loss_scale;
        st->good_steps = 0;
        st->flags = 0u;
        st->last_flags = 0u;
        st->skip = 0u;
        st->step_size = 0.f;
        st->inv_bc2_sqrt = 1.f;
        st->inv_scale = 1.f / loss_scale;
        st->loss_accum = 0.f;
    }
    if (t < kMaxD) st->mask[t] = 1.f;
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_adam(const FieldArgs& fa, float* params, float* grads, float* m, float* v, int64_t n,
                        float lr, float beta1, float beta2, float eps, int growth_interval,
                        cudaStream_t st, bool prologue) {
    if (prologue) {
        k_adam_prep<<<1, 32, 0, st>>>(fa.state, AdamHyper{lr, beta1, beta2, growth_interval});
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // live ranges: each level's reachable entries (rounded up to whole float4s),
    // then the dense block; touching ranges are merged
    AdamRanges rg{};
    const int64_t T = (int64_t)fa.Tmask + 1, F = fa.F;
    auto add = [&rg](int64_t b, int64_t e) {   // [b, e) in floats, multiples of 4
        if (e <= b) return;
        if (rg.n > 0 && rg.start4[rg.n - 1] + (rg.cum4[rg.n] - rg.cum4[rg.n - 1]) == b / 4) {
            rg.cum4[rg.n] += (e - b) / 4;
            return;
        }
        rg.start4[rg.n] = b / 4;
        rg.cum4[rg.n + 1] = rg.cum4[rg.n] + (e - b) / 4;
        rg.n++;
    };
    for (int l = 0; l < fa.L; l++) {
        int64_t live = T;
        if ((fa.dense_mask >> l) & 1u) {
            const int64_t s = (int64_t)fa.res[l] + 1;
            live = s * s * s < T ? s * s * s : T;
        }
        add(l * T * F, l * T * F + (((live * F + 3) / 4) * 4 < T * F ? ((live * F + 3) / 4) * 4 : T * F));
    }
    add(fa.n_table, n);
    const int64_t n4 = rg.cum4[rg.n];
    int64_t blocks = (n4 + 256 * kU - 1) / (256 * kU);
    int per_sm = 0;   // one resident wave
    if (fa.precision == NH_PREC_BF16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adam<__nv_bfloat16>, 256, 0);
    else if (fa.precision == NH_PREC_F16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adam<__half>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adam<float>, 256, 0);
    const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // blocks per range in proportion to its float4s, at least one each
    {
        int b0 = 0;
        for (int r = 0; r < rg.n; r++) {
            const int64_t len = rg.cum4[r + 1] - rg.cum4[r];
            int64_t nb = (len * blocks + n4 - 1) / n4;
            if (nb < 1) nb = 1;
            rg.block0[r] = b0;
            b0 += (int)nb;
        }
        rg.block0[rg.n] = b0;
        blocks = b0;
    }
    if (fa.precision == NH_PREC_BF16)
        k_adam<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(params, grads, m, v, rg,
            (__nv_bfloat16*)fa.tables_lp, fa.n_table, fa.state, beta1, beta2, eps);
    else if (fa.precision == NH_PREC_F16)
        k_adam<__half><<<(unsigned)blocks, 256, 0, st>>>(params, grads, m, v, rg, (__half*)fa.tables_lp,
            fa.n_table, fa.state, beta1, beta2, eps);
    else
        k_adam<float><<<(unsigned)blocks, 256, 0, st>>>(params, grads, m, v, rg, nullptr, 0, fa.state,
            beta1, beta2, eps);
    return cudaGetLastError();
}

cudaError_t launch_refresh_lowp(const float* params, void* lp, int64_t n, int precision, cudaStream_t st) {
    if (n == 0 || lp == nullptr || precision == NH_PREC_F32) return cudaSuccess;
    int64_t blocks = ((n >> 2) + 255) / 256;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    if (precision == NH_PREC_BF16)
        k_refresh<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(params, (__nv_bfloat16*)lp, n);
    else
        k_refresh<__half><<<(unsigned)blocks, 256, 0, st>>>(params, (__half*)lp, n);
    return cudaGetLastError();
}

cudaError_t launch_init_state(DeviceState* s, float loss_scale, cudaStream_t st) {
    k_init_state<<<1, 64, 0, st>>>(s, loss_scale);
    return cudaGetLastError();
}

}  // namespace nh
