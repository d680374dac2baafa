// Precision-independent launchers of the field kernels and the public dispatch on
// the table precision (the templated launchers live in nh_field_{f32,bf16,f16}.cu).
#include "nh_field.cuh"

namespace nh {

GridInfo& last_grid() {
    static GridInfo g{};
    return g;
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

extern template cudaError_t launch_ray_forward_tt<float>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, float*, cudaStream_t);
extern template cudaError_t launch_ray_forward_tt<__nv_bfloat16>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, float*, cudaStream_t);
extern template cudaError_t launch_ray_forward_tt<__half>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, float*, cudaStream_t);
extern template cudaError_t launch_ray_backward_tt<float>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, const float*, cudaStream_t);
extern template cudaError_t launch_ray_backward_tt<__nv_bfloat16>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, const float*, cudaStream_t);
extern template cudaError_t launch_ray_backward_tt<__half>(const FieldArgs&, const ViewArgs&, const int32_t*, int, int, const float*, cudaStream_t);
extern template cudaError_t launch_points_tt<float>(const FieldArgs&, int, const float*, const float*, float*, float*, int, float*, cudaStream_t);
extern template cudaError_t launch_points_tt<__nv_bfloat16>(const FieldArgs&, int, const float*, const float*, float*, float*, int, float*, cudaStream_t);
extern template cudaError_t launch_points_tt<__half>(const FieldArgs&, int, const float*, const float*, float*, float*, int, float*, cudaStream_t);
extern template cudaError_t launch_encode_points_tt<float>(const FieldArgs&, int, const float*, float*, cudaStream_t);
extern template cudaError_t launch_encode_points_tt<__nv_bfloat16>(const FieldArgs&, int, const float*, float*, cudaStream_t);
extern template cudaError_t launch_encode_points_tt<__half>(const FieldArgs&, int, const float*, float*, cudaStream_t);
extern template cudaError_t launch_query_volume_tt<float>(const FieldArgs&, int, float*, cudaStream_t);
extern template cudaError_t launch_query_volume_tt<__nv_bfloat16>(const FieldArgs&, int, float*, cudaStream_t);
extern template cudaError_t launch_query_volume_tt<__half>(const FieldArgs&, int, float*, cudaStream_t);

extern template cudaError_t launch_ray_train_tt<float>(const FieldArgs&, const ViewArgs&, const int32_t*, const float*, int, int, int, float*, float*, const AdamHyper*, cudaStream_t);
extern template cudaError_t launch_ray_train_tt<__nv_bfloat16>(const FieldArgs&, const ViewArgs&, const int32_t*, const float*, int, int, int, float*, float*, const AdamHyper*, cudaStream_t);
extern template cudaError_t launch_ray_train_tt<__half>(const FieldArgs&, const ViewArgs&, const int32_t*, const float*, int, int, int, float*, float*, const AdamHyper*, cudaStream_t);

cudaError_t launch_ray_train(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, const float* a_meas,
                             int R, int N, int loss_kind, float* loss_part, float* loss_out,
                             const AdamHyper* hyper, cudaStream_t st) {
    switch (fa.precision) {
        case NH_PREC_F32: return launch_ray_train_tt<float>(fa, va, pix, a_meas, R, N, loss_kind, loss_part, loss_out, hyper, st);
        case NH_PREC_BF16: return launch_ray_train_tt<__nv_bfloat16>(fa, va, pix, a_meas, R, N, loss_kind, loss_part, loss_out, hyper, st);
        case NH_PREC_F16: return launch_ray_train_tt<__half>(fa, va, pix, a_meas, R, N, loss_kind, loss_part, loss_out, hyper, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ray_forward(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, int R, int N,
                               float* ray_part, cudaStream_t st) {
    switch (fa.precision) {
        case NH_PREC_F32: return launch_ray_forward_tt<float>(fa, va, pix, R, N, ray_part, st);
        case NH_PREC_BF16: return launch_ray_forward_tt<__nv_bfloat16>(fa, va, pix, R, N, ray_part, st);
        case NH_PREC_F16: return launch_ray_forward_tt<__half>(fa, va, pix, R, N, ray_part, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ray_backward(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, int R, int N,
                                const float* dLdA, cudaStream_t st) {
    switch (fa.precision) {
        case NH_PREC_F32: return launch_ray_backward_tt<float>(fa, va, pix, R, N, dLdA, st);
        case NH_PREC_BF16: return launch_ray_backward_tt<__nv_bfloat16>(fa, va, pix, R, N, dLdA, st);
        case NH_PREC_F16: return launch_ray_backward_tt<__half>(fa, va, pix, R, N, dLdA, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_points(const FieldArgs& fa, int n, const float* xyz, const float* mu_gt, float* mu_out,
                          float* loss_part, int n_part, float* loss_out, cudaStream_t st) {
    switch (fa.precision) {
        case NH_PREC_F32: return launch_points_tt<float>(fa, n, xyz, mu_gt, mu_out, loss_part, n_part, loss_out, st);
        case NH_PREC_BF16: return launch_points_tt<__nv_bfloat16>(fa, n, xyz, mu_gt, mu_out, loss_part, n_part, loss_out, st);
        case NH_PREC_F16: return launch_points_tt<__half>(fa, n, xyz, mu_gt, mu_out, loss_part, n_part, loss_out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_encode_points(const FieldArgs& fa, int n, const float* xyz, float* h, cudaStream_t st) {
    switch (fa.precision) {
        case NH_PREC_F32: return launch_encode_points_tt<float>(fa, n, xyz, h, st);
        case NH_PREC_BF16: return launch_encode_points_tt<__nv_bfloat16>(fa, n, xyz, h, st);
        case NH_PREC_F16: return launch_encode_points_tt<__half>(fa, n, xyz, h, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_query_volume(const FieldArgs& fa, int D, float* out, cudaStream_t st) {
    switch (fa.precision) {
        case NH_PREC_F32: return launch_query_volume_tt<float>(fa, D, out, st);
        case NH_PREC_BF16: return launch_query_volume_tt<__nv_bfloat16>(fa, D, out, st);
        case NH_PREC_F16: return launch_query_volume_tt<__half>(fa, D, out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ray_loss(const float* ray_part, int R, int C, const float* a_meas, int loss_kind,
                            float* a_pred, float* dLdA, float* loss_out, DeviceState* state, bool,
                            cudaStream_t st) {
    k_ray_loss<<<1, 1024, 0, st>>>(ray_part, R, C, a_meas, loss_kind, a_pred, dLdA, loss_out, state);
    return cudaGetLastError();
}

int points_partials(int) { return 4096; }

void last_train_grid(int32_t out[6]) {
    const GridInfo& g = last_grid();
    out[0] = g.sms;
    out[1] = g.occupancy;
    out[2] = g.by_tmem;
    out[3] = g.blocks;
    out[4] = (int32_t)g.tmem_cols;
    out[5] = (int32_t)g.smem;
}

cudaError_t launch_sample_rays(const ViewArgs& va, const int32_t* pix, int R, int N, float* xyz, float* delta,
                               cudaStream_t st) {
    const long long n = (long long)R * N;
    if (n == 0) return cudaSuccess;
    k_sample_rays<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(va, pix, R, N, xyz, delta);
    return cudaGetLastError();
}

// Scatter stage alone: grads[l][idx_k][f] += w_k dh[p][l F + f] for n points, one
// point per lane, warps over 32 consecutive points (the layout of the training
// kernels' samples along a ray). Each lane stages its dL/dh row in shared memory in
// the XOR-swizzled order scatter_point reads.
template <int D>
__global__ void __launch_bounds__(128) k_scatter_points(FieldArgs fa, int n, const float* __restrict__ xyz,
                                                        const float* __restrict__ dh) {
    __shared__ __align__(16) float rows[4][32][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* row = rows[warp][lane];
    const long long ntask = ((long long)n + 31) / 32;
    for (long long task = (long long)blockIdx.x * 4 + warp; task < ntask; task += (long long)gridDim.x * 4) {
        const long long p = task * 32 + lane;
        const bool active = p < n;
        const long long pc = active ? p : (long long)n - 1;
        const float x[3] = {xyz[3 * pc], xyz[3 * pc + 1], xyz[3 * pc + 2]};
        __syncwarp();
#pragma unroll
        for (int k = 0; k < D; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(dh + pc * D + k);
            row[k ^ lane] = active ? v.x : 0.f;
            row[(k + 1) ^ lane] = active ? v.y : 0.f;
            row[(k + 2) ^ lane] = active ? v.z : 0.f;
            row[(k + 3) ^ lane] = active ? v.w : 0.f;
        }
        __syncwarp();
        scatter_point<D / 2>(fa, x, row, lane);
    }
}

cudaError_t launch_scatter_points(const FieldArgs& fa, int n, const float* xyz, const float* dh, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    long long blocks = ((long long)n + 127) / 128;
    if (blocks > (long long)num_sms() * 16) blocks = (long long)num_sms() * 16;
    NH_DISPATCH_D(fa, { k_scatter_points<D_><<<(unsigned)blocks, 128, 0, st>>>(fa, n, xyz, dh); });
    return cudaGetLastError();
}

cudaError_t launch_hash_corners(const FieldArgs& fa, int n, const float* xyz, uint32_t* idx, float* w,
                                cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_hash_corners<<<(n + 127) / 128, 128, 0, st>>>(fa, n, xyz, idx, w);
    return cudaGetLastError();
}

}  // namespace nh
