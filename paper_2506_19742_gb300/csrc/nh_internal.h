// Internal structures shared by the library's translation units (host and device).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/nhcbct.h"

namespace nh {

constexpr int kMaxLevels = 32;
constexpr int kMaxD = 64;

// Device state block at the start of the caller's `state` buffer.
struct DeviceState {
    int32_t  step;          // Adam step count t (steps actually applied)
    float    loss_scale;    // multiplies dL/dA before the backward
    int32_t  good_steps;    // finite steps since the last scale change
    uint32_t flags;         // NH_FLAG_NONFINITE raised by kernels of the current step
    uint32_t last_flags;    // flags of the last optimizer step (polled by the host)
    uint32_t skip;          // 1: the pending optimizer step is skipped
    float    step_size;     // lr / (1 - beta1^t)
    float    inv_bc2_sqrt;  // 1 / sqrt(1 - beta2^t)
    float    inv_scale;     // 1 / loss scale used by the pending step
    float    loss_accum;    // scratch for multi-kernel loss reductions
    float    pad[6];
    float    mask[kMaxD];   // channel mask applied after the LN affine step
};
static_assert(sizeof(DeviceState) == 64 + 4 * kMaxD, "state layout");

// One view of the scan: source s, detector centre c, detector axes u, v (float).
struct ViewArgs {
    float s[3], c[3], u[3], v[3];
    float du, dv;
    int32_t nu, nv;
    unsigned long long jitter;   // 0: midpoint samples; else the stratified-jitter seed
};

// Everything a field kernel needs, passed by value.
struct FieldArgs {
    const float* params;     // flat float32 parameter vector
    const void*  tables_lp;  // bf16 / f16 copy of the tables (or null)
    float*       grads;      // flat float32 gradient vector (same layout)
    DeviceState* state;
    int32_t  L, F, log2T;
    uint32_t Tmask;          // T - 1
    int32_t  D, H, W;        // D = L * F, H hidden layers of width W
    int32_t  norm;
    float    eps;
    uint32_t dense_mask;     // bit l set: level l is densely indexed
    int32_t  res[kMaxLevels];
    int64_t  n_table;        // L * T * F; the dense parameters follow
    int32_t  n_dense;        // gamma, beta, MLP weights and biases
    int32_t  off_beta;       // offsets relative to the dense base (gamma at 0)
    int32_t  off_mlp;
    int32_t  precision;
};

// Kernel launchers (one translation unit each). All return the launch error.
cudaError_t launch_ray_forward(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, int R,
                               int N, float* ray_part, cudaStream_t st);
cudaError_t launch_ray_loss(const float* ray_part, int R, int C, const float* a_meas, int loss_kind,
                            float* a_pred, float* dLdA, float* loss_out, DeviceState* state,
                            bool scale_by_loss_scale, cudaStream_t st);
cudaError_t launch_ray_backward(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, int R,
                                int N, const float* dLdA, cudaStream_t st);
// Fused forward + loss + backward (rays of at most kMaxFusedChunks chunks of 32
// samples); cudaErrorNotSupported for longer rays. loss_part: >= kTrainParts floats.
constexpr int kTrainParts = 4096;
constexpr int kMaxFusedChunks = 16;   // rays of up to 16 x 32 samples take the fused kernel
// hyper != null: the loss kernel also runs the optimizer's prologue (an Adam step
// follows, launched by launch_adam with prologue false).
struct AdamHyper;
cudaError_t launch_ray_train(const FieldArgs& fa, const ViewArgs& va, const int32_t* pix, const float* a_meas,
                             int R, int N, int loss_kind, float* loss_part, float* loss_out,
                             const AdamHyper* hyper, cudaStream_t st);
// query (mu_gt == null) or MCI fit step (loss written to loss_out, CTA partials in loss_part)
cudaError_t launch_points(const FieldArgs& fa, int n, const float* xyz, const float* mu_gt,
                          float* mu_out, float* loss_part, int n_part, float* loss_out,
                          cudaStream_t st);
int         points_partials(int n);
cudaError_t launch_adam(const FieldArgs& fa, float* params, float* grads, float* m, float* v,
                        int64_t n, float lr, float beta1, float beta2, float eps,
                        int growth_interval, cudaStream_t st, bool prologue = true);
cudaError_t launch_refresh_lowp(const float* params, void* lp, int64_t n, int precision,
                                cudaStream_t st);
cudaError_t launch_init_state(DeviceState* s, float loss_scale, cudaStream_t st);
cudaError_t launch_project(const ViewArgs& va, int view, const float* vol, int D, int oversample,
                           float* proj, cudaStream_t st);
cudaError_t launch_sample_rays(const ViewArgs& va, const int32_t* pix, int R, int N, float* xyz,
                               float* delta, cudaStream_t st);
cudaError_t launch_hash_corners(const FieldArgs& fa, int n, const float* xyz, uint32_t* idx,
                                float* w, cudaStream_t st);
cudaError_t launch_encode_points(const FieldArgs& fa, int n, const float* xyz, float* h,
                                 cudaStream_t st);
cudaError_t launch_query_volume(const FieldArgs& fa, int D, float* out, cudaStream_t st);
cudaError_t launch_scatter_points(const FieldArgs& fa, int n, const float* xyz, const float* dh,
                                  cudaStream_t st);
// roofline probes (nh_probe.cu)
cudaError_t launch_probe_l2_read(const void* buf, size_t bytes, int reps, float* sink, cudaStream_t st);
cudaError_t launch_probe_random_gather(const void* table, size_t n_entries, int entry_bytes, int64_t n_loads,
                                       float* sink, int64_t* n_done, cudaStream_t st);
cudaError_t launch_probe_random_red(float* table, size_t n_entries, int64_t n_ops, int64_t* n_done,
                                    cudaStream_t st);
cudaError_t launch_probe_random_red16(void* table, size_t n_entries, int fmt, int64_t n_ops, int64_t* n_done,
                                      cudaStream_t st);
size_t      mse_workspace_bytes();
// sms, occupancy (CTAs/SM by registers and shared memory), CTAs/SM by TMEM, grid,
// TMEM columns per CTA, dynamic shared memory bytes of the last training launch
void        last_train_grid(int32_t out[6]);
cudaError_t launch_mse(const float* a, const float* b, int64_t n, double* out, void* ws, cudaStream_t st);

}  // namespace nh
