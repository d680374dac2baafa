/*
 * nhcbct.h - C ABI of the GB300 NeRF-CBCT training library (libnhcbct.so).
 *
 * The library trains the field of "NeRF-based CBCT Reconstruction needs
 * Normalization and Initialization": a multiresolution hash encoder, the
 * Normalized Hash Encoder (a LayerNorm between encoder and network, Sec. 2.3)
 * and a small MLP that predicts attenuation mu(x, y, z). Cone-beam rays from a
 * known source and detector (Sec. 2.2) are sampled, mu is integrated with the
 * Beer-Lambert sum A = sum_i mu_i delta_i (Eq. 1), and the loss against the
 * measured projections (Eq. 3) is backpropagated into the MLP and, by
 * scatter-add, into the hash tables; Adam updates every parameter (Sec. 3.1).
 * Mapping Consistency Initialization pre-trains the field on voxel values
 * (Eq. 2, Sec. 2.4) and transfers only the LN and MLP weights (Sec. 2.1).
 *
 * Conventions
 *  - Every device buffer is owned by the caller (allocate, e.g., with PyTorch and
 *    pass the pointer). Handles own host metadata only; no call allocates or
 *    frees device memory, and nothing on the training path synchronizes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued on it and completes asynchronously.
 *  - Argument errors are reported synchronously as a negative nh_status and
 *    nothing is enqueued. Device-side conditions (non-finite loss or gradients)
 *    set flags that field_poll_status() reads; the optimizer then skips the step.
 *  - Lengths are in units of the volume side: the volume is the unit cube
 *    [0,1]^3 in normalized coordinates, so delta_i and A are dimensionless.
 *  - All float arrays are IEEE binary32 unless stated otherwise; device pointers
 *    must be 16-byte aligned, except the ray batch arrays (4-byte aligned).
 *  - Functions are thread-safe for distinct handles; calls on one field must be
 *    ordered by the caller (one stream, or events between streams).
 */
#ifndef NHCBCT_H
#define NHCBCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef int32_t nh_status;
#define NH_OK                  0
#define NH_ERR_INVALID_ARG    -1  /* null handle/pointer, value out of range          */
#define NH_ERR_CUDA           -2  /* a CUDA runtime call failed (see nh_last_error)   */
#define NH_ERR_SIZE_MISMATCH  -3  /* buffer or workspace smaller than required        */
#define NH_ERR_NONFINITE      -4  /* a non-finite value was detected; step skipped    */
#define NH_ERR_TIMEOUT        -5  /* reserved: a bounded device wait gave up          */
#define NH_ERR_UNSUPPORTED    -6  /* configuration valid but not compiled in          */
#define NH_ERR_ALIGNMENT      -7  /* a device pointer is not suitably aligned         */

/* Human-readable name of a status code (static string). */
const char* nh_status_string(nh_status s);
/* Copies the calling thread's last error detail into buf (NUL-terminated). */
nh_status nh_last_error(char* buf, size_t n);
/* Library ABI version (major * 100 + minor). */
int32_t nh_version(void);

/* ------------------------------------------------------------------ geometry
 * Circular cone-beam scan about the volume's z axis (the source and detector
 * positions are known, Sec. 2.2). View v is at angle
 *   theta_v = angle0 + v * span / n_views,
 * source s = c0 + (dso / side) (cos, sin, 0), detector centre
 * c0 - ((dsd - dso) / side) (cos, sin, 0), detector axes u = (-sin, cos, 0) and
 * v = (0, 0, 1), c0 = (1/2, 1/2, 1/2). Pixel id p = j * det_nu + i is the pixel
 * of column i, row j, centred ((i + 1/2) - nu/2) du, ((j + 1/2) - nv/2) dv from
 * the detector centre. Per-view constants are computed in double on the host and
 * rounded once to float.
 */
typedef struct nh_geometry nh_geometry;
typedef struct {
    int32_t n_views;
    double  angle0_rad, span_rad;
    double  dso_mm, dsd_mm;          /* source-origin, source-detector distance */
    int32_t det_nu, det_nv;          /* detector columns, rows                  */
    double  det_du_mm, det_dv_mm;    /* pixel pitch                             */
    double  vol_side_mm;             /* side of the cubic volume                */
} nh_geometry_desc;

/* Validates desc and builds the per-view table (host memory only; no device
 * allocation). *out receives a handle owned by the caller and released with
 * geometry_destroy. Errors (NH_ERR_INVALID_ARG): a null argument; n_views < 1;
 * a detector size outside 1..65536; a non-positive side, distance or pitch;
 * dsd <= dso; a non-finite angle; a source inside the volume's circumscribed
 * sphere (dso <= side * sqrt(3) / 2). */
nh_status geometry_create(const nh_geometry_desc* desc, nh_geometry** out);
/* Releases a handle from geometry_create (NULL is ignored). */
void      geometry_destroy(nh_geometry* g);
/* Host copy of the per-view table: n_views rows of 12 floats (s, c, u, v), then
 * du, dv (volume units). n_floats must be >= 12 * n_views + 2. */
nh_status geometry_view_table(const nh_geometry* g, float* host_out, size_t n_floats);

/* ------------------------------------------------------------------ field
 * Hash grid: L levels, F features, T = 2^log2_T entries per level; level
 * resolutions N_l = floor(base * exp(l (ln max - ln base) / (L - 1)) + 1e-9).
 * A level with (N_l + 1)^3 <= T is indexed densely, otherwise by the spatial
 * hash (x * 1) ^ (y * 2654435761) ^ (z * 805459861) mod T.
 * Normalization (Sec. 2.3): per-point LayerNorm of the L*F features (one
 * group, or one group per level), then affine gamma/beta and the channel mask.
 * MLP: hidden_layers Linear+ReLU layers of `width`, Linear to 1, sigmoid.
 *
 * Flat parameter vector (float32, one buffer; also the layout of grads/adam_m/
 * adam_v): tables [L][T][F] | gamma [D] | beta [D] | W_0 [width][D] | b_0 [width]
 * | ... | W_H [1][width] | b_H [1], D = L * F, H = hidden_layers.
 */
#define NH_NORM_NONE          0
#define NH_NORM_LN            1
#define NH_NORM_LN_PER_LEVEL  2
#define NH_PREC_F32   0   /* float32 tables, float32 FFMA MLP                     */
#define NH_PREC_BF16  1   /* bf16 table copy + bf16 tensor-core MLP, f32 master   */
#define NH_PREC_F16   2   /* f16 table copy + f16 tensor-core MLP, f32 master     */
#define NH_LOSS_MSE   0   /* mean over rays of (A - A_meas)^2                      */
#define NH_LOSS_L1    1   /* mean over rays of |A - A_meas| (Eq. 3)                */
#define NH_PART_HASH  1u  /* export/import parts */
#define NH_PART_LN    2u
#define NH_PART_MLP   4u
#define NH_PART_ADAM  8u  /* Adam moments of the selected parts */
#define NH_FLAG_NONFINITE 1u  /* a kernel saw a non-finite loss or gradient */
#define NH_FLAG_SKIPPED   2u  /* the last optimizer step was skipped        */

typedef struct nh_field nh_field;
typedef struct {
    int32_t n_levels, n_feat, log2_T, base_res, max_res;
    int32_t norm;               /* NH_NORM_*                                      */
    float   ln_eps;
    int32_t hidden_layers, width;
    int32_t precision;          /* NH_PREC_*                                      */
    int32_t loss;               /* NH_LOSS_*                                      */
    float   lr, beta1, beta2, adam_eps;
    float   loss_scale_init;    /* 1 for f32/bf16; e.g. 1024 for f16              */
    int32_t growth_interval;    /* 0: static loss scale; else double after this
                                   many finite steps, halve on overflow           */
} nh_field_desc;

typedef struct {
    uint64_t n_params;          /* floats in the flat parameter vector */
    uint64_t n_table_params;    /* L * T * F (first in the vector)     */
    uint64_t off_gamma, off_beta, off_mlp;   /* float offsets          */
    uint64_t bytes_params, bytes_grads, bytes_adam_m, bytes_adam_v;
    uint64_t bytes_tables_lp;   /* 0 for NH_PREC_F32                    */
    uint64_t bytes_state;       /* small device state block            */
} nh_field_sizes;

typedef struct {
    float* params;              /* bytes_params, float32 master weights        */
    float* grads;               /* bytes_grads; zero it with field_reset_state */
    float* adam_m;
    float* adam_v;
    void*  tables_lp;           /* bf16/f16 copy of the tables, or NULL (f32)  */
    void*  state;               /* bytes_state                                 */
} nh_field_buffers;

/* Sizes of every caller-owned buffer for this configuration. */
nh_status field_query_sizes(const nh_field_desc* desc, nh_field_sizes* out);
/* Binds a handle to caller-owned buffers (not initialised: see field_reset_state). */
nh_status field_create(const nh_field_desc* desc, const nh_field_buffers* buf, nh_field** out);
void      field_destroy(nh_field* f);                 /* never frees caller memory */
/* Zeroes grads, Adam moments, step count and flags; loss scale = init; channel
 * mask = ones; refreshes the low-precision table copy from params. */
nh_status field_reset_state(nh_field* f, void* stream);
/* Refreshes the low-precision table copy after the caller wrote params. */
nh_status field_refresh_lowp(nh_field* f, void* stream);
/* Channel mask m (Sec. 2.3: masking of noisy feature channels), n = L * F host floats. */
nh_status field_set_channel_mask(nh_field* f, const float* mask_host, int32_t n, void* stream);
/* FFT channel-mask selection (Sec. 2.3: some hash-feature channels carry noise, a
 * Fourier transform tells them apart, and they are masked during training; the
 * paper gives no grid, statistic or threshold). Each of the L * F channels of the
 * hash features h (before the normalization) is sampled at the voxel centres
 * (k + 1/2) / G of a G^3 grid, its mean over the grid removed and its 3-D DFT taken
 * (FP64); frac_dev[c] (double[L * F]) receives the share of its power at radial
 * frequencies |k| > cutoff (cycles per voxel; 0 for a channel without variance),
 * and the channel's mask is 0 where frac > threshold, else 1. mask_dev (float
 * [L * F], may be null) receives the mask; with apply != 0 it is also installed as
 * the field's channel mask (as field_set_channel_mask, on the stream). Sums run in
 * a fixed order: the same field gives the same fractions on every run. Supports
 * F = 2 with L = 8 or 16 (else NH_ERR_UNSUPPORTED); 2 <= G <= 128. ws: device
 * scratch of channel_mask_workspace_bytes(f, G) bytes (268 MB at G = 64, L * F =
 * 32), 256-byte aligned; frac_dev 8-byte aligned. Asynchronous on the stream;
 * allocates nothing. An occasional step between training steps. */
nh_status channel_mask_workspace_bytes(const nh_field* f, int32_t G, size_t* out);
nh_status field_select_channel_mask(nh_field* f, int32_t G, double cutoff, double threshold, int32_t apply,
                                    double* frac_dev, float* mask_dev, void* ws, size_t ws_bytes, void* stream);
nh_status field_level_resolutions(const nh_field* f, int32_t* out, int32_t n);
/* Export / import a subset of the parameters (MCI transfers NH_PART_LN |
 * NH_PART_MLP, Sec. 2.1). The packed order is HASH, LN (gamma, beta), MLP, then,
 * with NH_PART_ADAM, adam_m and adam_v of the same parts. Device-to-device. */
nh_status field_export_bytes(const nh_field* f, uint32_t parts, size_t* out);
nh_status field_export(const nh_field* f, uint32_t parts, void* dev_dst, size_t n_bytes, void* stream);
nh_status field_import(nh_field* f, uint32_t parts, const void* dev_src, size_t n_bytes, void* stream);
/* Synchronizes the stream and reads the state block: flags of the last optimizer
 * step (NH_FLAG_*), current loss scale, Adam step count. Any pointer may be NULL. */
nh_status field_poll_status(nh_field* f, void* stream, uint32_t* flags, float* loss_scale,
                            int32_t* step);

/* ------------------------------------------------------------------ training
 * A ray batch: one view, n_rays detector pixels (Sec. 3.1: one view per batch,
 * rays per view), n_samples samples per ray along [near, far] of the ray's
 * intersection with the volume ("sample points along the X-ray trajectories",
 * Sec. 2.1), delta = (far - near) / n_samples. Sample i sits at
 * t_i = near + (i + u_i) delta: u_i = 1/2 (midpoint rule) when jitter_seed is 0;
 * otherwise stratified jitter, u_i = (top 24 bits of output number
 * pix * n_samples + i + 1 of the SplitMix64 generator started at jitter_seed)
 * * 2^-24, so forward and backward of one batch see the same samples and a new
 * seed per step draws new ones. Rays that miss the volume predict A = 0 and
 * contribute no gradient.
 * pix: device int32[n_rays]; a_meas: device float[n_rays] (may be NULL where unused).
 * The result does not depend on the order of the rays in a batch beyond float
 * rounding, but the order sets which rays run side by side: pixels in ascending
 * id (detector raster order) put neighbouring rays, which read and update
 * neighbouring table entries, on the GPU at the same time and so raise the L2
 * hit rate. The fused step then runs about 6 % faster (paper-size FP32 field) to
 * 8 % faster (tables larger than the L2) than with the same pixels shuffled.
 */
typedef struct {
    int32_t        view;
    int32_t        n_rays;
    const int32_t* pix;
    const float*   a_meas;
    int32_t        n_samples;
    uint64_t       jitter_seed;   /* 0: midpoint samples */
} nh_ray_batch;

/* Workspace bytes needed by train_step / render_* / fit_points_step for a batch. */
nh_status step_workspace_bytes(const nh_field* f, int32_t n_rays, int32_t n_samples, size_t* out);

/* One training step: render (Eq. 1), loss vs a_meas (MSE or L1, Eq. 3) written to
 * loss_dev[0] (device float), backward into grads, Adam (Sec. 3.1). */
nh_status train_step(nh_field* f, const nh_geometry* g, const nh_ray_batch* b, float* loss_dev,
                     void* ws, size_t ws_bytes, void* stream);
/* train_step without the optimizer: forward, loss (written to loss_dev[0]) and
 * backward, ACCUMULATING into grads, so that several batches can be accumulated
 * before one optimizer_step. When every ray has at most 16 chunks of 32 samples
 * (n_samples <= 512) this is one fused kernel (plus the ordered loss sum) per
 * call, unless a CTA's activations would exceed tensor memory (more than four
 * hidden layers with rays of more than 8 chunks); then, as for longer rays, the
 * forward, loss and backward run as separate kernels, with the same results. */
nh_status accumulate_step(nh_field* f, const nh_geometry* g, const nh_ray_batch* b, float* loss_dev,
                          void* ws, size_t ws_bytes, void* stream);
/* The same step from HOST arrays (pinned memory for asynchrony): pix_host and
 * a_meas_host are copied into the workspace, and the loss is copied back to
 * loss_host, valid once the stream has synchronized. */
nh_status train_step_host(nh_field* f, const nh_geometry* g, int32_t view, int32_t n_rays,
                          const int32_t* pix_host, const float* a_meas_host, int32_t n_samples,
                          float* loss_host, void* ws, size_t ws_bytes, void* stream);
/* Forward only: a_pred_dev[r] = sum_i mu_i delta_i (Eq. 1). */
nh_status render_forward(const nh_field* f, const nh_geometry* g, const nh_ray_batch* b,
                         float* a_pred_dev, void* ws, size_t ws_bytes, void* stream);
/* render_forward for callers that cannot allocate device memory when they call.
 * Examples: plug-ins whose host framework owns every device allocation and hands
 * out none; fixed-budget real-time loops that forbid allocation after start-up;
 * latency-critical code that cannot afford cudaMalloc's implicit device-wide
 * synchronisation. The paper has no counterpart; this is a deployment convenience.
 * Instead of a caller workspace it uses one block of device memory built into the
 * library: 1 MiB (1048576 bytes), held on every GPU that uses the library until the
 * process exits. A batch whose scratch exceeds it (about 26000 rays at 192 samples
 * per ray) returns NH_ERR_SIZE_MISMATCH; n_rays < 0 or n_samples outside 1..2^20
 * returns NH_ERR_INVALID_ARG; neither enqueues anything. It calls no allocator. The
 * first call on a device (and the first after that device's context is destroyed
 * and created again, e.g. by cudaDeviceReset) looks the block's device address up
 * with cudaGetSymbolAddress; the address is tied to the context and cached per
 * device and context ID. Make that first call before any stream capture. All calls
 * share the block and it keeps the last call's contents; every value in it is
 * written before it is read, so nothing is cleared between calls. Calls whose GPU
 * work overlaps in time (other streams or threads) race on the block and must be
 * serialized by the caller. */
nh_status render_forward_noalloc(const nh_field* f, const nh_geometry* g, const nh_ray_batch* b,
                                 float* a_pred_dev, void* stream);
/* Backward only: ACCUMULATES into grads the gradient of sum_r dLdA[r] * A_r
 * (features are recomputed, not stored). No optimizer step. */
nh_status render_backward(nh_field* f, const nh_geometry* g, const nh_ray_batch* b,
                          const float* dLdA_dev, void* ws, size_t ws_bytes, void* stream);
/* Adam with the accumulated grads, then zeroes grads, over every parameter a step
 * can reach: all entries of hashed levels, the first (N_l + 1)^3 entries of a dense
 * level (its float count rounded up to a multiple of 4) and the LN / MLP block.
 * The other entries of a dense level are never read or written by any step, so
 * their gradients and moments stay zero and Adam would leave them unchanged; the
 * optimizer skips them and leaves their values, gradients and moments as they are
 * (27 % of the vector at T = 2^19 with 16 levels from 16 to 2048). */
nh_status optimizer_step(nh_field* f, void* stream);

/* MCI pre-training step (Eq. 2): loss = mean |mu_gt - M(x)| over n_pts points
 * xyz_dev (float[3 * n_pts], normalized coordinates), written to loss_dev[0];
 * backward and Adam as in train_step. */
nh_status fit_points_step(nh_field* f, int32_t n_pts, const float* xyz_dev, const float* mu_gt_dev,
                          float* loss_dev, void* ws, size_t ws_bytes, void* stream);
/* The voxel-loss forward and backward of fit_points_step without the optimizer:
 * ACCUMULATES the gradient of the Eq. 2 loss into grads and writes the loss. */
nh_status fit_points_backward(nh_field* f, int32_t n_pts, const float* xyz_dev, const float* mu_gt_dev,
                              float* loss_dev, void* ws, size_t ws_bytes, void* stream);
/* Workspace bytes for fit_points_step / fit_points_backward. */
nh_status points_workspace_bytes(const nh_field* f, int32_t n_pts, size_t* out);

/* ------------------------------------------------------------------ evaluation
 * mu = M(x) at n points (float[3n] in, float[n] out). */
nh_status query_points(const nh_field* f, int32_t n, const float* xyz_dev, float* mu_dev, void* stream);
/* mu at the D^3 voxel centres ((k + 1/2) / D), out_dev float[D^3] in [z][y][x] order. */
nh_status query_volume(const nh_field* f, int32_t D, float* out_dev, void* stream);

/* Mean squared difference of two float arrays, accumulated in double with a fixed
 * reduction order (deterministic): out_dev[0] = (1/n) sum (a - b)^2. With data in
 * [0, 1] the reconstruction PSNR of Sec. 3.2 is 10 log10(1 / mse). ws: device
 * scratch of at least 8192 bytes (8-byte aligned). */
nh_status volume_mse(const float* a_dev, const float* b_dev, int64_t n, double* out_dev, void* ws,
                     size_t ws_bytes, void* stream);

/* 3-D structural similarity (SSIM) of two D^3 volumes, the image-quality score
 * reported beside PSNR (Sec. 3.2, Fig. 7 and 8), with the settings of the SSIM
 * paper cited there (Wang, Bovik, Sheikh and Simoncelli 2004) taken to 3-D:
 * Gaussian window of standard deviation 1.5 voxels, 11 voxels per axis,
 * normalised to sum 1; C1 = (0.01 data_range)^2, C2 = (0.03 data_range)^2; the
 * local index (2 mu_x mu_y + C1)(2 sigma_xy + C2) /
 * ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)) at each of the M^3 window
 * positions wholly inside the volume, M = D - 10.
 *   x_dev, y_dev  float[D^3], [z][y][x] order, device, read only.
 *   D             11 .. 1024.
 *   data_range    > 0 and finite (1 for volumes in [0, 1]).
 *   mean_dev      double[1], device: the mean local index (the reported score).
 *   map_dev       double[M^3] [z][y][x], device, or NULL: the local index.
 *   ws            device scratch of ssim3d_workspace_bytes(D) bytes, caller-owned,
 *                 8-byte aligned (mean_dev and map_dev too).
 * Computed in FP64 with a fixed summation order: deterministic for a given D.
 * Errors: NH_ERR_INVALID_ARG (null input, D or data_range out of range),
 * NH_ERR_ALIGNMENT, NH_ERR_SIZE_MISMATCH (workspace too small), NH_ERR_CUDA. */
nh_status ssim3d(const float* x_dev, const float* y_dev, int32_t D, double data_range, double* mean_dev,
                 double* map_dev, void* ws, size_t ws_bytes, void* stream);
/* Workspace bytes for ssim3d at D (NH_ERR_INVALID_ARG outside 11 .. 1024). */
nh_status ssim3d_workspace_bytes(int32_t D, size_t* out);

/* ------------------------------------------------------------------ data synthesis
 * Forward projection of a voxel volume (the TIGRE projections of Sec. 3.1):
 * for every view and pixel, the clipped ray is cut into
 * n = ceil((far - near) * D * oversample) equal steps and the trilinearly
 * interpolated volume (voxel centres at (k + 1/2) / D, zero outside) is summed
 * at the step midpoints times the step. vol_dev float[D^3] [z][y][x];
 * proj_dev float[n_views * det_nv * det_nu] [view][row][col]. */
nh_status project(const nh_geometry* g, const float* vol_dev, int32_t D, int32_t oversample,
                  float* proj_dev, void* stream);

/* Launch configuration of the most recent training-kernel launch in this process
 * (diagnostics, no paper counterpart): out[0..5] = SM count, CTAs per SM allowed
 * by registers and shared memory, CTAs per SM allowed by tensor memory, grid size,
 * TMEM columns per CTA, dynamic shared memory bytes per CTA. n >= 6. */
nh_status launch_info(int32_t* out, int32_t n);

/* ------------------------------------------------------------------ stage probes
 * The individual stages of the fused kernels, exposed for bitwise tests.
 * sample_rays: positions float[3 * n_rays * n_samples] ([ray][sample][xyz]) and
 * delta float[n_rays] of the ray sampler (jitter_seed as in nh_ray_batch). */
nh_status sample_rays(const nh_geometry* g, int32_t view, int32_t n_rays, const int32_t* pix_dev,
                      int32_t n_samples, uint64_t jitter_seed, float* xyz_dev, float* delta_dev, void* stream);
/* hash_corners: for n points, corner indices uint32[n][L][8] and weights float[n][L][8]. */
nh_status hash_corners(const nh_field* f, int32_t n, const float* xyz_dev, uint32_t* idx_dev,
                       float* w_dev, void* stream);
/* encode_points: trilinear hash features float[n][L * F] (the gather stage). */
nh_status encode_points(const nh_field* f, int32_t n, const float* xyz_dev, float* h_dev, void* stream);
/* scatter_points: the hash scatter stage (Sec. 2.5 backward into the tables of the
 * hash encoding): for n points xyz_dev float[n][3] with upstream gradients dh_dev
 * float[n][L * F] (16-byte aligned), adds w_k * dh[p][l F + f] into the field's
 * float32 gradient table at every corner k of every level l. Accumulates; the
 * caller zeroes the gradients when it wants a fresh sum. Addition order is not
 * fixed (atomics). */
nh_status scatter_points(nh_field* f, int32_t n, const float* xyz_dev, const float* dh_dev, void* stream);

/* ------------------------------------------------------------------ roofline probes
 * No counterpart in the paper: kernels that measure the chip's capacity for the
 * access patterns of the gather and scatter stages, to be timed by the caller with
 * CUDA events on `stream`. They compute nothing of the method.
 * probe_l2_read: `reps` sweeps of 16-byte streaming reads over buf_dev (bytes a
 *   non-zero multiple of 16, 16-byte aligned); the L2 bandwidth when the buffer
 *   fits in L2 and the first sweep is not timed apart. sink_dev: one float that
 *   is written only to keep the loads live.
 * probe_random_gather: independent uniformly random loads of entry_bytes (4 or 8)
 *   from table_dev of n_entries (a power of two <= 2^32), eight in flight per
 *   thread; *n_done (host) receives the number issued (n_loads rounded up to the
 *   launch's granularity).
 * probe_random_red: uniformly random red.global.add.v2.f32 of 1e-30 into the
 *   float2 entries of table_dev (n_entries a power of two, 8-byte aligned); the
 *   table's values change. *n_done as above.
 * probe_random_red16: the same with packed 16-bit reductions (fmt NH_PREC_BF16:
 *   bf16x2, NH_PREC_F16: f16x2) into 4-byte entries (4-byte aligned): the scatter
 *   that 16-bit gradient tables would issue. */
nh_status probe_l2_read(const void* buf_dev, uint64_t bytes, int32_t reps, float* sink_dev, void* stream);
nh_status probe_random_gather(const void* table_dev, uint64_t n_entries, int32_t entry_bytes, int64_t n_loads,
                              float* sink_dev, int64_t* n_done, void* stream);
nh_status probe_random_red(float* table_dev, uint64_t n_entries, int64_t n_ops, int64_t* n_done, void* stream);
nh_status probe_random_red16(void* table_dev, uint64_t n_entries, int32_t fmt, int64_t n_ops, int64_t* n_done,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NHCBCT_H */
