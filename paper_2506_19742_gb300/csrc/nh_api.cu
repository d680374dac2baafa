// C ABI of libnhcbct: argument validation, handles (host metadata only), workspace
// layout and the launch sequence of each entry point. No call allocates device
// memory; every device buffer comes from the caller.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nh_eval.h"
#include "nh_adam_prep.cuh"
#include "nh_internal.h"
#include "nh_mask.h"

using namespace nh;

// ----------------------------------------------------------------------------- errors
static thread_local char t_err[512];

static nh_status fail(nh_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return s;
}

static nh_status cuda_fail(cudaError_t e, const char* where) {
    return fail(NH_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define NH_CUDA(call, where)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// NVTX range over one entry point, so that a profiler timeline shows the
// library's calls around their kernels (a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define NH_RANGE(name) NvtxRange nh_range_(name)
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

extern "C" const char* nh_status_string(nh_status s) {
    switch (s) {
        case NH_OK: return "NH_OK";
        case NH_ERR_INVALID_ARG: return "NH_ERR_INVALID_ARG";
        case NH_ERR_CUDA: return "NH_ERR_CUDA";
        case NH_ERR_SIZE_MISMATCH: return "NH_ERR_SIZE_MISMATCH";
        case NH_ERR_NONFINITE: return "NH_ERR_NONFINITE";
        case NH_ERR_TIMEOUT: return "NH_ERR_TIMEOUT";
        case NH_ERR_UNSUPPORTED: return "NH_ERR_UNSUPPORTED";
        case NH_ERR_ALIGNMENT: return "NH_ERR_ALIGNMENT";
        default: return "NH_ERR_UNKNOWN";
    }
}

extern "C" nh_status nh_last_error(char* buf, size_t n) {
    if (!buf || n == 0) return NH_ERR_INVALID_ARG;
    strncpy(buf, t_err, n - 1);
    buf[n - 1] = '\0';
    return NH_OK;
}

extern "C" int32_t nh_version(void) { return 101; }

// ----------------------------------------------------------------------------- geometry
struct nh_geometry {
    nh_geometry_desc desc;
    std::vector<float> tab;   // n_views x 12
    float du, dv;
};

// Per-view constants in double, rounded once to float (the order of operations is
// part of the bitwise contract with the CPU reference).
extern "C" nh_status geometry_create(const nh_geometry_desc* d, nh_geometry** out) {
    if (!d || !out) return fail(NH_ERR_INVALID_ARG, "geometry_create: null argument");
    *out = nullptr;
    if (d->n_views < 1 || d->det_nu < 1 || d->det_nv < 1 || d->det_nu > (1 << 16) || d->det_nv > (1 << 16))
        return fail(NH_ERR_INVALID_ARG, "geometry_create: bad view or detector count");
    if (!(d->vol_side_mm > 0) || !(d->dso_mm > 0) || !(d->dsd_mm > d->dso_mm) || !(d->det_du_mm > 0) ||
        !(d->det_dv_mm > 0) || !isfinite(d->angle0_rad) || !isfinite(d->span_rad))
        return fail(NH_ERR_INVALID_ARG, "geometry_create: bad distances or pitches");
    if (d->dso_mm / d->vol_side_mm <= 0.8660254037844387)
        return fail(NH_ERR_INVALID_ARG, "geometry_create: source inside the volume's circumsphere");
    nh_geometry* g = new (std::nothrow) nh_geometry;
    if (!g) return fail(NH_ERR_INVALID_ARG, "geometry_create: out of host memory");
    g->desc = *d;
    g->tab.resize((size_t)d->n_views * 12);
    const double dso = d->dso_mm / d->vol_side_mm;
    const double dsd = d->dsd_mm / d->vol_side_mm;
    const double ddet = dsd - dso;
    for (int v = 0; v < d->n_views; v++) {
        const double theta = d->angle0_rad + ((double)v * d->span_rad) / (double)d->n_views;
        const double ct = cos(theta), st = sin(theta);
        const double row[12] = {0.5 + dso * ct, 0.5 + dso * st, 0.5, 0.5 - ddet * ct, 0.5 - ddet * st, 0.5,
                                -st, ct, 0.0, 0.0, 0.0, 1.0};
        for (int k = 0; k < 12; k++) g->tab[(size_t)v * 12 + k] = (float)row[k];
    }
    g->du = (float)(d->det_du_mm / d->vol_side_mm);
    g->dv = (float)(d->det_dv_mm / d->vol_side_mm);
    *out = g;
    return NH_OK;
}

extern "C" void geometry_destroy(nh_geometry* g) { delete g; }

extern "C" nh_status geometry_view_table(const nh_geometry* g, float* out, size_t n) {
    if (!g || !out) return fail(NH_ERR_INVALID_ARG, "geometry_view_table: null argument");
    if (n < g->tab.size() + 2) return fail(NH_ERR_SIZE_MISMATCH, "geometry_view_table: need %zu floats", g->tab.size() + 2);
    memcpy(out, g->tab.data(), g->tab.size() * sizeof(float));
    out[g->tab.size()] = g->du;
    out[g->tab.size() + 1] = g->dv;
    return NH_OK;
}

static ViewArgs view_args(const nh_geometry* g, int view, uint64_t jitter = 0) {
    ViewArgs va;
    va.jitter = jitter;
    const float* r = &g->tab[(size_t)view * 12];
    for (int k = 0; k < 3; k++) {
        va.s[k] = r[k];
        va.c[k] = r[3 + k];
        va.u[k] = r[6 + k];
        va.v[k] = r[9 + k];
    }
    va.du = g->du;
    va.dv = g->dv;
    va.nu = g->desc.det_nu;
    va.nv = g->desc.det_nv;
    return va;
}

// ----------------------------------------------------------------------------- field
struct nh_field {
    nh_field_desc desc;
    nh_field_sizes sizes;
    nh_field_buffers buf;
    FieldArgs fa;
};

static nh_status compute_layout(const nh_field_desc* d, nh_field_sizes* s, FieldArgs* fa) {
    if (!d) return fail(NH_ERR_INVALID_ARG, "field: null descriptor");
    if (d->n_levels < 1 || d->n_levels > kMaxLevels) return fail(NH_ERR_INVALID_ARG, "field: n_levels must be 1..%d", kMaxLevels);
    if (d->n_feat != 2) return fail(NH_ERR_UNSUPPORTED, "field: only n_feat = 2 is compiled in");
    const int D = d->n_levels * d->n_feat;
    if (D != 16 && D != 32) return fail(NH_ERR_UNSUPPORTED, "field: n_levels * n_feat must be 16 or 32");
    if (d->log2_T < 4 || d->log2_T > 24) return fail(NH_ERR_INVALID_ARG, "field: log2_T must be 4..24");
    if (d->base_res < 1 || d->max_res < d->base_res || d->max_res > (1 << 20))
        return fail(NH_ERR_INVALID_ARG, "field: need 1 <= base_res <= max_res <= 2^20");
    if (d->n_levels == 1 && d->max_res != d->base_res)
        return fail(NH_ERR_INVALID_ARG, "field: a single level needs base_res == max_res");
    if (d->norm < NH_NORM_NONE || d->norm > NH_NORM_LN_PER_LEVEL) return fail(NH_ERR_INVALID_ARG, "field: bad norm");
    if (!(d->ln_eps > 0)) return fail(NH_ERR_INVALID_ARG, "field: ln_eps must be > 0");
    if (d->width != 32) return fail(NH_ERR_UNSUPPORTED, "field: only width = 32 is compiled in");
    if (d->hidden_layers < 1 || d->hidden_layers > 16) return fail(NH_ERR_INVALID_ARG, "field: hidden_layers must be 1..16");
    if (d->precision < NH_PREC_F32 || d->precision > NH_PREC_F16) return fail(NH_ERR_INVALID_ARG, "field: bad precision");
    if (d->loss != NH_LOSS_MSE && d->loss != NH_LOSS_L1) return fail(NH_ERR_INVALID_ARG, "field: bad loss");
    if (!(d->lr > 0) || !(d->beta1 >= 0 && d->beta1 < 1) || !(d->beta2 >= 0 && d->beta2 < 1) || !(d->adam_eps > 0))
        return fail(NH_ERR_INVALID_ARG, "field: bad Adam hyper-parameters");
    if (!(d->loss_scale_init >= 1) || d->growth_interval < 0) return fail(NH_ERR_INVALID_ARG, "field: bad loss scale");

    const uint64_t T = 1ull << d->log2_T;
    const uint64_t W = (uint64_t)d->width, H = (uint64_t)d->hidden_layers;
    memset(s, 0, sizeof(*s));
    s->n_table_params = (uint64_t)d->n_levels * T * d->n_feat;
    s->off_gamma = s->n_table_params;
    s->off_beta = s->off_gamma + D;
    s->off_mlp = s->off_beta + D;
    uint64_t mlp = W * D + W + (H - 1) * (W * W + W) + W + 1;
    s->n_params = s->off_mlp + mlp;
    {   // backward kernels: 8 warps keep 32 H TMEM columns per thread (two lane-quarter
        // groups, at most 512 columns), and shared memory holds dense params, mask,
        // gradient accumulators and 8 warps of transpose scratch
        if (2 * 32 * H > 512)
            return fail(NH_ERR_UNSUPPORTED, "field: hidden_layers = %d exceeds the 8 that tensor memory holds",
                        d->hidden_layers);
        const uint64_t nd4 = align_up(s->n_params - s->n_table_params, 4);
        const uint64_t scratch = 32 * (W + 1) + 32 * W;
        const uint64_t bytes = 4 * (2 * nd4 + kMaxD + 8 * scratch);
        if (bytes > 227 * 1024)
            return fail(NH_ERR_UNSUPPORTED, "field: hidden_layers = %d needs %llu bytes of shared memory",
                        d->hidden_layers, (unsigned long long)bytes);
    }
    const uint64_t np4 = align_up(s->n_params, 4);   // float4 passes: pad to 4
    s->bytes_params = s->bytes_grads = s->bytes_adam_m = s->bytes_adam_v = np4 * sizeof(float);
    s->bytes_tables_lp = d->precision == NH_PREC_F32 ? 0 : s->n_table_params * 2;
    s->bytes_state = align_up(sizeof(DeviceState), 256);
    if (s->n_params > (1ull << 31)) return fail(NH_ERR_INVALID_ARG, "field: too many parameters");

    if (fa) {
        memset(fa, 0, sizeof(*fa));
        fa->L = d->n_levels;
        fa->F = d->n_feat;
        fa->log2T = d->log2_T;
        fa->Tmask = (uint32_t)(T - 1);
        fa->D = D;
        fa->H = d->hidden_layers;
        fa->W = d->width;
        fa->norm = d->norm;
        fa->eps = d->ln_eps;
        fa->n_table = (int64_t)s->n_table_params;
        fa->n_dense = (int32_t)(s->n_params - s->n_table_params);
        fa->off_beta = D;
        fa->off_mlp = 2 * D;
        fa->precision = d->precision;
        // N_l = floor(base * exp(l (ln max - ln base) / (L - 1)) + 1e-9), in double
        const double step = d->n_levels > 1
            ? (log((double)d->max_res) - log((double)d->base_res)) / (double)(d->n_levels - 1) : 0.0;
        uint32_t dm = 0;
        for (int l = 0; l < d->n_levels; l++) {
            const int res = d->n_levels > 1 ? (int)floor((double)d->base_res * exp((double)l * step) + 1e-9)
                                            : d->base_res;
            fa->res[l] = res;
            const double v = (double)(res + 1);
            if (v * v * v <= (double)T) dm |= 1u << l;
        }
        fa->dense_mask = dm;
    }
    return NH_OK;
}

extern "C" nh_status field_query_sizes(const nh_field_desc* d, nh_field_sizes* out) {
    if (!out) return fail(NH_ERR_INVALID_ARG, "field_query_sizes: null out");
    return compute_layout(d, out, nullptr);
}

extern "C" nh_status field_create(const nh_field_desc* d, const nh_field_buffers* b, nh_field** out) {
    if (!d || !b || !out) return fail(NH_ERR_INVALID_ARG, "field_create: null argument");
    *out = nullptr;
    nh_field_sizes s;
    FieldArgs fa;
    nh_status st = compute_layout(d, &s, &fa);
    if (st != NH_OK) return st;
    if (!b->params || !b->grads || !b->adam_m || !b->adam_v || !b->state)
        return fail(NH_ERR_INVALID_ARG, "field_create: params, grads, adam_m, adam_v and state are required");
    if (d->precision != NH_PREC_F32 && !b->tables_lp)
        return fail(NH_ERR_INVALID_ARG, "field_create: tables_lp is required for bf16 / f16");
    const void* ptrs[] = {b->params, b->grads, b->adam_m, b->adam_v, b->state};
    for (const void* p : ptrs)
        if (!aligned(p, 16)) return fail(NH_ERR_ALIGNMENT, "field_create: buffers must be 16-byte aligned");
    if (b->tables_lp && !aligned(b->tables_lp, 16)) return fail(NH_ERR_ALIGNMENT, "field_create: tables_lp must be 16-byte aligned");
    nh_field* f = new (std::nothrow) nh_field;
    if (!f) return fail(NH_ERR_INVALID_ARG, "field_create: out of host memory");
    f->desc = *d;
    f->sizes = s;
    f->buf = *b;
    fa.params = b->params;
    fa.tables_lp = d->precision == NH_PREC_F32 ? nullptr : b->tables_lp;
    fa.grads = b->grads;
    fa.state = (DeviceState*)b->state;
    f->fa = fa;
    *out = f;
    return NH_OK;
}

extern "C" void field_destroy(nh_field* f) { delete f; }

static cudaStream_t S(void* s) { return (cudaStream_t)s; }

extern "C" nh_status field_reset_state(nh_field* f, void* stream) {
    if (!f) return fail(NH_ERR_INVALID_ARG, "field_reset_state: null field");
    const size_t bytes = f->sizes.bytes_grads;
    NH_CUDA(cudaMemsetAsync(f->buf.grads, 0, bytes, S(stream)), "field_reset_state grads");
    NH_CUDA(cudaMemsetAsync(f->buf.adam_m, 0, bytes, S(stream)), "field_reset_state adam_m");
    NH_CUDA(cudaMemsetAsync(f->buf.adam_v, 0, bytes, S(stream)), "field_reset_state adam_v");
    NH_CUDA(launch_init_state(f->fa.state, f->desc.loss_scale_init, S(stream)), "field_reset_state state");
    NH_CUDA(launch_refresh_lowp(f->buf.params, f->buf.tables_lp, (int64_t)f->sizes.n_table_params,
                                f->desc.precision, S(stream)), "field_reset_state refresh");
    return NH_OK;
}

extern "C" nh_status field_refresh_lowp(nh_field* f, void* stream) {
    if (!f) return fail(NH_ERR_INVALID_ARG, "field_refresh_lowp: null field");
    NH_CUDA(launch_refresh_lowp(f->buf.params, f->buf.tables_lp, (int64_t)f->sizes.n_table_params,
                                f->desc.precision, S(stream)), "field_refresh_lowp");
    return NH_OK;
}

extern "C" nh_status field_set_channel_mask(nh_field* f, const float* mask, int32_t n, void* stream) {
    if (!f || !mask) return fail(NH_ERR_INVALID_ARG, "field_set_channel_mask: null argument");
    if (n != f->fa.D) return fail(NH_ERR_SIZE_MISMATCH, "field_set_channel_mask: need %d values", f->fa.D);
    NH_CUDA(cudaMemcpyAsync(f->fa.state->mask, mask, sizeof(float) * n, cudaMemcpyHostToDevice, S(stream)),
            "field_set_channel_mask");
    NH_CUDA(cudaStreamSynchronize(S(stream)), "field_set_channel_mask sync");
    return NH_OK;
}

extern "C" nh_status channel_mask_workspace_bytes(const nh_field* f, int32_t G, size_t* out) {
    if (!f || !out) return fail(NH_ERR_INVALID_ARG, "channel_mask_workspace_bytes: null argument");
    if (G < 2 || G > kMaskMaxG) return fail(NH_ERR_INVALID_ARG, "channel_mask_workspace_bytes: G must be 2..%d", kMaskMaxG);
    *out = mask_workspace_bytes(G, f->fa.D);
    return NH_OK;
}

extern "C" nh_status field_select_channel_mask(nh_field* f, int32_t G, double cutoff, double threshold,
                                               int32_t apply, double* frac_dev, float* mask_dev, void* ws,
                                               size_t ws_bytes, void* stream) {
    NH_RANGE("field_select_channel_mask");
    if (!f || !frac_dev || !ws) return fail(NH_ERR_INVALID_ARG, "field_select_channel_mask: null argument");
    if (G < 2 || G > kMaskMaxG) return fail(NH_ERR_INVALID_ARG, "field_select_channel_mask: G must be 2..%d", kMaskMaxG);
    if (!(cutoff >= 0.0) || !isfinite(cutoff) || !isfinite(threshold))
        return fail(NH_ERR_INVALID_ARG, "field_select_channel_mask: need a finite cutoff >= 0 and a finite threshold");
    if (!mask_supported(f->fa))
        return fail(NH_ERR_UNSUPPORTED, "field_select_channel_mask: built for F = 2 with L = 8 or 16");
    if (!aligned(frac_dev, 8) || !aligned(mask_dev, 4) || !aligned(ws, 256))
        return fail(NH_ERR_ALIGNMENT, "field_select_channel_mask: misaligned buffer");
    const size_t need = mask_workspace_bytes(G, f->fa.D);
    if (ws_bytes < need) return fail(NH_ERR_SIZE_MISMATCH, "field_select_channel_mask: workspace needs %zu bytes", need);
    NH_CUDA(launch_select_mask(f->fa, G, cutoff, threshold, apply, frac_dev, mask_dev, ws, S(stream)),
            "field_select_channel_mask");
    return NH_OK;
}

extern "C" nh_status field_level_resolutions(const nh_field* f, int32_t* out, int32_t n) {
    if (!f || !out) return fail(NH_ERR_INVALID_ARG, "field_level_resolutions: null argument");
    if (n < f->fa.L) return fail(NH_ERR_SIZE_MISMATCH, "field_level_resolutions: need %d entries", f->fa.L);
    for (int l = 0; l < f->fa.L; l++) out[l] = f->fa.res[l];
    return NH_OK;
}

// Parts of the flat vector: HASH = [0, n_table), LN = [off_gamma, off_mlp), MLP = [off_mlp, n_params).
struct Span { uint64_t off, n; };
static int part_spans(const nh_field* f, uint32_t parts, Span* sp) {
    int k = 0;
    if (parts & NH_PART_HASH) sp[k++] = {0, f->sizes.n_table_params};
    if (parts & NH_PART_LN) sp[k++] = {f->sizes.off_gamma, f->sizes.off_mlp - f->sizes.off_gamma};
    if (parts & NH_PART_MLP) sp[k++] = {f->sizes.off_mlp, f->sizes.n_params - f->sizes.off_mlp};
    return k;
}

extern "C" nh_status field_export_bytes(const nh_field* f, uint32_t parts, size_t* out) {
    if (!f || !out) return fail(NH_ERR_INVALID_ARG, "field_export_bytes: null argument");
    if (parts & ~0xFu) return fail(NH_ERR_INVALID_ARG, "field_export_bytes: unknown part bits");
    Span sp[3];
    const int k = part_spans(f, parts, sp);
    uint64_t n = 0;
    for (int i = 0; i < k; i++) n += sp[i].n;
    if (parts & NH_PART_ADAM) n *= 3;
    *out = (size_t)n * sizeof(float);
    return NH_OK;
}

static nh_status copy_parts(const nh_field* f, uint32_t parts, void* dev, size_t n_bytes, bool to_field,
                            void* stream) {
    size_t need = 0;
    nh_status st = field_export_bytes(f, parts, &need);
    if (st != NH_OK) return st;
    if (!dev) return fail(NH_ERR_INVALID_ARG, "field_export/import: null buffer");
    if (n_bytes < need) return fail(NH_ERR_SIZE_MISMATCH, "field_export/import: need %zu bytes", need);
    Span sp[3];
    const int k = part_spans(f, parts, sp);
    float* bufs[3] = {f->buf.params, f->buf.adam_m, f->buf.adam_v};
    const int nb = (parts & NH_PART_ADAM) ? 3 : 1;
    char* p = (char*)dev;
    for (int b = 0; b < nb; b++) {
        for (int i = 0; i < k; i++) {
            const size_t bytes = sp[i].n * sizeof(float);
            float* fld = bufs[b] + sp[i].off;
            if (to_field)
                NH_CUDA(cudaMemcpyAsync(fld, p, bytes, cudaMemcpyDeviceToDevice, S(stream)), "field_import");
            else
                NH_CUDA(cudaMemcpyAsync(p, fld, bytes, cudaMemcpyDeviceToDevice, S(stream)), "field_export");
            p += bytes;
        }
    }
    return NH_OK;
}

extern "C" nh_status field_export(const nh_field* f, uint32_t parts, void* dst, size_t n, void* stream) {
    if (!f) return fail(NH_ERR_INVALID_ARG, "field_export: null field");
    return copy_parts(f, parts, dst, n, false, stream);
}

extern "C" nh_status field_import(nh_field* f, uint32_t parts, const void* src, size_t n, void* stream) {
    if (!f) return fail(NH_ERR_INVALID_ARG, "field_import: null field");
    nh_status st = copy_parts(f, parts, (void*)src, n, true, stream);
    if (st != NH_OK) return st;
    if (parts & NH_PART_HASH)
        NH_CUDA(launch_refresh_lowp(f->buf.params, f->buf.tables_lp, (int64_t)f->sizes.n_table_params,
                                    f->desc.precision, S(stream)), "field_import refresh");
    return NH_OK;
}

extern "C" nh_status field_poll_status(nh_field* f, void* stream, uint32_t* flags, float* scale, int32_t* step) {
    if (!f) return fail(NH_ERR_INVALID_ARG, "field_poll_status: null field");
    DeviceState h;
    NH_CUDA(cudaStreamSynchronize(S(stream)), "field_poll_status sync");
    NH_CUDA(cudaMemcpy(&h, f->fa.state, 64, cudaMemcpyDeviceToHost), "field_poll_status copy");
    if (flags) *flags = h.last_flags | h.flags;
    if (scale) *scale = h.loss_scale;
    if (step) *step = h.step;
    return NH_OK;
}

// ----------------------------------------------------------------------------- workspace
struct RayWs {
    int32_t* pix;
    float* a_meas;
    float* ray_part;
    float* a_pred;
    float* dLdA;
    float* loss;
    float* loss_part;   // per-CTA loss partials of the fused step
    size_t bytes;
};

static RayWs ray_ws(void* base, int R, int N) {
    const int C = (N + 31) / 32;
    RayWs w;
    size_t o = 0;
    char* b = (char*)base;
    w.pix = (int32_t*)(b + o); o = align_up(o + sizeof(int32_t) * (size_t)R, 256);
    w.a_meas = (float*)(b + o); o = align_up(o + sizeof(float) * (size_t)R, 256);
    w.ray_part = (float*)(b + o); o = align_up(o + sizeof(float) * (size_t)R * C, 256);
    w.a_pred = (float*)(b + o); o = align_up(o + sizeof(float) * (size_t)R, 256);
    w.dLdA = (float*)(b + o); o = align_up(o + sizeof(float) * (size_t)R, 256);
    w.loss = (float*)(b + o); o = align_up(o + sizeof(float) * 4, 256);
    w.loss_part = (float*)(b + o); o = align_up(o + sizeof(float) * kTrainParts, 256);
    w.bytes = o;
    return w;
}

extern "C" nh_status step_workspace_bytes(const nh_field* f, int32_t R, int32_t N, size_t* out) {
    if (!f || !out) return fail(NH_ERR_INVALID_ARG, "step_workspace_bytes: null argument");
    if (R < 0 || N < 1) return fail(NH_ERR_INVALID_ARG, "step_workspace_bytes: need n_rays >= 0, n_samples >= 1");
    *out = ray_ws(nullptr, R, N).bytes;
    return NH_OK;
}

extern "C" nh_status points_workspace_bytes(const nh_field* f, int32_t n, size_t* out) {
    if (!f || !out) return fail(NH_ERR_INVALID_ARG, "points_workspace_bytes: null argument");
    if (n < 0) return fail(NH_ERR_INVALID_ARG, "points_workspace_bytes: n < 0");
    *out = align_up(sizeof(float) * (size_t)points_partials(n), 256);
    return NH_OK;
}

static nh_status check_batch(const nh_field* f, const nh_geometry* g, const nh_ray_batch* b, void* ws,
                             size_t ws_bytes, bool need_meas, const char* who) {
    if (!f || !g || !b) return fail(NH_ERR_INVALID_ARG, "%s: null handle or batch", who);
    if (b->view < 0 || b->view >= g->desc.n_views) return fail(NH_ERR_INVALID_ARG, "%s: view out of range", who);
    if (b->n_rays < 0 || b->n_samples < 1 || b->n_samples > (1 << 20))
        return fail(NH_ERR_INVALID_ARG, "%s: need n_rays >= 0 and 1 <= n_samples <= 2^20", who);
    if (b->n_rays > 0 && !b->pix) return fail(NH_ERR_INVALID_ARG, "%s: null pix", who);
    if (need_meas && b->n_rays > 0 && !b->a_meas) return fail(NH_ERR_INVALID_ARG, "%s: null a_meas", who);
    if (!aligned(b->pix, 4) || !aligned(b->a_meas, 4)) return fail(NH_ERR_ALIGNMENT, "%s: batch arrays must be 4-byte aligned", who);
    const size_t need = ray_ws(nullptr, b->n_rays, b->n_samples).bytes;
    if (!ws) return fail(NH_ERR_INVALID_ARG, "%s: null workspace", who);
    if (!aligned(ws, 256)) return fail(NH_ERR_ALIGNMENT, "%s: workspace must be 256-byte aligned", who);
    if (ws_bytes < need) return fail(NH_ERR_SIZE_MISMATCH, "%s: workspace needs %zu bytes", who, need);
    return NH_OK;
}

// Forward, loss and backward of one batch, accumulating into grads (R > 0). With
// hyper (an optimizer step follows) the fused path's loss kernel also runs Adam's
// prologue, and *prologue_done is set so that the optimizer launches k_adam alone.
static nh_status run_accumulate(nh_field* f, const nh_geometry* g, int view, int R, const int32_t* pix,
                                const float* a_meas, int N, uint64_t jitter, float* loss_dev, const RayWs& w,
                                cudaStream_t st, const AdamHyper* hyper = nullptr, bool* prologue_done = nullptr) {
    const ViewArgs va = view_args(g, view, jitter);
    const int C = (N + 31) / 32;
    // whole rays fit a CTA: one fused forward + loss + backward kernel; it declines
    // (launching nothing) where a CTA's activations exceed tensor memory
    const cudaError_t fe = C <= kMaxFusedChunks
        ? launch_ray_train(f->fa, va, pix, a_meas, R, N, f->desc.loss, w.loss_part, loss_dev, hyper, st)
        : cudaErrorNotSupported;
    if (fe != cudaErrorNotSupported) {
        NH_CUDA(fe, "train_step fused");
        if (prologue_done) *prologue_done = hyper != nullptr;
    } else {
        NH_CUDA(launch_ray_forward(f->fa, va, pix, R, N, w.ray_part, st), "train_step forward");
        NH_CUDA(launch_ray_loss(w.ray_part, R, C, a_meas, f->desc.loss, w.a_pred, w.dLdA, loss_dev, f->fa.state,
                                true, st), "train_step loss");
        NH_CUDA(launch_ray_backward(f->fa, va, pix, R, N, w.dLdA, st), "train_step backward");
    }
    return NH_OK;
}

static nh_status run_train(nh_field* f, const nh_geometry* g, int view, int R, const int32_t* pix,
                           const float* a_meas, int N, uint64_t jitter, float* loss_dev, const RayWs& w,
                           cudaStream_t st) {
    if (R == 0) {   // empty batch: loss 0, no update
        if (loss_dev) NH_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), st), "train_step");
        return NH_OK;
    }
    const AdamHyper hyper{f->desc.lr, f->desc.beta1, f->desc.beta2, f->desc.growth_interval};
    bool prologue_done = false;
    const nh_status s = run_accumulate(f, g, view, R, pix, a_meas, N, jitter, loss_dev, w, st, &hyper,
                                       &prologue_done);
    if (s != NH_OK) return s;
    NH_CUDA(launch_adam(f->fa, f->buf.params, f->buf.grads, f->buf.adam_m, f->buf.adam_v,
                        (int64_t)align_up(f->sizes.n_params, 4), f->desc.lr, f->desc.beta1, f->desc.beta2,
                        f->desc.adam_eps, f->desc.growth_interval, st, !prologue_done), "train_step adam");
    return NH_OK;
}

extern "C" nh_status accumulate_step(nh_field* f, const nh_geometry* g, const nh_ray_batch* b, float* loss_dev,
                                     void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("accumulate_step");
    nh_status s = check_batch(f, g, b, ws, ws_bytes, true, "accumulate_step");
    if (s != NH_OK) return s;
    if (b->n_rays == 0) {
        if (loss_dev) NH_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), S(stream)), "accumulate_step");
        return NH_OK;
    }
    const RayWs w = ray_ws(ws, b->n_rays, b->n_samples);
    return run_accumulate(f, g, b->view, b->n_rays, b->pix, b->a_meas, b->n_samples, b->jitter_seed, loss_dev, w,
                          S(stream));
}

extern "C" nh_status train_step(nh_field* f, const nh_geometry* g, const nh_ray_batch* b, float* loss_dev,
                                void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("train_step");
    nh_status s = check_batch(f, g, b, ws, ws_bytes, true, "train_step");
    if (s != NH_OK) return s;
    const RayWs w = ray_ws(ws, b->n_rays, b->n_samples);
    return run_train(f, g, b->view, b->n_rays, b->pix, b->a_meas, b->n_samples, b->jitter_seed, loss_dev, w,
                     S(stream));
}

extern "C" nh_status train_step_host(nh_field* f, const nh_geometry* g, int32_t view, int32_t R,
                                     const int32_t* pix_host, const float* a_meas_host, int32_t N,
                                     float* loss_host, void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("train_step_host");
    nh_ray_batch b{view, R, pix_host, a_meas_host, N};
    nh_status s = check_batch(f, g, &b, ws, ws_bytes, true, "train_step_host");
    if (s != NH_OK) return s;
    if (!loss_host) return fail(NH_ERR_INVALID_ARG, "train_step_host: null loss_host");
    const RayWs w = ray_ws(ws, R, N);
    cudaStream_t st = S(stream);
    if (R > 0) {
        NH_CUDA(cudaMemcpyAsync(w.pix, pix_host, sizeof(int32_t) * R, cudaMemcpyHostToDevice, st), "train_step_host pix");
        NH_CUDA(cudaMemcpyAsync(w.a_meas, a_meas_host, sizeof(float) * R, cudaMemcpyHostToDevice, st), "train_step_host a_meas");
    }
    s = run_train(f, g, view, R, w.pix, w.a_meas, N, 0, w.loss, w, st);
    if (s != NH_OK) return s;
    NH_CUDA(cudaMemcpyAsync(loss_host, w.loss, sizeof(float), cudaMemcpyDeviceToHost, st), "train_step_host loss");
    return NH_OK;
}

extern "C" nh_status render_forward(const nh_field* f, const nh_geometry* g, const nh_ray_batch* b, float* a_pred,
                                    void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("render_forward");
    nh_status s = check_batch(f, g, b, ws, ws_bytes, false, "render_forward");
    if (s != NH_OK) return s;
    if (b->n_rays == 0) return NH_OK;
    if (!a_pred) return fail(NH_ERR_INVALID_ARG, "render_forward: null a_pred");
    const RayWs w = ray_ws(ws, b->n_rays, b->n_samples);
    const ViewArgs va = view_args(g, b->view, b->jitter_seed);
    const int C = (b->n_samples + 31) / 32;
    NH_CUDA(launch_ray_forward(f->fa, va, b->pix, b->n_rays, b->n_samples, w.ray_part, S(stream)), "render_forward");
    NH_CUDA(launch_ray_loss(w.ray_part, b->n_rays, C, nullptr, f->desc.loss, a_pred, nullptr, nullptr, f->fa.state,
                            false, S(stream)), "render_forward sum");
    return NH_OK;
}

extern "C" nh_status render_backward(nh_field* f, const nh_geometry* g, const nh_ray_batch* b, const float* dLdA,
                                     void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("render_backward");
    nh_status s = check_batch(f, g, b, ws, ws_bytes, false, "render_backward");
    if (s != NH_OK) return s;
    if (b->n_rays == 0) return NH_OK;
    if (!dLdA) return fail(NH_ERR_INVALID_ARG, "render_backward: null dLdA");
    const ViewArgs va = view_args(g, b->view, b->jitter_seed);
    NH_CUDA(launch_ray_backward(f->fa, va, b->pix, b->n_rays, b->n_samples, dLdA, S(stream)), "render_backward");
    return NH_OK;
}

extern "C" nh_status optimizer_step(nh_field* f, void* stream) {
    NH_RANGE("optimizer_step");
    if (!f) return fail(NH_ERR_INVALID_ARG, "optimizer_step: null field");
    NH_CUDA(launch_adam(f->fa, f->buf.params, f->buf.grads, f->buf.adam_m, f->buf.adam_v,
                        (int64_t)align_up(f->sizes.n_params, 4), f->desc.lr, f->desc.beta1, f->desc.beta2,
                        f->desc.adam_eps, f->desc.growth_interval, S(stream)), "optimizer_step");
    return NH_OK;
}

static nh_status run_fit(nh_field* f, int32_t n, const float* xyz, const float* mu_gt, float* loss_dev,
                         void* ws, size_t ws_bytes, void* stream, const char* who) {
    if (!f) return fail(NH_ERR_INVALID_ARG, "%s: null field", who);
    if (n < 0) return fail(NH_ERR_INVALID_ARG, "%s: n_pts < 0", who);
    if (n == 0) {
        if (loss_dev) NH_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), S(stream)), who);
        return NH_OK;
    }
    if (!xyz || !mu_gt) return fail(NH_ERR_INVALID_ARG, "%s: null points", who);
    if (!aligned(xyz, 4) || !aligned(mu_gt, 4)) return fail(NH_ERR_ALIGNMENT, "%s: misaligned points", who);
    size_t need = 0;
    points_workspace_bytes(f, n, &need);
    if (!ws) return fail(NH_ERR_INVALID_ARG, "%s: null workspace", who);
    if (!aligned(ws, 256)) return fail(NH_ERR_ALIGNMENT, "%s: workspace must be 256-byte aligned", who);
    if (ws_bytes < need) return fail(NH_ERR_SIZE_MISMATCH, "%s: workspace needs %zu bytes", who, need);
    NH_CUDA(launch_points(f->fa, n, xyz, mu_gt, nullptr, (float*)ws, points_partials(n), loss_dev, S(stream)),
            who);
    return NH_OK;
}

extern "C" nh_status fit_points_backward(nh_field* f, int32_t n, const float* xyz, const float* mu_gt,
                                         float* loss_dev, void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("fit_points_backward");
    return run_fit(f, n, xyz, mu_gt, loss_dev, ws, ws_bytes, stream, "fit_points_backward");
}

extern "C" nh_status fit_points_step(nh_field* f, int32_t n, const float* xyz, const float* mu_gt, float* loss_dev,
                                     void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("fit_points_step");
    nh_status s = run_fit(f, n, xyz, mu_gt, loss_dev, ws, ws_bytes, stream, "fit_points_step");
    if (s != NH_OK || n == 0) return s;
    NH_CUDA(launch_adam(f->fa, f->buf.params, f->buf.grads, f->buf.adam_m, f->buf.adam_v,
                        (int64_t)align_up(f->sizes.n_params, 4), f->desc.lr, f->desc.beta1, f->desc.beta2,
                        f->desc.adam_eps, f->desc.growth_interval, S(stream)), "fit_points_step adam");
    return NH_OK;
}

extern "C" nh_status query_points(const nh_field* f, int32_t n, const float* xyz, float* mu, void* stream) {
    NH_RANGE("query_points");
    if (!f) return fail(NH_ERR_INVALID_ARG, "query_points: null field");
    if (n < 0) return fail(NH_ERR_INVALID_ARG, "query_points: n < 0");
    if (n == 0) return NH_OK;
    if (!xyz || !mu) return fail(NH_ERR_INVALID_ARG, "query_points: null buffer");
    NH_CUDA(launch_points(f->fa, n, xyz, nullptr, mu, nullptr, 0, nullptr, S(stream)), "query_points");
    return NH_OK;
}

extern "C" nh_status query_volume(const nh_field* f, int32_t D, float* out, void* stream) {
    NH_RANGE("query_volume");
    if (!f || !out) return fail(NH_ERR_INVALID_ARG, "query_volume: null argument");
    if (D < 1 || D > 2048) return fail(NH_ERR_INVALID_ARG, "query_volume: D must be 1..2048");
    NH_CUDA(launch_query_volume(f->fa, D, out, S(stream)), "query_volume");
    return NH_OK;
}

extern "C" nh_status project(const nh_geometry* g, const float* vol, int32_t D, int32_t os, float* proj, void* stream) {
    NH_RANGE("project");
    if (!g || !vol || !proj) return fail(NH_ERR_INVALID_ARG, "project: null argument");
    if (D < 1 || D > 4096 || os < 1 || os > 64) return fail(NH_ERR_INVALID_ARG, "project: need 1 <= D <= 4096, 1 <= oversample <= 64");
    if (!aligned(vol, 4) || !aligned(proj, 4)) return fail(NH_ERR_ALIGNMENT, "project: misaligned buffer");
    for (int v = 0; v < g->desc.n_views; v++)
        NH_CUDA(launch_project(view_args(g, v), v, vol, D, os, proj, S(stream)), "project");
    return NH_OK;
}

extern "C" nh_status sample_rays(const nh_geometry* g, int32_t view, int32_t R, const int32_t* pix, int32_t N,
                                 uint64_t jitter_seed, float* xyz, float* delta, void* stream) {
    if (!g || (R > 0 && (!pix || !xyz || !delta))) return fail(NH_ERR_INVALID_ARG, "sample_rays: null argument");
    if (view < 0 || view >= g->desc.n_views || R < 0 || N < 1) return fail(NH_ERR_INVALID_ARG, "sample_rays: bad sizes");
    NH_CUDA(launch_sample_rays(view_args(g, view, jitter_seed), pix, R, N, xyz, delta, S(stream)), "sample_rays");
    return NH_OK;
}

extern "C" nh_status hash_corners(const nh_field* f, int32_t n, const float* xyz, uint32_t* idx, float* w,
                                  void* stream) {
    if (!f || (n > 0 && (!xyz || !idx || !w))) return fail(NH_ERR_INVALID_ARG, "hash_corners: null argument");
    if (n < 0) return fail(NH_ERR_INVALID_ARG, "hash_corners: n < 0");
    NH_CUDA(launch_hash_corners(f->fa, n, xyz, idx, w, S(stream)), "hash_corners");
    return NH_OK;
}

extern "C" nh_status encode_points(const nh_field* f, int32_t n, const float* xyz, float* h, void* stream) {
    if (!f || (n > 0 && (!xyz || !h))) return fail(NH_ERR_INVALID_ARG, "encode_points: null argument");
    if (n < 0) return fail(NH_ERR_INVALID_ARG, "encode_points: n < 0");
    NH_CUDA(launch_encode_points(f->fa, n, xyz, h, S(stream)), "encode_points");
    return NH_OK;
}

extern "C" nh_status scatter_points(nh_field* f, int32_t n, const float* xyz, const float* dh, void* stream) {
    if (!f || (n > 0 && (!xyz || !dh))) return fail(NH_ERR_INVALID_ARG, "scatter_points: null argument");
    if (n < 0) return fail(NH_ERR_INVALID_ARG, "scatter_points: n < 0");
    if (!aligned(dh, 16)) return fail(NH_ERR_ALIGNMENT, "scatter_points: dh must be 16-byte aligned");
    NH_CUDA(launch_scatter_points(f->fa, n, xyz, dh, S(stream)), "scatter_points");
    return NH_OK;
}

static bool pow2(uint64_t v) { return v != 0 && (v & (v - 1)) == 0; }

extern "C" nh_status probe_l2_read(const void* buf, uint64_t bytes, int32_t reps, float* sink, void* stream) {
    if (!buf || !sink) return fail(NH_ERR_INVALID_ARG, "probe_l2_read: null argument");
    if (reps < 1 || bytes == 0 || bytes % 16 != 0)
        return fail(NH_ERR_INVALID_ARG, "probe_l2_read: need reps >= 1 and a non-zero multiple of 16 bytes");
    if (!aligned(buf, 16)) return fail(NH_ERR_ALIGNMENT, "probe_l2_read: buffer must be 16-byte aligned");
    NH_CUDA(launch_probe_l2_read(buf, bytes, reps, sink, S(stream)), "probe_l2_read");
    return NH_OK;
}

extern "C" nh_status probe_random_gather(const void* table, uint64_t n_entries, int32_t entry_bytes, int64_t n_loads,
                                         float* sink, int64_t* n_done, void* stream) {
    if (!table || !sink || !n_done) return fail(NH_ERR_INVALID_ARG, "probe_random_gather: null argument");
    if (!pow2(n_entries) || n_entries > (uint64_t(1) << 32) || (entry_bytes != 4 && entry_bytes != 8) || n_loads < 0)
        return fail(NH_ERR_INVALID_ARG, "probe_random_gather: n_entries a power of two <= 2^32, entry_bytes 4 or 8");
    if (!aligned(table, (size_t)entry_bytes)) return fail(NH_ERR_ALIGNMENT, "probe_random_gather: misaligned table");
    NH_CUDA(launch_probe_random_gather(table, n_entries, entry_bytes, n_loads, sink, n_done, S(stream)),
            "probe_random_gather");
    return NH_OK;
}

extern "C" nh_status probe_random_red(float* table, uint64_t n_entries, int64_t n_ops, int64_t* n_done, void* stream) {
    if (!table || !n_done) return fail(NH_ERR_INVALID_ARG, "probe_random_red: null argument");
    if (!pow2(n_entries) || n_entries > (uint64_t(1) << 32) || n_ops < 0)
        return fail(NH_ERR_INVALID_ARG, "probe_random_red: n_entries a power of two <= 2^32");
    if (!aligned(table, 8)) return fail(NH_ERR_ALIGNMENT, "probe_random_red: table must be 8-byte aligned");
    NH_CUDA(launch_probe_random_red(table, n_entries, n_ops, n_done, S(stream)), "probe_random_red");
    return NH_OK;
}

extern "C" nh_status probe_random_red16(void* table, uint64_t n_entries, int32_t fmt, int64_t n_ops,
                                        int64_t* n_done, void* stream) {
    if (!table || !n_done) return fail(NH_ERR_INVALID_ARG, "probe_random_red16: null argument");
    if (!pow2(n_entries) || n_entries > (uint64_t(1) << 32) || n_ops < 0 || (fmt != NH_PREC_BF16 && fmt != NH_PREC_F16))
        return fail(NH_ERR_INVALID_ARG, "probe_random_red16: n_entries a power of two <= 2^32, fmt BF16 or F16");
    if (!aligned(table, 4)) return fail(NH_ERR_ALIGNMENT, "probe_random_red16: table must be 4-byte aligned");
    NH_CUDA(launch_probe_random_red16(table, n_entries, fmt, n_ops, n_done, S(stream)), "probe_random_red16");
    return NH_OK;
}

extern "C" nh_status volume_mse(const float* a, const float* b, int64_t n, double* out_dev, void* ws,
                                size_t ws_bytes, void* stream) {
    NH_RANGE("volume_mse");
    if (!a || !b || !out_dev || !ws) return fail(NH_ERR_INVALID_ARG, "volume_mse: null argument");
    if (n < 1) return fail(NH_ERR_INVALID_ARG, "volume_mse: n < 1");
    if (!aligned(ws, 8) || !aligned(out_dev, 8)) return fail(NH_ERR_ALIGNMENT, "volume_mse: misaligned buffer");
    if (ws_bytes < mse_workspace_bytes()) return fail(NH_ERR_SIZE_MISMATCH, "volume_mse: workspace needs %zu bytes",
                                                      mse_workspace_bytes());
    NH_CUDA(launch_mse(a, b, n, out_dev, ws, S(stream)), "volume_mse");
    return NH_OK;
}

extern "C" nh_status ssim3d_workspace_bytes(int32_t D, size_t* out) {
    if (!out) return fail(NH_ERR_INVALID_ARG, "ssim3d_workspace_bytes: null argument");
    if (D < 2 * kSsimRadius + 1 || D > kSsimMaxD)
        return fail(NH_ERR_INVALID_ARG, "ssim3d_workspace_bytes: D must be %d..%d", 2 * kSsimRadius + 1, kSsimMaxD);
    *out = ssim_workspace_bytes(D);
    return NH_OK;
}

extern "C" nh_status ssim3d(const float* x, const float* y, int32_t D, double data_range, double* mean_dev,
                            double* map_dev, void* ws, size_t ws_bytes, void* stream) {
    NH_RANGE("ssim3d");
    if (!x || !y || !mean_dev || !ws) return fail(NH_ERR_INVALID_ARG, "ssim3d: null argument");
    if (D < 2 * kSsimRadius + 1 || D > kSsimMaxD)
        return fail(NH_ERR_INVALID_ARG, "ssim3d: D must be %d..%d", 2 * kSsimRadius + 1, kSsimMaxD);
    if (!(data_range > 0.0) || !isfinite(data_range))
        return fail(NH_ERR_INVALID_ARG, "ssim3d: data_range must be positive and finite");
    if (!aligned(ws, 8) || !aligned(mean_dev, 8) || (map_dev && !aligned(map_dev, 8)))
        return fail(NH_ERR_ALIGNMENT, "ssim3d: misaligned buffer");
    if (ws_bytes < ssim_workspace_bytes(D))
        return fail(NH_ERR_SIZE_MISMATCH, "ssim3d: workspace needs %zu bytes", ssim_workspace_bytes(D));
    NH_CUDA(launch_ssim3d(x, y, D, data_range, mean_dev, map_dev, ws, S(stream)), "ssim3d");
    return NH_OK;
}

extern "C" nh_status launch_info(int32_t* out, int32_t n) {
    if (!out || n < 6) return fail(NH_ERR_INVALID_ARG, "launch_info: need 6 entries");
    last_train_grid(out);
    return NH_OK;
}

// ----------------------------------------------------------------------------- fixed-scratch forward
// render_forward_noalloc takes its scratch from this fixed block of device memory
// instead of a caller workspace. The block is part of the library image: every GPU
// on which the library is used holds it until the process exits. In host code the
// name g_fixed_ws only stands for the variable; its device address is looked up
// with cudaGetSymbolAddress, with the device current, once per device and context.
// A context torn down and created again (cudaDeviceReset) loads the module again,
// and the block may then sit at another address, so the cached address is keyed to
// the context's unique ID and looked up afresh when that ID changes.
constexpr size_t kFixedWsBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_fixed_ws[kFixedWsBytes];

namespace {
struct FixedSlot {
    unsigned long long ctx_id;   // context the address belongs to (0: none yet)
    void* ptr;
};
// Driver calls reached through the runtime's entry-point table, so the library
// needs no link against libcuda.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
}  // namespace

static std::mutex g_fixed_mu;
static FixedSlot g_fixed[64];
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;
static bool g_ctx_fns_looked_up = false;

// ID of the calling thread's current context, or 0 when it cannot be had.
static unsigned long long current_context_id() {
    if (!g_ctx_fns_looked_up) {
        g_ctx_fns_looked_up = true;
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess) {
            g_ctx_current = (CtxGetCurrentFn)a;
            g_ctx_id = (CtxGetIdFn)b;
        }
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

static nh_status fixed_workspace(void** out) {
    int dev = 0;
    NH_CUDA(cudaGetDevice(&dev), "render_forward_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(NH_ERR_UNSUPPORTED, "render_forward_noalloc: device ordinal %d >= 64", dev);
    std::lock_guard<std::mutex> lock(g_fixed_mu);
    const unsigned long long id = current_context_id();
    FixedSlot& slot = g_fixed[dev];
    if (!slot.ptr || id == 0 || slot.ctx_id != id) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_ws);
        if (e != cudaSuccess) return cuda_fail(e, "render_forward_noalloc: cudaGetSymbolAddress");
        // The lookup makes the device's primary context current if it was not yet.
        slot.ctx_id = id != 0 ? id : current_context_id();
        slot.ptr = p;
    }
    *out = slot.ptr;
    return NH_OK;
}

extern "C" nh_status render_forward_noalloc(const nh_field* f, const nh_geometry* g, const nh_ray_batch* b,
                                            float* a_pred, void* stream) {
    if (!f || !g || !b) return fail(NH_ERR_INVALID_ARG, "render_forward_noalloc: null handle or batch");
    if (b->n_rays < 0 || b->n_samples < 1 || b->n_samples > (1 << 20))
        return fail(NH_ERR_INVALID_ARG, "render_forward_noalloc: need n_rays >= 0 and 1 <= n_samples <= 2^20");
    const size_t need = ray_ws(nullptr, b->n_rays, b->n_samples).bytes;
    if (need > kFixedWsBytes)
        return fail(NH_ERR_SIZE_MISMATCH,
                    "render_forward_noalloc: %d rays x %d samples need %zu bytes of scratch, the fixed block "
                    "holds %zu; use render_forward with a caller workspace",
                    b->n_rays, b->n_samples, need, kFixedWsBytes);
    void* ws = nullptr;
    const nh_status s = fixed_workspace(&ws);
    if (s != NH_OK) return s;
    return render_forward(f, g, b, a_pred, ws, kFixedWsBytes, stream);
}
