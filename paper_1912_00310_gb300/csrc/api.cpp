// api.cpp -- the C ABI (include/llg.h): contexts, parameter setup, ensemble state, engine
// selection and host/device marshalling.  All arithmetic of a step runs in the CUDA engines.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "../../include/llg.h"
#include "llg_internal.h"

struct llg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nx = 0, ny = 0, nz = 0, b = 1;
    unsigned periodic = 0;
    double a0 = 0.0;
    bool has_material = false, has_sweep = false;
    llg::MaterialIn mat{};
    llg::ScalingIn sc{1, 858.0, 0.511, 1.0, 1.0, 1.0};
    llg::SweepIn sw{};
    double volume = 0.0;  // cell volume override (0: (b a0)^3)
    double disp = 0.0;    // easy-axis dispersion: cone half-angle (rad) about z, 0 = axis z
    float4 *d_axis = nullptr;  // [n_real][ncells] easy axes when disp > 0
    size_t axis_cap = 0;       // float4 entries
    bool axis_ok = false;      // d_axis holds the axes of (ax_seed, ax_real0, ax_n, ax_disp)
    uint32_t ax_seed = 0, ax_real0 = 0;
    int ax_n = 0;
    double ax_disp = 0.0;
    int engine = LLG_ENGINE_AUTO;
    int tune_kind = 0, tune_rods = 0, tune_rows = 0, tune_generic = 0, tune_balance = 1, tune_cpt = 0;
    long long adjoint_state_mb = 16384;  // budget for the adjoint's stored window states
    int grad_method = 0;                 // 0 reverse-mode adjoint, 1 forward-mode tangents
    long long chunk_steps = 1LL << 20;
    long long handoff_timeout_ms = 30000;  // balanced resident schedule: longest hand-off wait
    int withhold_handoff = 0;              // test hook: the hand-offs are never released
    // ensemble
    int n_real = 0;
    uint32_t seed = 0, real0 = 0;
    long long step = 0;
    float *d_m = nullptr;        // [n_real][ncells][3]
    size_t m_cap = 0;            // floats
    float *d_scratch = nullptr;  // plain engine: mt, acc, hth
    size_t scratch_cap = 0;
    float *d_samples = nullptr;  // staging for host sample buffers
    size_t samples_cap = 0;
    int *d_status = nullptr;
    unsigned *d_flags = nullptr;  // resident engine: hand-off flags of the balanced schedule
    size_t flags_cap = 0;
    float *d_slab = nullptr;      // streaming engine: two float4 ping-pong buffers + partial sums
    size_t slab_cap = 0;          // floats
    long long launches = 0;
};

namespace {

thread_local char g_err[512] = "";

llg_status fail(llg_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

llg_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(LLG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LLG_CUDA(call, what)                        \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

long long ncells_of(const llg_ctx *c) { return (long long)c->nx * c->ny * c->nz; }

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

llg_status derived_of(const llg_ctx *c, llg::Derived *d)
{
    if (!c->has_material) return fail(LLG_EINVAL, "material not set (llg_set_material)");
    if (!c->has_sweep) return fail(LLG_EINVAL, "sweep not set (llg_set_sweep)");
    char err[256];
    if (!llg::derive(c->b, c->a0, c->mat, c->sc, c->sw, d, err, sizeof err, c->volume)) return fail(LLG_EINVAL, "%s", err);
    return LLG_OK;
}

llg_status grow(float **buf, size_t *cap, size_t need_floats)
{
    if (*cap >= need_floats) return LLG_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(buf, need_floats * sizeof(float));
    if (e != cudaSuccess) {
        *buf = nullptr;
        cudaGetLastError();
        return fail(LLG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", need_floats * sizeof(float),
                    cudaGetErrorString(e));
    }
    *cap = need_floats;
    return LLG_OK;
}

// The easy axes of the ensemble in the dispersed-axis mode, drawn on the context's stream when
// the ensemble's keys or the dispersion changed; *out = NULL in the z-axis mode.
llg_status ensure_axes(llg_ctx *c, const float4 **out)
{
    *out = nullptr;
    if (!(c->disp > 0.0)) return LLG_OK;
    if (c->n_real < 1) return fail(LLG_EINVAL, "no ensemble (llg_reset first)");
    if (c->axis_ok && c->ax_seed == c->seed && c->ax_real0 == c->real0 && c->ax_n == c->n_real &&
        c->ax_disp == c->disp) {
        *out = c->d_axis;
        return LLG_OK;
    }
    const size_t need = (size_t)c->n_real * (size_t)ncells_of(c);
    if (c->axis_cap < need) {
        cudaFree(c->d_axis);
        c->d_axis = nullptr;
        c->axis_cap = 0;
        cudaError_t e = cudaMalloc(&c->d_axis, need * sizeof(float4));
        if (e != cudaSuccess) {
            c->d_axis = nullptr;
            cudaGetLastError();
            return fail(LLG_ENOMEM, "cudaMalloc of %zu bytes (easy axes) failed", need * sizeof(float4));
        }
        c->axis_cap = need;
    }
    const float w_max = (float)(1.0 - std::cos(c->disp));
    LLG_CUDA(llg::axis_fill(c->d_axis, c->n_real, (int)ncells_of(c), c->seed, c->real0, w_max, c->stream),
             "easy-axis draw");
    c->axis_ok = true;
    c->ax_seed = c->seed;
    c->ax_real0 = c->real0;
    c->ax_n = c->n_real;
    c->ax_disp = c->disp;
    *out = c->d_axis;
    return LLG_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int resolve_engine(const llg_ctx *c, const llg::KParams &kp, int n_real, llg::RodPlan *plan,
                   llg::SlabPlan *splan)
{
    const bool rod_ok =
        llg::rod_plan(kp, n_real, c->device, plan, c->tune_kind, c->tune_rods, c->tune_rows, c->tune_cpt);
    plan->generic = c->tune_generic != 0;
    plan->balance = c->tune_balance != 0;
    plan->handoff_timeout_ns = (unsigned long long)c->handoff_timeout_ms * 1000000ull;
    plan->withhold_handoff = c->withhold_handoff != 0;
    llg::SlabPlan tmp;
    const bool slab_ok = llg::slab_plan(kp, c->device, splan ? splan : &tmp);
    switch (c->engine) {
        case LLG_ENGINE_RESIDENT:
            return rod_ok ? LLG_ENGINE_RESIDENT : -1;
        case LLG_ENGINE_PLAIN:
            return LLG_ENGINE_PLAIN;
        case LLG_ENGINE_STREAM:
            return slab_ok ? LLG_ENGINE_STREAM : -1;
        default:
            return rod_ok ? LLG_ENGINE_RESIDENT : (slab_ok ? LLG_ENGINE_STREAM : LLG_ENGINE_PLAIN);
    }
}

}  // namespace

namespace llg {
void set_last_error(const char *msg) { std::snprintf(g_err, sizeof g_err, "%s", msg); }

llg_status ctx_view(llg_ctx *c, CtxView *v)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    Derived d;
    const llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    if (c->n_real > 0 && c->flags_cap < (size_t)c->n_real) {
        DeviceGuard g(c->device);
        cudaFree(c->d_flags);
        c->d_flags = nullptr;
        c->flags_cap = 0;
        LLG_CUDA(cudaMalloc(&c->d_flags, sizeof(unsigned) * (size_t)c->n_real), "cudaMalloc(flags)");
        c->flags_cap = (size_t)c->n_real;
    }
    v->device = c->device;
    v->stream = c->stream;
    v->n_real = c->n_real;
    v->d_m = c->d_m;
    v->d_status = c->d_status;
    v->d_flags = c->d_flags;
    v->step = c->step;
    v->steps_per_loop = d.steps_per_loop;
    v->kp = kparams_of(d, c->nx, c->ny, c->nz, c->periodic, c->sw.dt);
    v->kp.seed = c->seed;
    v->kp.real0 = c->real0;
    if (c->n_real > 0) {
        DeviceGuard g(c->device);
        const llg_status sa = ensure_axes(c, &v->kp.axis);
        if (sa != LLG_OK) return sa;
    }
    v->tune_kind = c->tune_kind;
    v->tune_rods = c->tune_rods;
    v->tune_rows = c->tune_rows;
    v->tune_generic = c->tune_generic != 0;
    v->tune_cpt = c->tune_cpt;
    v->chunk_steps = c->chunk_steps;
    return LLG_OK;
}

void ctx_add_steps(llg_ctx *c, long long n) { c->step += n; }

llg_status kparams_from_ctx(const llg_ctx *c, KParams *out)
{
    Derived d;
    const llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    if (c->disp > 0.0) return fail(LLG_EUNSUPPORTED, "the dispersed-axis mode keeps its axes in the context");
    *out = kparams_of(d, c->nx, c->ny, c->nz, c->periodic, c->sw.dt);
    return LLG_OK;
}

int ctx_device(const llg_ctx *c) { return c->device; }
}  // namespace llg

extern "C" {

const char *llg_last_error(void) { return g_err; }

llg_status llg_create_grid(llg_ctx **out, int nx, int ny, int nz, double a0_m, int b,
                           unsigned periodic_mask, int device, void *cuda_stream)
{
    if (!out) return fail(LLG_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(LLG_EINVAL, "grid sizes must be positive");
    if ((long long)nx * ny * nz > (1LL << 31)) return fail(LLG_EINVAL, "more than 2^31 cells");
    if (!(a0_m > 0.0) || b < 1) return fail(LLG_EINVAL, "a0 must be > 0 and b >= 1");
    if (periodic_mask > 7u) return fail(LLG_EINVAL, "periodic_mask uses bits 0-2 only");
    // The device is only checked when a driver is present, so that parameter setup and the
    // host-side queries also work on a machine without a GPU; the first call that needs the
    // GPU (llg_reset) reports ECUDA there.
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess) {
        if (device < 0 || device >= ndev)
            return fail(LLG_EINVAL, "device %d out of range (%d devices)", device, ndev);
    } else {
        cudaGetLastError();
        if (device < 0) return fail(LLG_EINVAL, "device must be >= 0");
    }
    llg_ctx *c = new (std::nothrow) llg_ctx();
    if (!c) return fail(LLG_ENOMEM, "context allocation failed");
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->a0 = a0_m;
    c->b = b;
    c->periodic = periodic_mask;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return LLG_OK;
}

void llg_destroy(llg_ctx *c)
{
    if (!c) return;
    if (!c->d_status && !c->d_m && !c->d_flags && !c->d_axis) {  // nothing was ever put on the device
        delete c;
        return;
    }
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_m);
    cudaFree(c->d_scratch);
    cudaFree(c->d_samples);
    cudaFree(c->d_status);
    cudaFree(c->d_flags);
    cudaFree(c->d_slab);
    cudaFree(c->d_axis);
    cudaGetLastError();
    delete c;
}

llg_status llg_set_stream(llg_ctx *c, void *cuda_stream)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    c->stream = (cudaStream_t)cuda_stream;
    return LLG_OK;
}

llg_status llg_set_material(llg_ctx *c, double A0, double Ms, double K0, const double u[3],
                            double alpha, double T)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (!(Ms > 0.0) || !(alpha >= 0.0) || !(T >= 0.0) || !(A0 >= 0.0) || !std::isfinite(K0))
        return fail(LLG_EINVAL, "need Ms > 0, alpha >= 0, T >= 0, A0 >= 0, finite K0");
    if (u) {
        const double n = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (!(n > 0.0)) return fail(LLG_EINVAL, "easy axis has zero length");
        if (std::fabs(u[0]) > 1e-12 * n || std::fabs(u[1]) > 1e-12 * n)
            return fail(LLG_EUNSUPPORTED, "only an easy axis along z is built (a dispersed axis: llg_set_axis_dispersion)");
    }
    c->mat = llg::MaterialIn{A0, Ms, K0, alpha, T};
    c->has_material = true;
    return LLG_OK;
}

llg_status llg_set_scaling(llg_ctx *c, int mode, double Tc, double delta, const double scale[3])
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (mode < 0 || mode > 2) return fail(LLG_EINVAL, "scaling mode must be 0, 1 or 2");
    if (!(Tc > 0.0)) return fail(LLG_EINVAL, "Tc must be > 0");
    double s[3] = {1.0, 1.0, 1.0};
    if (scale)
        for (int i = 0; i < 3; ++i) s[i] = scale[i];
    for (double v : s)
        if (!(v > 0.0) || !std::isfinite(v)) return fail(LLG_EINVAL, "scale factors must be > 0");
    c->sc = llg::ScalingIn{mode, Tc, delta, s[0], s[1], s[2]};
    return LLG_OK;
}

llg_status llg_set_sweep(llg_ctx *c, double H_start_Oe, double H_turn_Oe, double rate, double dt_s,
                         double sample_dH_Oe, int shape)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (shape != 0 && shape != 1) return fail(LLG_EINVAL, "shape must be 0 (triangle) or 1 (sinusoid)");
    if (!(dt_s > 0.0) || !(rate >= 0.0) || !(sample_dH_Oe > 0.0) || !std::isfinite(H_start_Oe) ||
        !std::isfinite(H_turn_Oe))
        return fail(LLG_EINVAL, "need dt > 0, rate >= 0, sample spacing > 0");
    llg::SweepIn sw{H_start_Oe, H_turn_Oe, rate, dt_s, sample_dH_Oe, shape};
    // validate now so that errors surface at the call that caused them
    const llg::MaterialIn mat = c->has_material ? c->mat : llg::MaterialIn{1e-11, 1e5, 0.0, 0.1, 0.0};
    llg::Derived d;
    char err[256];
    if (!llg::derive(c->b, c->a0, mat, c->sc, sw, &d, err, sizeof err, c->volume)) return fail(LLG_EINVAL, "%s", err);
    c->sw = sw;
    c->has_sweep = true;
    return LLG_OK;
}

llg_status llg_set_held_samples(llg_ctx *c, int64_t n_samples)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (n_samples < 1) return fail(LLG_EINVAL, "n_samples must be >= 1");
    if (!c->has_sweep) return fail(LLG_EINVAL, "sweep not set (llg_set_sweep)");
    llg::Derived d;
    llg::SweepIn sw = c->sw;
    sw.held_samples = n_samples;
    const llg::MaterialIn mat = c->has_material ? c->mat : llg::MaterialIn{1e-11, 1e5, 0.0, 0.1, 0.0};
    char err[256];
    if (!llg::derive(c->b, c->a0, mat, c->sc, sw, &d, err, sizeof err, c->volume)) return fail(LLG_EINVAL, "%s", err);
    if (d.steps_per_loop != 0) return fail(LLG_EINVAL, "a sample count is set only for a held (constant) field");
    c->sw.held_samples = n_samples;
    return LLG_OK;
}

llg_status llg_set_cell_volume(llg_ctx *c, double volume_m3)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (!(volume_m3 >= 0.0) || !std::isfinite(volume_m3)) return fail(LLG_EINVAL, "volume must be >= 0");
    c->volume = volume_m3;
    return LLG_OK;
}

llg_status llg_gk_flow(double Tstar0, double h0, double g0, double b, int64_t n_steps, double out[4])
{
    if (!out) return fail(LLG_EINVAL, "out is NULL");
    if (!(b >= 1.0) || n_steps < 1 || !(Tstar0 >= 0.0) || !(h0 >= 0.0) || !(g0 >= 0.0))
        return fail(LLG_EINVAL, "need b >= 1, n_steps >= 1 and non-negative T*, h, g");
    llg::gk_flow(Tstar0, h0, g0, b, n_steps, out);
    return LLG_OK;
}

llg_status llg_set_axis_dispersion(llg_ctx *c, double half_angle_rad)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (!(half_angle_rad >= 0.0) || !(half_angle_rad <= 0.5 * 3.141592653589793))
        return fail(LLG_EINVAL, "the dispersion half-angle must lie in [0, pi/2]");
    c->disp = half_angle_rad;
    return LLG_OK;
}

llg_status llg_get_axes(llg_ctx *c, float *u)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (!u) return fail(LLG_EINVAL, "u is NULL");
    if (c->n_real < 1 || !c->d_m) return fail(LLG_EINVAL, "no ensemble (llg_reset first)");
    DeviceGuard g(c->device);
    const size_t n = (size_t)c->n_real * (size_t)ncells_of(c);
    const float4 *ax = nullptr;
    llg_status s = ensure_axes(c, &ax);
    if (s != LLG_OK) return s;
    const bool dev = is_device_ptr(u);
    if (!ax) {  // z-axis mode
        if (dev) {
            LLG_CUDA(cudaMemsetAsync(u, 0, n * 3 * sizeof(float), c->stream), "cudaMemsetAsync(u)");
            LLG_CUDA(llg::fill_column(u, (int)n, 3, 2, 1.0f, c->stream), "fill +z");
        } else {
            for (size_t i = 0; i < n; ++i) {
                u[3 * i] = 0.f;
                u[3 * i + 1] = 0.f;
                u[3 * i + 2] = 1.f;
            }
        }
        return LLG_OK;
    }
    // float4 -> float3 rows through a strided 2-D copy
    LLG_CUDA(cudaMemcpy2DAsync(u, 3 * sizeof(float), ax, sizeof(float4), 3 * sizeof(float), n,
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
             "axis copy");
    if (!dev) LLG_CUDA(cudaStreamSynchronize(c->stream), "axis copy");
    return LLG_OK;
}

llg_status llg_set_engine(llg_ctx *c, int engine)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (engine < LLG_ENGINE_AUTO || engine > LLG_ENGINE_STREAM) return fail(LLG_EINVAL, "unknown engine %d", engine);
    c->engine = engine;
    return LLG_OK;
}

llg_status llg_set_tuning(llg_ctx *c, int key, int64_t value)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (value < 0) return fail(LLG_EINVAL, "tuning values must be >= 0");
    switch (key) {
        case LLG_TUNE_ROD_KIND:
            if (value > 3) return fail(LLG_EINVAL, "rod kernel kind must be 0, 1, 2 or 3");
            c->tune_kind = (int)value;
            return LLG_OK;
        case LLG_TUNE_RODS_PER_CTA:
            if (value > 4096) return fail(LLG_EINVAL, "rods per CTA too large");
            c->tune_rods = (int)value;
            return LLG_OK;
        case LLG_TUNE_ROWS_PER_THREAD:
            if (value > 4) return fail(LLG_EINVAL, "rows per thread must be 0..4");
            c->tune_rows = (int)value;
            return LLG_OK;
        case LLG_TUNE_GENERIC_KERNEL:
            c->tune_generic = value != 0;
            return LLG_OK;
        case LLG_TUNE_BALANCE:
            c->tune_balance = value != 0;
            return LLG_OK;
        case LLG_TUNE_ADJOINT_STATE_MB:
            if (value > (1LL << 22)) return fail(LLG_EINVAL, "at most 4 TB for the adjoint's states");
            c->adjoint_state_mb = value;
            return LLG_OK;
        case LLG_TUNE_CELLS_PER_THREAD:
            if (value != 0 && value != 1 && value != 2 && value != 4)
                return fail(LLG_EINVAL, "cells per thread must be 0 (automatic), 1, 2 or 4");
            c->tune_cpt = (int)value;
            return LLG_OK;
        case LLG_TUNE_GRAD_METHOD:
            if (value > 1) return fail(LLG_EINVAL, "gradient method must be 0 (adjoint) or 1 (tangent)");
            c->grad_method = (int)value;
            return LLG_OK;
        case LLG_TUNE_HANDOFF_TIMEOUT_MS:
            if (value < 1 || value > 3600000) return fail(LLG_EINVAL, "hand-off timeout must be 1 ms .. 1 h");
            c->handoff_timeout_ms = value;
            return LLG_OK;
        case LLG_TUNE_WITHHOLD_HANDOFF:
            c->withhold_handoff = value != 0;
            return LLG_OK;
        case LLG_TUNE_CHUNK_STEPS:
            if (value > (1LL << 30)) return fail(LLG_EINVAL, "at most 2^30 steps per launch");
            c->chunk_steps = value > 0 ? value : (1LL << 20);
            return LLG_OK;
        default:
            return fail(LLG_EINVAL, "unknown tuning key %d", key);
    }
}

llg_status llg_get_tuning(const llg_ctx *c, int key, int64_t *value)
{
    if (!c || !value) return fail(LLG_EINVAL, "NULL argument");
    switch (key) {
        case LLG_TUNE_ROD_KIND: *value = c->tune_kind; return LLG_OK;
        case LLG_TUNE_RODS_PER_CTA: *value = c->tune_rods; return LLG_OK;
        case LLG_TUNE_CHUNK_STEPS: *value = c->chunk_steps; return LLG_OK;
        case LLG_TUNE_ROWS_PER_THREAD: *value = c->tune_rows; return LLG_OK;
        case LLG_TUNE_GENERIC_KERNEL: *value = c->tune_generic; return LLG_OK;
        case LLG_TUNE_BALANCE: *value = c->tune_balance; return LLG_OK;
        case LLG_TUNE_ADJOINT_STATE_MB: *value = c->adjoint_state_mb; return LLG_OK;
        case LLG_TUNE_HANDOFF_TIMEOUT_MS: *value = c->handoff_timeout_ms; return LLG_OK;
        case LLG_TUNE_WITHHOLD_HANDOFF: *value = c->withhold_handoff; return LLG_OK;
        case LLG_TUNE_CELLS_PER_THREAD: *value = c->tune_cpt; return LLG_OK;
        case LLG_TUNE_GRAD_METHOD: *value = c->grad_method; return LLG_OK;
        default: return fail(LLG_EINVAL, "unknown tuning key %d", key);
    }
}

llg_status llg_reset(llg_ctx *c, uint32_t seed, int n_real, uint32_t real_offset)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (n_real < 1) return fail(LLG_EINVAL, "n_real must be >= 1");
    llg::Derived d;
    llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    DeviceGuard g(c->device);
    if (!c->d_status) LLG_CUDA(cudaMalloc(&c->d_status, sizeof(int)), "cudaMalloc(status)");
    const size_t n = (size_t)n_real * (size_t)ncells_of(c) * 3;
    s = grow(&c->d_m, &c->m_cap, n);
    if (s != LLG_OK) return s;
    // m = +z everywhere: fill the z components through the column helper (row stride 3)
    LLG_CUDA(cudaMemsetAsync(c->d_m, 0, n * sizeof(float), c->stream), "cudaMemsetAsync(m)");
    LLG_CUDA(llg::fill_column(c->d_m, (int)(n / 3), 3, 2, 1.0f, c->stream), "fill +z");
    LLG_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "cudaMemsetAsync(status)");
    c->n_real = n_real;
    c->seed = seed;
    c->real0 = real_offset;
    c->step = 0;
    return LLG_OK;
}

llg_status llg_advance(llg_ctx *c, int64_t n_steps, float *m_samples)
{
    llg::NvtxRange nvtx("llg_advance");
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (c->n_real < 1 || !c->d_m) return fail(LLG_EINVAL, "no ensemble (llg_reset first)");
    if (n_steps < 0) return fail(LLG_EINVAL, "n_steps must be >= 0");
    if (m_samples && !is_device_ptr(m_samples)) return fail(LLG_EINVAL, "m_samples must be device memory");
    llg::Derived d;
    llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    DeviceGuard g(c->device);
    llg::KParams kp = llg::kparams_of(d, c->nx, c->ny, c->nz, c->periodic, c->sw.dt);
    kp.seed = c->seed;
    kp.real0 = c->real0;
    s = ensure_axes(c, &kp.axis);
    if (s != LLG_OK) return s;
    llg::RodPlan plan{};
    llg::SlabPlan splan{};
    const int eng = resolve_engine(c, kp, c->n_real, &plan, &splan);
    if (eng < 0) return fail(LLG_EUNSUPPORTED, "the selected engine cannot hold a %dx%dx%d grid", c->nx, c->ny, c->nz);
    if (eng == LLG_ENGINE_RESIDENT) {
        if (c->flags_cap < (size_t)c->n_real) {
            cudaFree(c->d_flags);
            c->d_flags = nullptr;
            c->flags_cap = 0;
            LLG_CUDA(cudaMalloc(&c->d_flags, sizeof(unsigned) * (size_t)c->n_real), "cudaMalloc(flags)");
            c->flags_cap = (size_t)c->n_real;
        }
        const long long chunk = c->chunk_steps;
        for (long long done = 0; done < n_steps; done += chunk) {
            const long long k = n_steps - done < chunk ? n_steps - done : chunk;
            LLG_CUDA(llg::rod_advance(kp, plan, c->d_m, c->n_real, c->step + done, k, m_samples,
                                      c->d_status, c->d_flags, c->stream),
                     "resident engine launch");
            ++c->launches;
        }
    } else if (eng == LLG_ENGINE_STREAM) {
        const size_t padded = llg::slab_state_float4s(kp, c->n_real);
        const size_t need = 8 * padded + llg::slab_partial_floats(c->n_real);
        s = grow(&c->d_slab, &c->slab_cap, need);
        if (s != LLG_OK) return s;
        float4 *a = reinterpret_cast<float4 *>(c->d_slab);
        float4 *b = a + padded;
        LLG_CUDA(llg::slab_advance(kp, splan, c->d_m, c->n_real, c->step, n_steps, m_samples, c->d_status, a, b,
                                   c->d_slab + 8 * padded, c->stream, &c->launches),
                 "streaming engine launch");
    } else {
        const size_t per = (size_t)c->n_real * (size_t)ncells_of(c) * 3;
        s = grow(&c->d_scratch, &c->scratch_cap, 3 * per);
        if (s != LLG_OK) return s;
        LLG_CUDA(llg::plain_advance(kp, c->d_m, c->d_scratch, c->d_scratch + per, c->d_scratch + 2 * per,
                                    c->n_real, c->step, n_steps, m_samples, c->d_status, c->stream,
                                    &c->launches),
                 "plain engine launch");
    }
    c->step += n_steps;
    return LLG_OK;
}

llg_status llg_sync(llg_ctx *c, double timeout_s)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    DeviceGuard g(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "stream");
        if (timeout_s > 0.0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) return fail(LLG_ETIMEOUT, "stream still busy after %.3f s", el);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int st = 0;
    if (!c->d_status) return LLG_OK;
    LLG_CUDA(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (st & 2) return fail(LLG_ETIMEOUT, "a resident-engine hand-off wait gave up");
    if (st & 4) return fail(LLG_ETIMEOUT, "a streaming-engine staging wait gave up");
    if (st) return fail(LLG_ENONFINITE, "a non-finite magnetisation was sampled");
    return LLG_OK;
}

llg_status llg_run_loops(llg_ctx *c, uint32_t seed, int n_real, uint32_t real_offset, float *m_samples,
                         llg_loop_stats *stats)
{
    llg::NvtxRange nvtx("llg_run_loops");
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (!m_samples) return fail(LLG_EINVAL, "m_samples is required");
    llg::Derived d;
    llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    if (d.steps_per_loop <= 0) return fail(LLG_EINVAL, "a loop needs a swept field (rate > 0)");
    s = llg_reset(c, seed, n_real, real_offset);
    if (s != LLG_OK) return s;
    DeviceGuard g(c->device);
    const bool dev = is_device_ptr(m_samples);
    float *dst = m_samples;
    const size_t ns = (size_t)n_real * (size_t)d.n_samples;
    if (!dev) {
        s = grow(&c->d_samples, &c->samples_cap, ns);
        if (s != LLG_OK) return s;
        dst = c->d_samples;
    }
    LLG_CUDA(llg::fill_column(dst, n_real, d.n_samples, 0, 1.0f, c->stream), "sample 0");
    s = llg_advance(c, d.steps_per_loop, dst);
    if (s != LLG_OK) return s;
    if (!dev) {
        LLG_CUDA(cudaMemcpyAsync(m_samples, dst, ns * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
                 "samples to host");
    }
    if (stats || !dev) {
        s = llg_sync(c, 0.0);
        if (s != LLG_OK) return s;
    }
    if (stats) {
        std::vector<float> host;
        const float *hs = m_samples;
        if (dev) {
            host.resize(ns);
            LLG_CUDA(cudaMemcpy(host.data(), m_samples, ns * sizeof(float), cudaMemcpyDeviceToHost), "samples");
            hs = host.data();
        }
        std::vector<double> H((size_t)d.n_samples);
        s = llg_sample_fields(c, H.data());
        if (s != LLG_OK) return s;
        s = llg_loop_stats_host(hs, n_real, d.n_samples, H.data(), d.n_half / d.sample_every, c->sc.mode,
                                d.zeta, c->sc.delta, stats, nullptr);
        if (s != LLG_OK) return fail(s, "loop statistics failed");
    }
    return LLG_OK;
}

llg_status llg_get_state(llg_ctx *c, float *m, int64_t *step)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (c->n_real < 1) return fail(LLG_EINVAL, "no ensemble");
    if (step) *step = c->step;
    if (!m) return LLG_OK;
    DeviceGuard g(c->device);
    const size_t bytes = (size_t)c->n_real * (size_t)ncells_of(c) * 3 * sizeof(float);
    const bool dev = is_device_ptr(m);
    LLG_CUDA(cudaMemcpyAsync(m, c->d_m, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
             "state copy out");
    if (!dev) LLG_CUDA(cudaStreamSynchronize(c->stream), "state copy out");
    return LLG_OK;
}

llg_status llg_set_state(llg_ctx *c, const float *m, int64_t step)
{
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (c->n_real < 1) return fail(LLG_EINVAL, "no ensemble (llg_reset first)");
    if (!m || step < 0) return fail(LLG_EINVAL, "need a state and step >= 0");
    DeviceGuard g(c->device);
    const size_t bytes = (size_t)c->n_real * (size_t)ncells_of(c) * 3 * sizeof(float);
    const bool dev = is_device_ptr(m);
    LLG_CUDA(cudaMemcpyAsync(c->d_m, m, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
             "state copy in");
    if (!dev) LLG_CUDA(cudaStreamSynchronize(c->stream), "state copy in");
    c->step = step;
    return LLG_OK;
}

// Loss of the window's mean loop and its weights dL/dmbar_k (objective 0: mismatch against
// target; 1: signed trapezoid area), from the realisation means mbar of samples k_first ...
static double window_loss(const llg::Derived &d, const llg::SweepIn &sw, int objective, const double *target,
                          long long k_first, long long K, const std::vector<double> &mbar, std::vector<double> &wk)
{
    const long long se = d.sample_every;
    std::vector<double> Hk((size_t)K);
    for (long long k = 0; k < K; ++k) Hk[(size_t)k] = llg::field_Oe(d, sw, (k_first + k) * se);
    wk.assign((size_t)K, 0.0);
    double L = 0.0;
    if (objective == 0) {
        for (long long k = 0; k < K; ++k) {
            const double err = mbar[(size_t)k] - target[k_first + k];
            L += err * err / (double)K;
            wk[(size_t)k] = 2.0 * err / (double)K;
        }
    } else {
        for (long long k = 0; k + 1 < K; ++k) {
            const double dH = Hk[(size_t)k + 1] - Hk[(size_t)k];
            L += 0.5 * (mbar[(size_t)k] + mbar[(size_t)k + 1]) * dH;
            wk[(size_t)k] += 0.5 * dH;
            wk[(size_t)k + 1] += 0.5 * dH;
        }
    }
    return L;
}

// The forward-mode method: one pass carrying dm/d(s_K, s_alpha, s_Ms) (k_tangent.cu), the
// derivatives of the simulation coefficients taken here in FP64.
static llg_status tangent_grad(llg_ctx *c, const llg::Derived &d, const llg::KParams &kp, long long N, int objective,
                               const double *target, long long k_first, long long K, size_t state, double *loss_out,
                               double grad_out[3])
{
    if (!llg::tangent_supported(kp, c->device))
        return fail(LLG_EUNSUPPORTED, "the tangent method handles rods of at most 1408 cells with free faces");
    if (K > 0x7fffffffLL) return fail(LLG_EINVAL, "too many samples in the window");
    const double sK = c->sc.sK, sA = c->sc.sAlpha, sM = c->sc.sMs;
    const double alpha = d.alpha, a = c->sw.dt * d.g1;
    const double dcoef[15] = {0.0, 0.0, -d.c_ex / sM,                                  // c_ex
                              d.c_an / sK, 0.0, -d.c_an / sM,                          // c_an
                              0.0, alpha / sA, 0.0,                                    // alpha
                              0.0, -2.0 * alpha * a / (1.0 + alpha * alpha) * alpha / sA, 0.0,  // a
                              0.0, 0.5 / sA, -0.5 / sM};                               // dsigma / sigma
    float *work = nullptr, *smp = nullptr, *dsmp = nullptr;
    cudaError_t e = cudaMalloc(&work, sizeof(float) * state);
    if (e == cudaSuccess) e = cudaMalloc(&smp, sizeof(float) * (size_t)c->n_real * (size_t)K);
    if (e == cudaSuccess) e = cudaMalloc(&dsmp, sizeof(float) * 3 * (size_t)c->n_real * (size_t)K);
    auto cleanup = [&]() {
        cudaFree(work);
        cudaFree(smp);
        cudaFree(dsmp);
    };
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(LLG_ENOMEM, "tangent buffers: %s", cudaGetErrorString(e));
    }
    const cudaStream_t st = c->stream;
    std::vector<float> hs((size_t)c->n_real * (size_t)K), hd(3 * hs.size());
    e = cudaMemcpyAsync(work, c->d_m, sizeof(float) * state, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = llg::tangent_forward(kp, dcoef, c->n_real, c->step, N, k_first, (int)K, work, smp, dsmp, c->d_status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), smp, sizeof(float) * hs.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), dsmp, sizeof(float) * hd.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "tangent pass");
    std::vector<double> mbar((size_t)K, 0.0), wk;
    double dm[3] = {0.0, 0.0, 0.0};
    std::vector<double> dmb((size_t)K * 3, 0.0);
    for (long long k = 0; k < K; ++k)
        for (int r = 0; r < c->n_real; ++r) {
            const size_t i = (size_t)r * (size_t)K + (size_t)k;
            mbar[(size_t)k] += hs[i];
            for (int j = 0; j < 3; ++j) dmb[(size_t)k * 3 + j] += hd[3 * i + j];
        }
    for (long long k = 0; k < K; ++k) {
        mbar[(size_t)k] /= c->n_real;
        for (int j = 0; j < 3; ++j) dmb[(size_t)k * 3 + j] /= c->n_real;
    }
    const double L = window_loss(d, c->sw, objective, target, k_first, K, mbar, wk);
    for (long long k = 0; k < K; ++k)
        for (int j = 0; j < 3; ++j) dm[j] += wk[(size_t)k] * dmb[(size_t)k * 3 + j];
    for (int j = 0; j < 3; ++j) grad_out[j] = dm[j];
    if (loss_out) *loss_out = L;
    return LLG_OK;
}

llg_status llg_loop_area_grad(llg_ctx *c, int64_t n_steps, int objective, const double *target,
                              int64_t ckpt_every, double *loss_out, double grad_out[3])
{
    llg::NvtxRange nvtx("llg_loop_area_grad");
    if (!c) return fail(LLG_EINVAL, "ctx is NULL");
    if (c->n_real < 1 || !c->d_m) return fail(LLG_EINVAL, "no ensemble (llg_reset first)");
    if (n_steps < 1 || ckpt_every < 1 || ckpt_every > (1 << 20)) return fail(LLG_EINVAL, "need n_steps >= 1, 1 <= ckpt_every <= 2^20");
    if (objective != 0 && objective != 1) return fail(LLG_EINVAL, "objective must be 0 (mismatch) or 1 (area)");
    if (objective == 0 && !target) return fail(LLG_EINVAL, "the mismatch objective needs a target");
    llg::Derived d;
    llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    DeviceGuard g(c->device);
    llg::KParams kp = llg::kparams_of(d, c->nx, c->ny, c->nz, c->periodic, c->sw.dt);
    kp.seed = c->seed;
    kp.real0 = c->real0;
    s = ensure_axes(c, &kp.axis);
    if (s != LLG_OK) return s;
    const long long step0 = c->step, N = n_steps, C = ckpt_every;
    const long long S = (N + C - 1) / C;
    const long long se = d.sample_every;
    const long long k_first = step0 / se + 1, k_last = (step0 + N) / se;
    const long long K = k_last >= k_first ? k_last - k_first + 1 : 0;
    if (K < 1) return fail(LLG_EINVAL, "the window holds no sample");
    if (k_last >= d.n_samples && d.n_half > 0) return fail(LLG_EINVAL, "the window runs past the end of the loop");
    const size_t state = (size_t)c->n_real * (size_t)ncells_of(c) * 3;
    if (c->grad_method == 1) return tangent_grad(c, d, kp, n_steps, objective, target, k_first, K, state, loss_out,
                                                 grad_out);
    if (!llg::adjoint_supported(kp, c->device))
        return fail(LLG_EUNSUPPORTED, "the adjoint handles rods of at most 1024 cells with free faces");
    llg::RodPlan plan{};
    if (!llg::rod_plan(kp, c->n_real, c->device, &plan, 1, 0, 0))
        return fail(LLG_EUNSUPPORTED, "no resident forward plan for this grid");
    const long long ns_total = std::max<long long>(d.n_samples, k_last + 1);
    // store the whole window's states when they fit the budget and a quarter of the free memory
    bool store_all = false;
    {
        const double bytes = (double)sizeof(float) * (double)state * (double)N;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = 0;
        }
        store_all = S <= 65535 && N <= 0x7fffffffLL && bytes <= (double)c->adjoint_state_mb * 1048576.0 &&
                    bytes <= 0.25 * (double)free_b;
    }
    float *ckpt = nullptr, *seg = nullptr, *lam = nullptr, *work = nullptr, *smp = nullptr;
    double *w = nullptr, *partial = nullptr;
    auto cleanup = [&]() {
        cudaFree(ckpt);
        cudaFree(seg);
        cudaFree(lam);
        cudaFree(work);
        cudaFree(smp);
        cudaFree(w);
        cudaFree(partial);
    };
    cudaError_t e = cudaMalloc(&ckpt, sizeof(float) * state * (size_t)S);
    if (e == cudaSuccess && store_all && cudaMalloc(&seg, sizeof(float) * state * (size_t)N) != cudaSuccess) {
        cudaGetLastError();  // no room for the whole window: reverse segment by segment
        seg = nullptr;
        store_all = false;
    }
    if (e == cudaSuccess && !store_all) e = cudaMalloc(&seg, sizeof(float) * state * (size_t)std::min(C, N));
    if (e == cudaSuccess) e = cudaMalloc(&lam, sizeof(float) * state);
    if (e == cudaSuccess) e = cudaMalloc(&work, sizeof(float) * state);
    if (e == cudaSuccess) e = cudaMalloc(&smp, sizeof(float) * (size_t)c->n_real * (size_t)ns_total);
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * (size_t)K);
    if (e == cudaSuccess) e = cudaMalloc(&partial, sizeof(double) * 5 * (size_t)c->n_real);
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(LLG_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
    }
    llg::KParams kps = kp;
    kps.n_samples = ns_total;
    const cudaStream_t st = c->stream;
    // forward pass with a checkpoint at the start of every segment
    e = cudaMemcpyAsync(work, c->d_m, sizeof(float) * state, cudaMemcpyDeviceToDevice, st);
    for (long long sg = 0; sg < S && e == cudaSuccess; ++sg) {
        e = cudaMemcpyAsync(ckpt + (size_t)sg * state, work, sizeof(float) * state, cudaMemcpyDeviceToDevice, st);
        const long long len = std::min(C, N - sg * C);
        if (e == cudaSuccess)
            e = llg::rod_advance(kps, plan, work, c->n_real, step0 + sg * C, len, smp, c->d_status, nullptr, st);
    }
    std::vector<float> hs((size_t)c->n_real * (size_t)ns_total);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.data(), smp, sizeof(float) * hs.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "adjoint forward");
    }
    // loss and its weights on the realisation-mean samples
    std::vector<double> mbar((size_t)K, 0.0), wk;
    for (long long k = 0; k < K; ++k) {
        double sum = 0.0;
        for (int r = 0; r < c->n_real; ++r) sum += hs[(size_t)r * ns_total + (size_t)(k_first + k)];
        mbar[(size_t)k] = sum / c->n_real;
    }
    const double L = window_loss(d, c->sw, objective, target, k_first, K, mbar, wk);
    e = cudaMemcpyAsync(w, wk.data(), sizeof(double) * (size_t)K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(lam, 0, sizeof(float) * state, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(partial, 0, sizeof(double) * 5 * (size_t)c->n_real, st);
    if (store_all) {
        if (e == cudaSuccess) e = llg::adjoint_recompute_all(kps, c->n_real, step0, N, (int)C, ckpt, seg, st);
        if (e == cudaSuccess)
            e = llg::adjoint_backward_all(kps, c->n_real, step0, N, k_first, (int)K, seg, lam, w, partial, st);
    } else {
        for (long long sg = S - 1; sg >= 0 && e == cudaSuccess; --sg) {
            const long long len = std::min(C, N - sg * C);
            e = llg::adjoint_segment(kps, c->n_real, step0 + sg * C, (int)len, step0 + N, k_first, (int)K,
                                     ckpt + (size_t)sg * state, seg, lam, w, partial, st);
        }
    }
    std::vector<double> hp((size_t)c->n_real * 5);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint backward");
    double gs[5] = {0, 0, 0, 0, 0};
    for (int r = 0; r < c->n_real; ++r)
        for (int k = 0; k < 5; ++k) gs[k] += hp[(size_t)r * 5 + k];
    // chain rule to the scale factors: alpha = alpha0 s_alpha (in the torque, in a = dt g1 with
    // g1 = g0/(1 + alpha^2), and in sigma ~ sqrt(alpha / Ms)); c_ex ~ 1/s_Ms; c_an ~ s_K/s_Ms
    const double alpha = d.alpha, a = c->sw.dt * d.g1;
    const double da_dalpha = -2.0 * alpha * a / (1.0 + alpha * alpha);
    const double sK = c->sc.sK, sA = c->sc.sAlpha, sM = c->sc.sMs;
    grad_out[0] = gs[3] * d.c_an / sK;
    grad_out[1] = (gs[0] + gs[1] * da_dalpha) * (alpha / sA) + gs[4] / (2.0 * sA);
    grad_out[2] = -(gs[2] * d.c_ex + gs[3] * d.c_an) / sM - gs[4] / (2.0 * sM);
    if (loss_out) *loss_out = L;
    return LLG_OK;
}

int64_t llg_num_cells(const llg_ctx *c) { return c ? ncells_of(c) : -1; }

int64_t llg_num_samples(const llg_ctx *c)
{
    llg::Derived d;
    if (!c || derived_of(c, &d) != LLG_OK) return -1;
    return d.n_samples;
}

int64_t llg_steps_per_loop(const llg_ctx *c)
{
    llg::Derived d;
    if (!c || derived_of(c, &d) != LLG_OK) return -1;
    return d.steps_per_loop;
}

int64_t llg_sample_every(const llg_ctx *c)
{
    llg::Derived d;
    if (!c || derived_of(c, &d) != LLG_OK) return -1;
    return d.sample_every;
}

int64_t llg_current_step(const llg_ctx *c) { return c ? c->step : -1; }

int llg_active_engine(const llg_ctx *c)
{
    llg::Derived d;
    if (!c || derived_of(c, &d) != LLG_OK) return -1;
    llg::KParams kp = llg::kparams_of(d, c->nx, c->ny, c->nz, c->periodic, c->sw.dt);
    llg::RodPlan plan{};
    return resolve_engine(c, kp, c->n_real > 0 ? c->n_real : 1, &plan, nullptr);
}

llg_status llg_get_coefficients(const llg_ctx *c, double out[LLG_NCOEFF])
{
    if (!c || !out) return fail(LLG_EINVAL, "NULL argument");
    llg::Derived d;
    llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    const double v[LLG_NCOEFF] = {d.zeta, d.A, d.K, d.Ms, d.alpha, d.a, d.V, d.g0, d.g1, d.ag1,
                                  d.c_ex, d.c_an, d.sigma, d.H_start_Am, d.slope_Am, d.m_rescale};
    std::memcpy(out, v, sizeof v);
    return LLG_OK;
}

llg_status llg_sample_fields(const llg_ctx *c, double *H_Oe)
{
    if (!c || !H_Oe) return fail(LLG_EINVAL, "NULL argument");
    llg::Derived d;
    llg_status s = derived_of(c, &d);
    if (s != LLG_OK) return s;
    for (long long k = 0; k < d.n_samples; ++k) H_Oe[k] = llg::field_Oe(d, c->sw, k * d.sample_every);
    return LLG_OK;
}

}  // extern "C"
