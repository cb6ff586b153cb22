// llg_internal.h -- declarations shared by the host runtime (api.cpp, scaling.cpp, loops.cpp)
// and the CUDA engines (k_plain.cu, k_rod.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/llg.h"

namespace llg {

// NVTX range around one C-ABI call (header-only NVTX3: no cost unless a profiler is attached), so
// that timelines and ncu ranges show which call issued which launches.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Simulation-level coefficients of one job, derived on the host in FP64 (scaling.cpp).
struct Derived {
    double zeta, A, K, Ms, alpha, a, V;
    double g0, g1, ag1, c_ex, c_an, sigma;
    double H_start_Am, H_turn_Am, slope_Am;  // slope: A/m per step of the triangle coordinate
    long long n_half;                         // steps from H_start to H_turn (0: constant)
    long long sample_every;                   // steps between samples
    long long n_samples;                      // samples of one full loop
    long long steps_per_loop;
    double m_rescale;
    int shape;                                // 0 triangle, 1 cosine
    long long period;                         // steps per field cycle
};

// Per-job parameters handed to the kernels (FP32 coefficients).
struct KParams {
    int nx, ny, nz, ncells;
    unsigned periodic;        // bit0 x, bit1 y, bit2 z
    float c_ex, c_an, sigma;  // A/m
    float neg_dt_g1;          // -dt g1   (predictor)
    float neg_hdt_g1;         // -dt g1/2 (corrector)
    float alpha;
    float H0, slope;          // triangle sweep, A/m and A/m per step
    long long n_half;
    int shape;                // 0 triangle, 1 cosine
    float amp;                // cosine amplitude, A/m
    long long period;         // cosine period in steps
    uint32_t seed;
    uint32_t real0;           // key of realisation 0 of this ensemble
    long long sample_every;   // 0: no sampling
    long long n_samples;      // columns of the sample array
    // per-cell easy axes [n_real][ncells] (x, y, z, 0) of the dispersed-axis mode, or NULL for
    // the axis z in every cell; indexed by the rod's position in this ensemble
    const float4 *axis;
};

// Host helpers (scaling.cpp)
double zeta_of(double b, double T, double Tc);
// Fill d from the context's material, scaling and sweep; returns false with a message in err.
struct MaterialIn {
    double A0, Ms, K0, alpha, T;
};
struct ScalingIn {
    int mode;
    double Tc, delta, sK, sAlpha, sMs;
};
struct SweepIn {
    double H_start_Oe, H_turn_Oe, rate_Oe_per_ns, dt, sample_dH_Oe;
    int shape;
    long long held_samples = 1;  // sample columns of a held (constant) field
};
// volume_m3 > 0 overrides the cell volume (b a0)^3 of the thermal field (a single block whose
// volume is not a cube of the cell edge).
bool derive(int b, double a0, const MaterialIn &m, const ScalingIn &s, const SweepIn &w, Derived *d,
            char *err, size_t errlen, double volume_m3 = 0.0);
// Field (Oe) at step n of a derived sweep (host, FP64).
double field_Oe(const Derived &d, const SweepIn &w, long long n);
KParams kparams_of(const Derived &d, int nx, int ny, int nz, unsigned periodic, double dt);
// Grinstein-Koch flow from l = 0 to ln b: out = {T*, h, g, zeta} (host, FP64).
void gk_flow(double Ts0, double h0, double g0, double b, long long n_steps, double out[4]);

// ---- plain engine (k_plain.cu): state in global memory, two launches per step --------------
// m, mt: [n_real][ncells][3]; acc, hth: same shape (scratch).
// The field of step n (predictor) and n + 1 (corrector) is evaluated on the device.
cudaError_t plain_predictor(const KParams &p, const float *m, float *mt, float *acc, float *hth,
                            int n_real, long long n, cudaStream_t st);
cudaError_t plain_corrector(const KParams &p, float *m, const float *mt, const float *acc,
                            const float *hth, int n_real, long long n, cudaStream_t st);
// samples[r][k] = mean over cells of m_z; sets *status = 1 on a non-finite mean.
cudaError_t plain_sample(const KParams &p, const float *m, int n_real, long long k, float *samples,
                         int *status, cudaStream_t st);
// Host-side driver of the plain engine over n_steps from step0 (one predictor and one corrector
// launch per step, a reduction launch per sample).
cudaError_t plain_advance(const KParams &p, float *m, float *mt, float *acc, float *hth, int n_real,
                          long long step0, long long n_steps, float *samples, int *status,
                          cudaStream_t st, long long *launches);

// a[r * ld + col] = v for r in [0, rows)
cudaError_t fill_column(float *a, int rows, long long ld, long long col, float v, cudaStream_t st);
// ax[r][c] = easy_axis(seed, real0 + r, c, w_max) for r < n_real, c < ncells
cudaError_t axis_fill(float4 *ax, int n_real, int ncells, uint32_t seed, uint32_t real0, float w_max,
                      cudaStream_t st);

// ---- resident engine (k_rod.cu): rods in shared memory for the whole launch ------------------
struct RodPlan {
    int kind;          // 1: two-phase (small rods, several per CTA); 2: plane-pipelined (one per CTA);
                       // 3: rows (the b = 2, 4, 8 rods, a thread per x-row, several rods per CTA)
    int rods_per_cta;  // kind 1
    int threads;
    int rows_per_thread;  // kind 2
    int cells_per_thread; // kind 1
    size_t smem_bytes;
    int ctas;
    bool generic = false;  // kind 2: use the runtime-nx kernel even where a specialised one exists
    bool balance = true;   // kind 2: balance rod-steps over a co-resident grid (needs flags)
    unsigned long long handoff_timeout_ns = 30000000000ull;  // kind 2 balanced: longest hand-off wait
    bool withhold_handoff = false;  // test hook: balanced producers never release (waits run out)
};
// Choose a launch plan for n_real rods of this grid on device `dev`; returns false if no
// resident kernel can hold the rod.
// force_kind / force_rods: 0 = automatic.
bool rod_plan(const KParams &p, int n_real, int dev, RodPlan *plan, int force_kind = 0,
              int force_rods = 0, int force_rows = 0, int force_cpt = 0);
// Two-phase kernel (k_rod_small.cu): whether the grid and sweep have a compile-time instance,
// the largest CTA for cpt cells per thread, and the launch of n_steps (< 2^31) steps.
bool twophase_shaped(const KParams &p);
// Row kernel (k_rod_small.cu, plan kind 3): the b = 2, 4, 8 rods with a compile-time instance,
// its largest CTA, the shared memory of one rod, and the launch.
bool rows_supported(const KParams &p);
int rows_max_threads(const KParams &p);
size_t rows_rod_bytes(const KParams &p);
cudaError_t rows_advance(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0, int n_steps,
                         float *samples, int *status, cudaStream_t st);
int twophase_max_threads(const KParams &p, int cpt);
cudaError_t twophase_advance(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0,
                             int n_steps, float *samples, int *status, cudaStream_t st);
// flags: n_real words of device scratch for the balanced schedule's hand-offs (may be NULL:
// then no balancing).  status bit 0: non-finite sample; bit 1: a hand-off wait gave up.
cudaError_t rod_advance(const KParams &p, const RodPlan &plan, float *m, int n_real,
                        long long step0, long long n_steps, float *samples, int *status,
                        unsigned *flags, cudaStream_t st);

// ---- streaming engine (k_slab.cu): one fused Heun step per launch over HBM ----------------
struct SlabPlan {
    int tiles_x, tiles_y, TXmax, TYmax, cols_per_thread, threads;
    size_t smem_bytes;
};
bool slab_plan(const KParams &p, int dev, SlabPlan *plan);
// buf_a, buf_b: slab_state_float4s(p, n_real) float4 each (the padded layout
// [n_real][nz][ny + 4][nx + 4]); partial: slab_partial_floats(n_real) floats.
// status bit 2 (value 4): a staging wait of the streaming kernel gave up.
size_t slab_state_float4s(const KParams &p, int n_real);
cudaError_t slab_advance(const KParams &p, const SlabPlan &plan, float *m, int n_real, long long step0,
                         long long n_steps, float *samples, int *status, float4 *buf_a, float4 *buf_b,
                         float *partial, cudaStream_t st, long long *launches);
size_t slab_partial_floats(int n_real);

// ---- adjoint (k_adjoint.cu): one launch per checkpoint segment, rods of at most 1024 cells -----
bool adjoint_supported(const KParams &p, int dev);
// ckpt: state at seg_start; seg: scratch of seg_len states; lam: dL/d(state at seg_start +
// seg_len) in, dL/d(state at seg_start) out; w: loss weights of the window's samples k_first..;
// partial: [n_real][5] FP64 accumulators (g_alpha, g_a, g_cex, g_can, sigma g_sigma).
cudaError_t adjoint_segment(const KParams &p, int n_real, long long seg_start, int seg_len, long long win_end,
                            long long k_first, int n_k, const float *ckpt, float *seg, float *lam,
                            const double *w, double *partial, cudaStream_t st);
// The same reverse pass with the whole window's states stored: states[j] (j < n_steps, each
// n_real * ncells * 3 floats) = the state before step step0 + j, recomputed for all checkpoint
// segments in one launch (ckpt: one state per ckpt_every steps), then walked back in one launch.
cudaError_t adjoint_recompute_all(const KParams &p, int n_real, long long step0, long long n_steps, int ckpt_every,
                                  const float *ckpt, float *states, cudaStream_t st);
cudaError_t adjoint_backward_all(const KParams &p, int n_real, long long step0, long long n_steps, long long k_first,
                                 int n_k, const float *states, float *lam, const double *w, double *partial,
                                 cudaStream_t st);

// ---- tangent gradient (k_tangent.cu): one pass, a CTA per rod and parameter, <= 1408 cells -----
bool tangent_supported(const KParams &p, int dev);
// dcoef: the derivatives of (c_ex, c_an, alpha, a = dt g1) and dsigma/sigma with respect to
// (s_K, s_alpha, s_Ms), five groups of three.  m_work (advanced in place), samples [n_real][n_k]
// and dsamples [n_real][n_k][3] for the samples k_first .. k_first + n_k - 1 of the window.
cudaError_t tangent_forward(const KParams &p, const double dcoef[15], int n_real, long long step0, long long n_steps,
                            long long k_first, int n_k, float *m_work, float *samples, float *dsamples, int *status,
                            cudaStream_t st);

// ---- host runtime helpers (api.cpp) ---------------------------------------------------------
// Store a message for llg_last_error() on this thread.
void set_last_error(const char *msg);
}  // namespace llg

namespace llg {
// Kernel parameters of a context's grid, material, scaling and sweep (host-side derivation
// only; seed and real0 are left zero).  Returns LLG_OK or the setup error (message stored).
llg_status kparams_from_ctx(const llg_ctx *ctx, KParams *out);
// The CUDA device ordinal a context was created for.
int ctx_device(const llg_ctx *ctx);

// A context's ensemble and launch settings, for the batching layer and the autotuner.  Makes
// sure the hand-off flags of the resident engine exist when there is an ensemble.
struct CtxView {
    int device;
    cudaStream_t stream;
    int n_real;
    float *d_m;
    int *d_status;
    unsigned *d_flags;
    long long step, steps_per_loop;
    KParams kp;  // with the ensemble's seed and real0
    int tune_kind, tune_rods, tune_rows, tune_cpt;
    bool tune_generic;
    long long chunk_steps;  // steps per launch
};
llg_status ctx_view(llg_ctx *ctx, CtxView *out);
void ctx_add_steps(llg_ctx *ctx, long long n);
}  // namespace llg
