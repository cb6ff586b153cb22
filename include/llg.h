/*
 * llg.h -- C ABI of the GB300 stochastic-LLG hysteresis-loop library.
 *
 * The library time-steps the stochastic Landau-Lifshitz-Gilbert equation (Eq. 1 of Behbahani,
 * Plumer & Saika-Voivod, "Coarse-graining in micromagnetic simulations of dynamic hysteresis
 * loops", arXiv:1912.00310) on cubic grids of macrospin cells and builds averaged M(H) loops over
 * many independent noise realisations (the realisation count paragraph after the field-sweep
 * definition), at any coarse-graining level b with the parameter map of Eqs. 8-13.
 *
 * Conventions
 *   - SI units, except fields, which are in Oe at the API (as in the paper; 1 Oe = 1000/4pi A/m).
 *   - A cell index is  x + nx * (y + ny * z).  A state is float m[n_real][ncells][3] of unit
 *     vectors (AoS).  A sample array is float m_samples[n_real][n_samples].
 *   - Every call that enqueues GPU work does so on the context's CUDA stream (set at creation
 *     or with llg_set_stream; NULL means the legacy default stream) and returns without waiting,
 *     unless it says otherwise.  Pointers documented as "device" must be device memory of the
 *     context's device; pointers documented as "host or device" are classified with
 *     cudaPointerGetAttributes and copied through library-owned device buffers when on the host
 *     (such calls synchronise the stream).
 *   - No call throws.  Each returns an llg_status; on failure llg_last_error() holds a message
 *     (thread-local, valid until the next failing call on the same thread).
 *   - The library allocates device memory for the ensemble state and its own scratch with
 *     cudaMalloc; the context owns it and llg_destroy frees it.  Output buffers are owned by the
 *     caller.
 *   - Thread safety: a context must not be used from two threads at once.  Distinct contexts
 *     are independent.
 */
#ifndef LLG_H
#define LLG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct llg_ctx llg_ctx;

typedef enum llg_status {
    LLG_OK = 0,
    LLG_EINVAL = 1,        /* bad argument or call order                                    */
    LLG_ENOMEM = 2,        /* device or host allocation failed                              */
    LLG_ECUDA = 3,         /* a CUDA runtime call failed (message carries cudaGetErrorString) */
    LLG_ENONFINITE = 4,    /* a non-finite magnetisation was found                          */
    LLG_ETIMEOUT = 5,      /* llg_sync gave up waiting                                      */
    LLG_EUNSUPPORTED = 6   /* valid request that no engine of this build handles            */
} llg_status;

/* Integration engines (all compute the same Heun step; they differ only in where the state
 * lives between steps). */
typedef enum llg_engine {
    LLG_ENGINE_AUTO = 0,      /* resident when the grid fits on chip, else streaming          */
    LLG_ENGINE_RESIDENT = 1,  /* persistent kernel, whole rods in shared memory, one launch  */
    LLG_ENGINE_PLAIN = 2,     /* global-memory state, a predictor and a corrector launch per step */
    LLG_ENGINE_STREAM = 3     /* HBM stencil for grids larger than shared memory             */
} llg_engine;

/* Loop observables of one ensemble (raw = at level b; "0" = mapped back to the unscaled system
 * with H0 = H / zeta (Eq. 10) and m0 = rescale * m (Eq. 11 or Eq. 13)). */
typedef struct llg_loop_stats {
    double Hc_Oe, Hc_se_Oe;        /* coercive field (|Hc_down| + |Hc_up|) / 2, jackknife SE */
    double area_Oe, area_se_Oe;    /* |closed integral of m dH| (trapezoid), jackknife SE     */
    double Hc_down_Oe, Hc_up_Oe;   /* zero crossings of the mean loop on each branch         */
    double zeta, m_rescale;        /* factors of the selected scaling mode                   */
    double Hc0_Oe, area0_Oe;       /* rescaled coercive field and area                       */
} llg_loop_stats;

/* Number of doubles written by llg_get_coefficients. */
#define LLG_NCOEFF 16

/* ---------------------------------------------------------------------------------------- */
/* Context                                                                                   */
/* ---------------------------------------------------------------------------------------- */

/* Create a grid of nx * ny * nz cubic cells of edge b * a0_m (the rod of the simulation-cell
 * paragraph is 8x24x56 cells of a0 = 0.839 nm at b = 1 and (8/b)x(24/b)x(56/b) at level b).
 * periodic_mask: bit 0 x, bit 1 y, bit 2 z; free faces otherwise.  device: CUDA ordinal.
 * cuda_stream: a cudaStream_t (may be NULL).  *out receives the context.
 * Errors: EINVAL (non-positive sizes, b < 1, a0 <= 0, more than 2^31 cells), ECUDA. */
llg_status llg_create_grid(llg_ctx **out, int nx, int ny, int nz, double a0_m, int b,
                           unsigned periodic_mask, int device, void *cuda_stream);

/* Free all device memory of the context (waits for its stream).  NULL is ignored. */
void llg_destroy(llg_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *llg_last_error(void);

/* Replace the stream on which the context enqueues work. */
llg_status llg_set_stream(llg_ctx *ctx, void *cuda_stream);

/* Material parameters of the unscaled (b = 1) system, material paragraph and Eq. 1:
 * A0 exchange stiffness (J/m), Ms saturation magnetisation (A/m), K0 uniaxial anisotropy
 * (J/m^3) along the unit vector u, alpha Gilbert damping, T temperature (K).  The engines of this
 * build support u = +z or -z only (EUNSUPPORTED otherwise); the paper's 5-degree dispersion of
 * the axis is set by llg_set_axis_dispersion.  Errors: EINVAL (Ms <= 0, alpha < 0, T < 0, A0 < 0,
 * |u| = 0). */
llg_status llg_set_material(llg_ctx *ctx, double A0, double Ms, double K0, const double u[3],
                            double alpha, double T_kelvin);

/* Coarse-graining map, Eqs. 8-13.  mode 0: A and K unchanged (Fig. 2a); mode 1: A(b) = zeta A0,
 * K(b) = zeta^3 K0 and m0 = zeta m (Eqs. 8-11); mode 2: as mode 1 with m0 = (delta zeta + 1 -
 * delta) m (Eq. 13).  zeta(b) = t/b + 1 - t, t = T / Tc.  scale = {s_K, s_alpha, s_Ms} multiplies
 * K(b), alpha and Ms (NULL means {1, 1, 1}).  Default: mode 1, Tc = 858 K, delta = 0.511.
 * Errors: EINVAL (mode outside 0..2, Tc <= 0, a scale factor <= 0). */
llg_status llg_set_scaling(llg_ctx *ctx, int mode, double Tc_kelvin, double delta,
                           const double scale[3]);

/* Zeeman field along z (the field-sweep paragraph): a triangle wave H_start -> H_turn -> H_start
 * at |dH/dt| = rate (Oe/ns), time step dt_s (s), one M(H) sample every sample_dH_Oe of sweep.
 * A full loop is 2 |H_start - H_turn| / (rate dt) steps and 2 |H_start - H_turn| / sample_dH + 1
 * samples, sample k taken after step k * sample_every (sample 0 is the initial state).
 * rate = 0 (or H_start = H_turn) holds the field at H_start; sample_dH then counts steps.
 * shape: 0 = triangle; 1 = the paper's sinusoidal field H_max sin(2 pi f t) with H_max = H_start,
 * SR = rate = 4 H_max f (the field-sweep paragraph), started at its maximum, i.e.
 * H = H_max cos(2 pi n / period) with period = 4 H_max / (rate dt) steps (H_turn is ignored);
 * sample_dH then sets the sample interval sample_dH / (rate dt) steps.
 * Errors: EINVAL (dt <= 0, rate < 0, the span or the sample spacing not a whole number of steps
 * to 1e-6 relative; for the sinusoid, a period that is not an even whole number of steps and of
 * sample intervals). */
llg_status llg_set_sweep(llg_ctx *ctx, double H_start_Oe, double H_turn_Oe, double rate_Oe_per_ns,
                         double dt_s, double sample_dH_Oe, int shape);

/* For a held field (rate 0 in llg_set_sweep): n_samples sample columns, sample k taken after step
 * k * sample_every (sample_dH of llg_set_sweep counts steps), for time averages at equilibrium
 * (the temperature dependence of the magnetisation behind Eq. 12 and Fig. 3).  A later
 * llg_set_sweep resets it to 1.  Errors: EINVAL (n_samples < 1, no sweep, a swept field). */
llg_status llg_set_held_samples(llg_ctx *ctx, int64_t n_samples);

/* Cell volume (m^3) of the thermal field in place of (b a0)^3, for the paper's single-block
 * limit: the whole rod as one rectangular-prism macrospin of volume 10752 a0^3 at b = 22 (the
 * simulation-cell paragraph).  0 restores (b a0)^3.  Errors: EINVAL (negative). */
llg_status llg_set_cell_volume(llg_ctx *ctx, double volume_m3);

/* Easy-axis dispersion (the material paragraph's 5-degree spread of the anisotropy axis, modelling
 * lattice disorder): with half_angle_rad > 0 every cell of every realisation gets its own easy
 * axis, uniform over the solid angle of the cone of that half-angle about z, drawn from
 * Philox4x32-10 with key (seed, realisation) and counter (cell, 0, 0, 1), so it is fixed by the
 * ensemble's seed and realisation numbers like the thermal field (the thermal draws use counter
 * word 3 = 0).  The anisotropy field of a cell is then c_an (m.u) u.  The axes are drawn on the
 * context's stream at the next launch after a reset and kept in device memory (16 bytes per
 * cell and realisation).  0 (the default) restores the axis z everywhere.  Every engine, the
 * batching layer and llg_loop_area_grad honour it; llg_plain_advance_noalloc rejects it
 * (EUNSUPPORTED).  Errors: EINVAL (outside [0, pi/2]). */
llg_status llg_set_axis_dispersion(llg_ctx *ctx, double half_angle_rad);

/* The easy axes of the current ensemble, u [n_real][ncells][3] (x, y, z; host or device memory,
 * caller-owned; the z axis in every cell when no dispersion is set).  A host copy is complete on
 * return; a device copy is ordered on the context's stream.  Errors: EINVAL (no ensemble). */
llg_status llg_get_axes(llg_ctx *ctx, float *u);

/* The Grinstein-Koch flow of the reduced parameters (Eqs. 4-7) integrated numerically from
 * l = 0 to l = ln b (classical Runge-Kutta, n_steps equal steps, host FP64):
 * with Ts the reduced temperature T star = k_B T Lambda / A, h = mu0 Ms H / (A Lambda^2) and
 * g = K / (A Lambda^2), Lambda = 2 pi / a: d(Ts)/dl = (F - 1) Ts, dh/dl = 2 h,
 * dg/dl = (2 - 2F) g, F = Ts / (2 pi (1 + h + g)).
 * out = {Ts(ln b), h(ln b), g(ln b), zeta(ln b) = exp(-integral of F)}.  The scaling modes use
 * the closed form zeta = t/b + 1 - t that this flow reduces to when h = g = 0 (t = Ts(0) / 2 pi);
 * this call measures the difference for a material.  Needs no context or GPU.
 * Errors: EINVAL (b < 1, n_steps < 1, a negative parameter). */
llg_status llg_gk_flow(double Tstar0, double h0, double g0, double b, int64_t n_steps, double out[4]);

/* Select the integration engine (llg_engine).  Errors: EINVAL, EUNSUPPORTED (the engine cannot
 * hold this grid: checked at the next reset/advance). */
llg_status llg_set_engine(llg_ctx *ctx, int engine);

/* Launch-shape overrides of the resident engine (0 = automatic, the default):
 *   LLG_TUNE_ROD_KIND      1 two-phase kernel, 2 plane-pipelined kernel, 3 row kernel (the
 *                          b = 2, 4, 8 rods of the paper's ladder: a thread per x-row)
 *   LLG_TUNE_RODS_PER_CTA  rods per CTA of the two-phase and row kernels
 *   LLG_TUNE_CHUNK_STEPS   Heun steps per launch (default 2^20; llg_autotune sets it so the
 *                          launch overhead stays near 1% of a launch)
 *   LLG_TUNE_ROWS_PER_THREAD  rows per thread of the plane-pipelined kernel (1..4)
 *   LLG_TUNE_GENERIC_KERNEL   1: the runtime-size plane-pipelined kernel even where a kernel
 *                             specialised for the plane count exists
 *   LLG_TUNE_BALANCE          0: one rod per CTA even when the rods do not fill whole waves
 *                             (default 1: rod-steps balanced over a co-resident grid)
 *   LLG_TUNE_ADJOINT_STATE_MB device memory (MB, default 16384) that llg_loop_area_grad may hold
 *                             for the whole window's states (12 bytes per cell, realisation and
 *                             step); within it every checkpoint segment is recomputed in one
 *                             launch and the window reversed in another, beyond it (or with 0)
 *                             segment by segment.  The states, and so the loss, are the same
 *                             either way; the gradient's FP32 partial sums may be grouped
 *                             differently where a segment boundary splits a 64-step block
 *                             (measured: bitwise equal with aligned segments; FP32 blocks differ
 *                             from a per-step FP64 accumulation by at most 2e-8 relative).
 *   LLG_TUNE_CELLS_PER_THREAD cells per thread of the two-phase kernel (0 automatic, 1, 2, 4;
 *                             the b = 4 and b = 8 rods get 768 / cells-per-thread threads per CTA
 *                             at most, other grids 768)
 *   LLG_TUNE_GRAD_METHOD      llg_loop_area_grad's method: 0 the reverse-mode adjoint (default),
 *                             1 forward-mode tangents (one pass carrying dm/d(s_K, s_alpha, s_Ms);
 *                             no checkpoints or stored window; the same loss and, to FP32
 *                             rounding, the same gradient)
 *   LLG_TUNE_HANDOFF_TIMEOUT_MS  longest wait (ms, default 30000, 1 .. 3600000) of a CTA of the
 *                             balanced schedule for the CTA that runs the first part of a rod it
 *                             finishes; on expiry the CTA skips its remaining segments, and the
 *                             next llg_sync returns ETIMEOUT (the ensemble is then incomplete:
 *                             reset or restore it)
 *   LLG_TUNE_WITHHOLD_HANDOFF 1: failure-path test hook -- the balanced schedule's producers do
 *                             not signal their hand-offs, so every wait runs out (default 0)
 * The arithmetic, and so the trajectory, does not depend on these.  Errors: EINVAL (unknown
 * key, negative value); EUNSUPPORTED at the next advance if the shape cannot hold the grid. */
#define LLG_TUNE_ROD_KIND 1
#define LLG_TUNE_RODS_PER_CTA 2
#define LLG_TUNE_CHUNK_STEPS 3
#define LLG_TUNE_ROWS_PER_THREAD 4
#define LLG_TUNE_GENERIC_KERNEL 5
#define LLG_TUNE_BALANCE 6
#define LLG_TUNE_ADJOINT_STATE_MB 7
#define LLG_TUNE_HANDOFF_TIMEOUT_MS 8
#define LLG_TUNE_WITHHOLD_HANDOFF 9
#define LLG_TUNE_CELLS_PER_THREAD 10
#define LLG_TUNE_GRAD_METHOD 11
llg_status llg_set_tuning(llg_ctx *ctx, int key, int64_t value);

/* The current value of a tuning key (as set, by llg_set_tuning or llg_autotune; 0 = automatic).
 * Errors: EINVAL (unknown key, NULL argument). */
llg_status llg_get_tuning(const llg_ctx *ctx, int key, int64_t *value);

/* ---------------------------------------------------------------------------------------- */
/* Ensemble runs                                                                             */
/* ---------------------------------------------------------------------------------------- */

/* Start an ensemble of n_real realisations r = 0..n_real-1 with noise keys
 * (seed, real_offset + r): every cell m = +z (saturated along the initial field), step 0.
 * Allocates the state (n_real * ncells * 12 bytes).  Errors: EINVAL (n_real < 1, material or
 * sweep not set), ENOMEM, ECUDA. */
llg_status llg_reset(llg_ctx *ctx, uint32_t seed, int n_real, uint32_t real_offset);

/* Advance the ensemble by n_steps Heun steps of Eq. 1 with the Brown thermal field: per step n
 * and cell i, three standard normals from Philox4x32-10 (key = (seed, realisation), counter =
 * (i, n mod 2^32, n >> 32, 0)) and Box-Muller on 24-bit uniforms, times
 * sigma = sqrt(2 alpha kB T / (gamma0 mu0 Ms V dt)); predictor m~ = |m + dt f(m, t_n)|^-1 (...),
 * corrector m <- normalise(m + dt/2 (f(m, t_n) + f(m~, t_n+1))) with the same thermal field.
 * m_samples: device [n_real][n_samples] (llg_num_samples) or NULL; the cell-averaged m_z after
 * every step index that is a multiple of sample_every and below n_samples * sample_every is
 * written at its sample column; other columns are left untouched.  Asynchronous.
 * Errors: EINVAL (no ensemble, n_steps < 0), EUNSUPPORTED, ECUDA. */
llg_status llg_advance(llg_ctx *ctx, int64_t n_steps, float *m_samples);

/* One full loop per realisation: llg_reset(seed, n_real, real_offset), sample 0 = 1 (the +z
 * start), then llg_advance(llg_steps_per_loop).  m_samples: host or device
 * [n_real][n_samples] (caller-owned, required).  stats (host, optional): when given, the call
 * synchronises and fills the loop observables of the mean loop.  Errors: as llg_reset and
 * llg_advance. */
llg_status llg_run_loops(llg_ctx *ctx, uint32_t seed, int n_real, uint32_t real_offset,
                         float *m_samples, llg_loop_stats *stats);

/* Copy the ensemble state out to m (host or device [n_real][ncells][3]) and its step index
 * (optional).  Synchronises when m is host memory. */
llg_status llg_get_state(llg_ctx *ctx, float *m, int64_t *step);

/* Replace the ensemble state from m (host or device [n_real][ncells][3], unit vectors) at step
 * index `step`.  Resuming at step n with the same keys reproduces the uninterrupted run
 * bitwise (the noise is a function of (seed, realisation, cell, step) only). */
llg_status llg_set_state(llg_ctx *ctx, const float *m, int64_t step);

/* Wait for the context's stream, giving up after timeout_s seconds (<= 0: wait forever) with
 * LLG_ETIMEOUT.  Errors from earlier asynchronous work surface here as ECUDA. */
llg_status llg_sync(llg_ctx *ctx, double timeout_s);

/* Uneven batch (the realisation ensembles of the loop paragraph, for several b, sweep rates and
 * damping values at once): advance every job -- a context with an ensemble from llg_reset --
 * by min(max_steps, the steps left in its loop) Heun steps with the resident engine, all jobs in
 * one launch: a CUDA graph with one kernel node per job on independent branches, ordered
 * longest first, launched on jobs[0]'s stream after the work queued on every job's stream.  A
 * request of more steps than the jobs' smallest LLG_TUNE_CHUNK_STEPS runs as several such graph
 * launches; the instantiated graph of a job set is cached (a few per process) and refreshed in
 * place with cudaGraphExecUpdate.
 * m_samples (optional) [n_jobs] device sample arrays, one per job, as for llg_advance.
 * steps_done (optional, host) [n_jobs] receives the steps each job advanced.  Asynchronous.
 * Errors: EINVAL (no ensemble, jobs on different devices), EUNSUPPORTED (a grid the resident
 * engine cannot hold), ECUDA. */
llg_status llg_run_batch(llg_ctx *const *jobs, int n_jobs, int64_t max_steps,
                         float *const *m_samples, int64_t *steps_done);

/* Choose the resident engine's launch shape for this context by timing the candidates (rows per
 * thread of the plane-pipelined kernel; rods per CTA and cells per thread of the two-phase
 * kernel) for trial_steps Heun steps each on a scratch copy of the ensemble (allocated and freed
 * here), and set them with llg_set_tuning; also set the steps per launch (LLG_TUNE_CHUNK_STEPS)
 * from the measured time of a one-step launch, so that the launch overhead stays near 1% of a
 * launch.  Results are cached for the life of the process per (device, grid, realisation
 * count, sweep shape, whether the sweep and sample counts fit 32 bits, dispersed axes, periodic
 * faces), and a cached shape is used only while it still plans for the context.  The ensemble
 * itself is not advanced.  best_rate (optional) receives the fastest
 * cell-steps/s.  Synchronises.  Errors: EINVAL (no ensemble), ENOMEM, EUNSUPPORTED. */
llg_status llg_autotune(llg_ctx *ctx, int64_t trial_steps, double *best_rate);

/* Pathwise gradient of a loop loss with respect to the calibration scale factors
 * (s_K, s_alpha, s_Ms) of llg_set_scaling (the coarse-grained parameters of Eqs. 8-9 are fitted
 * to a finer loop), with the thermal normals of every (realisation, cell, step) held fixed.
 * The window is the n_steps Heun steps from the ensemble's current step; the ensemble is not
 * advanced.  Samples of the window: the realisation means mbar_k of the cell-averaged m_z after
 * the steps k * sample_every in (step, step + n_steps].
 *   objective 0: L = (1/K) sum_k (mbar_k - target[k])^2, target host array indexed by the global
 *                sample number (length llg_num_samples)
 *   objective 1: L = sum_k (mbar_k + mbar_k+1)/2 (H_k+1 - H_k), the signed area under the
 *                window's mean loop (target unused)
 * Method (LLG_TUNE_GRAD_METHOD 0, the default): a forward pass with the resident engine storing
 * the state every ckpt_every steps, then, segment by segment from the last, a kernel that
 * recomputes the segment's states from its checkpoint and runs the reverse-mode adjoint of the
 * Heun step back through them (one CTA per realisation; rods of at most 1024 cells with free
 * faces).  Method 1: one forward pass carrying the tangents dm/d(s_K, s_alpha, s_Ms) beside the
 * state (one CTA per realisation and parameter; rods of at most 1408 cells with free faces, the
 * b = 2 rod included; ckpt_every unused).  Either allocates its scratch for the duration of the call and
 * synchronises.
 * loss_out (optional) receives L; grad_out receives dL/d(s_K, s_alpha, s_Ms).
 * Errors: EINVAL (no ensemble, no sample in the window, window past the loop end),
 * EUNSUPPORTED (grid), ENOMEM, ECUDA. */
llg_status llg_loop_area_grad(llg_ctx *ctx, int64_t n_steps, int objective, const double *target,
                              int64_t ckpt_every, double *loss_out, double grad_out[3]);

/* ---------------------------------------------------------------------------------------- */
/* Queries and host-side loop analysis                                                       */
/* ---------------------------------------------------------------------------------------- */

int64_t llg_num_cells(const llg_ctx *ctx);
int64_t llg_num_samples(const llg_ctx *ctx);      /* samples of one full loop             */
int64_t llg_steps_per_loop(const llg_ctx *ctx);   /* 2 * steps from H_start to H_turn     */
int64_t llg_sample_every(const llg_ctx *ctx);     /* steps between samples                */
int64_t llg_current_step(const llg_ctx *ctx);
int llg_active_engine(const llg_ctx *ctx);        /* engine the next advance will use     */

/* Simulation-level coefficients (FP64) in this order: zeta, A(b), K(b), Ms, alpha, a, V,
 * gamma0 = mu0 ge, gamma1 = gamma0/(1+alpha^2), alpha*gamma1, c_ex = 2A/(mu0 Ms a^2),
 * c_an = 2K/(mu0 Ms), sigma, H_start (A/m), dH per step (A/m), m_rescale. */
llg_status llg_get_coefficients(const llg_ctx *ctx, double out[LLG_NCOEFF]);

/* Field (Oe) of every sample of one full loop: H_Oe host [llg_num_samples]. */
llg_status llg_sample_fields(const llg_ctx *ctx, double *H_Oe);

/* Loop observables of host samples [n_real][n_samples] taken at fields H_Oe [n_samples], the
 * descending branch ending at sample k_turn: mean loop, coercive field from the first zero
 * crossing on each branch (linear interpolation), trapezoid area, delete-one jackknife standard
 * errors (paragraph on the Fig. 2 loops: "one standard error"), and the rescaled values for
 * scaling mode / zeta / delta (Eqs. 10, 11, 13).  mean_out (optional) host [n_samples].
 * Errors: EINVAL. */
llg_status llg_loop_stats_host(const float *m_samples, int n_real, int64_t n_samples,
                               const double *H_Oe, int64_t k_turn, int mode, double zeta,
                               double delta, llg_loop_stats *out, double *mean_out);

/* The same observables for an ensemble whose realisations are split over several processes
 * (one per GPU; the realisations of the loop paragraph are independent).  The exchange is two
 * small sums across processes:
 *   1. llg_loop_moments on each process: per-sample sums sum_out [n_samples] (and, optional,
 *      sums of squares sumsq_out) of its own realisations, in FP64 (zeros for a process holding
 *      none: n_real 0, m_samples may be NULL); the processes add them and their realisation
 *      counts (n_total);
 *   2. llg_loop_jackknife_terms on each process: given the global sums sum_all, the delete-one
 *      jackknife terms of its own n_local realisations, out = {sum d_Hc, sum d_Hc^2, sum d_area,
 *      sum d_area^2} with d = (statistic of the mean loop without that realisation) - (statistic
 *      of the full mean loop); the processes add the four numbers;
 *   3. llg_loop_stats_from_sums: the observables of the global mean loop and their jackknife
 *      standard errors from the global sums and terms (jk NULL: no standard errors).
 * Over one process this is llg_loop_stats_host (which is implemented this way).  All host memory;
 * no GPU needed.  Errors: EINVAL. */
llg_status llg_loop_moments(const float *m_samples, int n_real, int64_t n_samples, double *sum_out,
                            double *sumsq_out);
llg_status llg_loop_jackknife_terms(const float *m_samples, int n_local, int64_t n_samples,
                                    const double *sum_all, int n_total, const double *H_Oe,
                                    int64_t k_turn, double out[4]);
llg_status llg_loop_stats_from_sums(const double *sum_all, int n_total, int64_t n_samples,
                                    const double *H_Oe, int64_t k_turn, const double jk[4], int mode,
                                    double zeta, double delta, llg_loop_stats *out, double *mean_out);

/* Specific loss power (the SR/alpha paragraph's heating figure): a loop of area area_Oe (the
 * closed integral of m dH, Oe) dissipates mu0 Ms area per cycle and unit volume (H in A/m), so at
 * frequency f_hz the power per mass is f mu0 Ms (1000/4pi) area / rho, here in W/g with the
 * density rho_kg_m3 in kg/m^3.  Errors: EINVAL (f < 0, Ms <= 0, rho <= 0, non-finite area). */
llg_status llg_specific_loss_power(double f_hz, double Ms, double area_Oe, double rho_kg_m3,
                                   double *W_per_g);

/* Measured issue rates of the SM's 32-bit lanes on `device` (the ALU roofline denominator of the
 * resident and streaming kernels, which are bound by 32-bit lane operations): out[0] FP32
 * fused multiply-adds per second (eight independent chains per thread, 64 warps per SM), out[1]
 * the median SM clock (MHz) during that kernel, from the SM cycle counter against the global
 * timer, out[2] lane operations per second of the noise generator's integer mix (Philox rounds,
 * counted as in the algorithmic lane-op count: a 32x32->64 product = 2, a 3-input xor = 2),
 * out[3] the SM clock during that kernel.  Best of five timed launches of about 10-50 ms each;
 * synchronises; allocates a few KB.  No clock or other device setting is changed.
 * Errors: EINVAL (device), ECUDA. */
llg_status llg_measure_alu_peak(int device, double out[4]);

/* ---------------------------------------------------------------------------------------- */
/* Allocation-free advance (no counterpart in the paper)                                     */
/* ---------------------------------------------------------------------------------------- */

/* Largest n_real * ncells that llg_plain_advance_noalloc accepts.  Its scratch (9 floats per
 * cell-realisation plus a 256-byte header, about 9.4 MB) is a fixed array inside the library
 * that every GPU which loads the library holds until the process exits. */
#define LLG_NOALLOC_MAX_CELL_REALISATIONS 262144

/* The plain engine (a predictor and a corrector launch per Heun step, as llg_advance with
 * LLG_ENGINE_PLAIN) for callers that cannot allocate device memory: code running while its
 * stream is captured into a CUDA graph, programs whose device memory belongs to an allocator
 * that must account for every byte, and loops that cannot accept the device synchronisation a
 * cudaMalloc may cause.  It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * lives in the library's fixed device array described above, and the context is used only for
 * its host-side parameters (grid, material, scaling, sweep; its own device buffers are untouched).
 *   m          device [n_real][ncells][3], the state, advanced in place from step index step0
 *   seed, real_offset  noise keys (seed, real_offset + r) as in llg_reset
 *   m_samples  device [n_real][llg_num_samples] or NULL, written as llg_advance does
 *   cuda_stream  stream for the work; the call is asynchronous unless status_out is given
 *   status_out host or NULL: when given, the call waits for the stream and stores 1 if a
 *              non-finite sample was seen, else 0.  It must be NULL while the stream is being
 *              captured (the read-back and the wait are not capturable): EINVAL otherwise.
 * The work runs on the current device, which must be the context's device; m and m_samples must
 * be memory of that device (EINVAL otherwise, checked before anything is enqueued).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture begins.  All calls share
 * the one array and the status word is cleared at the start of each call, so calls whose GPU work
 * overlaps (other streams, other host threads) race and must be serialised by the caller.
 * Errors: EINVAL (n_real * ncells above LLG_NOALLOC_MAX_CELL_REALISATIONS, bad arguments, setup
 * incomplete, wrong current device, buffers not on it, status_out during capture), ECUDA. */
llg_status llg_plain_advance_noalloc(const llg_ctx *ctx, float *m, int n_real, uint32_t seed,
                                     uint32_t real_offset, int64_t step0, int64_t n_steps,
                                     float *m_samples, void *cuda_stream, int *status_out);

#ifdef __cplusplus
}
#endif

#endif /* LLG_H */
