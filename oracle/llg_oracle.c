/*
 * llg_oracle.c -- plain, slow FP64 CPU oracle for the stochastic LLG hysteresis-loop path of
 * Behbahani, Plumer & Saika-Voivod, "Coarse-graining in micromagnetic simulations of dynamic
 * hysteresis loops" (arXiv:1912.00310).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes, in the paper's order and notation:
 *   - Eq. 1 (LLG in Landau-Lifshitz form): dM/dt = -g1 M x H_eff - (alpha g1/Ms) M x (M x H_eff),
 *     g1 = mu0 ge / (1 + alpha^2), ge = 1.76e11 rad/(s T).  Written for the unit vector m = M/Ms.
 *   - H_eff = exchange (6-neighbour cubic stencil) + uniaxial anisotropy along u + Zeeman field
 *     along z + Brown thermal field (material paragraph; thermal-field paragraph after Eq. 1).
 *   - Coarse-graining (Eqs. 8-13): zeta(b) = t/b + 1 - t, t = T/Tc; A(b) = zeta A0,
 *     K(b) = zeta^3 K0; H0 = H(b)/zeta; M0 = zeta M(b) (Eq. 11) or the delta-corrected
 *     M0 = delta zeta M(b) + (1 - delta) M(b) (Eq. 13).
 *   - Loop observables: m_H = z component of the cell-averaged unit magnetisation, averaged over
 *     independent realisations; coercive field with one standard error; loop area.
 * Readings where the paper is silent (all listed in the design notes): thermal-field variance
 * sigma^2 = 2 alpha kB T / (g0 mu0 Ms V dt) with g0 = mu0 ge; Heun predictor-corrector with
 * renormalisation of predictor and corrector and one thermal draw per step; exchange field
 * (2A/(mu0 Ms a^2)) sum_j m_j with free faces; Philox4x32-10 noise keyed by (seed, realisation)
 * with counter (cell, step_lo, step_hi, 0) and Box-Muller on 24-bit uniforms.
 *
 * Precision: double throughout.  Parallelism: one POSIX thread per group of realisations
 * (realisations are independent; results do not depend on the thread count).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_MU0 (4.0e-7 * ORC_PI)          /* vacuum permeability, T m / A            */
#define ORC_GE 1.76e11                      /* electron gyromagnetic ratio, rad/(s T)  */
#define ORC_KB 1.380649e-23                 /* Boltzmann constant, J/K                 */
#define ORC_OE_TO_AM (1000.0 / (4.0 * ORC_PI)) /* 1 Oe in A/m                          */

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",   */
/* SC'11).  A 4x32-bit counter is mixed with a 2x32-bit key by ten rounds; each round multiplies */
/* counter words 0 and 2 by the two Philox multipliers, swaps the halves, xors in the key, and  */
/* the key is advanced by the two Weyl constants between rounds.                                 */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t prod0 = (uint64_t)mult0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)mult1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Uniform in (0,1) from the top 24 bits of a 32-bit word: (floor(x / 256) + 1/2) / 2^24. */
double orc_uniform24(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Three standard normals for (seed, realisation, cell, step): Box-Muller on the pairs
 * (u0, u1) -> (n0, n1) and (u2, u3) -> n2 (the fourth normal is not used). */
void orc_thermal_normals(uint32_t seed, uint32_t real, uint32_t cell, uint64_t step, double n[3])
{
    uint32_t ctr[4] = {cell, (uint32_t)step, (uint32_t)(step >> 32), 0u};
    uint32_t key[2] = {seed, real};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u0 = orc_uniform24(x[0]), u1 = orc_uniform24(x[1]);
    double u2 = orc_uniform24(x[2]), u3 = orc_uniform24(x[3]);
    double r01 = sqrt(-2.0 * log(u0));
    double r23 = sqrt(-2.0 * log(u2));
    n[0] = r01 * cos(2.0 * ORC_PI * u1);
    n[1] = r01 * sin(2.0 * ORC_PI * u1);
    n[2] = r23 * cos(2.0 * ORC_PI * u3);
}

/* ------------------------------------------------------------------------------------------ */
/* Coarse-graining map, Eqs. 8-13.                                                             */
/* ------------------------------------------------------------------------------------------ */
double orc_zeta(double b, double T, double Tc)
{
    double t = T / Tc;
    return t / b + 1.0 - t;
}

/* Exchange length of the renormalised material, l_ex,b = sqrt(2 zeta A0 / (mu0 Ms^2)). */
double orc_exchange_length(double zeta, double A0, double Ms)
{
    return sqrt(2.0 * zeta * A0 / (ORC_MU0 * Ms * Ms));
}

/* Factor that maps a simulated m_H at level b back to the unscaled system: Eq. 11 for
 * mode 1 (zeta), Eq. 13 for mode 2 (delta zeta + 1 - delta); mode 0 leaves m unchanged. */
double orc_m_rescale(int mode, double zeta, double delta)
{
    if (mode == 1) return zeta;
    if (mode == 2) return delta * zeta + (1.0 - delta);
    return 1.0;
}

/* Grinstein-Koch flow of the reduced parameters with l = ln b (Eqs. 4-7), writing Ts for the
 * reduced temperature T star:
 *   d(Ts)/dl = (-1 + F) Ts,  dh/dl = 2 h,  dg/dl = (2 - 2 F) g,  F = Ts / (2 pi (1 + h + g)),
 * and the magnetisation factor zeta(l) = exp(-integral_0^l F dl').  Classical fourth-order
 * Runge-Kutta over n equal steps of l from 0 to ln b, the integral of F carried as a fourth
 * state variable.  out = {Ts(l), h(l), g(l), zeta(l)}. */
static void gk_derivative(const double y[4], double d[4])
{
    const double F = y[0] / (2.0 * ORC_PI * (1.0 + y[1] + y[2]));
    d[0] = (-1.0 + F) * y[0];
    d[1] = 2.0 * y[1];
    d[2] = (2.0 - 2.0 * F) * y[2];
    d[3] = F;
}

void orc_gk_flow(double Ts0, double h0, double g0, double b, int64_t n, double out[4])
{
    double y[4] = {Ts0, h0, g0, 0.0};
    const double dl = log(b) / (double)n;
    for (int64_t s = 0; s < n; ++s) {
        double k1[4], k2[4], k3[4], k4[4], t[4];
        gk_derivative(y, k1);
        for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * dl * k1[i];
        gk_derivative(t, k2);
        for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * dl * k2[i];
        gk_derivative(t, k3);
        for (int i = 0; i < 4; ++i) t[i] = y[i] + dl * k3[i];
        gk_derivative(t, k4);
        for (int i = 0; i < 4; ++i) y[i] += dl / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    out[0] = y[0];
    out[1] = y[1];
    out[2] = y[2];
    out[3] = exp(-y[3]);
}

/* ------------------------------------------------------------------------------------------ */
/* Problem description.  All quantities are the simulation-level values (already rescaled).    */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    unsigned periodic;   /* bit0 x, bit1 y, bit2 z */
    double a;            /* cell edge, m                                  */
    double volume;       /* cell volume, m^3 (a^3 for cubic cells)        */
    double A;            /* exchange stiffness, J/m                       */
    double K;            /* uniaxial anisotropy, J/m^3                    */
    double Ms;           /* saturation magnetisation, A/m                 */
    double alpha;        /* Gilbert damping                               */
    double T;            /* temperature, K                                */
    double u[3];         /* easy axis (unit vector)                       */
    double dt;           /* time step, s                                  */
    double H_start_Oe;   /* field at step 0                               */
    double H_turn_Oe;    /* field at the turning point                    */
    int64_t n_half;      /* steps from H_start to H_turn (0: constant)    */
    int shape;           /* 0 triangle, 1 sinusoid of amplitude H_start   */
    int64_t period;      /* sinusoid: steps per cycle, 1/(f dt)           */
    double disp;         /* easy-axis dispersion: half-angle (rad) of the cone about z in which
                            each cell's axis lies (0: every cell has the axis u) */
} orc_problem;

typedef struct {
    double g0, g1, ag1;  /* mu0 ge, g1 = g0/(1+alpha^2), alpha g1 */
    double c_ex;         /* 2A / (mu0 Ms a^2), A/m                 */
    double c_an;         /* 2K / (mu0 Ms), A/m                     */
    double sigma;        /* thermal-field standard deviation, A/m  */
} orc_coeffs;

void orc_coefficients(const orc_problem *p, double out[6])
{
    double g0 = ORC_MU0 * ORC_GE;
    out[0] = g0;
    out[1] = g0 / (1.0 + p->alpha * p->alpha);
    out[2] = p->alpha * out[1];
    out[3] = 2.0 * p->A / (ORC_MU0 * p->Ms * p->a * p->a);
    out[4] = 2.0 * p->K / (ORC_MU0 * p->Ms);
    out[5] = (p->T > 0.0)
                 ? sqrt(2.0 * p->alpha * ORC_KB * p->T / (g0 * ORC_MU0 * p->Ms * p->volume * p->dt))
                 : 0.0;
}

static orc_coeffs coeffs_of(const orc_problem *p)
{
    double c[6];
    orc_coefficients(p, c);
    orc_coeffs r = {c[0], c[1], c[2], c[3], c[4], c[5]};
    return r;
}

/* Zeeman field along z at step n, in Oe.  shape 0: a triangle wave from H_start to H_turn and
 * back, with n_half steps per half period.  shape 1: the sinusoidal field of the field-sweep
 * paragraph, H_max sin(2 pi f t) with H_max = H_start and f = 1/(period dt), taken a quarter
 * cycle on so that each loop starts at +H_max like the triangle; t is n dt reduced modulo the
 * period. */
double orc_field_Oe(const orc_problem *p, int64_t n)
{
    if (p->shape == 1) {
        int64_t ph = n % p->period;
        return p->H_start_Oe * sin(2.0 * ORC_PI * (double)ph / (double)p->period + 0.5 * ORC_PI);
    }
    if (p->n_half <= 0) return p->H_start_Oe;
    int64_t period = 2 * p->n_half;
    int64_t ph = n % period;
    int64_t tri = ph <= p->n_half ? ph : period - ph;
    return p->H_start_Oe + (p->H_turn_Oe - p->H_start_Oe) * ((double)tri / (double)p->n_half);
}

static int64_t ncells_of(const orc_problem *p) { return (int64_t)p->nx * p->ny * p->nz; }

/* Easy axis of one cell of one realisation.  With disp = 0 it is the material axis u.  With
 * disp > 0 it models the lattice disorder of the material paragraph (a 5 degree dispersion of
 * the anisotropy axis): a direction uniform over the solid angle of the cone of half-angle disp
 * about z, drawn once per (seed, realisation, cell) from Philox4x32-10 with counter
 * (cell, 0, 0, 1) (the thermal draws use the tag word 0): for a uniform point of a spherical cap,
 * 1 - cos(theta) is uniform on [0, 1 - cos(disp)] and the azimuth is uniform. */
void orc_easy_axis(const orc_problem *p, uint32_t seed, uint32_t real, uint32_t cell, double u[3])
{
    if (!(p->disp > 0.0)) {
        u[0] = p->u[0];
        u[1] = p->u[1];
        u[2] = p->u[2];
        return;
    }
    uint32_t ctr[4] = {cell, 0u, 0u, 1u};
    uint32_t key[2] = {seed, real};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    const double one_minus_cos = orc_uniform24(x[0]) * (1.0 - cos(p->disp));
    const double phi = 2.0 * ORC_PI * orc_uniform24(x[1]);
    const double cos_t = 1.0 - one_minus_cos;
    const double sin_t = sqrt(one_minus_cos * (2.0 - one_minus_cos));
    u[0] = sin_t * cos(phi);
    u[1] = sin_t * sin(phi);
    u[2] = cos_t;
}

/* Axes of all cells of one realisation, [N][3]. */
static void easy_axes(const orc_problem *p, uint32_t seed, uint32_t real, double *ax)
{
    const int64_t N = ncells_of(p);
    for (int64_t i = 0; i < N; ++i) orc_easy_axis(p, seed, real, (uint32_t)i, ax + 3 * i);
}

/* Effective field at cell (x,y,z) of state m (unit vectors), field Hz (A/m) along z, thermal
 * field hth, easy axes ax [N][3]. */
static void effective_field(const orc_problem *p, const orc_coeffs *c, const double *m, int x, int y,
                            int z, double Hz, const double *hth, const double *ax, double H[3])
{
    double s[3] = {0.0, 0.0, 0.0};
    const int dims[3] = {p->nx, p->ny, p->nz};
    const int pos[3] = {x, y, z};
    for (int axis = 0; axis < 3; ++axis) {
        for (int dir = -1; dir <= 1; dir += 2) {
            int q[3] = {pos[0], pos[1], pos[2]};
            q[axis] += dir;
            if (q[axis] < 0 || q[axis] >= dims[axis]) {
                if (!(p->periodic & (1u << axis))) continue; /* free face: no neighbour */
                q[axis] = (q[axis] + dims[axis]) % dims[axis];
            }
            int64_t j = q[0] + (int64_t)p->nx * (q[1] + (int64_t)p->ny * q[2]);
            s[0] += m[3 * j + 0];
            s[1] += m[3 * j + 1];
            s[2] += m[3 * j + 2];
        }
    }
    int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
    const double *mi = m + 3 * i, *u = ax + 3 * i;
    double mu = mi[0] * u[0] + mi[1] * u[1] + mi[2] * u[2];
    for (int k = 0; k < 3; ++k) H[k] = c->c_ex * s[k] + c->c_an * mu * u[k] + hth[k];
    H[2] += Hz;
}

/* Right-hand side of Eq. 1 for the unit vector: f = -g1 m x H - alpha g1 m x (m x H). */
static void llg_rhs(const orc_coeffs *c, const double m[3], const double H[3], double f[3])
{
    double mxH[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
    double mxmxH[3] = {m[1] * mxH[2] - m[2] * mxH[1], m[2] * mxH[0] - m[0] * mxH[2],
                       m[0] * mxH[1] - m[1] * mxH[0]};
    for (int k = 0; k < 3; ++k) f[k] = -c->g1 * mxH[k] - c->ag1 * mxmxH[k];
}

static void normalise(double v[3])
{
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n;
    v[1] /= n;
    v[2] /= n;
}

typedef struct {
    double *mt, *f0, *hth;
    double *ax;  /* easy axes of the realisation being stepped */
} work_buffers;

/* One Heun step n -> n+1 of one realisation, in place on m. */
static void heun_step(const orc_problem *p, const orc_coeffs *c, uint32_t seed, uint32_t real,
                      int64_t n, double *m, work_buffers *w)
{
    const int64_t N = ncells_of(p);
    const double Hn = orc_field_Oe(p, n) * ORC_OE_TO_AM;
    const double Hn1 = orc_field_Oe(p, n + 1) * ORC_OE_TO_AM;
    /* thermal field, drawn once per step and used by both stages */
    for (int64_t i = 0; i < N; ++i) {
        double xi[3];
        if (c->sigma > 0.0) {
            orc_thermal_normals(seed, real, (uint32_t)i, (uint64_t)n, xi);
        } else {
            xi[0] = xi[1] = xi[2] = 0.0;
        }
        for (int k = 0; k < 3; ++k) w->hth[3 * i + k] = c->sigma * xi[k];
    }
    /* predictor: mt = normalise(m + dt f(m, t_n)) */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
                double H[3];
                effective_field(p, c, m, x, y, z, Hn, w->hth + 3 * i, w->ax, H);
                llg_rhs(c, m + 3 * i, H, w->f0 + 3 * i);
                for (int k = 0; k < 3; ++k) w->mt[3 * i + k] = m[3 * i + k] + p->dt * w->f0[3 * i + k];
                normalise(w->mt + 3 * i);
            }
    /* corrector: m <- normalise(m + dt/2 (f(m, t_n) + f(mt, t_{n+1}))) */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
                double H[3], f1[3];
                effective_field(p, c, w->mt, x, y, z, Hn1, w->hth + 3 * i, w->ax, H);
                llg_rhs(c, w->mt + 3 * i, H, f1);
                for (int k = 0; k < 3; ++k)
                    m[3 * i + k] = m[3 * i + k] + 0.5 * p->dt * (w->f0[3 * i + k] + f1[k]);
                normalise(m + 3 * i);
            }
}

/* ------------------------------------------------------------------------------------------ */
/* Ensemble driver.                                                                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const orc_problem *p;
    uint32_t seed;
    int n_real;
    uint32_t real0;
    int64_t step0, n_steps;
    double *m_state;     /* [n_real][N][3] */
    int64_t sample_every;
    int64_t n_samples;   /* columns of samples */
    double *samples;     /* [n_real][n_samples], indexed by global sample number */
    double *mz_timeavg;  /* [n_real] or NULL: mean of cell-averaged m_z over all steps after
                            burn_in (state after each step) */
    int64_t burn_in;
    int next_real;
    pthread_mutex_t lock;
} run_job;

static double mean_mz(const double *m, int64_t N)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += m[3 * i + 2];
    return s / (double)N;
}

static void run_one(run_job *job, int r)
{
    const orc_problem *p = job->p;
    const int64_t N = ncells_of(p);
    orc_coeffs c = coeffs_of(p);
    work_buffers w;
    w.mt = (double *)malloc(sizeof(double) * 3 * N);
    w.f0 = (double *)malloc(sizeof(double) * 3 * N);
    w.hth = (double *)malloc(sizeof(double) * 3 * N);
    w.ax = (double *)malloc(sizeof(double) * 3 * N);
    easy_axes(p, job->seed, job->real0 + (uint32_t)r, w.ax);
    double *m = job->m_state + (int64_t)r * N * 3;
    double acc = 0.0;
    int64_t acc_n = 0;
    for (int64_t s = 0; s < job->n_steps; ++s) {
        int64_t n = job->step0 + s;
        heun_step(p, &c, job->seed, job->real0 + (uint32_t)r, n, m, &w);
        int64_t done = n + 1;
        if (job->samples && job->sample_every > 0 && done % job->sample_every == 0) {
            int64_t k = done / job->sample_every;
            if (k < job->n_samples) job->samples[(int64_t)r * job->n_samples + k] = mean_mz(m, N);
        }
        if (job->mz_timeavg && s >= job->burn_in) {
            acc += mean_mz(m, N);
            ++acc_n;
        }
    }
    if (job->mz_timeavg) job->mz_timeavg[r] = acc_n ? acc / (double)acc_n : 0.0;
    free(w.mt);
    free(w.f0);
    free(w.hth);
    free(w.ax);
}

static void *run_worker(void *arg)
{
    run_job *job = (run_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int r = job->next_real++;
        pthread_mutex_unlock(&job->lock);
        if (r >= job->n_real) break;
        run_one(job, r);
    }
    return NULL;
}

/* Advance n_real realisations (keys (seed, real0 + r)) from step0 by n_steps Heun steps.
 * m_state [n_real][nx*ny*nz][3] is updated in place.  If samples is given, the cell-averaged m_z
 * after every step whose index (step0 + s + 1) is a multiple of sample_every is stored at column
 * (step index / sample_every).  If mz_timeavg is given, it receives, per realisation, the mean
 * of the cell-averaged m_z over the steps s >= burn_in of this call.  Returns 0. */
int orc_run(const orc_problem *p, uint32_t seed, int n_real, uint32_t real0, int64_t step0,
            int64_t n_steps, double *m_state, int64_t sample_every, int64_t n_samples,
            double *samples, double *mz_timeavg, int64_t burn_in, int n_threads)
{
    run_job job;
    job.p = p;
    job.seed = seed;
    job.n_real = n_real;
    job.real0 = real0;
    job.step0 = step0;
    job.n_steps = n_steps;
    job.m_state = m_state;
    job.sample_every = sample_every;
    job.n_samples = n_samples;
    job.samples = samples;
    job.mz_timeavg = mz_timeavg;
    job.burn_in = burn_in;
    job.next_real = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_real) n_threads = n_real;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, run_worker, &job);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
    return 0;
}

/* Total energy (J) of a state at field H (Oe along z): exchange per nearest-neighbour pair
 * 2 A a (1 - m_i . m_j), anisotropy -K V (m.u)^2 with the material axis u (no dispersion),
 * Zeeman -mu0 Ms V H m_z.  The effective field of Eq. 1 is -(1/(mu0 Ms V)) dE/dm_i of this
 * energy. */
double orc_energy(const orc_problem *p, const double *m, double H_Oe)
{
    const double H = H_Oe * ORC_OE_TO_AM;
    double e = 0.0;
    const int dims[3] = {p->nx, p->ny, p->nz};
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
                const double *mi = m + 3 * i;
                int pos[3] = {x, y, z};
                for (int axis = 0; axis < 3; ++axis) { /* each pair once: the +1 neighbour */
                    int q[3] = {pos[0], pos[1], pos[2]};
                    q[axis] += 1;
                    if (q[axis] >= dims[axis]) {
                        if (!(p->periodic & (1u << axis))) continue; /* free face */
                        q[axis] = 0; /* periodic: the wrapped bond is a bond of its own */
                    }
                    int64_t j = q[0] + (int64_t)p->nx * (q[1] + (int64_t)p->ny * q[2]);
                    const double *mj = m + 3 * j;
                    e += 2.0 * p->A * p->a * (1.0 - (mi[0] * mj[0] + mi[1] * mj[1] + mi[2] * mj[2]));
                }
                double mu = mi[0] * p->u[0] + mi[1] * p->u[1] + mi[2] * p->u[2];
                e -= p->K * p->volume * mu * mu;
                e -= ORC_MU0 * p->Ms * p->volume * H * mi[2];
            }
    return e;
}

/* ------------------------------------------------------------------------------------------ */
/* Loop observables (sample spacing in field, mean loop over realisations).                   */
/* ------------------------------------------------------------------------------------------ */

/* Coercive field of one mean loop m[0..n-1] at fields H[0..n-1], the loop starting at
 * positive saturation and turning at sample k_turn: the first zero crossing after the start on
 * the descending branch and the first after the turning point on the ascending branch, each by
 * linear interpolation; Hc = (|Hc_down| + |Hc_up|) / 2.  Returns NAN when a branch has no
 * crossing. */
static double crossing(const double *H, const double *m, int64_t k0, int64_t k1, int descending)
{
    for (int64_t k = k0; k < k1; ++k) {
        double a = m[k], b = m[k + 1];
        int hit = descending ? (a > 0.0 && b <= 0.0) : (a < 0.0 && b >= 0.0);
        if (hit) {
            double f = a / (a - b);
            return H[k] + f * (H[k + 1] - H[k]);
        }
    }
    return NAN;
}

double orc_coercive_field(const double *H, const double *m, int64_t n, int64_t k_turn,
                          double *hc_down, double *hc_up)
{
    double d = crossing(H, m, 0, k_turn, 1);
    double u = crossing(H, m, k_turn, n - 1, 0);
    if (hc_down) *hc_down = d;
    if (hc_up) *hc_up = u;
    return 0.5 * (fabs(d) + fabs(u));
}

/* Loop area |closed integral of m dH| by the trapezoid rule over consecutive samples. */
double orc_loop_area(const double *H, const double *m, int64_t n)
{
    double s = 0.0;
    for (int64_t k = 0; k + 1 < n; ++k) s += 0.5 * (m[k] + m[k + 1]) * (H[k + 1] - H[k]);
    return fabs(s);
}

/* Mean loop, coercive field and area with delete-one jackknife standard errors over the
 * realisations.  samples [n_real][n].  out: {Hc, Hc_se, area, area_se, Hc_down, Hc_up}.
 * mean_out [n] (optional) receives the mean loop. */
void orc_loop_stats(const double *H, const double *samples, int n_real, int64_t n, int64_t k_turn,
                    double *out, double *mean_out)
{
    double *mean = (double *)calloc((size_t)n, sizeof(double));
    double *loo = (double *)malloc(sizeof(double) * (size_t)n);
    for (int r = 0; r < n_real; ++r)
        for (int64_t k = 0; k < n; ++k) mean[k] += samples[(int64_t)r * n + k];
    for (int64_t k = 0; k < n; ++k) mean[k] /= (double)n_real;
    double hd, hu;
    double hc = orc_coercive_field(H, mean, n, k_turn, &hd, &hu);
    double area = orc_loop_area(H, mean, n);
    double hc_se = NAN, area_se = NAN;
    if (n_real > 1) {
        double *jh = (double *)malloc(sizeof(double) * (size_t)n_real);
        double *ja = (double *)malloc(sizeof(double) * (size_t)n_real);
        double mh = 0.0, ma = 0.0;
        for (int r = 0; r < n_real; ++r) {
            for (int64_t k = 0; k < n; ++k)
                loo[k] = (mean[k] * n_real - samples[(int64_t)r * n + k]) / (double)(n_real - 1);
            jh[r] = orc_coercive_field(H, loo, n, k_turn, NULL, NULL);
            ja[r] = orc_loop_area(H, loo, n);
            mh += jh[r];
            ma += ja[r];
        }
        mh /= n_real;
        ma /= n_real;
        double vh = 0.0, va = 0.0;
        for (int r = 0; r < n_real; ++r) {
            vh += (jh[r] - mh) * (jh[r] - mh);
            va += (ja[r] - ma) * (ja[r] - ma);
        }
        hc_se = sqrt((double)(n_real - 1) / n_real * vh);
        area_se = sqrt((double)(n_real - 1) / n_real * va);
        free(jh);
        free(ja);
    }
    out[0] = hc;
    out[1] = hc_se;
    out[2] = area;
    out[3] = area_se;
    out[4] = hd;
    out[5] = hu;
    if (mean_out) memcpy(mean_out, mean, sizeof(double) * (size_t)n);
    free(mean);
    free(loo);
}

/* Specific loss power (W/g) from a loop area S in Oe: f mu0 (1000/4 pi) Ms S / rho, with rho in
 * g/cm^3 (energy per cycle per volume times frequency, divided by the density). */
double orc_specific_loss_power(double f_hz, double Ms, double S_Oe, double rho_g_cm3)
{
    double w_per_m3 = f_hz * ORC_MU0 * ORC_OE_TO_AM * Ms * S_Oe;
    return w_per_m3 / (rho_g_cm3 * 1.0e6);
}

/* ------------------------------------------------------------------------------------------ */
/* Gradient of a loop-mismatch loss with respect to the calibration scale factors              */
/* (s_K, s_alpha, s_Ms), by forward-mode differentiation of the discrete Heun map.             */
/*                                                                                             */
/* The scale factors multiply K(b), alpha (everywhere it appears: g1, alpha g1 and the thermal */
/* variance) and Ms (in the exchange and anisotropy fields and the thermal variance; m stays a */
/* unit vector).  The thermal normals of each (realisation, cell, step) are fixed (pathwise,   */
/* common random numbers).  Every quantity carries its value and its derivatives along the    */
/* three scale factors; the arithmetic is the same as heun_step's.                             */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double v, d[3];
} dual;

static dual dconst(double v)
{
    dual r = {v, {0.0, 0.0, 0.0}};
    return r;
}
static dual dadd(dual a, dual b)
{
    dual r = {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
    return r;
}
static dual dsub(dual a, dual b)
{
    dual r = {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
    return r;
}
static dual dmul(dual a, dual b)
{
    dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
static dual ddiv(dual a, dual b)
{
    dual r;
    r.v = a.v / b.v;
    for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
static dual dsqrt(dual a)
{
    dual r;
    r.v = sqrt(a.v);
    for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] / (2.0 * r.v);
    return r;
}
static dual dscale(double s, dual a)
{
    dual r = {s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2]}};
    return r;
}

typedef struct {
    dual x, y, z;
} dvec;

static dvec dv_add(dvec a, dvec b)
{
    dvec r = {dadd(a.x, b.x), dadd(a.y, b.y), dadd(a.z, b.z)};
    return r;
}
static dvec dv_scale(dual s, dvec a)
{
    dvec r = {dmul(s, a.x), dmul(s, a.y), dmul(s, a.z)};
    return r;
}
static dvec dv_cross(dvec a, dvec b)
{
    dvec r = {dsub(dmul(a.y, b.z), dmul(a.z, b.y)), dsub(dmul(a.z, b.x), dmul(a.x, b.z)),
              dsub(dmul(a.x, b.y), dmul(a.y, b.x))};
    return r;
}
static dvec dv_normalise(dvec a)
{
    dual n = dsqrt(dadd(dadd(dmul(a.x, a.x), dmul(a.y, a.y)), dmul(a.z, a.z)));
    dvec r = {ddiv(a.x, n), ddiv(a.y, n), ddiv(a.z, n)};
    return r;
}

typedef struct {
    dual c_ex, c_an, g1, ag1, sigma;
} dcoeffs;

/* Coefficients of Eq. 1 and of the thermal field as functions of the three scale factors. */
static dcoeffs dual_coefficients(const orc_problem *p, const double scale[3])
{
    dual sK = {scale[0], {1.0, 0.0, 0.0}};
    dual sA = {scale[1], {0.0, 1.0, 0.0}};
    dual sM = {scale[2], {0.0, 0.0, 1.0}};
    dual K = dscale(p->K, sK), alpha = dscale(p->alpha, sA), Ms = dscale(p->Ms, sM);
    const double g0 = ORC_MU0 * ORC_GE;
    dcoeffs c;
    c.c_ex = ddiv(dconst(2.0 * p->A / (ORC_MU0 * p->a * p->a)), Ms);
    c.c_an = ddiv(dscale(2.0 / ORC_MU0, K), Ms);
    c.g1 = ddiv(dconst(g0), dadd(dconst(1.0), dmul(alpha, alpha)));
    c.ag1 = dmul(alpha, c.g1);
    c.sigma = p->T > 0.0 ? dsqrt(ddiv(dscale(2.0 * ORC_KB * p->T / (g0 * ORC_MU0 * p->volume * p->dt), alpha), Ms))
                         : dconst(0.0);
    return c;
}

static dvec dual_field(const orc_problem *p, const dcoeffs *c, const dvec *m, int x, int y, int z,
                       double Hz, dvec hth, const double *ax)
{
    dvec s = {dconst(0.0), dconst(0.0), dconst(0.0)};
    const int dims[3] = {p->nx, p->ny, p->nz};
    const int pos[3] = {x, y, z};
    for (int axis = 0; axis < 3; ++axis) {
        for (int dir = -1; dir <= 1; dir += 2) {
            int q[3] = {pos[0], pos[1], pos[2]};
            q[axis] += dir;
            if (q[axis] < 0 || q[axis] >= dims[axis]) {
                if (!(p->periodic & (1u << axis))) continue;
                q[axis] = (q[axis] + dims[axis]) % dims[axis];
            }
            int64_t j = q[0] + (int64_t)p->nx * (q[1] + (int64_t)p->ny * q[2]);
            s = dv_add(s, m[j]);
        }
    }
    int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
    /* anisotropy field c_an (m.u) u of the cell's easy axis u */
    const double *u = ax + 3 * i;
    dual mu = dadd(dadd(dscale(u[0], m[i].x), dscale(u[1], m[i].y)), dscale(u[2], m[i].z));
    dual a = dmul(c->c_an, mu);
    dvec H = dv_add(dv_scale(c->c_ex, s), hth);
    H.x = dadd(H.x, dscale(u[0], a));
    H.y = dadd(H.y, dscale(u[1], a));
    H.z = dadd(H.z, dadd(dscale(u[2], a), dconst(Hz)));
    return H;
}

static dvec dual_rhs(const dcoeffs *c, dvec m, dvec H)
{
    dvec mxH = dv_cross(m, H);
    dvec mxmxH = dv_cross(m, mxH);
    dvec r = dv_add(dv_scale(dscale(-1.0, c->g1), mxH), dv_scale(dscale(-1.0, c->ag1), mxmxH));
    return r;
}

typedef struct {
    const orc_problem *p;
    const double *scale;
    uint32_t seed, real0;
    int n_real;
    int64_t step0, n_steps, sample_every;
    const double *m0;      /* [n_real][N][3] */
    dual *mean_samples;    /* [n_samples_window], sums over realisations (each thread adds) */
    int64_t k_first, n_k;  /* sample numbers in the window */
    int next_real;
    pthread_mutex_t lock;
} grad_job;

static void *grad_worker(void *arg)
{
    grad_job *J = (grad_job *)arg;
    const orc_problem *p = J->p;
    const int64_t N = ncells_of(p);
    const dcoeffs c = dual_coefficients(p, J->scale);
    const double dt = p->dt;
    dvec *m = (dvec *)malloc(sizeof(dvec) * (size_t)N);
    dvec *mt = (dvec *)malloc(sizeof(dvec) * (size_t)N);
    dvec *f0 = (dvec *)malloc(sizeof(dvec) * (size_t)N);
    dvec *hth = (dvec *)malloc(sizeof(dvec) * (size_t)N);
    double *ax = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    dual *local = (dual *)calloc((size_t)J->n_k, sizeof(dual));
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int r = J->next_real++;
        pthread_mutex_unlock(&J->lock);
        if (r >= J->n_real) break;
        easy_axes(p, J->seed, J->real0 + (uint32_t)r, ax);
        for (int64_t i = 0; i < N; ++i) {
            const double *mi = J->m0 + ((int64_t)r * N + i) * 3;
            m[i].x = dconst(mi[0]);
            m[i].y = dconst(mi[1]);
            m[i].z = dconst(mi[2]);
        }
        for (int64_t s = 0; s < J->n_steps; ++s) {
            const int64_t n = J->step0 + s;
            const double Hn = orc_field_Oe(p, n) * ORC_OE_TO_AM, Hn1 = orc_field_Oe(p, n + 1) * ORC_OE_TO_AM;
            for (int64_t i = 0; i < N; ++i) {
                double xi[3];
                orc_thermal_normals(J->seed, J->real0 + (uint32_t)r, (uint32_t)i, (uint64_t)n, xi);
                hth[i].x = dscale(xi[0], c.sigma);
                hth[i].y = dscale(xi[1], c.sigma);
                hth[i].z = dscale(xi[2], c.sigma);
            }
            for (int z = 0; z < p->nz; ++z)
                for (int y = 0; y < p->ny; ++y)
                    for (int x = 0; x < p->nx; ++x) {
                        int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
                        dvec H = dual_field(p, &c, m, x, y, z, Hn, hth[i], ax);
                        f0[i] = dual_rhs(&c, m[i], H);
                        mt[i] = dv_normalise(dv_add(m[i], dv_scale(dconst(dt), f0[i])));
                    }
            for (int z = 0; z < p->nz; ++z)
                for (int y = 0; y < p->ny; ++y)
                    for (int x = 0; x < p->nx; ++x) {
                        int64_t i = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
                        dvec H = dual_field(p, &c, mt, x, y, z, Hn1, hth[i], ax);
                        dvec f1 = dual_rhs(&c, mt[i], H);
                        m[i] = dv_normalise(dv_add(m[i], dv_scale(dconst(0.5 * dt), dv_add(f0[i], f1))));
                    }
            const int64_t done = n + 1;
            if (J->sample_every > 0 && done % J->sample_every == 0) {
                const int64_t k = done / J->sample_every - J->k_first;
                if (k >= 0 && k < J->n_k) {
                    dual acc = dconst(0.0);
                    for (int64_t i = 0; i < N; ++i) acc = dadd(acc, m[i].z);
                    local[k] = dadd(local[k], dscale(1.0 / (double)N, acc));
                }
            }
        }
    }
    pthread_mutex_lock(&J->lock);
    for (int64_t k = 0; k < J->n_k; ++k) J->mean_samples[k] = dadd(J->mean_samples[k], local[k]);
    pthread_mutex_unlock(&J->lock);
    free(m);
    free(mt);
    free(f0);
    free(hth);
    free(ax);
    free(local);
    return NULL;
}

/* Loss L = (1/K) sum_k (mbar_k - target[k])^2 over the samples k of the window
 * (step0, step0 + n_steps] (sample k after step k * sample_every), mbar_k the realisation mean of
 * the cell-averaged m_z, starting from m0 [n_real][N][3] at step0, at the given scale factors.
 * out[0] = L, out[1..3] = dL/d(s_K, s_alpha, s_Ms); mean_out [K] (optional) = mbar_k.
 * target is indexed by the global sample number.  Returns the number K of samples used. */
int64_t orc_loss_grad(const orc_problem *p, const double scale[3], uint32_t seed, int n_real,
                      uint32_t real0, int64_t step0, int64_t n_steps, const double *m0,
                      int64_t sample_every, const double *target, double *out, double *mean_out,
                      int n_threads)
{
    const int64_t k_first = step0 / sample_every + 1;
    const int64_t k_last = (step0 + n_steps) / sample_every;
    const int64_t n_k = k_last >= k_first ? k_last - k_first + 1 : 0;
    grad_job J;
    J.p = p;
    J.scale = scale;
    J.seed = seed;
    J.real0 = real0;
    J.n_real = n_real;
    J.step0 = step0;
    J.n_steps = n_steps;
    J.sample_every = sample_every;
    J.m0 = m0;
    J.mean_samples = (dual *)calloc((size_t)(n_k > 0 ? n_k : 1), sizeof(dual));
    J.k_first = k_first;
    J.n_k = n_k;
    J.next_real = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_real) n_threads = n_real;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, grad_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    dual L = dconst(0.0);
    for (int64_t k = 0; k < n_k; ++k) {
        dual mbar = dscale(1.0 / (double)n_real, J.mean_samples[k]);
        if (mean_out) mean_out[k] = mbar.v;
        dual e = dsub(mbar, dconst(target[k_first + k]));
        L = dadd(L, dmul(e, e));
    }
    if (n_k > 0) L = dscale(1.0 / (double)n_k, L);
    out[0] = L.v;
    out[1] = L.d[0];
    out[2] = L.d[1];
    out[3] = L.d[2];
    free(J.mean_samples);
    return n_k;
}
