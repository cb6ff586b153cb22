// scaling.cpp -- host FP64 parameter setup of one job: the coarse-graining map (Eqs. 8-13), the
// coefficients of Eq. 1 and of the Brown thermal field, the triangle and sinusoidal field sweeps and
// the numerical Grinstein-Koch flow (Eqs. 4-7).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "llg_internal.h"

namespace llg {

namespace {
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kMu0 = 4.0e-7 * kPi;           // T m / A
constexpr double kGammaE = 1.76e11;             // rad / (s T), Eq. 1
constexpr double kBoltzmann = 1.380649e-23;     // J / K
constexpr double kAmPerOe = 1000.0 / (4.0 * kPi);

// Whole number of steps in x, or -1 when x is not within 1e-6 relative of one.
long long whole_steps(double x)
{
    const double r = std::nearbyint(x);
    if (!(std::fabs(x - r) <= 1e-6 * std::fmax(1.0, std::fabs(x)))) return -1;
    return (long long)r;
}
}  // namespace

// zeta(b) = t/b + 1 - t with t = T/Tc (text after Eq. 11).
double zeta_of(double b, double T, double Tc)
{
    const double t = T / Tc;
    return t / b + (1.0 - t);
}

bool derive(int b, double a0, const MaterialIn &mat, const ScalingIn &sc, const SweepIn &sw,
            Derived *d, char *err, size_t errlen, double volume_m3)
{
    const bool cg = sc.mode == 1 || sc.mode == 2;
    d->zeta = cg ? zeta_of((double)b, mat.T, sc.Tc) : 1.0;
    // Eqs. 8-9 (A(b) = zeta A0, K(b) = zeta^3 K0) and the calibration scale factors.
    d->A = d->zeta * mat.A0;
    d->K = d->zeta * d->zeta * d->zeta * mat.K0 * sc.sK;
    d->Ms = mat.Ms * sc.sMs;
    d->alpha = mat.alpha * sc.sAlpha;
    d->a = b * a0;
    d->V = volume_m3 > 0.0 ? volume_m3 : d->a * d->a * d->a;
    // Eq. 1 gyromagnetic factors
    d->g0 = kMu0 * kGammaE;
    d->g1 = d->g0 / (1.0 + d->alpha * d->alpha);
    d->ag1 = d->alpha * d->g1;
    // exchange (6-neighbour stencil, bond energy 2 A a (1 - m_i.m_j)) and uniaxial anisotropy
    d->c_ex = 2.0 * d->A / (kMu0 * d->Ms * d->a * d->a);
    d->c_an = 2.0 * d->K / (kMu0 * d->Ms);
    // Brown thermal field: per component, per cell and step, variance
    // 2 alpha kB T / (gamma0 mu0 Ms V dt)
    d->sigma = mat.T > 0.0
                   ? std::sqrt(2.0 * d->alpha * kBoltzmann * mat.T / (d->g0 * kMu0 * d->Ms * d->V * sw.dt))
                   : 0.0;
    d->shape = sw.shape;
    d->period = 0;
    // sinusoidal sweep (the paper's H_max sin(2 pi f t), started at its maximum:
    // H = H_max cos(2 pi n / period)), SR = 4 H_max f
    d->H_start_Am = sw.H_start_Oe * kAmPerOe;
    d->H_turn_Am = sw.H_turn_Oe * kAmPerOe;
    if (sw.shape == 1) {
        if (!(sw.H_start_Oe > 0.0) || !(sw.rate_Oe_per_ns > 0.0)) {
            std::snprintf(err, errlen, "the sinusoidal sweep needs an amplitude H_start > 0 and a rate > 0");
            return false;
        }
        const double per_step = sw.rate_Oe_per_ns * 1e9 * sw.dt;  // Oe of nominal sweep per step
        d->period = whole_steps(4.0 * sw.H_start_Oe / per_step);
        d->sample_every = whole_steps(sw.sample_dH_Oe / per_step);
        if (d->period <= 0 || d->sample_every <= 0 || d->period % d->sample_every != 0 || d->period % 2 != 0) {
            std::snprintf(err, errlen, "the period 4 H_max / (rate dt) must be an even whole number of steps "
                                       "and a whole number of sample intervals");
            return false;
        }
        d->n_half = d->period / 2;  // half a cycle: the descending branch
        d->slope_Am = 0.0;
        d->steps_per_loop = d->period;
        d->n_samples = d->period / d->sample_every + 1;
        d->m_rescale = sc.mode == 1 ? d->zeta : (sc.mode == 2 ? sc.delta * d->zeta + (1.0 - sc.delta) : 1.0);
        return true;
    }
    // triangle sweep
    const double span = std::fabs(sw.H_start_Oe - sw.H_turn_Oe);
    if (sw.rate_Oe_per_ns > 0.0 && span > 0.0) {
        const double per_step = sw.rate_Oe_per_ns * 1e9 * sw.dt;  // Oe per step
        d->n_half = whole_steps(span / per_step);
        if (d->n_half <= 0) {
            std::snprintf(err, errlen, "sweep span %.9g Oe is not a whole number of %.9g Oe steps",
                          span, per_step);
            return false;
        }
        d->sample_every = whole_steps(sw.sample_dH_Oe / per_step);
        if (d->sample_every <= 0) {
            std::snprintf(err, errlen, "sample spacing %.9g Oe is not a whole number of %.9g Oe steps",
                          sw.sample_dH_Oe, per_step);
            return false;
        }
        d->slope_Am = (d->H_turn_Am - d->H_start_Am) / (double)d->n_half;
        d->steps_per_loop = 2 * d->n_half;
        if (d->steps_per_loop % d->sample_every != 0) {
            std::snprintf(err, errlen, "a loop of %lld steps is not a whole number of samples",
                          d->steps_per_loop);
            return false;
        }
        d->n_samples = d->steps_per_loop / d->sample_every + 1;
    } else {
        // constant field; sample_dH counts steps
        d->n_half = 0;
        d->slope_Am = 0.0;
        d->sample_every = whole_steps(sw.sample_dH_Oe);
        if (d->sample_every <= 0) d->sample_every = 1;
        d->steps_per_loop = 0;
        d->n_samples = std::max(1LL, sw.held_samples);  // sample k after step k * sample_every
    }
    // Eq. 11 (mode 1) or Eq. 13 (mode 2) rescale of m back to the unscaled system
    d->m_rescale = sc.mode == 1 ? d->zeta : (sc.mode == 2 ? sc.delta * d->zeta + (1.0 - sc.delta) : 1.0);
    return true;
}

KParams kparams_of(const Derived &d, int nx, int ny, int nz, unsigned periodic, double dt)
{
    KParams p{};
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.ncells = nx * ny * nz;
    p.periodic = periodic;
    p.c_ex = (float)d.c_ex;
    p.c_an = (float)d.c_an;
    p.sigma = (float)d.sigma;
    p.neg_dt_g1 = (float)(-dt * d.g1);
    p.neg_hdt_g1 = (float)(-0.5 * dt * d.g1);
    p.alpha = (float)d.alpha;
    p.H0 = (float)d.H_start_Am;
    p.slope = (float)d.slope_Am;
    p.n_half = d.shape == 1 ? 0 : d.n_half;
    p.shape = d.shape;
    p.amp = (float)d.H_start_Am;
    p.period = d.period;
    p.sample_every = d.sample_every;
    p.n_samples = d.n_samples;
    return p;
}

// Grinstein-Koch flow (Eqs. 4-7) in l = ln b, fourth-order Runge-Kutta with n_steps equal steps;
// state {T*, h, g, I} with I the running integral of F, zeta = exp(-I).
void gk_flow(double Ts0, double h0, double g0, double b, long long n_steps, double out[4])
{
    struct S {
        double Ts, h, g, I;
    };
    auto rate = [](const S &s) {
        const double F = s.Ts / (2.0 * kPi * (1.0 + s.h + s.g));
        return S{(F - 1.0) * s.Ts, 2.0 * s.h, 2.0 * (1.0 - F) * s.g, F};
    };
    auto step = [](const S &s, const S &k, double c) {
        return S{s.Ts + c * k.Ts, s.h + c * k.h, s.g + c * k.g, s.I + c * k.I};
    };
    const double dl = std::log(b) / (double)n_steps;
    S s{Ts0, h0, g0, 0.0};
    for (long long i = 0; i < n_steps; ++i) {
        const S k1 = rate(s);
        const S k2 = rate(step(s, k1, 0.5 * dl));
        const S k3 = rate(step(s, k2, 0.5 * dl));
        const S k4 = rate(step(s, k3, dl));
        const S sum{k1.Ts + 2.0 * (k2.Ts + k3.Ts) + k4.Ts, k1.h + 2.0 * (k2.h + k3.h) + k4.h,
                    k1.g + 2.0 * (k2.g + k3.g) + k4.g, k1.I + 2.0 * (k2.I + k3.I) + k4.I};
        s = step(s, sum, dl / 6.0);
    }
    out[0] = s.Ts;
    out[1] = s.h;
    out[2] = s.g;
    out[3] = std::exp(-s.I);
}

double field_Oe(const Derived &d, const SweepIn &w, long long n)
{
    if (d.shape == 1) {
        const long long ph = n % d.period;
        return w.H_start_Oe * std::cos(2.0 * kPi * (double)ph / (double)d.period);
    }
    if (d.n_half <= 0) return w.H_start_Oe;
    const long long ph = n % (2 * d.n_half);
    const long long tri = ph <= d.n_half ? ph : 2 * d.n_half - ph;
    return w.H_start_Oe + (w.H_turn_Oe - w.H_start_Oe) * ((double)tri / (double)d.n_half);
}

}  // namespace llg
