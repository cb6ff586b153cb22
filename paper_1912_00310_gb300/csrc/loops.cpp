// loops.cpp -- host-side loop observables of the library: mean M(H) loop over realisations,
// coercive field from the zero crossings of the mean loop (with one standard error, as quoted
// for the Fig. 2 loops), loop area, and the rescale to the unscaled system (Eqs. 10, 11, 13).
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/llg.h"
#include "llg_internal.h"

namespace llg {
namespace {

// Field of the first sign change of m in samples [k0, k1] (descending: + to -, else - to +),
// linearly interpolated; NaN when there is none.
double first_crossing(const double *H, const double *m, int64_t k0, int64_t k1, bool descending)
{
    for (int64_t k = k0; k < k1; ++k) {
        const double a = m[k], b = m[k + 1];
        const bool cross = descending ? (a > 0.0 && b <= 0.0) : (a < 0.0 && b >= 0.0);
        if (cross) return H[k] + (H[k + 1] - H[k]) * (a / (a - b));
    }
    return NAN;
}

struct LoopValues {
    double hc, down, up, area;
};

LoopValues evaluate(const double *H, const double *m, int64_t n, int64_t k_turn)
{
    LoopValues v;
    v.down = first_crossing(H, m, 0, k_turn, true);
    v.up = first_crossing(H, m, k_turn, n - 1, false);
    v.hc = 0.5 * (std::fabs(v.down) + std::fabs(v.up));
    double s = 0.0;
    for (int64_t k = 0; k + 1 < n; ++k) s += (H[k + 1] - H[k]) * 0.5 * (m[k] + m[k + 1]);
    v.area = std::fabs(s);
    return v;
}

}  // namespace
}  // namespace llg

namespace llg {
namespace {

void finish(const LoopValues &all, double hc_se, double area_se, int mode, double zeta, double delta,
            llg_loop_stats *out)
{
    out->Hc_Oe = all.hc;
    out->Hc_se_Oe = hc_se;
    out->area_Oe = all.area;
    out->area_se_Oe = area_se;
    out->Hc_down_Oe = all.down;
    out->Hc_up_Oe = all.up;
    out->zeta = zeta;
    out->m_rescale = mode == 1 ? zeta : (mode == 2 ? delta * zeta + 1.0 - delta : 1.0);
    const double hs = mode == 0 ? 1.0 : zeta;  // H0 = H(b) / zeta (Eq. 10)
    out->Hc0_Oe = all.hc / hs;
    out->area0_Oe = all.area * out->m_rescale / hs;
}

// Delete-one jackknife terms of the realisations in m_samples against an ensemble whose
// per-sample sums over all n_total realisations are sum_all: with theta_(r) the statistic of the
// mean loop without realisation r and theta the statistic of the full mean loop,
// out = {sum_r d_hc, sum_r d_hc^2, sum_r d_area, sum_r d_area^2}, d = theta_(r) - theta (shifted by
// theta so that the variance is formed without cancellation).
void jackknife_terms(const float *m_samples, int n_local, int64_t n_samples, const double *sum_all, int n_total,
                     const double *H_Oe, int64_t k_turn, double out[4])
{
    std::vector<double> mean((size_t)n_samples), loo((size_t)n_samples);
    for (int64_t k = 0; k < n_samples; ++k) mean[(size_t)k] = sum_all[k] / n_total;
    const LoopValues all = evaluate(H_Oe, mean.data(), n_samples, k_turn);
    for (int i = 0; i < 4; ++i) out[i] = 0.0;
    for (int r = 0; r < n_local; ++r) {
        for (int64_t k = 0; k < n_samples; ++k)
            loo[(size_t)k] = (sum_all[k] - m_samples[(size_t)r * n_samples + k]) / (n_total - 1);
        const LoopValues v = evaluate(H_Oe, loo.data(), n_samples, k_turn);
        const double dh = v.hc - all.hc, da = v.area - all.area;
        out[0] += dh;
        out[1] += dh * dh;
        out[2] += da;
        out[3] += da * da;
    }
}

// Jackknife standard error sqrt((n-1)/n sum_r (theta_(r) - mean_r theta_(r))^2) from the shifted
// sums of jackknife_terms.
double jackknife_se(double s1, double s2, int n)
{
    const double ss = s2 - s1 * s1 / n;
    return std::sqrt(std::max(0.0, ss) * (n - 1) / n);
}

}  // namespace
}  // namespace llg

extern "C" llg_status llg_loop_moments(const float *m_samples, int n_real, int64_t n_samples, double *sum_out,
                                       double *sumsq_out)
{
    if (!sum_out || n_real < 0 || (n_real > 0 && !m_samples) || n_samples < 1) {
        llg::set_last_error("need samples (unless n_real is 0), n_real >= 0, n_samples >= 1 and an output array");
        return LLG_EINVAL;
    }
    for (int64_t k = 0; k < n_samples; ++k) {
        sum_out[k] = 0.0;
        if (sumsq_out) sumsq_out[k] = 0.0;
    }
    for (int r = 0; r < n_real; ++r)
        for (int64_t k = 0; k < n_samples; ++k) {
            const double v = m_samples[(size_t)r * n_samples + k];
            sum_out[k] += v;
            if (sumsq_out) sumsq_out[k] += v * v;
        }
    return LLG_OK;
}

extern "C" llg_status llg_loop_jackknife_terms(const float *m_samples, int n_local, int64_t n_samples,
                                               const double *sum_all, int n_total, const double *H_Oe,
                                               int64_t k_turn, double out[4])
{
    if (!sum_all || !H_Oe || !out || n_local < 0 || (n_local > 0 && !m_samples) || n_total < 2 ||
        n_local > n_total || n_samples < 2 || k_turn < 1 || k_turn >= n_samples) {
        llg::set_last_error("bad arguments to llg_loop_jackknife_terms");
        return LLG_EINVAL;
    }
    llg::jackknife_terms(m_samples, n_local, n_samples, sum_all, n_total, H_Oe, k_turn, out);
    return LLG_OK;
}

extern "C" llg_status llg_loop_stats_from_sums(const double *sum_all, int n_total, int64_t n_samples,
                                               const double *H_Oe, int64_t k_turn, const double jk[4], int mode,
                                               double zeta, double delta, llg_loop_stats *out, double *mean_out)
{
    if (!sum_all || !H_Oe || !out || n_total < 1 || n_samples < 2 || k_turn < 1 || k_turn >= n_samples ||
        mode < 0 || mode > 2) {
        llg::set_last_error("bad arguments to llg_loop_stats_from_sums");
        return LLG_EINVAL;
    }
    std::vector<double> mean((size_t)n_samples);
    for (int64_t k = 0; k < n_samples; ++k) mean[(size_t)k] = sum_all[k] / n_total;
    const llg::LoopValues all = llg::evaluate(H_Oe, mean.data(), n_samples, k_turn);
    double hc_se = NAN, area_se = NAN;
    if (n_total > 1 && jk) {
        hc_se = llg::jackknife_se(jk[0], jk[1], n_total);
        area_se = llg::jackknife_se(jk[2], jk[3], n_total);
    }
    llg::finish(all, hc_se, area_se, mode, zeta, delta, out);
    if (mean_out)
        for (int64_t k = 0; k < n_samples; ++k) mean_out[k] = mean[(size_t)k];
    return LLG_OK;
}

extern "C" llg_status llg_loop_stats_host(const float *m_samples, int n_real, int64_t n_samples,
                                          const double *H_Oe, int64_t k_turn, int mode, double zeta,
                                          double delta, llg_loop_stats *out, double *mean_out)
{
    if (!m_samples || !H_Oe || !out || n_real < 1 || n_samples < 2 || k_turn < 1 ||
        k_turn >= n_samples || mode < 0 || mode > 2) {
        llg::set_last_error("bad arguments to llg_loop_stats_host");
        return LLG_EINVAL;
    }
    // the single-process case of the distributed reduction: sums, jackknife terms, statistics
    std::vector<double> sum((size_t)n_samples);
    llg_loop_moments(m_samples, n_real, n_samples, sum.data(), nullptr);
    double jk[4] = {0.0, 0.0, 0.0, 0.0};
    if (n_real > 1) llg::jackknife_terms(m_samples, n_real, n_samples, sum.data(), n_real, H_Oe, k_turn, jk);
    return llg_loop_stats_from_sums(sum.data(), n_real, n_samples, H_Oe, k_turn, n_real > 1 ? jk : nullptr, mode,
                                    zeta, delta, out, mean_out);
}

extern "C" llg_status llg_specific_loss_power(double f_hz, double Ms, double area_Oe, double rho_kg_m3,
                                              double *W_per_g)
{
    if (!W_per_g || !(f_hz >= 0.0) || !(Ms > 0.0) || !(rho_kg_m3 > 0.0) || !std::isfinite(area_Oe)) {
        llg::set_last_error("need f >= 0, Ms > 0, rho > 0, a finite area and an output");
        return LLG_EINVAL;
    }
    // energy per cycle and volume mu0 Ms |closed integral of m dH| (H in A/m: 1 Oe = 1000/4pi A/m),
    // times the frequency, per mass
    const double mu0 = 4e-7 * 3.14159265358979323846;
    const double w_per_m3 = f_hz * mu0 * Ms * area_Oe * (1000.0 / (4.0 * 3.14159265358979323846));
    *W_per_g = w_per_m3 / rho_kg_m3 / 1000.0;
    return LLG_OK;
}
