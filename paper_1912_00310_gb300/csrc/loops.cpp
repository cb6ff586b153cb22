// loops.cpp -- host-side loop observables of the library: mean M(H) loop over realisations,
// coercive field from the zero crossings of the mean loop (with one standard error, as quoted
// for the Fig. 2 loops), loop area, and the rescale to the unscaled system (Eqs. 10, 11, 13).
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

extern "C" llg_status llg_loop_stats_host(const float *m_samples, int n_real, int64_t n_samples,
                                          const double *H_Oe, int64_t k_turn, int mode, double zeta,
                                          double delta, llg_loop_stats *out, double *mean_out)
{
    if (!m_samples || !H_Oe || !out || n_real < 1 || n_samples < 2 || k_turn < 1 ||
        k_turn >= n_samples || mode < 0 || mode > 2)
        return LLG_EINVAL;
    std::vector<double> sum((size_t)n_samples, 0.0), mean((size_t)n_samples), loo((size_t)n_samples);
    for (int r = 0; r < n_real; ++r)
        for (int64_t k = 0; k < n_samples; ++k) sum[(size_t)k] += m_samples[(size_t)r * n_samples + k];
    for (int64_t k = 0; k < n_samples; ++k) mean[(size_t)k] = sum[(size_t)k] / n_real;
    const llg::LoopValues all = llg::evaluate(H_Oe, mean.data(), n_samples, k_turn);
    double hc_se = NAN, area_se = NAN;
    if (n_real > 1) {
        std::vector<double> jh((size_t)n_real), ja((size_t)n_real);
        for (int r = 0; r < n_real; ++r) {
            for (int64_t k = 0; k < n_samples; ++k)
                loo[(size_t)k] = (sum[(size_t)k] - m_samples[(size_t)r * n_samples + k]) / (n_real - 1);
            const llg::LoopValues v = llg::evaluate(H_Oe, loo.data(), n_samples, k_turn);
            jh[(size_t)r] = v.hc;
            ja[(size_t)r] = v.area;
        }
        double mh = 0.0, ma = 0.0;
        for (int r = 0; r < n_real; ++r) {
            mh += jh[(size_t)r];
            ma += ja[(size_t)r];
        }
        mh /= n_real;
        ma /= n_real;
        double vh = 0.0, va = 0.0;
        for (int r = 0; r < n_real; ++r) {
            vh += (jh[(size_t)r] - mh) * (jh[(size_t)r] - mh);
            va += (ja[(size_t)r] - ma) * (ja[(size_t)r] - ma);
        }
        hc_se = std::sqrt(vh * (n_real - 1) / n_real);
        area_se = std::sqrt(va * (n_real - 1) / n_real);
    }
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
    if (mean_out)
        for (int64_t k = 0; k < n_samples; ++k) mean_out[k] = mean[(size_t)k];
    return LLG_OK;
}
