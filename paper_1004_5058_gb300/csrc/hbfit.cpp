// Herschel-Bulkley fit sigma = sigma_Y + A S^beta of a flow curve (the law the
// paper fits to its stress/shear scatter, section "Numerical Results").
//
// Variable projection: for a fixed beta the model is linear in (sigma_Y, A), so
// the best pair is the least-squares line through (x_i = S_i^beta, sigma_i).
// The residual sum of squares rss(beta) is minimised by a scan over
// [beta_lo, beta_hi] followed by golden-section refinement around the best scan
// point.  Host FP64.
#include <cmath>
#include <vector>

#include "lbhb.h"

namespace {

struct Fit {
    double sy, a, rss;
};

Fit linear_for_beta(const double* S, const double* sig, int n, double beta)
{
    double xm = 0.0, ym = 0.0;
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) {
        x[i] = std::pow(S[i], beta);
        xm += x[i];
        ym += sig[i];
    }
    xm /= n;
    ym /= n;
    double sxx = 0.0, sxy = 0.0;
    for (int i = 0; i < n; ++i) {
        sxx += (x[i] - xm) * (x[i] - xm);
        sxy += (x[i] - xm) * (sig[i] - ym);
    }
    Fit f;
    f.a = sxx > 0.0 ? sxy / sxx : 0.0;
    f.sy = ym - f.a * xm;
    f.rss = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = sig[i] - f.sy - f.a * x[i];
        f.rss += r * r;
    }
    return f;
}

}  // namespace

extern "C" lb_status lb_hb_fit(const double* shear_rate, const double* sigma, int n, double beta_lo,
                               double beta_hi, double* out)
{
    if (!shear_rate || !sigma || !out || n < 3) return LB_ERR_INVALID;
    if (!(beta_lo > 0.0) || !(beta_hi > beta_lo) || !std::isfinite(beta_hi)) return LB_ERR_INVALID;
    for (int i = 0; i < n; ++i)
        if (!(shear_rate[i] > 0.0) || !std::isfinite(shear_rate[i]) || !std::isfinite(sigma[i])) return LB_ERR_INVALID;
    const int scan = 4000;
    double best_b = beta_lo, best_r = INFINITY;
    for (int k = 0; k <= scan; ++k) {
        const double b = beta_lo + (beta_hi - beta_lo) * k / scan;
        const double r = linear_for_beta(shear_rate, sigma, n, b).rss;
        if (r < best_r) {
            best_r = r;
            best_b = b;
        }
    }
    const double step = (beta_hi - beta_lo) / scan;
    double lo = std::fmax(beta_lo, best_b - step), hi = std::fmin(beta_hi, best_b + step);
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double c = hi - gr * (hi - lo), d = lo + gr * (hi - lo);
    double fc = linear_for_beta(shear_rate, sigma, n, c).rss, fd = linear_for_beta(shear_rate, sigma, n, d).rss;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * (1.0 + std::fabs(lo)); ++it) {
        if (fc < fd) {
            hi = d;
            d = c;
            fd = fc;
            c = hi - gr * (hi - lo);
            fc = linear_for_beta(shear_rate, sigma, n, c).rss;
        } else {
            lo = c;
            c = d;
            fc = fd;
            d = lo + gr * (hi - lo);
            fd = linear_for_beta(shear_rate, sigma, n, d).rss;
        }
    }
    double b = 0.5 * (lo + hi);
    Fit f = linear_for_beta(shear_rate, sigma, n, b);
    if (!(f.rss <= best_r)) {
        b = best_b;
        f = linear_for_beta(shear_rate, sigma, n, b);
    }
    out[0] = f.sy;
    out[1] = f.a;
    out[2] = b;
    out[3] = f.rss;
    return LB_OK;
}
