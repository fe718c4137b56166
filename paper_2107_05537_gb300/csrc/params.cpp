// Chi-square tail and upper quantile for integer degrees of freedom
// (Lemma 1: r'^2/r^2 ~ chi^2(m); Lemma 3: upper quantile chi^2_alpha(m);
// Eq. 9: t^2 = chi^2_{alpha1}(m), t^2 = c^2 chi^2_{1-alpha2}(m)).
//
// For integer m the tail has a finite closed form (repeated integration by
// parts of the Gamma(m/2, 2) density):
//   m = 2h:    Pr[X > x] = e^{-x/2} sum_{i=0}^{h-1} (x/2)^i / i!
//   m = 2h+1:  Pr[X > x] = erfc(sqrt(x/2))
//                          + e^{-x/2} sum_{i=1}^{h} (x/2)^{i-1/2} / Gamma(i+1/2)
// Every term is positive, so the sums lose no accuracy.  The quantile is
// found by safeguarded Newton steps on the density, then bisection down to
// adjacent doubles.
#include <cmath>

#include "pmlsh_impl.h"

double pm_chi2_sf(double x, int m)
{
    if (!(x > 0.0)) return 1.0;
    const double y = 0.5 * x;
    const double ey = std::exp(-y);
    if ((m & 1) == 0) {
        double term = 1.0, sum = 1.0;
        for (int i = 1; i < m / 2; i++) {
            term *= y / i;
            sum += term;
        }
        return ey * sum;
    }
    double sum = 0.0;
    double term = 2.0 * std::sqrt(y) / std::sqrt(M_PI);  // y^{1/2} / Gamma(3/2)
    for (int i = 1; i <= m / 2; i++) {
        sum += term;
        term *= y / (i + 0.5);
    }
    return std::erfc(std::sqrt(y)) + ey * sum;
}

static double chi2_pdf(double x, int m)
{
    if (!(x > 0.0)) return 0.0;
    double a = 0.5 * m;
    return std::exp((a - 1.0) * std::log(x) - 0.5 * x - a * std::log(2.0) - std::lgamma(a));
}

double pm_chi2_upper_quantile(double alpha, int m)
{
    if (!(alpha > 0.0 && alpha < 1.0) || m < 1) return NAN;
    double lo = 0.0, hi = 2.0 * m + 10.0;
    while (pm_chi2_sf(hi, m) > alpha) { lo = hi; hi *= 2.0; }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 60; it++) {
        double f = pm_chi2_sf(x, m) - alpha;      // decreasing in x
        if (f > 0.0) lo = x; else hi = x;
        double p = chi2_pdf(x, m);
        double nx = p > 0.0 ? x + f / p : 0.5 * (lo + hi);
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (nx == x) break;
        x = nx;
    }
    // finish by bisection so that [lo, hi] are adjacent doubles
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (pm_chi2_sf(mid, m) > alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}
