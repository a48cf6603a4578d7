// Host-side Trotter-schedule helpers of the C ABI: the magnitude ordering of
// the cluster operators (Section 2.3) and the Trotter-error extrapolation
// E(M) = alpha (1/M)^beta + gamma (Section 3.2, Fig. 3).  No device use.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/uccsd.h"

namespace {

// For a fixed exponent the model is linear in (alpha, gamma): u_m = M_m^-beta,
// alpha = cov(u, E) / var(u), gamma = mean(E) - alpha mean(u).  Returns the
// residual sum of squares, evaluated from the residuals themselves.
double fit_linear(int n, const double *M, const double *E, double beta, double *alpha,
                  double *gamma) {
    std::vector<double> u(n);
    double mu = 0.0, me = 0.0;
    for (int m = 0; m < n; ++m) {
        u[m] = std::pow(M[m], -beta);
        mu += u[m];
        me += E[m];
    }
    mu /= n;
    me /= n;
    double suu = 0.0, sue = 0.0;
    for (int m = 0; m < n; ++m) {
        suu += (u[m] - mu) * (u[m] - mu);
        sue += (u[m] - mu) * (E[m] - me);
    }
    const double a = suu > 0.0 ? sue / suu : 0.0;
    const double g = me - a * mu;
    double rss = 0.0;
    for (int m = 0; m < n; ++m) {
        const double r = a * u[m] + g - E[m];
        rss += r * r;
    }
    *alpha = a;
    *gamma = g;
    return rss;
}

}  // namespace

extern "C" {

uccsd_status uccsd_magnitude_order(int K, const int32_t *ijab, const double *t, int32_t *ijab_out,
                                   int32_t *perm) {
    if (K < 0 || (K > 0 && (!ijab || !t || !ijab_out))) return UCCSD_ERR_ARG;
    for (int k = 0; k < K; ++k)
        if (!std::isfinite(t[k])) return UCCSD_ERR_ARG;
    std::vector<int32_t> idx(K);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [t](int32_t a, int32_t b) { return std::fabs(t[a]) > std::fabs(t[b]); });
    std::vector<int32_t> rows(4 * size_t(K));
    for (int k = 0; k < K; ++k) std::memcpy(&rows[4 * size_t(k)], ijab + 4 * size_t(idx[k]), 16);
    if (K > 0) std::memcpy(ijab_out, rows.data(), rows.size() * sizeof(int32_t));
    if (perm && K > 0) std::memcpy(perm, idx.data(), idx.size() * sizeof(int32_t));
    return UCCSD_OK;
}

uccsd_status uccsd_trotter_extrapolate(int n, const int *M, const double *E, double *out) {
    if (n < 3 || !M || !E || !out) return UCCSD_ERR_ARG;
    std::vector<double> Md(n);
    for (int m = 0; m < n; ++m) {
        if (M[m] < 1 || !std::isfinite(E[m])) return UCCSD_ERR_ARG;
        Md[m] = double(M[m]);
    }
    int distinct = 0;
    {
        std::vector<int> s(M, M + n);
        std::sort(s.begin(), s.end());
        distinct = int(std::unique(s.begin(), s.end()) - s.begin());
    }
    if (distinct < 3) return UCCSD_ERR_ARG;
    // Variable projection: minimise the residual over beta alone.  A scan of
    // log-spaced exponents in [1e-3, 64] brackets the best minimum; golden-
    // section search then narrows the bracket to rounding level.
    const int n_scan = 2001;
    const double lo = std::log(1e-3), hi = std::log(64.0);
    auto beta_at = [&](int i) { return std::exp(lo + (hi - lo) * i / (n_scan - 1)); };
    double a, g;
    int best = 0;
    double best_rss = HUGE_VAL;
    for (int i = 0; i < n_scan; ++i) {
        const double r = fit_linear(n, Md.data(), E, beta_at(i), &a, &g);
        if (r < best_rss) {
            best_rss = r;
            best = i;
        }
    }
    double x0 = beta_at(std::max(best - 1, 0)), x3 = beta_at(std::min(best + 1, n_scan - 1));
    const double rg = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = x3 - rg * (x3 - x0), x2 = x0 + rg * (x3 - x0);
    double f1 = fit_linear(n, Md.data(), E, x1, &a, &g);
    double f2 = fit_linear(n, Md.data(), E, x2, &a, &g);
    for (int it = 0; it < 200 && (x3 - x0) > 1e-15 * x3; ++it) {
        if (f1 <= f2) {
            x3 = x2;
            x2 = x1;
            f2 = f1;
            x1 = x3 - rg * (x3 - x0);
            f1 = fit_linear(n, Md.data(), E, x1, &a, &g);
        } else {
            x0 = x1;
            x1 = x2;
            f1 = f2;
            x2 = x0 + rg * (x3 - x0);
            f2 = fit_linear(n, Md.data(), E, x2, &a, &g);
        }
    }
    const double beta = f1 <= f2 ? x1 : x2;
    fit_linear(n, Md.data(), E, beta, &a, &g);
    out[0] = a;
    out[1] = beta;
    out[2] = g;
    return UCCSD_OK;
}

}  // extern "C"
