// Zolotarev's best rational approximation of t^(-1/2), the coefficients of the EVD-free
// transform (host code, FP64, computed once per process).
//
// Zolotarev (1877) gave the best uniform rational approximation of sign(x) on
// [-1, -delta] U [delta, 1]: x R(x^2) with
//     R(t) = M prod_{l=1}^{n-1} (t + c_{2l}) / prod_{l=1}^{n} (t + c_{2l-1}),
//     c_j = delta^2 sn^2(j K' / (2n); k') / cn^2(j K' / (2n); k'),  k'^2 = 1 - delta^2,
// K' = K(k') the complete elliptic integral of the first kind and sn, cn the Jacobi elliptic
// functions.  Since sign(x) = x / sqrt(x^2), R(t) approximates t^(-1/2) on [delta^2, 1] with
// the same relative error, which falls like exp(-pi^2 n / ln(4 / delta)).  In partial
// fractions R(t) = sum_l beta_l / (t + p_l), p_l = c_{2l-1} > 0 and (for t^(-1/2), a Stieltjes
// function) every beta_l > 0.  M is fixed by equioscillation: the extremes of sqrt(t) R(t) on
// the interval are 1 -/+ err.
//
// The elliptic functions follow the arithmetic-geometric mean method (Abramowitz & Stegun
// 16.4, descending Landen transformation): K(m) = pi / (2 AGM(1, sqrt(1 - m))), and sn, cn
// from the amplitude recovered through the AGM's stored terms.
#include <math.h>

#include <mutex>

#include "kernels.h"
#include "letkf.h"

namespace lk {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Complete elliptic integral of the first kind, parameter m = k^2 < 1.
double ellip_k(double m) {
    double a = 1.0, b = sqrt(1.0 - m);
    for (int i = 0; i < 64 && fabs(a - b) > 1e-16 * a; ++i) {
        const double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return kPi / (2.0 * a);
}

// Jacobi elliptic functions sn(u | m), cn(u | m) by the AGM / descending Landen method.
void ellip_sncn(double u, double m, double *sn, double *cn) {
    double a[40], c[40];
    a[0] = 1.0;
    double b = sqrt(1.0 - m);
    c[0] = sqrt(m);
    int n = 0;
    while (n < 38 && fabs(c[n]) > 1e-16) {
        a[n + 1] = 0.5 * (a[n] + b);
        c[n + 1] = 0.5 * (a[n] - b);
        b = sqrt(a[n] * b);
        ++n;
    }
    double phi = ldexp(a[n] * u, n);
    for (int j = n; j > 0; --j) phi = 0.5 * (asin(c[j] * sin(phi) / a[j]) + phi);
    *sn = sin(phi);
    *cn = cos(phi);
}

}  // namespace

// Poles p_l and residues beta_l of the n-term approximation on [1/kappa, 1]; returns the
// largest relative error |sqrt(t) R(t) - 1| found on a fine logarithmic grid of the interval.
double zolotarev_rsqrt(double kappa, int n, double *poles, double *residues) {
    const double d2 = 1.0 / kappa, kp2 = 1.0 - d2;
    const double Kp = ellip_k(kp2);
    double c[2 * kMaxZoloPoles];
    for (int j = 1; j <= 2 * n - 1; ++j) {
        double sn, cn;
        ellip_sncn(j * Kp / (2.0 * n), kp2, &sn, &cn);
        c[j - 1] = d2 * sn * sn / (cn * cn);
    }
    // sqrt(t) prod (t + c_2l) / prod (t + c_2l-1) on the grid: its extremes fix M
    auto shape = [&](double t) {
        double v = sqrt(t);
        for (int l = 1; l <= n - 1; ++l) v *= t + c[2 * l - 1];
        for (int l = 1; l <= n; ++l) v /= t + c[2 * l - 2];
        return v;
    };
    const int G = 20000;
    double lo = 1e300, hi = -1e300;
    for (int g = 0; g <= G; ++g) {
        const double t = d2 * pow(kappa, (double)g / G);
        const double v = shape(t);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    const double M = 2.0 / (lo + hi);
    for (int l = 0; l < n; ++l) {
        const double p = c[2 * l];
        double r = M;
        for (int j = 1; j <= n - 1; ++j) r *= c[2 * j - 1] - p;
        for (int j = 0; j < n; ++j)
            if (j != l) r /= c[2 * j] - p;
        poles[l] = p;
        residues[l] = r;
    }
    double err = 0.0;
    for (int g = 0; g <= 4 * G; ++g) {
        const double t = d2 * pow(kappa, (double)g / (4 * G));
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += residues[l] / (t + poles[l]);
        err = fmax(err, fabs(sqrt(t) * s - 1.0));
    }
    return err;
}

// The approximations the EVD-free transform chooses from: the smallest n whose error stays
// near 1e-8 (well below FP32 rounding) for condition numbers up to kappa_max.
const ZoloTable &zolo_table() {
    static ZoloTable t;
    static std::once_flag once;
    std::call_once(once, [] {
        const double kmax[kZoloSets] = {1e2, 1e3, 1e4, 1e5, 1e6};
        const int nn[kZoloSets] = {8, 10, 12, 14, 16};
        for (int s = 0; s < kZoloSets; ++s) {
            double p[kMaxZoloPoles], r[kMaxZoloPoles];
            zolotarev_rsqrt(kmax[s], nn[s], p, r);
            t.kappa_max[s] = (float)kmax[s];
            t.n[s] = nn[s];
            for (int l = 0; l < kMaxZoloPoles; ++l) {
                t.pole[s][l] = l < nn[s] ? (float)p[l] : 0.0f;
                t.res[s][l] = l < nn[s] ? (float)r[l] : 0.0f;
            }
        }
    });
    return t;
}

}  // namespace lk

extern "C" double letkf_rational_coefficients(double kappa_max, int32_t n, double *poles,
                                              double *residues) {
    if (!(kappa_max > 1.0) || !(kappa_max < 1e12) || n < 1 || n > lk::kMaxZoloPoles || !poles ||
        !residues)
        return -1.0;
    return lk::zolotarev_rsqrt(kappa_max, n, poles, residues);
}
