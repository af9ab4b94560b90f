// Line profiles and redistribution functions for the host-built tables of the
// two-level atom (frequency table, partial-redistribution matrix).  Plain C++:
// evaluated once per handle, never on the device.
#pragma once

#include <cmath>

#include "voigt.cuh"

namespace mg3d {

// Adaptive Gauss-Kronrod (7-15 points) quadrature of f on [a, b] to an
// absolute tolerance tol, with a depth limit; the Kronrod nodes and weights
// are the standard published ones.
template <typename F>
double gk15(const F &f, double a, double b, double *err) {
    static const double xk[8] = {0.991455371120812639206854697526329,
                                 0.949107912342758524526189684047851,
                                 0.864864423359769072789712788640926,
                                 0.741531185599394439863864773280788,
                                 0.586087235467691130294144845693013,
                                 0.405845151377397166906606412076961,
                                 0.207784955007898467600689403773245,
                                 0.000000000000000000000000000000000};
    static const double wk[8] = {0.022935322010529224963732008058970,
                                 0.063092092629978553290700663189204,
                                 0.104790010322250183839876322541518,
                                 0.140653259715525918745189590510238,
                                 0.169004726639267902826583426598550,
                                 0.190350578064785409913256402421014,
                                 0.204432940075298892414161999234649,
                                 0.209482141084727828012999174891714};
    static const double wg[4] = {0.129484966168869693270611432679082,
                                 0.279705391489276667901467771423780,
                                 0.381830050505118944950369775488975,
                                 0.417959183673469387755102040816327};
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    const double fc = f(c);
    double rk = wk[7] * fc, rg = wg[3] * fc;
    for (int j = 0; j < 7; ++j) {
        const double d = h * xk[j];
        const double s = f(c - d) + f(c + d);
        rk += wk[j] * s;
        if (j % 2 == 1) rg += wg[j / 2] * s;
    }
    *err = std::fabs((rk - rg) * h);
    return rk * h;
}

// Bisects until the Gauss-Kronrod difference of a piece is below its share
// of tol (a difference that bounds the error of the 15-point result by far
// for smooth integrands), at most 20 levels deep.
template <typename F>
double bisect_gk(const F &f, double a, double b, double tol, int depth) {
    double err;
    const double v = gk15(f, a, b, &err);
    if (err <= tol || depth >= 20) return v;
    const double m = 0.5 * (a + b);
    return bisect_gk(f, a, m, 0.5 * tol, depth + 1) + bisect_gk(f, m, b, 0.5 * tol, depth + 1);
}

// Integral of f on [a, b] to a relative accuracy of about rel (and an
// absolute floor abs_floor), starting from the one-piece estimate.
template <typename F>
double integrate_adaptive(const F &f, double a, double b, double rel = 1e-13,
                          double abs_floor = 1e-300) {
    double err;
    const double v0 = gk15(f, a, b, &err);
    const double tol = std::fmax(rel * std::fabs(v0), abs_floor);
    if (err <= tol) return v0;
    return bisect_gk(f, a, b, tol, 0);
}

// Voigt function H(a, v) = (a/pi) int exp(-y^2)/((v - y)^2 + a^2) dy, written
// with y = v + a tan(t) as (1/pi) int_{-pi/2}^{pi/2} exp(-(v + a tan t)^2) dt
// (a smooth integrand); H(0, v) = exp(-v^2).  Even in v.
inline double voigt_H(double a, double v) {
    v = std::fabs(v);
    if (a <= 0.0) return std::exp(-v * v);
    auto f = [&](double t) {
        const double y = v + a * std::tan(t);
        return std::exp(-y * y);
    };
    // only |y| <= 8 contributes (exp(-64) ~ 1.6e-28 relative to the peak): the
    // t interval that maps onto it, split where y = 0
    const double t1 = std::atan((-8.0 - v) / a), t2 = std::atan((8.0 - v) / a);
    const double tp = std::atan(-v / a);
    return (integrate_adaptive(f, t1, tp) + integrate_adaptive(f, tp, t2)) /
           3.14159265358979323846;
}

// The coefficients of the rational Voigt function, computed once.
inline const VoigtTable &voigt_coefficients() {
    static const VoigtTable table = [] {
        VoigtTable t;
        voigt_table(&t);
        return t;
    }();
    return table;
}

// Hummer's angle-averaged R_II (damping a > 0): the average over the
// scattering angle g (weight sin g / 2) of R_II for fixed g,
//   (1/2pi) int_0^pi exp(-[(x - x')/(2 sin(g/2))]^2)
//                    H(a/cos(g/2), (x + x')/(2 cos(g/2))) dg;
// for a = 0 the closed form erfc(max(|x|, |x'|))/2 (R_I-A).  The integrand's
// H is the rational expansion (damping a/cos(g/2) >= a, relative error
// below 5e-14 + 2e-14/a), about a hundred times cheaper than the quadrature
// form, which matters for the n_freq^2/2 table entries.
inline double redistribution_r2a(double x, double xp, double a) {
    if (a <= 0.0) return 0.5 * std::erfc(std::fmax(std::fabs(x), std::fabs(xp)));
    const double pi = 3.14159265358979323846;
    const VoigtTable &tab = voigt_coefficients();
    auto f = [&](double g) {
        const double s = std::sin(0.5 * g), c = std::cos(0.5 * g);
        if (s <= 0.0 || c <= 0.0) return 0.0;
        const double d = (x - xp) / (2.0 * s);
        return std::exp(-d * d) * voigt_H_rational(tab, a / c, (x + xp) / (2.0 * c));
    };
    return integrate_adaptive(f, 0.0, pi) / (2.0 * pi);
}

}  // namespace mg3d
