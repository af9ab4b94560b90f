// Voigt function H(a, x) = Re w(x + i a), a > 0, from Weideman's rational
// expansion of the Faddeeva function (J. A. C. Weideman, SIAM J. Numer.
// Anal. 31 (1994) 1497).  For Im z > 0, w(z) = (i/pi) int exp(-t^2)/(z - t) dt.
// Writing exp(-t^2) = f(t)/(L^2 + t^2) with f(t) = (L^2 + t^2) exp(-t^2) and
// expanding f in the Fourier series of theta, t = L tan(theta/2), so that
// ((L + it)/(L - it))^n = exp(i n theta), every term integrates in closed
// form by residues:
//   w(z) = q/sqrt(pi) + 2 q^2 sum_{n>=1} a_n Z^(n-1),
//   q = 1/(L - iz),  Z = (L + iz)/(L - iz),
//   a_n = (1/2pi) int_{-pi}^{pi} f(L tan(theta/2)) cos(n theta) d theta
// (the n = 0 term gives q/sqrt(pi); negative n contribute nothing).  The
// series is cut after kVoigtTerms terms with Weideman's L = (N/sqrt 2)^(1/2);
// the coefficients come from the periodic trapezoid rule on the host, once.
// With z = x + i a, D = (L + a)^2 + x^2:
//   q = ((L + a) + i x)/D,   Z = ((L^2 - a^2 - x^2) + 2 i L x)/D,
// so one evaluation is a division, a few products and a complex Horner loop.
// Plain arithmetic only: the same code runs on the host and on the device.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define MG3D_HD __host__ __device__
#else
#define MG3D_HD
#endif

namespace mg3d {

constexpr int kVoigtTerms = 40;

struct VoigtTable {
    double L;
    double a[kVoigtTerms];   // a[n - 1] = a_n, n = 1..kVoigtTerms
};

// The coefficients by the periodic trapezoid rule on M midpoints in theta
// (spectrally accurate: f is smooth and vanishes with all derivatives at
// theta = +-pi).
inline void voigt_table(VoigtTable *t) {
    const double pi = 3.14159265358979323846;
    const int M = 1024;
    const double L = std::sqrt(kVoigtTerms / std::sqrt(2.0));
    t->L = L;
    for (int n = 0; n < kVoigtTerms; ++n) t->a[n] = 0.0;
    for (int k = 0; k < M; ++k) {
        const double th = -pi + (k + 0.5) * (2.0 * pi / M);
        const double s = L * std::tan(0.5 * th);
        const double f = (L * L + s * s) * std::exp(-s * s);
        if (f == 0.0) continue;
        for (int n = 1; n <= kVoigtTerms; ++n) t->a[n - 1] += f * std::cos(n * th);
    }
    for (int n = 0; n < kVoigtTerms; ++n) t->a[n] /= M;
}

// H(a, x) for a > 0 (not meant for a = 0, where H = exp(-x^2) is tiny in
// the wings while the expansion's error is absolute).
MG3D_HD inline double voigt_H_rational(const VoigtTable &t, double a, double x) {
    const double L = t.L;
    const double la = L + a;
    const double dinv = 1.0 / (la * la + x * x);
    const double qr = la * dinv, qi = x * dinv;
    const double zr = (L * L - a * a - x * x) * dinv, zi = 2.0 * L * x * dinv;
    double pr = t.a[kVoigtTerms - 1], pi_ = 0.0;
    for (int n = kVoigtTerms - 2; n >= 0; --n) {
        const double r = pr * zr - pi_ * zi + t.a[n];
        pi_ = pr * zi + pi_ * zr;
        pr = r;
    }
    // Re(2 p q^2) + Re(q)/sqrt(pi), q^2 = (qr^2 - qi^2) + 2 i qr qi
    const double q2r = qr * qr - qi * qi, q2i = 2.0 * qr * qi;
    return 2.0 * (pr * q2r - pi_ * q2i) + qr * 0.56418958354775628695;
}

}  // namespace mg3d
