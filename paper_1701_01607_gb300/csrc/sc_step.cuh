// Linear short-characteristics step shared by the sweep kernels.
#pragma once

#include <cuda_runtime.h>

#include "mg3d_internal.h"

namespace mg3d {

// Linear short-characteristics weights for optical path x:
//   I = I_up exp(-x) + w_up S_up + w_0 S_0,
//   u = (1 - exp(-x))/x, w_0 = 1 - u, w_up = u - exp(-x).
// Below a threshold the closed forms cancel, so Taylor series are used.  The
// FP32 variant uses the hardware exp2 approximation (__expf): its error grows
// with x, but exp(-x) then multiplies a term that is already negligible.
template <typename T>
struct ScWeights;

// Row band of a global row: ya / rows by multiplication with
// magic = ceil(2^32 / rows), exact for ya, rows < 2^16 (checked exhaustively
// for rows up to 2048 and sampled above).  Grids are limited to ny < 2^16.
__host__ __device__ inline unsigned long long band_magic(int rows) {
    return ((1ull << 32) + (unsigned long long)rows - 1) / (unsigned long long)rows;
}
__device__ __forceinline__ int band_of(int ya, unsigned long long magic) {
    return (int)(((unsigned long long)(unsigned)ya * magic) >> 32);
}

// 1/x in the formal-solution precision: FP64 correctly rounded; FP32 the
// hardware approximation (within 2 ulp), ample for the FP32 formal solution.
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
// 1/x of an optical path for the closed-form weights, which use it only where
// x is above the series threshold (far from 0 and from overflow).  FP64: the
// hardware approximation (about 23 correct bits) refined by two Newton-Raphson
// steps r <- r + r (1 - x r), each of which doubles the correct bits, in place
// of an IEEE division with its range checks.
__device__ __forceinline__ float sc_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double sc_rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// e^{-x} for x >= 0 by the table-driven method of Tang (ACM TOMS 15, 1989):
// -x = (256 m + j) ln2/256 + r with integer m, j in [0, 256) and
// |r| <= ln2/512, so e^{-x} = 2^m 2^{j/256} e^r.  The reduction uses a
// two-part ln2/256 whose high part (34 significant bits) times any |n| < 2^19
// is exact; e^r - 1 is its Taylor polynomial of degree 4 (truncation < 4e-17
// relative); 2^{j/256} comes from a 256-entry table and 2^m is applied by
// adding m to the exponent field.  Results below e^{-708} are flushed to zero.
struct ExpNegTable {
    const double *tab;   // [kExpTab] 2^{j/256}
    double l1, l2;       // ln2/256 = l1 + l2
};

__device__ __forceinline__ double exp_neg(double x, const ExpNegTable e) {
    const bool flush = x > 708.0;
    x = flush ? 0.0 : x;
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    const double t = fma(x, -369.3299304675746, magic);  // -x * 256/ln2, rounded to an integer
    const int n = __double2loint(t);
    const double nd = t - magic;
    double r = fma(-nd, e.l1, -x);
    r = fma(-nd, e.l2, r);
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    const double q = p * r;                      // e^r - 1
    const double tj = e.tab[n & (kExpTab - 1)];
    const double v = fma(tj, q, tj);             // 2^{j/256} e^r, in [0.99, 2.01)
    const long long bits = __double_as_longlong(v) + ((long long)(n >> 8) << 52);
    return flush ? 0.0 : __longlong_as_double(bits);
}

// exp_neg with the range test on the high word of x (an integer compare on
// the integer pipe instead of an FP64 compare): x >= 708, infinite or NaN
// gives 0 (0x40862000 is the high word of 708.0; a non-negative double orders
// like its bit pattern).  The reduction and polynomial are exp_neg's; for x
// past the test the intermediate values are discarded.
__device__ __forceinline__ double exp_neg_hi(double x, const ExpNegTable e) {
    const bool flush = __double2hiint(x) >= 0x40862000;
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    const double t = fma(x, -369.3299304675746, magic);
    const int n = __double2loint(t);
    const double nd = t - magic;
    double r = fma(-nd, e.l1, -x);
    r = fma(-nd, e.l2, r);
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    const double q = p * r;
    const double tj = e.tab[n & (kExpTab - 1)];
    const double v = fma(tj, q, tj);
    const long long bits = __double_as_longlong(v) + ((long long)(n >> 8) << 52);
    return __longlong_as_double(flush ? 0ll : bits);
}

// closed() has no branch, so a caller can evaluate several independent steps
// back to back and patch the small-x ones with series() afterwards; eval()
// takes one form or the other per lane.
template <>
struct ScWeights<double> {
    // inv_x = 1/x, formed by the caller as (1/dtau0)(1/phi): one division per
    // node and ray instead of one per frequency.
    static __device__ __forceinline__ void closed(double x, double inv_x, const ExpNegTable et,
                                                  double &ex, double &w0, double &wup,
                                                  double &u) {
        ex = exp_neg(x, et);
        u = fma(-ex, inv_x, inv_x);   // (1 - e^-x)/x
        w0 = 1.0 - u;
        wup = u - ex;
    }
    static __device__ __forceinline__ bool small(double x) { return x < 1e-3; }
    // coefficients as products with rounded reciprocals (a division would
    // expand to an iteration with a slow-path branch per evaluation)
    static __device__ __forceinline__ void series(double x, double &w0, double &wup, double &u) {
        w0 = x * (0.5 - x * (1.0 / 6.0 - x * (1.0 / 24.0 - x * (1.0 / 120.0 - x * (1.0 / 720.0)))));
        wup = x * (0.5 - x * (1.0 / 3.0 - x * (1.0 / 8.0 - x * (1.0 / 30.0 - x * (1.0 / 144.0)))));
        u = 1.0 - w0;
    }
    // one of the two forms per lane (the closed form's three operations are
    // skipped where the series applies)
    static __device__ __forceinline__ void eval(double x, double inv_x, const ExpNegTable et,
                                                double &ex, double &w0, double &wup, double &u) {
        ex = exp_neg(x, et);
        if (small(x)) {
            series(x, w0, wup, u);
        } else {
            u = fma(-ex, inv_x, inv_x);
            w0 = 1.0 - u;
            wup = u - ex;
        }
    }
};

template <>
struct ScWeights<float> {
    static __device__ __forceinline__ void closed(float x, float inv_x, const ExpNegTable,
                                                  float &ex, float &w0, float &wup, float &u) {
        ex = __expf(-x);
        u = fmaf(-ex, inv_x, inv_x);   // (1 - e^-x)/x
        w0 = 1.0f - u;
        wup = u - ex;
    }
    static __device__ __forceinline__ bool small(float x) { return x < 0.1f; }
    static __device__ __forceinline__ void series(float x, float &w0, float &wup, float &u) {
        w0 = x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f - x * (1.0f / 120.0f - x * (1.0f / 720.0f)))));
        wup = x * (0.5f - x * (1.0f / 3.0f - x * (1.0f / 8.0f - x * (1.0f / 30.0f - x * (1.0f / 144.0f)))));
        u = 1.0f - w0;
    }
    static __device__ __forceinline__ void eval(float x, float inv_x, const ExpNegTable et,
                                                float &ex, float &w0, float &wup, float &u) {
        closed(x, inv_x, et, ex, w0, wup, u);
        if (small(x)) series(x, w0, wup, u);
    }
};

// Monotone cubic Hermite upwind interpolation (the Hermite-spline option of
// Sec. 3; Auer 2003).  The slope at a node of a uniform periodic row, in
// units of one cell, is the harmonic mean 2ab/(a+b) of its two adjacent
// secants a and b when they have the same strict sign, else 0 (Fritsch &
// Butland 1984); the cubic on [0, 1] through p0, p1 with slopes d0, d1 at t
// is c0 p0 + c1 d0 + c2 p1 + c3 d1 with the Hermite basis c of t.  Rows are
// interpolated along x, then the four row values along y.
// Branch-free: the division always runs (on 1 where the slope is 0), so a
// warp whose lanes disagree on the sign test does not split.
template <typename T>
__device__ __forceinline__ T mono_slope(T a, T b) {
    const bool same = (a > T(0) && b > T(0)) || (a < T(0) && b < T(0));
    const T q = T(2) * a * b * rcp(same ? a + b : T(1));
    return same ? q : T(0);
}

template <typename T>
struct HermiteBasis {
    T c0, c1, c2, c3;
    __device__ __forceinline__ explicit HermiteBasis(T t) {
        const T t2 = t * t, t3 = t2 * t;
        c0 = T(2) * t3 - T(3) * t2 + T(1);
        c1 = t3 - T(2) * t2 + t;
        c2 = T(3) * t2 - T(2) * t3;
        c3 = t3 - t2;
    }
    // the cubic from values and slopes
    __device__ __forceinline__ T at(T p0, T d0, T p1, T d1) const {
        return c0 * p0 + c1 * d0 + c2 * p1 + c3 * d1;
    }
    // the cubic between q1 and q2 of four consecutive values
    __device__ __forceinline__ T through4(T q0, T q1, T q2, T q3) const {
        return at(q1, mono_slope(q1 - q0, q2 - q1), q2, mono_slope(q2 - q1, q3 - q2));
    }
};

}  // namespace mg3d
