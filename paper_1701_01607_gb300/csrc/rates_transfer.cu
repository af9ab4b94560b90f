// Rate equations (FP64) and FAS grid transfer.
//
// Rate kernel (Eqs. 2-4, 5, 9): per node, the partial sums of the sweep are
// added in slot order into Jeff = Jbar - Lambda* S and U = 1 - Lambda*.  The
// preconditioned radiative rates of MALI (Rybicki & Hummer 1991) are
//   P_lu = B_lu Jeff + C_lu,   P_ul = A_ul U + B_ul Jeff + C_ul
// (intensity unit 2 h nu^3/c^2, so B_ul = A_ul, B_lu = g_u/g_l A_ul), and
// with row 0 replaced by particle conservation (Eq. 3)
//   Gamma n = [ n_l + n_u ; n_u P_ul - n_l P_lu ].
// The MALI update solves Gamma n_new = f by eliminating n_l = f0 - n_u; the
// residual of Eq. 5 is f - Gamma n; the tau-corrected right-hand side of
// Eq. 9 adds Gamma n on the coarse grid to the restricted residual.
//
// Grid transfer (Sec. 4.4-4.6): full-weighting restriction over 27 nodes
// (periodic in x and y; on the two boundary planes the z stencil is the
// plane itself, so the boundary heights stay fixed), trilinear interpolation
// (linear in physical height for z), and the relative correction of
// Eqs. 10-11 with the 10 % rule for negative populations (Sec. 4.10).
#include "mg3d_internal.h"

namespace mg3d {

static int grid_for(long n, int threads) {
    long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152L * 32) b = 152L * 32;
    return (int)b;
}

__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}

// Block-wide max of a non-negative double, then one atomicMax on its bits
// (the bit patterns of non-negative doubles order like the values).
__device__ __forceinline__ void block_max_to(double v, unsigned long long *dst) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0 && v > 0.0) atomicMax(dst, dbits(v));
    }
}

__device__ __forceinline__ unsigned block_count(unsigned c) {
    __shared__ unsigned cnt[32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) cnt[wid] = c;
    __syncthreads();
    unsigned tot = 0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) tot += cnt[i];
    }
    return tot;  // valid in thread 0
}

template <typename TP>
__global__ void __launch_bounds__(256) rates_kernel(const RateArgs a) {
    const TP *__restrict__ pj = (const TP *)a.pj;
    const TP *__restrict__ pu = (const TP *)a.pu;
    const long nvox = a.nvox;
    double cmax = 0.0;
    unsigned neg = 0, bad = 0;
    // uniform trip count so that every thread reaches the block reductions
    const long stride = (long)gridDim.x * blockDim.x;
    for (long base = (long)blockIdx.x * blockDim.x; base < nvox; base += stride) {
        const long v = base + threadIdx.x;
        if (v >= nvox) continue;
        double J = 0.0, U = 1.0;
        if (!a.zero_radiation) {
            U = 0.0;
            for (int s = 0; s < a.nslots; ++s) {
                J += (double)pj[(long)s * nvox + v];
                U += (double)pu[(long)s * nvox + v];
            }
        }
        if (a.mode == kRateReduce) {
            a.out[v] = J;
            a.out[nvox + v] = U;
            continue;
        }
        const double A = a.a_ul;
        const double P_lu = a.g_ratio * A * J + a.c_lu[v];
        const double P_ul = A * U + A * J + a.c_ul[v];
        const double f0 = a.f ? a.f[v] : a.n_tot[v];
        const double f1 = a.f ? a.f[nvox + v] : 0.0;
        if (a.mode == kRateSolve) {
            const double nu_new = (f1 + f0 * P_lu) / (P_lu + P_ul);
            const double nl_new = f0 - nu_new;
            const double nl_old = a.n[v], nu_old = a.n[nvox + v];
            a.n[v] = nl_new;
            a.n[nvox + v] = nu_new;
            const double cl = fabs(nl_new - nl_old) / fabs(nl_new);
            const double cu = fabs(nu_new - nu_old) / fabs(nu_new);
            if (!(isfinite(nl_new) && isfinite(nu_new) && isfinite(cl) && isfinite(cu))) {
                ++bad;
            } else {
                cmax = fmax(cmax, fmax(cl, cu));
            }
            neg += (nl_new <= 0.0) + (nu_new <= 0.0);
        } else {
            const double nl = a.n[v], nu = a.n[nvox + v];
            const double w0 = nl + nu;
            const double w1 = nu * P_ul - nl * P_lu;
            if (a.mode == kRateResidual) {
                a.out[v] = f0 - w0;
                a.out[nvox + v] = f1 - w1;
            } else {
                a.out[v] += w0;
                a.out[nvox + v] += w1;
            }
        }
    }
    if (a.mode == kRateSolve && a.scal) {
        block_max_to(cmax, a.scal);
        unsigned tn = block_count(neg);
        unsigned tb = block_count(bad);
        if (threadIdx.x == 0) {
            if (tn) atomicAdd(a.scal + 1, (unsigned long long)tn);
            if (tb) atomicAdd(a.scal + 2, (unsigned long long)tb);
        }
    }
}

cudaError_t launch_rates(const RateArgs &a, cudaStream_t st) {
    const int th = 256;
    if (a.prec == 0)
        rates_kernel<double><<<grid_for(a.nvox, th), th, 0, st>>>(a);
    else
        rates_kernel<float><<<grid_for(a.nvox, th), th, 0, st>>>(a);
    return cudaGetLastError();
}

__global__ void collisions_up_kernel(long nvox, double g_ratio, double theta,
                                     const double *__restrict__ T,
                                     const double *__restrict__ c_ul, double *__restrict__ c_lu) {
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x)
        c_lu[v] = c_ul[v] * g_ratio * exp(-theta / T[v]);
}

cudaError_t launch_collisions_up(long nvox, double g_ratio, double theta, const double *T,
                                 const double *c_ul, double *c_lu, cudaStream_t st) {
    collisions_up_kernel<<<grid_for(nvox, 256), 256, 0, st>>>(nvox, g_ratio, theta, T, c_ul,
                                                              c_lu);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- restriction

// mode 0: full weighting (27 nodes), 1: half weighting (centre 1/2, six axis
// neighbours 1/12 each; on the boundary planes centre 1/2 and four in-plane
// neighbours 1/8 each), 2: injection.
template <typename V>
__global__ void restrict_kernel(int ncomp, int nxf, int nyf, int nzf, int mode,
                                const V *__restrict__ fine, V *__restrict__ coarse) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = (nzf + 1) / 2;
    const long nvc = (long)nxc * nyc * nzc, nvf = (long)nxf * nyf * nzf;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < nvc;
         c += (long)gridDim.x * blockDim.x) {
        const int I = (int)(c % nxc);
        const int J = (int)((c / nxc) % nyc);
        const int K = (int)(c / ((long)nxc * nyc));
        const bool boundary = (K == 0) || (K == nzc - 1);
        int xs[3], ys[3];
        const double wh[3] = {0.25, 0.5, 0.25};
        for (int d = 0; d < 3; ++d) {
            int xi = 2 * I + d - 1, yi = 2 * J + d - 1;
            xs[d] = xi < 0 ? xi + nxf : (xi >= nxf ? xi - nxf : xi);
            ys[d] = yi < 0 ? yi + nyf : (yi >= nyf ? yi - nyf : yi);
        }
        const long plane = (long)nxf * nyf;
        for (int comp = 0; comp < ncomp; ++comp) {
            const V *F = fine + comp * nvf;
            double acc = 0.0;
            if (mode == 2) {
                acc = F[(long)(2 * K) * plane + (long)ys[1] * nxf + xs[1]];
            } else if (mode == 1) {
                const V *P = F + (long)(2 * K) * plane;
                const double ctr = P[(long)ys[1] * nxf + xs[1]];
                const double inplane = (double)P[(long)ys[1] * nxf + xs[0]] +
                                       (double)P[(long)ys[1] * nxf + xs[2]] +
                                       (double)P[(long)ys[0] * nxf + xs[1]] +
                                       (double)P[(long)ys[2] * nxf + xs[1]];
                if (boundary) {
                    acc = 0.5 * ctr + inplane / 8.0;
                } else {
                    const double zpair =
                        (double)F[(long)(2 * K - 1) * plane + (long)ys[1] * nxf + xs[1]] +
                        (double)F[(long)(2 * K + 1) * plane + (long)ys[1] * nxf + xs[1]];
                    acc = 0.5 * ctr + (inplane + zpair) / 12.0;
                }
            } else {
                for (int dz = 0; dz < 3; ++dz) {
                    double wz;
                    int kf;
                    if (boundary) {
                        if (dz != 1) continue;
                        wz = 1.0;
                        kf = 2 * K;
                    } else {
                        wz = wh[dz];
                        kf = 2 * K + dz - 1;
                    }
                    const V *P = F + (long)kf * plane;
                    for (int dy = 0; dy < 3; ++dy) {
                        const V *R = P + (long)ys[dy] * nxf;
                        const double wy = wz * wh[dy];
                        acc += wy * (0.25 * (double)R[xs[0]] + 0.5 * (double)R[xs[1]] +
                                     0.25 * (double)R[xs[2]]);
                    }
                }
            }
            coarse[comp * nvc + c] = (V)acc;
        }
    }
}

cudaError_t launch_restrict(int ncomp, int nxf, int nyf, int nzf, const double *fine,
                            double *coarse, cudaStream_t st, int mode) {
    const long nvc = (long)(nxf / 2) * (nyf / 2) * ((nzf + 1) / 2);
    restrict_kernel<double><<<grid_for(nvc, 256), 256, 0, st>>>(ncomp, nxf, nyf, nzf, mode,
                                                                  fine, coarse);
    return cudaGetLastError();
}

cudaError_t launch_restrict_prec(int prec, int ncomp, int nxf, int nyf, int nzf,
                                 const void *fine, void *coarse, cudaStream_t st) {
    const long nvc = (long)(nxf / 2) * (nyf / 2) * ((nzf + 1) / 2);
    if (prec == 0)
        restrict_kernel<double><<<grid_for(nvc, 256), 256, 0, st>>>(
            ncomp, nxf, nyf, nzf, 0, (const double *)fine, (double *)coarse);
    else
        restrict_kernel<float><<<grid_for(nvc, 256), 256, 0, st>>>(
            ncomp, nxf, nyf, nzf, 0, (const float *)fine, (float *)coarse);
    return cudaGetLastError();
}

// -------------------------------------------------------------- prolongation

// Coarse corners and weights of fine node (i, j, k).  tz[k] is the weight of
// the upper coarse plane for an odd fine plane k (linear in height).
struct Corners {
    long idx[8];
    double w[8];
};

__device__ __forceinline__ void corners(long f, int nxc, int nyc, int nzc,
                                        const double *__restrict__ tz, Corners &cr) {
    const int nxf = 2 * nxc, nyf = 2 * nyc;
    const int i = (int)(f % nxf);
    const int j = (int)((f / nxf) % nyf);
    const int k = (int)(f / ((long)nxf * nyf));
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int i1 = (i & 1) ? (i0 + 1 == nxc ? 0 : i0 + 1) : i0;
    const int j1 = (j & 1) ? (j0 + 1 == nyc ? 0 : j0 + 1) : j0;
    const int k1 = (k & 1) ? k0 + 1 : k0;
    const double wx1 = (i & 1) ? 0.5 : 0.0, wy1 = (j & 1) ? 0.5 : 0.0;
    const double wz1 = (k & 1) ? tz[k] : 0.0;
    const int xs[2] = {i0, i1}, ys[2] = {j0, j1}, zs[2] = {k0, k1};
    const double wxs[2] = {1.0 - wx1, wx1}, wys[2] = {1.0 - wy1, wy1},
                 wzs[2] = {1.0 - wz1, wz1};
    int c = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) {
                cr.idx[c] = ((long)zs[a] * nyc + ys[b]) * nxc + xs[d];
                cr.w[c] = wzs[a] * wys[b] * wxs[d];
                ++c;
            }
}

template <typename V>
__global__ void prolong_kernel(int ncomp, int nxc, int nyc, int nzc,
                               const double *__restrict__ tz, const V *__restrict__ coarse,
                               V *__restrict__ fine) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    const long nvc = (long)nxc * nyc * nzc;
    for (long f = blockIdx.x * (long)blockDim.x + threadIdx.x; f < nvf;
         f += (long)gridDim.x * blockDim.x) {
        Corners cr;
        corners(f, nxc, nyc, nzc, tz, cr);
        for (int comp = 0; comp < ncomp; ++comp) {
            const V *C = coarse + comp * nvc;
            double acc = 0.0;
            for (int c = 0; c < 8; ++c) acc += cr.w[c] * (double)C[cr.idx[c]];
            fine[comp * nvf + f] = (V)acc;
        }
    }
}

// n_fine <- n_fine (1 + I(e)), e = (n_after - n_before)/n_before on the
// coarse grid (Eqs. 10-11); a result <= 0 becomes 0.1 n_fine (Sec. 4.10).
__global__ void __launch_bounds__(256) prolong_correct_kernel(
    int ncomp, int nxc, int nyc, int nzc, const double *__restrict__ tz,
    const double *__restrict__ n_after, const double *__restrict__ n_before,
    double *__restrict__ n_fine, unsigned long long *scal) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    const long nvc = (long)nxc * nyc * nzc;
    unsigned neg = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long base = (long)blockIdx.x * blockDim.x; base < nvf; base += stride) {
        const long f = base + threadIdx.x;
        if (f >= nvf) continue;
        Corners cr;
        corners(f, nxc, nyc, nzc, tz, cr);
        for (int comp = 0; comp < ncomp; ++comp) {
            const double *Aa = n_after + comp * nvc;
            const double *Bb = n_before + comp * nvc;
            double ie = 0.0;
            for (int c = 0; c < 8; ++c) {
                const long id = cr.idx[c];
                ie += cr.w[c] * ((Aa[id] - Bb[id]) / Bb[id]);
            }
            const double old = n_fine[comp * nvf + f];
            double nw = old * (1.0 + ie);
            if (nw <= 0.0) {
                nw = 0.1 * old;
                ++neg;
            }
            n_fine[comp * nvf + f] = nw;
        }
    }
    unsigned tn = block_count(neg);
    if (threadIdx.x == 0 && tn && scal) atomicAdd(scal + 3, (unsigned long long)tn);
}

// ------------------------------------ monotone cubic Hermite prolongation
// The other interpolation operator of Sec. 4.5: monotone cubic Hermite
// (Auer 2003) in successive 1D passes along x and y (periodic, uniform) and
// then z (at the physical heights).  On an odd index of an axis the fine
// node lies between two coarse nodes and takes the cubic through them, with
// slopes from their neighbours: the harmonic mean of the two adjacent
// secants where they have the same strict sign, else 0 (Fritsch & Butland
// 1984), weighted by the spacings in z, where the end nodes take the
// shape-preserving three-point slope.  On an even index the fine node keeps
// the coarse value along that axis.  A fine node reads the 4 x 4 x 4 coarse
// nodes around it, and each pass stays between the two coarse values of its
// interval.

__device__ __forceinline__ double mono_slope_unit(double a, double b) {
    return ((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0)) ? 2.0 * a * b / (a + b) : 0.0;
}

// cubic through q1, q2 at the midpoint, unit spacing
__device__ __forceinline__ double hermite_half(double q0, double q1, double q2, double q3) {
    const double d1 = mono_slope_unit(q1 - q0, q2 - q1);
    const double d2 = mono_slope_unit(q2 - q1, q3 - q2);
    return 0.5 * (q1 + q2) + 0.125 * (d1 - d2);
}

__device__ __forceinline__ int sign_of(double v) { return (v > 0.0) - (v < 0.0); }

__device__ __forceinline__ double slope_inner(double dm, double dp, double hm, double hp) {
    if (!((dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0))) return 0.0;
    const double w1 = 2.0 * hp + hm, w2 = hp + 2.0 * hm;
    return (w1 + w2) / (w1 / dm + w2 / dp);
}

// slope at an end node from the secant d0 of its interval (length h0) and
// the next one, d1 (length h1)
__device__ __forceinline__ double slope_end(double d0, double d1, double h0, double h1) {
    const double s = ((2.0 * h0 + h1) * d0 - h0 * d1) / (h0 + h1);
    if (sign_of(s) != sign_of(d0)) return 0.0;
    if (sign_of(d0) != sign_of(d1) && fabs(s) > 3.0 * fabs(d0)) return 3.0 * d0;
    return s;
}

// x then y pass on coarse plane kk for fine column (i, j); get(kk, y, x)
// returns a coarse value
template <typename Get>
__device__ __forceinline__ double hermite_xy(const Get &get, int kk, int i, int j, int nxc,
                                             int nyc) {
    auto xrow = [&](int yy) -> double {
        const int i0 = i >> 1;
        if (!(i & 1)) return get(kk, yy, i0);
        const int im = i0 == 0 ? nxc - 1 : i0 - 1;
        const int i1 = i0 + 1 == nxc ? 0 : i0 + 1;
        const int i2 = i1 + 1 == nxc ? 0 : i1 + 1;
        return hermite_half(get(kk, yy, im), get(kk, yy, i0), get(kk, yy, i1), get(kk, yy, i2));
    };
    const int j0 = j >> 1;
    if (!(j & 1)) return xrow(j0);
    const int jm = j0 == 0 ? nyc - 1 : j0 - 1;
    const int j1 = j0 + 1 == nyc ? 0 : j0 + 1;
    const int j2 = j1 + 1 == nyc ? 0 : j1 + 1;
    return hermite_half(xrow(jm), xrow(j0), xrow(j1), xrow(j2));
}

// the fine value at fine node f; zf: the fine grid's heights (coarse plane
// m at zf[2m])
template <typename Get>
__device__ double hermite_fine(const Get &get, long f, int nxc, int nyc, int nzc,
                               const double *__restrict__ zf) {
    const int nxf = 2 * nxc, nyf = 2 * nyc;
    const int i = (int)(f % nxf);
    const int j = (int)((f / nxf) % nyf);
    const int k = (int)(f / ((long)nxf * nyf));
    const int K = k >> 1;
    if (!(k & 1)) return hermite_xy(get, K, i, j, nxc, nyc);
    const double zK = zf[2 * K], zK1 = zf[2 * K + 2];
    const double h = zK1 - zK;
    const double qK = hermite_xy(get, K, i, j, nxc, nyc);
    const double qK1 = hermite_xy(get, K + 1, i, j, nxc, nyc);
    const double dK = (qK1 - qK) / h;
    double sK = dK, sK1 = dK;
    if (nzc > 2) {
        double dm = 0.0, hm = 0.0;
        if (K > 0) {
            hm = zK - zf[2 * K - 2];
            dm = (qK - hermite_xy(get, K - 1, i, j, nxc, nyc)) / hm;
        }
        double dp = 0.0, hp = 0.0;
        if (K + 2 < nzc) {
            hp = zf[2 * K + 4] - zK1;
            dp = (hermite_xy(get, K + 2, i, j, nxc, nyc) - qK1) / hp;
        }
        sK = K > 0 ? slope_inner(dm, dK, hm, h) : slope_end(dK, dp, h, hp);
        sK1 = K + 2 < nzc ? slope_inner(dK, dp, h, hp) : slope_end(dK, dm, h, hm);
    }
    const double t = (zf[k] - zK) / h, t2 = t * t, t3 = t2 * t;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * qK + (t3 - 2.0 * t2 + t) * h * sK +
           (-2.0 * t3 + 3.0 * t2) * qK1 + (t3 - t2) * h * sK1;
}

template <typename V>
__global__ void __launch_bounds__(256) prolong_hermite_kernel(
    int ncomp, int nxc, int nyc, int nzc, const double *__restrict__ zf,
    const V *__restrict__ coarse, V *__restrict__ fine) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    const long nvc = (long)nxc * nyc * nzc;
    for (long f = blockIdx.x * (long)blockDim.x + threadIdx.x; f < nvf;
         f += (long)gridDim.x * blockDim.x) {
        for (int comp = 0; comp < ncomp; ++comp) {
            const V *C = coarse + comp * nvc;
            auto get = [&](int kk, int yy, int xx) -> double {
                return (double)C[((long)kk * nyc + yy) * nxc + xx];
            };
            fine[comp * nvf + f] = (V)hermite_fine(get, f, nxc, nyc, nzc, zf);
        }
    }
}

// e = (n_after - n_before)/n_before written over n_before (Eq. 10)
__global__ void rel_correction_kernel(long len, const double *__restrict__ n_after,
                                      double *__restrict__ n_before) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < len;
         i += (long)gridDim.x * blockDim.x)
        n_before[i] = (n_after[i] - n_before[i]) / n_before[i];
}

// n_fine <- n_fine (1 + I(e)) with the Hermite I, and the 10 % rule
__global__ void __launch_bounds__(256) prolong_correct_hermite_kernel(
    int ncomp, int nxc, int nyc, int nzc, const double *__restrict__ zf,
    const double *__restrict__ e, double *__restrict__ n_fine, unsigned long long *scal) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    const long nvc = (long)nxc * nyc * nzc;
    unsigned neg = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long base = (long)blockIdx.x * blockDim.x; base < nvf; base += stride) {
        const long f = base + threadIdx.x;
        if (f >= nvf) continue;
        for (int comp = 0; comp < ncomp; ++comp) {
            const double *E = e + comp * nvc;
            auto get = [&](int kk, int yy, int xx) -> double {
                return E[((long)kk * nyc + yy) * nxc + xx];
            };
            const double ie = hermite_fine(get, f, nxc, nyc, nzc, zf);
            const double old = n_fine[comp * nvf + f];
            double nw = old * (1.0 + ie);
            if (nw <= 0.0) {
                nw = 0.1 * old;
                ++neg;
            }
            n_fine[comp * nvf + f] = nw;
        }
    }
    unsigned tn = block_count(neg);
    if (threadIdx.x == 0 && tn && scal) atomicAdd(scal + 3, (unsigned long long)tn);
}

cudaError_t launch_prolong(int interp, int ncomp, int nxc, int nyc, int nzc, const double *tz,
                           const double *zf, const double *coarse, double *fine,
                           cudaStream_t st) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    if (interp)
        prolong_hermite_kernel<double><<<grid_for(nvf, 256), 256, 0, st>>>(ncomp, nxc, nyc, nzc,
                                                                         zf, coarse, fine);
    else
        prolong_kernel<double><<<grid_for(nvf, 256), 256, 0, st>>>(ncomp, nxc, nyc, nzc, tz,
                                                                     coarse, fine);
    return cudaGetLastError();
}

cudaError_t launch_prolong_prec(int interp, int prec, int ncomp, int nxc, int nyc, int nzc,
                                const double *tz, const double *zf, const void *coarse,
                                void *fine, cudaStream_t st) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    if (interp && prec == 0)
        prolong_hermite_kernel<double><<<grid_for(nvf, 256), 256, 0, st>>>(
            ncomp, nxc, nyc, nzc, zf, (const double *)coarse, (double *)fine);
    else if (interp)
        prolong_hermite_kernel<float><<<grid_for(nvf, 256), 256, 0, st>>>(
            ncomp, nxc, nyc, nzc, zf, (const float *)coarse, (float *)fine);
    else if (prec == 0)
        prolong_kernel<double><<<grid_for(nvf, 256), 256, 0, st>>>(
            ncomp, nxc, nyc, nzc, tz, (const double *)coarse, (double *)fine);
    else
        prolong_kernel<float><<<grid_for(nvf, 256), 256, 0, st>>>(
            ncomp, nxc, nyc, nzc, tz, (const float *)coarse, (float *)fine);
    return cudaGetLastError();
}

cudaError_t launch_prolong_correct(int interp, int ncomp, int nxc, int nyc, int nzc,
                                   const double *tz, const double *zf, const double *n_after,
                                   double *n_before, double *n_fine, unsigned long long *scal,
                                   cudaStream_t st) {
    const long nvf = (long)(2 * nxc) * (2 * nyc) * (2 * nzc - 1);
    if (interp) {
        const long len = (long)ncomp * nxc * nyc * nzc;
        rel_correction_kernel<<<grid_for(len, 256), 256, 0, st>>>(len, n_after, n_before);
        prolong_correct_hermite_kernel<<<grid_for(nvf, 256), 256, 0, st>>>(
            ncomp, nxc, nyc, nzc, zf, n_before, n_fine, scal);
        return cudaGetLastError();
    }
    prolong_correct_kernel<<<grid_for(nvf, 256), 256, 0, st>>>(ncomp, nxc, nyc, nzc, tz,
                                                                 n_after, n_before, n_fine,
                                                                 scal);
    return cudaGetLastError();
}

// C = max |n_new - n_old| / |n_new| into scal[0]; non-finite into scal[2].
__global__ void __launch_bounds__(256) max_rel_change_kernel(long len,
                                                             const double *__restrict__ a,
                                                             const double *__restrict__ b,
                                                             unsigned long long *scal) {
    double m = 0.0;
    unsigned bad = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long base = (long)blockIdx.x * blockDim.x; base < len; base += stride) {
        const long i = base + threadIdx.x;
        if (i >= len) continue;
        const double c = fabs(a[i] - b[i]) / fabs(a[i]);
        if (isfinite(c)) m = fmax(m, c);
        else ++bad;
    }
    block_max_to(m, scal);
    unsigned tb = block_count(bad);
    if (threadIdx.x == 0 && tb) atomicAdd(scal + 2, (unsigned long long)tb);
}

cudaError_t launch_max_rel_change(long len, const double *n_new, const double *n_old,
                                  unsigned long long *scal, cudaStream_t st) {
    max_rel_change_kernel<<<grid_for(len, 256), 256, 0, st>>>(len, n_new, n_old, scal);
    return cudaGetLastError();
}

}  // namespace mg3d
