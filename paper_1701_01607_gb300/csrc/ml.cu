// Multi-level atom: opacity per frequency and node, the plane sweep with all
// rays of a hemisphere in one thread block, and the N x N rate equations.
//
// Opacity (Eq. 1, Sec. 2.1, Sec. 3).  Every frequency point belongs to one
// transition (lower l, upper u); with the grey LTE background chi_c:
//   chi = chi_t + chi_c,  S = (eta_t + chi_c B_nu) / chi,
//   sc = chi_c B_nu / chi = S - eta_t / chi (the part of S the transition's
//        populations do not set),
//   oc = chi_c / chi = 1 - chi_t / chi (the opacity share they do not set),
// each formed directly, not as a difference.
// Line:        chi_t = kappa (n_l g_u/g_l - n_u) phi,  eta_t = kappa rho^3 n_u phi,
//              phi = exp(-(x/d)^2)/(sqrt(pi) d), d = sqrt(T/t_ref), B at line centre.
// Bound-free:  chi_t = kappa y^-3 (n_l - n_u G E),  eta_t = kappa y^-3 n_u G E (rho y)^3,
//              G = n_l*/n_u*, E = exp(-theta_ref rho y/T).
//
// Sweep.  One thread-block cluster per (frequency, group of rays of one
// hemisphere: 12, 6, 4, 3, 2 or 1 rays); its blocks split the plane in row
// bands and each holds the intensity planes of the group's rays, double
// buffered.  A thread owns a node and walks the group's rays, so the angle
// sums
//   Jx = sum_r w_r (I - w0 eta_t/chi),   Ux = sum_r w_r (1 - w0 chi_t/chi)
// over the group are complete in registers and written once per group; the
// radiative sums below add the groups in order.  They are accumulated as
//   Jx = sum (I - w0 S) + sc sum w0,   Ux = sum (1 - w0) + oc sum w0,
// where I - w0 S = I_up e^-x + w_up S_up and 1 - w0 = u come from the step
// itself: every term is non-negative, so in FP32 no cancellation between
// I and w0 eta_t/chi (nearly equal in an optically thick line) degrades
// them.  The MALI rates of a scattering-dominated line depend on the small
// difference J - Lambda* S, so this order keeps the FP32 formal solution
// accurate there.
//
// Rates (Rybicki & Hummer 1992, diagonal operator).  Per node, for a line:
//   Jbar = sum wphi Jx, Ubar = sum wphi Ux (wphi: trapezoid x profile,
//   normalised per node), P_lu += B_lu Jbar, P_ul += A_ul Ubar + B_ul Jbar;
// for a bound-free continuum (qa = beta w_y y^-4):
//   P_lc += sum qa Jx,   P_cl += G sum qa E ((rho y)^3 Ux + Jx);
// plus collisions; row 0 is particle conservation (Eq. 3); the N x N system
// is solved by Gaussian elimination with partial pivoting.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "mg3d.h"
#include "mg3d_internal.h"
#include "sc_step.cuh"
#include "voigt.cuh"

namespace cg = cooperative_groups;

namespace mg3d {

static int grid_for(long n, int threads) {
    long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152L * 32) b = 152L * 32;
    return (int)b;
}

__device__ __forceinline__ double planck_rho(double rho, double theta_ref, double T) {
    return rho * rho * rho / expm1(theta_ref * rho / T);
}

// ------------------------------------------------------------------ opacity

// exp(-x), x >= 0, in the opacity's precision: the sweep's table-driven FP64
// exp, or the FP32 library exp for the FP32 formal solution.
__device__ __forceinline__ double opac_exp(double x, const ExpNegTable &et) {
    return exp_neg(x, et);
}
__device__ __forceinline__ float opac_exp(float x, const ExpNegTable &) { return expf(-x); }

// Line profile exp(-dd2) di / sqrt(pi) in the formal-solution precision.
__device__ __forceinline__ double ml_doppler(double dd2, double di, const ExpNegTable &et) {
    return exp_neg(dd2, et) * di * 0.56418958354775628;
}
__device__ __forceinline__ float ml_doppler(float dd2, float di, const ExpNegTable &) {
    return __expf(-dd2) * di * 0.564189584f;
}

// A line's profile at a node of Doppler width d = 1/inv_d reference widths,
// per reference width: the Doppler profile in the formal-solution precision,
// or for a damped line (damping a at t_ref; the node's parameter a/d, since
// the damping width does not scale with temperature) H(a/d, x/d)/(sqrt(pi) d)
// from the rational Voigt function in FP64, rounded once.
template <typename T>
__device__ __forceinline__ T ml_line_phi(const FreqInfo &q, double inv_d, T pnorm,
                                         const VoigtTable *vt, const ExpNegTable &et) {
    const double xd = q.xy * inv_d;
    if (q.adamp > 0.0)
        return (T)(voigt_H_rational(*vt, q.adamp * inv_d, xd) * 0.5641895835477563 * inv_d);
    return opac_exp((T)(xd * xd), et) * pnorm;
}

// One thread per node walks the chunk's frequencies, so per-node quantities
// (temperature, Doppler width, background) and per-transition ones
// (populations, the line-centre Planck function) are formed once.  The
// profile and the source terms are evaluated in the formal-solution
// precision T; population differences in FP64.
template <typename T>
__global__ void ml_opacity_kernel(const MlOpacityArgs a) {
    __shared__ double tab[kExpTab];
    for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) tab[i] = a.exp_tab[i];
    __syncthreads();
    const ExpNegTable et{tab, a.exp_l1, a.exp_l2};
    const double rsqpi = 0.5641895835477563;  // 1/sqrt(pi)
    const long nvox = a.nvox;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x) {
        const double Tg = a.T[v];
        const double cc = a.chi_c[v];
        const double inv_d = sqrt(a.t_ref / Tg);   // 1/d, d = sqrt(T/t_ref)
        const T pnorm = (T)(rsqpi * inv_d);
        int lo = -1, up = -1;
        double nl = 0.0, nu = 0.0, G = 0.0, rho_b = -1.0;
        T B = 0;
        for (int fl = 0; fl < a.nfreq; ++fl) {
            const FreqInfo q = a.fi[a.f0 + fl];
            if (q.lo != lo || q.up != up) {
                lo = q.lo;
                up = q.up;
                nl = a.n[(long)lo * nvox + v];
                nu = a.n[(long)up * nvox + v];
                G = a.saha[(long)lo * nvox + v];
                rho_b = -1.0;
            }
            T chi_t, eta_t;
            if (q.kind == 0) {
                if (q.rho != rho_b) {
                    rho_b = q.rho;
                    B = (T)planck_rho(q.rho, a.theta_ref, Tg);
                }
                const T phi = ml_line_phi<T>(q, inv_d, pnorm, a.voigt, et);
                chi_t = (T)q.kappa * phi * (T)(q.gr * nl - nu);
                eta_t = (T)(q.kappa * q.rho * q.rho * q.rho) * (T)nu * phi;
            } else {
                const double y = q.xy;
                const T E = opac_exp((T)(a.theta_ref * q.rho * y / Tg), et);
                const double ry = q.rho * y;
                const T alpha = (T)(q.kappa / (y * y * y));
                chi_t = alpha * ((T)nl - (T)(nu * G) * E);
                eta_t = alpha * (T)(nu * G * ry * ry * ry) * E;
                B = (T)planck_rho(ry, a.theta_ref, Tg);
                rho_b = -1.0;
            }
            const long i = (long)fl * nvox + v;
            if (a.moving) {
                // ray-independent parts; a line's profile is applied per ray
                // in the sweep (continua do not shift)
                T ca = chi_t, ea = eta_t;
                if (q.kind == 0) {
                    ca = (T)q.kappa * (T)(q.gr * nl - nu);
                    ea = (T)(q.kappa * q.rho * q.rho * q.rho) * (T)nu;
                }
                T cb = (T)cc, eb = (T)cc * B;
                if (a.sigma_c) {
                    const T sg = (T)a.sigma_c[v];
                    cb += sg;
                    eb += sg * ((const T *)a.jbg)[(long)(a.f0 + fl) * nvox + v];
                }
                ((T *)a.chi)[i] = ca;
                ((T *)a.S)[i] = ea;
                ((T *)a.oc)[i] = cb;
                ((T *)a.sc)[i] = eb;
                continue;
            }
            // the background's opacity and emissivity (continuum, and
            // coherent scattering of the previous mean intensity)
            T chi_b = (T)cc, eta_b = (T)cc * B;
            if (a.sigma_c) {
                const T sg = (T)a.sigma_c[v];
                chi_b += sg;
                eta_b += sg * ((const T *)a.jbg)[(long)(a.f0 + fl) * nvox + v];
            }
            T rho = T(1);
            bool prd = false;
            if (a.prd_index) {
                // partial redistribution: the line's emission profile is rho phi,
                // so its emissivity and the transition's shares scale by rho
                const int pr = a.prd_index[a.f0 + fl];
                if (pr >= 0) {
                    rho = (T)a.prd_rho[(long)pr * nvox + v];
                    prd = true;
                }
            }
            const T chi = chi_t + chi_b;
            const T inv = T(1) / chi;
            ((T *)a.chi)[i] = chi;
            ((T *)a.S)[i] = (rho * eta_t + eta_b) * inv;
            // the parts of S and chi the transition does not set, formed
            // directly: S - rho eta_t/chi and 1 - chi_t/chi.  For a PRD
            // frequency oc = 1 - rho chi_t/chi takes either sign and its
            // weighted sum over the line nearly cancels, so the sweep gets
            // oc = 0 (Ux = sum w u) and the radiative sums add the local
            // term in FP64 (prd_oc)
            ((T *)a.sc)[i] = eta_b * inv;
            ((T *)a.oc)[i] = prd ? T(0) : chi_b * inv;
        }
    }
}

// ------------------------------------------------ partial redistribution

// Partial redistribution of a line (the next step Sec. 6 names; the reading
// of the two-level case generalised): the angle-averaged Doppler
// redistribution R_I-A at a node of Doppler width d,
//   R0(x', x) = erfc(max(|x|, |x'|)/d) / (2 d^2),
// scaled symmetrically, R = diag(c) R0 diag(c), so that its discrete
// marginals sum_f' wq_f' R(f', f) are the node's profile phi_f (wq: the
// line's trapezoid weights normalised by sum w phi).  R0 depends on its two
// frequencies only through the larger |x|, so with the frequencies sorted by
// |x| a product R0^T v is, for a frequency of group k (equal |x|),
//   g_k sum_{groups <= k} v + sum_{groups > k} g v,   g = erfc(|x|/d)/(2 d^2):
// a prefix and a suffix sum, O(n) per node instead of O(n^2).
constexpr int kMaxPrdFreq = kMaxPrdLineFreq;

// out_s = sum_a R0(a, s) v_a for the line's sorted frequencies s (v, out in
// sorted order; g per group; suf scratch of ngrp + 1 entries).
__device__ inline void prd_r0_product(int nf, int ngrp, const int *__restrict__ gs,
                                      const double *g, const double *v, double *out,
                                      double *suf) {
    // suffix sums over groups above k
    suf[ngrp] = 0.0;
    for (int k = ngrp - 1; k >= 0; --k) {
        double sg = 0.0;
        for (int s = gs[k]; s < gs[k + 1]; ++s) sg += v[s];
        suf[k] = suf[k + 1] + g[k] * sg;
    }
    double pre = 0.0;
    for (int k = 0; k < ngrp; ++k) {
        for (int s = gs[k]; s < gs[k + 1]; ++s) pre += v[s];
        const double m = g[k] * pre + suf[k + 1];
        for (int s = gs[k]; s < gs[k + 1]; ++s) out[s] = m;
    }
}

// The line's profile at the node (sorted order), its normalised weights and
// the R0 group values.
__device__ inline void prd_line_setup(const PrdLine &L, const FreqInfo *__restrict__ fi,
                                      const int *__restrict__ ord, const int *__restrict__ gs,
                                      double d, double *phi, double *wq, double *g) {
    const double inv_d = 1.0 / d;
    double norm = 0.0;
    for (int s = 0; s < L.nf; ++s) {
        const FreqInfo q = fi[ord[L.ord0 + s]];
        const double xd = q.xy * inv_d;
        phi[s] = exp(-xd * xd) * 0.56418958354775628 * inv_d;
        norm += q.w * phi[s];
    }
    for (int s = 0; s < L.nf; ++s) wq[s] = fi[ord[L.ord0 + s]].w / norm;
    for (int k = 0; k < L.ngrp; ++k) {
        const double ax = fabs(fi[ord[L.ord0 + gs[k]]].xy);
        g[k] = 0.5 * erfc(ax * inv_d) * inv_d * inv_d;
    }
}

__global__ void __launch_bounds__(128) ml_prd_scale_kernel(long nvox, int n_prd,
                                                           const PrdLine *__restrict__ pl,
                                                           const FreqInfo *__restrict__ fi,
                                                           const int *__restrict__ ord,
                                                           const int *__restrict__ grp,
                                                           double t_ref,
                                                           const double *__restrict__ T,
                                                           double *__restrict__ scale) {
    double phi[kMaxPrdFreq], wq[kMaxPrdFreq], c[kMaxPrdFreq], v[kMaxPrdFreq], m[kMaxPrdFreq];
    double g[kMaxPrdFreq + 1], suf[kMaxPrdFreq + 1];
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < nvox;
         x += (long)gridDim.x * blockDim.x) {
        const double d = sqrt(T[x] / t_ref);
        for (int l = 0; l < n_prd; ++l) {
            const PrdLine L = pl[l];
            const int *gs = grp + L.grp0;
            prd_line_setup(L, fi, ord, gs, d, phi, wq, g);
            for (int s = 0; s < L.nf; ++s) c[s] = 1.0;
            for (int it = 0; it < 200; ++it) {
                for (int s = 0; s < L.nf; ++s) v[s] = wq[s] * c[s];
                prd_r0_product(L.nf, L.ngrp, gs, g, v, m, suf);
                for (int s = 0; s < L.nf; ++s) c[s] = sqrt(c[s] * phi[s] / m[s]);
            }
            for (int s = 0; s < L.nf; ++s)
                scale[(long)(L.pf0 + ord[L.ord0 + s] - L.f_begin) * nvox + x] = c[s];
        }
    }
}

template <typename TP>
__global__ void __launch_bounds__(128) ml_prd_rho_kernel(const MlPrdArgs a) {
    double phi[kMaxPrdFreq], wq[kMaxPrdFreq], v[kMaxPrdFreq], m[kMaxPrdFreq];
    double g[kMaxPrdFreq + 1], suf[kMaxPrdFreq + 1];
    const TP *__restrict__ jbg = (const TP *)a.jbg;
    const long nvox = a.nvox;
    const int N = a.n_levels;
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < nvox;
         x += (long)gridDim.x * blockDim.x) {
        const double Tg = a.T[x];
        const double d = sqrt(Tg / a.t_ref), inv_d = 1.0 / d;
        // plain rates of the lagged field: collisions plus every transition's
        // radiative rates with J (no local operator)
        double P[kMaxLevels][kMaxLevels];
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) P[i][j] = i == j ? 0.0 : a.c[((long)i * N + j) * nvox + x];
        for (int t = 0; t < a.n_trans; ++t) {
            const TransInfo tr = a.ti[t];
            if (tr.kind == 0) {
                double s0 = 0.0, s1 = 0.0;
                for (int f = tr.f_begin; f < tr.f_end; ++f) {
                    const FreqInfo q = a.fi[f];
                    const double xd = q.xy * inv_d;
                    const double wphi = q.w * exp(-xd * xd) * 0.56418958354775628 * inv_d;
                    s0 += wphi;
                    s1 += wphi * (double)jbg[(long)f * nvox + x];
                }
                const double Jb = s1 / s0;
                const double b_ul = tr.coef / (tr.rho * tr.rho * tr.rho);
                P[tr.lo][tr.up] += tr.gr * b_ul * Jb;
                P[tr.up][tr.lo] += tr.coef + b_ul * Jb;
            } else {
                const double G = a.saha[(long)tr.lo * nvox + x];
                double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                for (int f = tr.f_begin; f < tr.f_end; ++f) {
                    const FreqInfo q = a.fi[f];
                    const double y = q.xy;
                    const double qa = tr.coef * q.w / (y * y * y * y);
                    const double E = exp(-a.theta_ref * tr.rho * y / Tg);
                    const double ry = tr.rho * y;
                    const double J = (double)jbg[(long)f * nvox + x];
                    s0 += qa * J;
                    s1 += qa * E * J;
                    s2 += qa * E * ry * ry * ry;
                }
                P[tr.lo][tr.up] += s0;
                P[tr.up][tr.lo] += G * (s2 + s1);
            }
        }
        for (int l = 0; l < a.n_prd; ++l) {
            const PrdLine L = a.pl[l];
            const int *gs = a.grp + L.grp0;
            prd_line_setup(L, a.fi, a.ord, gs, d, phi, wq, g);
            double Jbar = 0.0;
            for (int s = 0; s < L.nf; ++s) {
                const int f = a.ord[L.ord0 + s];
                const double J = (double)jbg[(long)f * nvox + x];
                const double cs = a.scale[(long)(L.pf0 + f - L.f_begin) * nvox + x];
                Jbar += wq[s] * phi[s] * J;
                v[s] = wq[s] * cs * J;
            }
            double inflow = 0.0;
            for (int j = 0; j < N; ++j)
                if (j != L.up) inflow += a.n[(long)j * nvox + x] * P[j][L.up];
            const double excite = a.n[(long)L.lo * nvox + x] * L.gr * L.b_ul * Jbar;
            const double frad = excite / inflow;
            prd_r0_product(L.nf, L.ngrp, gs, g, v, m, suf);
            // the line's opacity at the node (as the opacity step forms it)
            // for 1 - rho chi_t/chi, the local term of the line's U
            const double nlo = a.n[(long)L.lo * nvox + x], nup = a.n[(long)L.up * nvox + x];
            const double chi_b = a.chi_c[x] + (a.sigma_c ? a.sigma_c[x] : 0.0);
            for (int s = 0; s < L.nf; ++s) {
                const int f = a.ord[L.ord0 + s];
                const long row = (long)(L.pf0 + f - L.f_begin) * nvox + x;
                double r = 1.0;
                if (Jbar > 0.0) {
                    const double Af = a.scale[row] * m[s];
                    r = 1.0 + L.gamma * frad * (Af / (phi[s] * Jbar) - 1.0);
                }
                a.rho[row] = r;
                const FreqInfo q = a.fi[f];
                const double chi_t = q.kappa * phi[s] * (q.gr * nlo - nup);
                a.oc[row] = (chi_b + (1.0 - r) * chi_t) / (chi_t + chi_b);
            }
        }
    }
}

cudaError_t launch_ml_prd_scale(long nvox, int n_prd, const PrdLine *pl, const FreqInfo *fi,
                                const int *ord, const int *grp, double t_ref, const double *T,
                                double *scale, cudaStream_t st) {
    ml_prd_scale_kernel<<<grid_for(nvox, 128), 128, 0, st>>>(nvox, n_prd, pl, fi, ord, grp, t_ref,
                                                              T, scale);
    return cudaGetLastError();
}

cudaError_t launch_ml_prd_rho(const MlPrdArgs &a, cudaStream_t st) {
    if (a.prec == MG3D_PREC_F64)
        ml_prd_rho_kernel<double><<<grid_for(a.nvox, 128), 128, 0, st>>>(a);
    else
        ml_prd_rho_kernel<float><<<grid_for(a.nvox, 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
__global__ void ml_bottom_kernel(long nplane, int nfreq, const FreqInfo *__restrict__ fi,
                                 double theta_ref, const double *__restrict__ Tg,
                                 T *__restrict__ ib) {
    const long total = nplane * nfreq;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        const int f = (int)(i / nplane);
        const long p = i - (long)f * nplane;
        const FreqInfo q = fi[f];
        const double rho = q.kind == 0 ? q.rho : q.rho * q.xy;
        ib[i] = (T)planck_rho(rho, theta_ref, Tg[p]);
    }
}

// -------------------------------------------------------------------- sweep

// HERM: monotone cubic Hermite upwind interpolation (the Hermite-spline
// option of Sec. 3): per ray and local row the table holds the four upwind
// rows ya-1 .. ya+2 of the intensity and slope planes and of chi, S; each
// finished plane gets its x-slopes after a block barrier; chi and S take
// theirs from dchi, dS.
//
// MODE kSweepMoving (a velocity field): along ray r a line's profile at a node
// is phi((x - u_r) / d) / (d sqrt(pi)), so chi, S and the transition shares
// are formed per node, ray and frequency from the ray-independent parts the
// opacity kernel wrote, and kept in opacity and source planes next to the
// intensity planes, from which the next step interpolates the upwind values;
// the angle sums carry the ray's normalised profile weight inside the ray
// sum.
template <typename T, int MODE>
__device__ __forceinline__ void ml_sweep_body(const MlSweepArgs<T> &a, int f, int slot) {
    constexpr bool HERM = MODE == kSweepHermite, VEL = MODE == kSweepMoving;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    // slot = (hemisphere, ray group); hemisphere 0: rays 0-11 (up), 1: 12-23
    const int rpb = a.rpb, groups = 12 / rpb;
    const int hemi = slot / groups;
    const int r0 = hemi * 12 + (slot - hemi * groups) * rpb;
    const bool up = hemi == 0;
    const int nx = a.nx, ny = a.ny, nz = a.nz, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = max(0, min(rows, ny - y0));
    const int band = myrows * nx;
    const long nplane = (long)nx * ny;
    const long nvox = nplane * nz;
    const T *__restrict__ chif = a.chi + (long)f * nvox;
    const T *__restrict__ Sf = a.S + (long)f * nvox;
    const T *__restrict__ scf = a.sc + (long)f * nvox;
    const T *__restrict__ ocf = a.oc + (long)f * nvox;
    T *__restrict__ jxo = a.jx + ((long)slot * a.nfreq + f) * nvox;
    T *__restrict__ uxo = a.ux + ((long)slot * a.nfreq + f) * nvox;
    T *__restrict__ jmo = a.jm ? a.jm + ((long)slot * a.nfreq + f) * nvox : nullptr;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const long raystride = (long)rows * nx;
    const long bufstride = rpb * raystride;
    // per step and (ray, local row): the upwind rows of the intensity planes
    // (here or in a peer block) and of chi, S on the upwind plane
    struct RowRef {
        const T *pa, *pb;
        int ra, rb;
    };
    struct RowRef4 {
        const T *p[4], *d[4];
        int r[4];
    };
    T *dbuf = buf + 2 * bufstride;  // slope planes (HERM)
    // VEL: opacity planes at buf + 2 bufstride, source planes at buf + 4 bufstride,
    // the same offsets from the intensity planes in every block of the cluster
    const long coff = 2 * bufstride, soff = 4 * bufstride;
    RowRef *rowref =
        reinterpret_cast<RowRef *>(buf + (HERM ? 4 : (VEL ? 6 : 2)) * bufstride);
    RowRef4 *rowref4 = reinterpret_cast<RowRef4 *>(rowref);
    __shared__ double exp_tab[kExpTab];
    if (sizeof(T) == 8) {
        for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) exp_tab[i] = a.exp_tab[i];
        __syncthreads();
    }
    const ExpNegTable et{exp_tab, a.exp_l1, a.exp_l2};
    const T wray = T(1.0 / kRays);
    const unsigned long long rmagic = band_magic(rows);
    // per-ray constants of the current step (the upwind offset is the same
    // for every node of a plane): bilinear weights, half path, corner offsets
    __shared__ T g_w[12][4];        // bilinear weights, or the x and y Hermite
    __shared__ T g_wy[12][4];       // bases (HERM)
    __shared__ T g_hs[12];
    __shared__ int g_ix[12];
    const T *__restrict__ dchif = HERM ? a.dchi + (long)f * nvox : nullptr;
    const T *__restrict__ dSf = HERM ? a.dS + (long)f * nvox : nullptr;
    // VEL: this frequency's line (or -1), offset and weight
    const int vl = VEL ? a.vline[a.f0 + f] : -1;
    const T vxf = VEL ? a.vx[a.f0 + f] : T(0), vwf = VEL ? a.vwq[a.f0 + f] : T(0);
    // chi, S, sc, oc and the profile weight of node v for ray r0 + j
    auto moving_terms = [&](long v, int j, T &chi, T &S, T &sc, T &oc, T &wr) {
        const T A = chif[v], E = Sf[v], cb = ocf[v], eb = scf[v];
        T prof = T(1);
        wr = T(1);
        if (vl >= 0) {
            const long rv = (long)(r0 + j) * nvox + v;
            const T di = a.dinv[v];
            const T dd = (vxf - a.uproj[rv]) * di;
            prof = ml_doppler(dd * dd, di, et);
            wr = vwf * prof * a.vnorm[(long)vl * kRays * nvox + rv];
        }
        const T ct = A * prof, et_ = E * prof;
        chi = ct + cb;
        const T inv = T(1) / chi;
        S = (et_ + eb) * inv;
        sc = eb * inv;
        oc = cb * inv;
    };

    for (int t = 0; t < nz; ++t) {
        const int k = up ? t : nz - 1 - t;
        T *cur = buf + (t & 1) * bufstride;
        if (t == 0 && VEL) {
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                const T Ib = up ? a.ib[(long)f * nplane + (long)y * nx + x] : T(0);
                const long v = (long)k * nplane + (long)y * nx + x;
                T jacc = 0, uacc = 0;
                for (int j = 0; j < rpb; ++j) {
                    T chi, S, sc, oc, wr;
                    moving_terms(v, j, chi, S, sc, oc, wr);
                    const long i = j * raystride + (long)yl * nx + x;
                    cur[i] = Ib;
                    cur[coff + i] = chi;
                    cur[soff + i] = S;
                    jacc += wr * Ib;
                    uacc += wr;
                }
                jxo[v] = wray * jacc;
                uxo[v] = wray * uacc;
                if (jmo) jmo[v] = T(rpb) * wray * Ib;
            }
        } else if (t == 0) {
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                const T Ib = up ? a.ib[(long)f * nplane + (long)y * nx + x] : T(0);
                for (int j = 0; j < rpb; ++j) cur[j * raystride + (long)yl * nx + x] = Ib;
                const long v = (long)k * nplane + (long)y * nx + x;
                jxo[v] = T(rpb) * wray * Ib;
                uxo[v] = T(rpb) * wray;
                if (jmo) jmo[v] = T(rpb) * wray * Ib;
            }
        } else {
            const T *prev = buf + ((t - 1) & 1) * bufstride;
            if (threadIdx.x < rpb) {
                const StepGeom o = a.geom[(long)(r0 + threadIdx.x) * nz + t];
                const T tx = (T)o.tx, ty = (T)o.ty;
                if constexpr (HERM) {
                    const HermiteBasis<T> bx(tx), by(ty);
                    g_w[threadIdx.x][0] = bx.c0;
                    g_w[threadIdx.x][1] = bx.c1;
                    g_w[threadIdx.x][2] = bx.c2;
                    g_w[threadIdx.x][3] = bx.c3;
                    g_wy[threadIdx.x][0] = by.c0;
                    g_wy[threadIdx.x][1] = by.c1;
                    g_wy[threadIdx.x][2] = by.c2;
                    g_wy[threadIdx.x][3] = by.c3;
                } else {
                    g_w[threadIdx.x][0] = (T(1) - tx) * (T(1) - ty);
                    g_w[threadIdx.x][1] = tx * (T(1) - ty);
                    g_w[threadIdx.x][2] = (T(1) - tx) * ty;
                    g_w[threadIdx.x][3] = tx * ty;
                }
                g_hs[threadIdx.x] = T(0.5) * (T)o.s;
                g_ix[threadIdx.x] = o.ix0;
            }
            for (int i = threadIdx.x; i < rpb * myrows; i += blockDim.x) {
                const int j = i / myrows, yl = i - j * myrows;
                int ya = y0 + yl + a.geom[(long)(r0 + j) * nz + t].iy0;
                if (ya >= ny) ya -= ny;
                const int yb = (ya + 1 == ny) ? 0 : ya + 1;
                if constexpr (HERM) {
                    const T *dprev = dbuf + ((t - 1) & 1) * bufstride;
                    int yr[4] = {ya == 0 ? ny - 1 : ya - 1, ya, yb, yb + 1 == ny ? 0 : yb + 1};
                    RowRef4 r4;
                    for (int m = 0; m < 4; ++m) {
                        const int b = band_of(yr[m], rmagic);
                        const long ro = j * raystride + (long)(yr[m] - b * rows) * nx;
                        r4.p[m] = (b == rank ? prev : cluster.map_shared_rank(prev, b)) + ro;
                        r4.d[m] = (b == rank ? dprev : cluster.map_shared_rank(dprev, b)) + ro;
                        r4.r[m] = yr[m] * nx;
                    }
                    rowref4[j * rows + yl] = r4;
                } else {
                    const int ba = band_of(ya, rmagic), bb = band_of(yb, rmagic);
                    const T *Pa = (ba == rank) ? prev : cluster.map_shared_rank(prev, ba);
                    const T *Pb = (bb == rank) ? prev : cluster.map_shared_rank(prev, bb);
                    RowRef r;
                    r.pa = Pa + j * raystride + (long)(ya - ba * rows) * nx;
                    r.pb = Pb + j * raystride + (long)(yb - bb * rows) * nx;
                    r.ra = ya * nx;
                    r.rb = yb * nx;
                    rowref[j * rows + yl] = r;
                }
            }
            __syncthreads();
            const int kp = up ? k - 1 : k + 1;
            const T *__restrict__ chip = chif + (long)kp * nplane;
            const T *__restrict__ Sp = Sf + (long)kp * nplane;
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                const long v = (long)k * nplane + (long)y * nx + x;
                const T chi_loc = chif[v], S_loc = Sf[v], sc = scf[v], oc = ocf[v];
                // sc and oc are the node's: sum I - w0 S, 1 - w0, w0 (and I
                // for the mean intensity) over the rays, then
                // Jx = sum (I - w0 S) + sc sum w0, Ux = sum u + oc sum w0
                T sum_i = 0, sum_p = 0, sum_u = 0, sum_w0 = 0;
                if constexpr (VEL) {
                    T jacc = 0, uacc = 0;
                    for (int j = 0; j < rpb; ++j) {
                        const T w00 = g_w[j][0], w10 = g_w[j][1], w01 = g_w[j][2],
                                w11 = g_w[j][3];
                        int xa = x + g_ix[j];
                        if (xa >= nx) xa -= nx;
                        const int xb = (xa + 1 == nx) ? 0 : xa + 1;
                        const RowRef r = rowref[j * rows + yl];
                        const T *Pa = r.pa, *Pb = r.pb;
                        auto bil = [&](long o) {
                            return w00 * Pa[o + xa] + w10 * Pa[o + xb] + w01 * Pb[o + xa] +
                                   w11 * Pb[o + xb];
                        };
                        const T I_up = bil(0), chi_up = bil(coff), S_up = bil(soff);
                        T chi, S, sc_r, oc_r, wr;
                        moving_terms(v, j, chi, S, sc_r, oc_r, wr);
                        const T x_tau = (chi_up + chi) * g_hs[j];
                        T ex, w0, wup, u;
                        ScWeights<T>::eval(x_tau, sc_rcp(x_tau), et, ex, w0, wup, u);
                        const T part = I_up * ex + wup * S_up;   // I - w0 S
                        const T I = part + w0 * S;
                        const long i = j * raystride + (long)yl * nx + x;
                        cur[i] = I;
                        cur[coff + i] = chi;
                        cur[soff + i] = S;
                        sum_i += I;
                        jacc += wr * (part + w0 * sc_r);
                        uacc += wr * (u + w0 * oc_r);
                    }
                    jxo[v] = wray * jacc;
                    uxo[v] = wray * uacc;
                    if (jmo) jmo[v] = wray * sum_i;
                    continue;
                }
                if constexpr (HERM) {
                    for (int j = 0; j < rpb; ++j) {
                        int xa = x + g_ix[j];
                        if (xa >= nx) xa -= nx;
                        const int xb = (xa + 1 == nx) ? 0 : xa + 1;
                        const RowRef4 &r4 = rowref4[j * rows + yl];
                        const T c0 = g_w[j][0], c1 = g_w[j][1], c2 = g_w[j][2], c3 = g_w[j][3];
                        const T e0 = g_wy[j][0], e1 = g_wy[j][1], e2 = g_wy[j][2], e3 = g_wy[j][3];
                        // x pass on four rows, then y pass through their values
                        auto up2d = [&](auto value_row, auto slope_row) {
                            T gq[4];
#pragma unroll
                            for (int m = 0; m < 4; ++m) {
                                const T *v = value_row(m), *d = slope_row(m);
                                gq[m] = c0 * v[xa] + c1 * d[xa] + c2 * v[xb] + c3 * d[xb];
                            }
                            return e0 * gq[1] + e1 * mono_slope(gq[1] - gq[0], gq[2] - gq[1]) +
                                   e2 * gq[2] + e3 * mono_slope(gq[2] - gq[1], gq[3] - gq[2]);
                        };
                        const T *dchip = dchif + (long)kp * nplane, *dSp = dSf + (long)kp * nplane;
                        const T chi_up = up2d([&](int m) { return chip + r4.r[m]; },
                                              [&](int m) { return dchip + r4.r[m]; });
                        const T S_up = up2d([&](int m) { return Sp + r4.r[m]; },
                                            [&](int m) { return dSp + r4.r[m]; });
                        const T I_up = up2d([&](int m) { return r4.p[m]; },
                                            [&](int m) { return r4.d[m]; });
                        const T x_tau = (chi_up + chi_loc) * g_hs[j];
                        T ex, w0, wup, u;
                        ScWeights<T>::eval(x_tau, sc_rcp(x_tau), et, ex, w0, wup, u);
                        const T part = I_up * ex + wup * S_up;   // I - w0 S
                        const T I = part + w0 * S_loc;
                        cur[j * raystride + (long)yl * nx + x] = I;
                        sum_i += I;
                        sum_p += part;
                        sum_u += u;
                        sum_w0 += w0;
                    }
                } else
                for (int j = 0; j < rpb; ++j) {
                    const T w00 = g_w[j][0], w10 = g_w[j][1], w01 = g_w[j][2], w11 = g_w[j][3];
                    int xa = x + g_ix[j];
                    if (xa >= nx) xa -= nx;
                    const int xb = (xa + 1 == nx) ? 0 : xa + 1;
                    const RowRef r = rowref[j * rows + yl];
                    const T *ca = chip + r.ra, *cb = chip + r.rb;
                    const T *sa = Sp + r.ra, *sb = Sp + r.rb;
                    const T chi_up = w00 * ca[xa] + w10 * ca[xb] + w01 * cb[xa] + w11 * cb[xb];
                    const T S_up = w00 * sa[xa] + w10 * sa[xb] + w01 * sb[xa] + w11 * sb[xb];
                    const T *Pa = r.pa, *Pb = r.pb;
                    const T I_up = w00 * Pa[xa] + w10 * Pa[xb] + w01 * Pb[xa] + w11 * Pb[xb];
                    const T x_tau = (chi_up + chi_loc) * g_hs[j];
                    T ex, w0, wup, u;
                    ScWeights<T>::eval(x_tau, sc_rcp(x_tau), et, ex, w0, wup, u);
                    const T part = I_up * ex + wup * S_up;   // I - w0 S
                    const T I = part + w0 * S_loc;
                    cur[j * raystride + (long)yl * nx + x] = I;
                    sum_i += I;
                    sum_p += part;
                    sum_u += u;
                    sum_w0 += w0;
                }
                jxo[v] = wray * (sum_p + sc * sum_w0);
                uxo[v] = wray * (sum_u + oc * sum_w0);
                if (jmo) jmo[v] = wray * sum_i;
            }
        }
        if constexpr (HERM) {
            // x-slopes of the new planes; a band holds whole rows
            __syncthreads();
            T *dcur = dbuf + (t & 1) * bufstride;
            for (int i = threadIdx.x; i < rpb * band; i += blockDim.x) {
                const int j = i / band, q = i - j * band;
                const int yl = q / nx, x = q - yl * nx;
                const int xm = x == 0 ? nx - 1 : x - 1, xp = x + 1 == nx ? 0 : x + 1;
                const T *row = cur + j * raystride + (long)yl * nx;
                dcur[j * raystride + (long)yl * nx + x] =
                    mono_slope(row[x] - row[xm], row[xp] - row[x]);
            }
        }
        cluster.sync();
    }
}

template <typename T, int MAXT, int MODE>
__global__ void __launch_bounds__(MAXT) ml_sweep_kernel(const MlSweepArgs<T> a) {
    ml_sweep_body<T, MODE>(a, blockIdx.y, blockIdx.z);
}

// Batched: item y = (problem, ray-group slot as ray, frequency as group).
template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT) ml_sweep_batch_kernel(
    const MlSweepArgs<T> *__restrict__ args, const BatchItem *__restrict__ items) {
    const BatchItem it = items[blockIdx.y];
    const MlSweepArgs<T> a = args[it.member];
    ml_sweep_body<T, kSweepLinear>(a, it.group, it.ray);
}

size_t ml_sweep_smem_bytes(int prec, int rows, int nx, int rpb, int herm, int moving) {
    const size_t elem = prec == MG3D_PREC_F64 ? sizeof(double) : sizeof(float);
    // moving: intensity, opacity and source planes and the 24-byte table
    if (moving) return 6ull * rpb * rows * nx * elem + 24ull * rpb * rows;
    // intensity planes (and their slope planes), then the per-(ray, row)
    // upwind row table: two pointers and two offsets (24 bytes), or eight
    // pointers and four offsets (80 bytes); the planes end on an 8-byte
    // boundary
    if (herm) return 4ull * rpb * rows * nx * elem + 80ull * rpb * rows;
    return 2ull * rpb * rows * nx * elem + 24ull * rpb * rows;
}

template <typename T, int MAXT, int MODE>
static cudaError_t launch_ml_sweep_t(const MlSweepArgs<T> &a, int bands, int threads,
                                     cudaStream_t st) {
    const size_t smem = ml_sweep_smem_bytes(sizeof(T) == 8 ? MG3D_PREC_F64 : MG3D_PREC_F32,
                                            a.rows, a.nx, a.rpb, MODE == kSweepHermite ? 1 : 0,
                                            MODE == kSweepMoving ? 1 : 0);
    if (MODE == kSweepHermite && (!a.dchi || !a.dS)) return cudaErrorInvalidValue;
    if (MODE == kSweepMoving && (!a.vx || !a.vwq || !a.vline || !a.vnorm || !a.uproj || !a.dinv))
        return cudaErrorInvalidValue;
    // one fixed limit for every launch, so graph replays never meet a lower one
    cudaError_t e = cudaFuncSetAttribute(ml_sweep_kernel<T, MAXT, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSweepSmem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(bands, a.nfreq, 2 * (12 / a.rpb));
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = bands;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = bands > 1 ? 1 : 0;  // one band: a plain launch
    return cudaLaunchKernelEx(&cfg, ml_sweep_kernel<T, MAXT, MODE>, a);
}

template <typename T, int MAXT>
static cudaError_t launch_ml_sweep_batch_t(const MlSweepArgs<T> *args, const BatchItem *items,
                                           int n_items, int bands, int threads, size_t smem,
                                           cudaStream_t st) {
    // one fixed limit for every launch, so graph replays never meet a lower one
    cudaError_t e = cudaFuncSetAttribute(ml_sweep_batch_kernel<T, MAXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSweepSmem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(bands, n_items, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = bands;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = bands > 1 ? 1 : 0;  // one band: a plain launch
    return cudaLaunchKernelEx(&cfg, ml_sweep_batch_kernel<T, MAXT>, args, items);
}

cudaError_t launch_ml_sweep_batch(int prec, const void *args, const BatchItem *items,
                                  int n_items, int bands, int threads, size_t smem,
                                  cudaStream_t st) {
    if (prec == MG3D_PREC_F64)
        return threads <= 256
                   ? launch_ml_sweep_batch_t<double, 256>((const MlSweepArgs<double> *)args,
                                                          items, n_items, bands, threads, smem, st)
                   : launch_ml_sweep_batch_t<double, 512>((const MlSweepArgs<double> *)args,
                                                          items, n_items, bands, threads, smem, st);
    return threads <= 256
               ? launch_ml_sweep_batch_t<float, 256>((const MlSweepArgs<float> *)args, items,
                                                     n_items, bands, threads, smem, st)
               : launch_ml_sweep_batch_t<float, 512>((const MlSweepArgs<float> *)args, items,
                                                     n_items, bands, threads, smem, st);
}

template <typename T>
static cudaError_t launch_ml_sweep_any(const MlSweepArgs<T> &a, int bands, int threads,
                                       cudaStream_t st) {
    if (a.herm && a.moving) return cudaErrorInvalidValue;
    if (a.herm)
        return threads <= 256 ? launch_ml_sweep_t<T, 256, kSweepHermite>(a, bands, threads, st)
                              : launch_ml_sweep_t<T, 512, kSweepHermite>(a, bands, threads, st);
    if (a.moving)
        return threads <= 256 ? launch_ml_sweep_t<T, 256, kSweepMoving>(a, bands, threads, st)
                              : launch_ml_sweep_t<T, 512, kSweepMoving>(a, bands, threads, st);
    return threads <= 256 ? launch_ml_sweep_t<T, 256, kSweepLinear>(a, bands, threads, st)
                          : launch_ml_sweep_t<T, 512, kSweepLinear>(a, bands, threads, st);
}

// Moving atmospheres: per ray and node the projected velocity u = mu_r . v,
// per node 1/d = sqrt(t_ref/T), and per line, ray and node the inverse of
// sum_f w_f phi((x_f - u)/d)/(d sqrt(pi)) over the line's frequencies (lines
// numbered in transition order).
template <typename T>
__global__ void ml_vel_prep_kernel(long nvox, int ntrans, const TransInfo *__restrict__ ti,
                                   const FreqInfo *__restrict__ fi, const double *__restrict__ mu,
                                   const double *__restrict__ vel, const double *__restrict__ Tg,
                                   double t_ref, T *__restrict__ uproj, T *__restrict__ dinv,
                                   T *__restrict__ vnorm) {
    const long total = (long)kRays * nvox;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / nvox);
        const long v = i - (long)r * nvox;
        const double u = mu[3 * r] * vel[v] + mu[3 * r + 1] * vel[nvox + v] +
                         mu[3 * r + 2] * vel[2 * nvox + v];
        const double di = sqrt(t_ref / Tg[v]);
        uproj[i] = (T)u;
        if (r == 0) dinv[v] = (T)di;
        int l = 0;
        for (int t = 0; t < ntrans; ++t) {
            const TransInfo tr = ti[t];
            if (tr.kind != 0) continue;
            double sum = 0.0;
            for (int f = tr.f_begin; f < tr.f_end; ++f) {
                const double dd = (fi[f].xy - u) * di;
                sum += fi[f].w * exp(-dd * dd) * di * 0.56418958354775628;
            }
            vnorm[((long)l * kRays + r) * nvox + v] = (T)(1.0 / sum);
            ++l;
        }
    }
}

cudaError_t launch_ml_vel_prep(int prec, long nvox, int ntrans, const TransInfo *ti,
                               const FreqInfo *fi, const double *mu, const double *vel,
                               const double *T, double t_ref, void *uproj, void *dinv,
                               void *vnorm, cudaStream_t st) {
    const long total = (long)kRays * nvox;
    const int th = 256;
    const long b = std::min<long>((total + th - 1) / th, 152L * 32);
    if (prec == MG3D_PREC_F64)
        ml_vel_prep_kernel<double><<<(int)b, th, 0, st>>>(nvox, ntrans, ti, fi, mu, vel, T, t_ref,
                                                          (double *)uproj, (double *)dinv,
                                                          (double *)vnorm);
    else
        ml_vel_prep_kernel<float><<<(int)b, th, 0, st>>>(nvox, ntrans, ti, fi, mu, vel, T, t_ref,
                                                         (float *)uproj, (float *)dinv,
                                                         (float *)vnorm);
    return cudaGetLastError();
}

cudaError_t launch_ml_sweep_f64(const MlSweepArgs<double> &a, int bands, int threads,
                                cudaStream_t st) {
    return launch_ml_sweep_any<double>(a, bands, threads, st);
}

cudaError_t launch_ml_sweep_f32(const MlSweepArgs<float> &a, int bands, int threads,
                                cudaStream_t st) {
    return launch_ml_sweep_any<float>(a, bands, threads, st);
}

// -------------------------------------------------------------------- rates

__device__ __forceinline__ unsigned long long dbits_ml(double x) {
    return (unsigned long long)__double_as_longlong(x);
}

// Radiative sums of the transitions over the chunk's frequencies, added to
// acc (frequencies in increasing order within a chunk, chunks in order).
template <typename TP>
__global__ void ml_accum_kernel(const MlAccumArgs a) {
    __shared__ double tab[kExpTab];
    for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) tab[i] = a.exp_tab[i];
    __syncthreads();
    const ExpNegTable et{tab, a.exp_l1, a.exp_l2};
    const TP *__restrict__ jx = (const TP *)a.jx;
    const TP *__restrict__ ux = (const TP *)a.ux;
    const long nvox = a.nvox;
    const long hstride = (long)a.nfreq * nvox;
    const int f1 = a.f0 + a.nfreq;
    // J, U of frequency f at node v: the ray-group slots added in order
    auto sums = [&](int f, long v, double &J, double &U) {
        const long i = (long)(f - a.f0) * nvox + v;
        J = (double)jx[i];
        U = (double)ux[i];
        for (int s = 1; s < a.nslots; ++s) {
            J += (double)jx[(long)s * hstride + i];
            U += (double)ux[(long)s * hstride + i];
        }
    };
    const double rsqpi = 0.5641895835477563;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x) {
        const double Tg = a.T[v];
        for (int t = 0; t < a.n_trans; ++t) {
            const TransInfo tr = a.ti[t];
            const int fb = max(tr.f_begin, a.f0), fe = min(tr.f_end, f1);
            if (fb >= fe) continue;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            if (tr.kind == 0) {
                const double inv_d = sqrt(a.t_ref / Tg);
                for (int f = fb; f < fe; ++f) {
                    if (a.moving && !a.zero_radiation) {
                        // the per-ray profile weights are inside J and U already
                        double J, U;
                        sums(f, v, J, U);
                        s0 += f == tr.f_begin ? 1.0 : 0.0;
                        s1 += J;
                        s2 += U;
                        continue;
                    }
                    const FreqInfo q = a.fi[f];
                    // profile in the formal-solution precision, sums in FP64
                    double wphi;
                    if (q.adamp > 0.0) {
                        wphi = q.w * (double)ml_line_phi<TP>(q, inv_d, TP(0), a.voigt, et);
                    } else {
                        const double xd = q.xy * inv_d;
                        wphi = q.w * (double)opac_exp((TP)(xd * xd), et) * rsqpi * inv_d;
                    }
                    double J = 0.0, U = 1.0;
                    if (!a.zero_radiation) {
                        sums(f, v, J, U);
                        const int pr = a.prd_index ? a.prd_index[f] : -1;
                        if (pr >= 0) {
                            // U = sum_r w_r (1 - w0 (1 - oc)) = oc + (1 - oc) sum_r w_r u_r
                            const double oc = a.prd_oc[(long)pr * nvox + v];
                            U = oc + (1.0 - oc) * U;
                        }
                    }
                    s0 += wphi;
                    s1 += wphi * J;
                    s2 += wphi * U;
                }
            } else {
                for (int f = fb; f < fe; ++f) {
                    const FreqInfo q = a.fi[f];
                    const double y = q.xy;
                    const double qa = tr.coef * q.w / (y * y * y * y);
                    const double E = (double)opac_exp((TP)(a.theta_ref * tr.rho * y / Tg), et);
                    const double ry = tr.rho * y;
                    double J = 0.0, U = 1.0;
                    if (!a.zero_radiation) sums(f, v, J, U);
                    s0 += qa * J;
                    s1 += qa * E * J;
                    s2 += qa * E * ry * ry * ry * U;
                }
            }
            double *acc = a.acc + (long)t * kAccTerms * nvox + v;
            acc[0] += s0;
            acc[nvox] += s1;
            acc[2 * nvox] += s2;
        }
        // background field of the chunk's frequencies: the new mean intensity
        if (a.jbg && !a.zero_radiation) {
            const TP *__restrict__ jm = (const TP *)a.jm;
            for (int fl = 0; fl < a.nfreq; ++fl) {
                const long i = (long)fl * nvox + v;
                double J = (double)jm[i];
                for (int s = 1; s < a.nslots; ++s) J += (double)jm[(long)s * hstride + i];
                ((TP *)a.jbg)[(long)(a.f0 + fl) * nvox + v] = (TP)J;
            }
        }
    }
}

__global__ void __launch_bounds__(128) ml_rates_kernel(const MlRateArgs a) {
    const long nvox = a.nvox;
    const int N = a.n_levels;
    double cmax = 0.0;
    unsigned neg = 0, bad = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long base = (long)blockIdx.x * blockDim.x; base < nvox; base += stride) {
        const long v = base + threadIdx.x;
        if (v >= nvox) continue;
        double P[kMaxLevels][kMaxLevels];
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) P[i][j] = i == j ? 0.0 : a.c[((long)i * N + j) * nvox + v];
        for (int t = 0; t < a.n_trans; ++t) {
            const TransInfo tr = a.ti[t];
            const double *acc = a.acc + (long)t * kAccTerms * nvox + v;
            if (tr.kind == 0) {
                const double norm = acc[0];
                const double Jb = acc[nvox] / norm, Ub = acc[2 * nvox] / norm;
                const double b_ul = tr.coef / (tr.rho * tr.rho * tr.rho);
                P[tr.lo][tr.up] += tr.gr * b_ul * Jb;
                P[tr.up][tr.lo] += tr.coef * Ub + b_ul * Jb;
            } else {
                const double G = a.saha[(long)tr.lo * nvox + v];
                P[tr.lo][tr.up] += acc[0];
                P[tr.up][tr.lo] += G * (acc[2 * nvox] + acc[nvox]);
            }
        }
        // W(n) = M n: row 0 conservation, row i: n_i sum_j P_ij - sum_j n_j P_ji
        double M[kMaxLevels][kMaxLevels + 1];
        for (int j = 0; j < N; ++j) M[0][j] = 1.0;
        for (int i = 1; i < N; ++i) {
            double out_i = 0.0;
            for (int j = 0; j < N; ++j)
                if (j != i) out_i += P[i][j];
            for (int j = 0; j < N; ++j) M[i][j] = j == i ? out_i : -P[j][i];
        }
        double fv[kMaxLevels];
        for (int i = 0; i < N; ++i)
            fv[i] = a.f ? a.f[(long)i * nvox + v] : (i == 0 ? a.n_tot[v] : 0.0);
        if (a.mode == kRateSolve) {
            for (int i = 0; i < N; ++i) M[i][N] = fv[i];
            for (int c = 0; c < N; ++c) {
                int piv = c;
                double best = fabs(M[c][c]);
                for (int r = c + 1; r < N; ++r)
                    if (fabs(M[r][c]) > best) {
                        best = fabs(M[r][c]);
                        piv = r;
                    }
                if (piv != c)
                    for (int j = c; j <= N; ++j) {
                        const double tmp = M[c][j];
                        M[c][j] = M[piv][j];
                        M[piv][j] = tmp;
                    }
                const double inv = 1.0 / M[c][c];
                for (int r = c + 1; r < N; ++r) {
                    const double fac = M[r][c] * inv;
                    for (int j = c; j <= N; ++j) M[r][j] -= fac * M[c][j];
                }
            }
            double xsol[kMaxLevels];
            for (int i = N - 1; i >= 0; --i) {
                double acc = M[i][N];
                for (int j = i + 1; j < N; ++j) acc -= M[i][j] * xsol[j];
                xsol[i] = acc / M[i][i];
            }
            bool finite = true;
            double cl = 0.0;
            for (int i = 0; i < N; ++i) {
                const double old = a.n[(long)i * nvox + v];
                a.n[(long)i * nvox + v] = xsol[i];
                const double ci = fabs(xsol[i] - old) / fabs(xsol[i]);
                if (!(isfinite(xsol[i]) && isfinite(ci))) finite = false;
                else cl = fmax(cl, ci);
                neg += xsol[i] <= 0.0;
            }
            if (finite) cmax = fmax(cmax, cl);
            else ++bad;
        } else {
            for (int i = 0; i < N; ++i) {
                double w = 0.0;
                for (int j = 0; j < N; ++j) w += M[i][j] * a.n[(long)j * nvox + v];
                if (a.mode == kRateResidual) a.out[(long)i * nvox + v] = fv[i] - w;
                else a.out[(long)i * nvox + v] += w;
            }
        }
    }
    if (a.mode == kRateSolve && a.scal) {
        __shared__ double red[32];
        __shared__ unsigned cnt[2][32];
        double m = cmax;
        for (int o = 16; o > 0; o >>= 1) {
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            neg += __shfl_xor_sync(0xffffffffu, neg, o);
            bad += __shfl_xor_sync(0xffffffffu, bad, o);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            red[wid] = m;
            cnt[0][wid] = neg;
            cnt[1][wid] = bad;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int nw = (blockDim.x + 31) >> 5;
            double mm = 0.0;
            unsigned tn = 0, tb = 0;
            for (int i = 0; i < nw; ++i) {
                mm = fmax(mm, red[i]);
                tn += cnt[0][i];
                tb += cnt[1][i];
            }
            if (mm > 0.0) atomicMax(a.scal, dbits_ml(mm));
            if (tn) atomicAdd(a.scal + 1, (unsigned long long)tn);
            if (tb) atomicAdd(a.scal + 2, (unsigned long long)tb);
        }
    }
}

cudaError_t launch_ml_opacity(const MlOpacityArgs &a, cudaStream_t st) {
    if (a.prec == MG3D_PREC_F64)
        ml_opacity_kernel<double><<<grid_for(a.nvox, 256), 256, 0, st>>>(a);
    else
        ml_opacity_kernel<float><<<grid_for(a.nvox, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ml_bottom(int prec, long nplane, int nfreq, const FreqInfo *fi,
                             double theta_ref, const double *T, void *ib, cudaStream_t st) {
    const long total = nplane * nfreq;
    if (prec == MG3D_PREC_F64)
        ml_bottom_kernel<double><<<grid_for(total, 256), 256, 0, st>>>(nplane, nfreq, fi,
                                                                       theta_ref, T, (double *)ib);
    else
        ml_bottom_kernel<float><<<grid_for(total, 256), 256, 0, st>>>(nplane, nfreq, fi,
                                                                      theta_ref, T, (float *)ib);
    return cudaGetLastError();
}

cudaError_t launch_ml_accum(const MlAccumArgs &a, cudaStream_t st) {
    if (a.prec == MG3D_PREC_F64)
        ml_accum_kernel<double><<<grid_for(a.nvox, 128), 128, 0, st>>>(a);
    else
        ml_accum_kernel<float><<<grid_for(a.nvox, 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ml_rates(const MlRateArgs &a, cudaStream_t st) {
    ml_rates_kernel<<<grid_for(a.nvox, 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mg3d
