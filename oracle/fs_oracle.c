/*
 * CPU oracle: short-characteristics formal solution in plain FP64 loops.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes (Sec. 3, "Computational setup"; Eq. 1): the transfer
 * equation dI/dtau = S - I is integrated cell by cell with the short
 * characteristics method of Kunasz & Auer (1988).
 * For a node on plane k and a ray with direction (mux, muy, muz) the short
 * characteristic runs back to the neighbouring plane upwind (k-1 for muz > 0,
 * k+1 for muz < 0).  Where it crosses that plane, I, chi and S are
 * interpolated, periodic in x and y (Sec. 4.2), with one of the two schemes
 * Sec. 3 names:
 *   interp = 0: linear -- bilinear between the four surrounding nodes;
 *   interp = 1: Hermite spline -- monotone cubic Hermite interpolation
 *     (Auer 2003) along x on the four rows around the crossing point, then
 *     along y through the four results (a 4 x 4 stencil).  The slope at a
 *     node is the harmonic mean of the two neighbouring secants when they
 *     have the same sign and zero otherwise (Fritsch & Butland 1984), so the
 *     interpolant stays between the two nodes of each interval.
 * Along the characteristic of length s = |dz|/|muz| the optical
 * depth is the trapezoid dtau = (chi_up + chi_0) s / 2 and S is linear in tau,
 * which gives
 *     I_0 = I_up exp(-dtau) + w_up S_up + w_0 S_0,
 *     w_0  = 1 - (1 - exp(-dtau))/dtau,   w_up = (1 - exp(-dtau))/dtau - exp(-dtau).
 * Boundary conditions (Sec. 4.2): rays entering through the bottom plane
 * start with the given I_bottom (the Planck function at the local gas
 * temperature), rays entering through the top start with I_top (zero).
 *
 * Accumulated per node, with the quadrature weight w_r of each ray and the
 * per-node frequency weight wphi (frequency quadrature weight times line
 * profile):
 *     Jbar  = sum w_r wphi I                 (mean intensity, profile-averaged)
 *     Jeff  = sum w_r wphi (I - w_0 S_0)     (Jbar minus the local part)
 *     U     = sum w_r wphi (1 - w_0)         (so that the diagonal operator
 *                                             Lambda* = sum w_r wphi w_0 = sum w_r wphi - U)
 * The diagonal of the Lambda operator is exactly w_0 at each node and ray,
 * because the upwind intensity depends only on nodes of other planes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static long node_index(long x, long y, long k, long nx, long ny)
{
    return (k * ny + y) * nx + x;
}

static long periodic(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Weights of the linear short-characteristics step.  For small dtau the
 * closed forms lose digits to cancellation, so below 1e-3 the Taylor series
 * of w_0 and w_up (five terms each) are used instead. */
static void sc_weights(double dtau, double *ex, double *w0, double *wup)
{
    double e = exp(-dtau);
    *ex = e;
    if (dtau < 1e-3) {
        double t = dtau;
        *w0 = t * (0.5 - t * (1.0 / 6.0 - t * (1.0 / 24.0 - t * (1.0 / 120.0 - t / 720.0))));
        *wup = t * (0.5 - t * (1.0 / 3.0 - t * (1.0 / 8.0 - t * (1.0 / 30.0 - t / 144.0))));
    } else {
        double u = (1.0 - e) / dtau;
        *w0 = 1.0 - u;
        *wup = u - e;
    }
}

static double bilinear(const double *plane, long nx, long ny, double xu, double yu)
{
    double fx0 = floor(xu), fy0 = floor(yu);
    double tx = xu - fx0, ty = yu - fy0;
    long x0 = periodic((long)fx0, nx), x1 = periodic((long)fx0 + 1, nx);
    long y0 = periodic((long)fy0, ny), y1 = periodic((long)fy0 + 1, ny);
    double f00 = plane[y0 * nx + x0], f10 = plane[y0 * nx + x1];
    double f01 = plane[y1 * nx + x0], f11 = plane[y1 * nx + x1];
    return (1.0 - tx) * (1.0 - ty) * f00 + tx * (1.0 - ty) * f10
         + (1.0 - tx) * ty * f01 + tx * ty * f11;
}

/* Monotone slope at a node of a uniform periodic row from its two secants
 * (in units of one cell): the harmonic mean 2 a b / (a + b) when a and b have
 * the same strict sign, else zero. */
static double harmonic_slope(double a, double b)
{
    if ((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0))
        return 2.0 * a * b / (a + b);
    return 0.0;
}

/* Cubic Hermite on [0, 1] from end values p0, p1 and end slopes d0, d1 (per
 * unit of t), at t. */
static double hermite01(double p0, double p1, double d0, double d1, double t)
{
    double t2 = t * t, t3 = t2 * t;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * p0 + (t3 - 2.0 * t2 + t) * d0
         + (-2.0 * t3 + 3.0 * t2) * p1 + (t3 - t2) * d1;
}

/* Monotone cubic Hermite through q[0..3] (uniform spacing) on the interval
 * between q[1] and q[2], at fraction t. */
static double hermite4(const double *q, double t)
{
    double d1 = harmonic_slope(q[1] - q[0], q[2] - q[1]);
    double d2 = harmonic_slope(q[2] - q[1], q[3] - q[2]);
    return hermite01(q[1], q[2], d1, d2, t);
}

static double bicubic_hermite(const double *plane, long nx, long ny, double xu, double yu)
{
    double fx0 = floor(xu), fy0 = floor(yu);
    double tx = xu - fx0, ty = yu - fy0;
    double col[4], row[4];
    for (int j = 0; j < 4; ++j) {
        long y = periodic((long)fy0 - 1 + j, ny);
        for (int i = 0; i < 4; ++i)
            row[i] = plane[y * nx + periodic((long)fx0 - 1 + i, nx)];
        col[j] = hermite4(row, tx);
    }
    return hermite4(col, ty);
}

static double upwind_value(const double *plane, long nx, long ny, double xu, double yu,
                           int interp)
{
    return interp ? bicubic_hermite(plane, nx, ny, xu, yu) : bilinear(plane, nx, ny, xu, yu);
}

/*
 * Formal solution for all rays and frequencies.
 *   chi, S, wphi : [nfreq][nz][ny][nx]
 *   I_bottom, I_top : [nfreq][ny][nx]
 *   mu : [nrays][3] direction cosines, wray : [nrays]
 * Outputs (zeroed here) Jbar, Jeff, U : [nz][ny][nx]; I_out, if not NULL,
 * receives every intensity as [nrays][nfreq][nz][ny][nx].  interp selects the
 * upwind interpolation (0 linear, 1 monotone cubic Hermite).
 * Returns 0, or -1 on a bad argument.
 */
int orc_formal_solution(long nx, long ny, long nz, double dx, double dy,
                        const double *z, long nrays, const double *mu,
                        const double *wray, long nfreq, const double *chi,
                        const double *S, const double *wphi,
                        const double *I_bottom, const double *I_top,
                        double *Jbar, double *Jeff, double *U, double *I_out, int interp)
{
    if (nx < 1 || ny < 1 || nz < 2 || nrays < 1 || nfreq < 1 || dx <= 0 || dy <= 0 ||
        interp < 0 || interp > 1)
        return -1;
    long nplane = nx * ny, nvox = nplane * nz;
    memset(Jbar, 0, sizeof(double) * nvox);
    memset(Jeff, 0, sizeof(double) * nvox);
    memset(U, 0, sizeof(double) * nvox);
    double *Iprev = malloc(sizeof(double) * nplane);
    double *Icur = malloc(sizeof(double) * nplane);
    double *W0 = malloc(sizeof(double) * nplane);
    if (!Iprev || !Icur || !W0) {
        free(Iprev);
        free(Icur);
        free(W0);
        return -1;
    }
    for (long r = 0; r < nrays; ++r) {
        double mx = mu[3 * r], my = mu[3 * r + 1], mz = mu[3 * r + 2];
        int up = mz > 0.0;
        for (long f = 0; f < nfreq; ++f) {
            const double *chif = chi + f * nvox, *Sf = S + f * nvox, *wf = wphi + f * nvox;
            for (long step = 0; step < nz; ++step) {
                long k = up ? step : nz - 1 - step;
                if (step == 0) {
                    /* entering boundary: the intensity is prescribed, so the
                     * node's own source function does not enter (w_0 = 0) */
                    const double *bc = (up ? I_bottom : I_top) + f * nplane;
                    for (long y = 0; y < ny; ++y)
                        for (long x = 0; x < nx; ++x) {
                            Icur[y * nx + x] = bc[y * nx + x];
                            W0[y * nx + x] = 0.0;
                        }
                } else {
                    long kp = up ? k - 1 : k + 1;
                    double s = fabs(z[k] - z[kp]) / fabs(mz);
                    const double *chip = chif + kp * nplane, *Sp = Sf + kp * nplane;
                    for (long y = 0; y < ny; ++y) {
                        for (long x = 0; x < nx; ++x) {
                            /* upwind crossing point, in units of cells */
                            double xu = (double)x - s * mx / dx;
                            double yu = (double)y - s * my / dy;
                            double I_up = upwind_value(Iprev, nx, ny, xu, yu, interp);
                            double chi_up = upwind_value(chip, nx, ny, xu, yu, interp);
                            double S_up = upwind_value(Sp, nx, ny, xu, yu, interp);
                            long v = node_index(x, y, k, nx, ny);
                            double dtau = 0.5 * (chi_up + chif[v]) * s;
                            double ex, w0, wup;
                            sc_weights(dtau, &ex, &w0, &wup);
                            Icur[y * nx + x] = I_up * ex + wup * S_up + w0 * Sf[v];
                            W0[y * nx + x] = w0;
                        }
                    }
                }
                /* accumulate this plane */
                for (long y = 0; y < ny; ++y) {
                    for (long x = 0; x < nx; ++x) {
                        long v = node_index(x, y, k, nx, ny);
                        double I = Icur[y * nx + x], w0 = W0[y * nx + x];
                        double w = wray[r] * wf[v];
                        Jbar[v] += w * I;
                        Jeff[v] += w * (I - w0 * Sf[v]);
                        U[v] += w * (1.0 - w0);
                        if (I_out)
                            I_out[((r * nfreq + f) * nz + k) * nplane + y * nx + x] = I;
                    }
                }
                double *t = Iprev;
                Iprev = Icur;
                Icur = t;
            }
        }
    }
    free(Iprev);
    free(Icur);
    free(W0);
    return 0;
}

/*
 * The same formal solution with the rays spread over `nthreads` host threads
 * (OpenMP, when the file is compiled with it; otherwise one thread): each ray
 * runs orc_formal_solution above on its own, into its own partial sums, and
 * the partial sums are then added in ray order.  It exists to time the
 * oracle on all cores of a host (the bench's CPU baseline); the sums differ
 * from the serial ones only in their association (rounding).  Same
 * arguments as orc_formal_solution without I_out; returns 0, or -1 on a bad
 * argument or a failed allocation.
 */
int orc_formal_solution_threads(long nx, long ny, long nz, double dx, double dy,
                                const double *z, long nrays, const double *mu,
                                const double *wray, long nfreq, const double *chi,
                                const double *S, const double *wphi,
                                const double *I_bottom, const double *I_top,
                                double *Jbar, double *Jeff, double *U, int interp, int nthreads)
{
    if (nrays < 1 || nthreads < 1 || nx < 1 || ny < 1 || nz < 2)
        return -1;
    long nvox = nx * ny * nz;
    double *part = malloc(sizeof(double) * 3 * (size_t)nrays * (size_t)nvox);
    if (!part)
        return -1;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(| : bad)
#endif
    for (long r = 0; r < nrays; ++r) {
        double *p = part + 3 * r * nvox;
        bad |= orc_formal_solution(nx, ny, nz, dx, dy, z, 1, mu + 3 * r, wray + r, nfreq, chi,
                                   S, wphi, I_bottom, I_top, p, p + nvox, p + 2 * nvox, NULL,
                                   interp) != 0;
    }
    if (!bad) {
        for (long v = 0; v < nvox; ++v) {
            double jb = 0.0, je = 0.0, u = 0.0;
            for (long r = 0; r < nrays; ++r) {
                const double *p = part + 3 * r * nvox;
                jb += p[v];
                je += p[nvox + v];
                u += p[2 * nvox + v];
            }
            Jbar[v] = jb;
            Jeff[v] = je;
            U[v] = u;
        }
    }
    free(part);
    return bad ? -1 : 0;
}

/* Threads the OpenMP runtime offers (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Formal solution with per-frequency angle sums, for atoms with several
 * transitions and a background continuum (Sec. 2.1; MALI with the diagonal
 * operator of Rybicki & Hummer 1992).  Each frequency belongs to one
 * transition t; at every node and frequency the total opacity chi and
 * source function S drive the transfer, while the transition's own share
 * enters the preconditioning:
 *     sl = eta_t / chi   (the part of S the transition's new populations set)
 *     fl = chi_t / chi   (the transition's share of the opacity)
 * Returned per frequency and node (zeroed here):
 *     Jx = sum_r w_r (I - w_0 sl),     Ux = sum_r w_r (1 - w_0 fl),
 * and, when Jm is not NULL, the mean intensity Jm = sum_r w_r I.
 * Shapes: chi, S, sl, fl, Jx, Ux, Jm [nfreq][nz][ny][nx]; I_bottom, I_top
 * [nfreq][ny][nx].  interp as for orc_formal_solution.  Returns 0, or -1 on
 * a bad argument.
 */
int orc_formal_solution_nu(long nx, long ny, long nz, double dx, double dy,
                           const double *z, long nrays, const double *mu,
                           const double *wray, long nfreq, const double *chi,
                           const double *S, const double *sl, const double *fl,
                           const double *I_bottom, const double *I_top,
                           double *Jx, double *Ux, double *Jm, int interp)
{
    if (nx < 1 || ny < 1 || nz < 2 || nrays < 1 || nfreq < 1 || dx <= 0 || dy <= 0 ||
        interp < 0 || interp > 1)
        return -1;
    long nplane = nx * ny, nvox = nplane * nz;
    memset(Jx, 0, sizeof(double) * nvox * nfreq);
    memset(Ux, 0, sizeof(double) * nvox * nfreq);
    if (Jm) memset(Jm, 0, sizeof(double) * nvox * nfreq);
    double *Iprev = malloc(sizeof(double) * nplane);
    double *Icur = malloc(sizeof(double) * nplane);
    double *W0 = malloc(sizeof(double) * nplane);
    if (!Iprev || !Icur || !W0) {
        free(Iprev);
        free(Icur);
        free(W0);
        return -1;
    }
    for (long r = 0; r < nrays; ++r) {
        double mx = mu[3 * r], my = mu[3 * r + 1], mz = mu[3 * r + 2];
        int up = mz > 0.0;
        for (long f = 0; f < nfreq; ++f) {
            const double *chif = chi + f * nvox, *Sf = S + f * nvox;
            const double *slf = sl + f * nvox, *flf = fl + f * nvox;
            double *Jf = Jx + f * nvox, *Uf = Ux + f * nvox;
            for (long step = 0; step < nz; ++step) {
                long k = up ? step : nz - 1 - step;
                if (step == 0) {
                    const double *bc = (up ? I_bottom : I_top) + f * nplane;
                    for (long q = 0; q < nplane; ++q) {
                        Icur[q] = bc[q];
                        W0[q] = 0.0;
                    }
                } else {
                    long kp = up ? k - 1 : k + 1;
                    double s = fabs(z[k] - z[kp]) / fabs(mz);
                    const double *chip = chif + kp * nplane, *Sp = Sf + kp * nplane;
                    for (long y = 0; y < ny; ++y) {
                        for (long x = 0; x < nx; ++x) {
                            double xu = (double)x - s * mx / dx;
                            double yu = (double)y - s * my / dy;
                            double I_up = upwind_value(Iprev, nx, ny, xu, yu, interp);
                            double chi_up = upwind_value(chip, nx, ny, xu, yu, interp);
                            double S_up = upwind_value(Sp, nx, ny, xu, yu, interp);
                            long v = node_index(x, y, k, nx, ny);
                            double dtau = 0.5 * (chi_up + chif[v]) * s;
                            double ex, w0, wup;
                            sc_weights(dtau, &ex, &w0, &wup);
                            Icur[y * nx + x] = I_up * ex + wup * S_up + w0 * Sf[v];
                            W0[y * nx + x] = w0;
                        }
                    }
                }
                for (long q = 0; q < nplane; ++q) {
                    long v = k * nplane + q;
                    Jf[v] += wray[r] * (Icur[q] - W0[q] * slf[v]);
                    Uf[v] += wray[r] * (1.0 - W0[q] * flf[v]);
                    if (Jm) Jm[f * nvox + v] += wray[r] * Icur[q];
                }
                double *t = Iprev;
                Iprev = Icur;
                Icur = t;
            }
        }
    }
    free(Iprev);
    free(Icur);
    free(W0);
    return 0;
}
