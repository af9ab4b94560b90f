// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace mg3d {

struct VoigtTable;   // voigt.cuh

constexpr int kRays = 24;          // A4 quadrature, 12 up and 12 down
constexpr int kMaxBands = 16;      // thread blocks per cluster sharing a plane (beyond
                                   // 8: non-portable cluster size, checked per shape)
constexpr int kPortableBands = 8;  // cap for shapes chosen without a measurement
constexpr int kMaxSweepThreads = 512;
constexpr size_t kMaxSweepSmem = 200 * 1024;
constexpr int kExpTab = 256;       // entries 2^{j/256} of the FP64 exp table

// Upwind geometry of one sweep step of one ray.  The short characteristic of
// every node on the plane crosses the upwind plane at the same horizontal
// offset, so the bilinear weights and the integer corner offsets are
// constants of (ray, step).  ix0/iy0 are already reduced modulo nx/ny.
struct StepGeom {
    int ix0, iy0;
    double tx, ty;   // fractional position inside the upwind cell, [0, 1)
    double s;        // path length of the short characteristic
};

// Launch shape of the sweep on one level.
struct SweepShape {
    int ng;       // frequencies per thread block
    int ngroups;  // ceil(nfreq / ng)
    int bands;    // thread blocks per cluster; each holds `rows` rows
    int rows;     // ceil(ny / bands)
    int threads;  // threads per block
    int lean = 0; // register budget: 0 full, 1: 1024 resident threads per SM (64
                  // registers), 2: three 256-thread blocks per SM (85 registers)
    int stage = 1; // 1: chi0/S rows staged in shared memory one step ahead
    int herm = 0;  // 1: monotone cubic Hermite upwind interpolation (unstaged)
    int vel = 0;   // 1: moving atmosphere, ray-dependent profiles (unstaged)
    int prd = 0;   // 1: partial redistribution, frequency-dependent S (unstaged)
    int plane = 0; // shifted-plane sweep (plane_sweep.cuh) with np slots of two
                   // frequencies: 1 cluster barriers, 2 transaction-counted stores
    int np = 0;    //    frequencies per group (ng = 2 np table positions per group)
};

// Per (ray, step t) constants of the shifted-plane sweep (plane_sweep.cuh),
// in the formal-solution precision: the bilinear weights of the upwind
// corners and half the path length of step t (t >= 1), and the shift of the
// plane written at step t, i.e. the corner offsets (ix0, iy0) of step t+1
// (t <= nz-2).
template <typename T>
struct alignas(16) PlaneStep {
    T w00, w10, w01, w11;
    T half_s;
    int sx, sy;   // (16-byte aligned and padded: loaded as whole vectors)
};

// Slot flags of the shifted-plane sweep.
namespace plane {
constexpr int kHasB = 1;    // the slot has a second frequency
constexpr int kShared = 2;  // the second frequency has the first one's phi
}  // namespace plane

// One slot of the shifted-plane sweep: two frequencies (a, b) of a group.
template <typename T>
struct PlaneSlot {
    T phi_a, phi_b;      // profile values
    T iphi_a, iphi_b;    // their inverses
    T wphi_a, wphi_b;    // ray weight x frequency weight x profile (0: no frequency b)
    T wu_a, wu_b;        // weight of u: wphi_a + wphi_b when a and b share phi, else own
    int flags;           // bit 0: frequency b present; bit 1: b has a's phi
};

// Arguments of the shifted-plane sweep kernel (plane_sweep.cuh).
template <typename T>
struct PlaneArgs {
    int nx, ny, nz, rows, bands, ngroups;
    int nslot_last;                      // active slots of the last group (0: all NP)
    unsigned up_mask;                    // bit r set when ray r points up
    unsigned long long rmagic, xmagic;   // band_magic(rows), band_magic(nx)
    const T *chi0, *S, *bbot;            // [nvox], [nvox], [nx*ny]
    const PlaneStep<T> *steps;           // [kRays][nz]
    const PlaneSlot<T> *slots;           // [ngroups][NP]
    T *pj, *pu;                          // [kRays*ngroups][nvox] partial Jeff and U
    const double *exp_tab;               // FP64 exp table (FP64 sweeps)
    double exp_l1, exp_l2;
    unsigned *status;                    // kPlaneStatus* bits (async scheme), nullable
};

// Status bits of the shifted-plane sweep: a bounded wait for a plane's bytes
// ran out (the launch's results are not valid).
constexpr unsigned kPlaneStatusWait = 1u;

// Slot counts (frequency pairs per group) the shifted-plane sweep is built for.
constexpr int kPlaneNp[] = {1, 2, 3, 5, 8};
constexpr int kPlaneNpCount = 5;
constexpr size_t kMaxPlaneSmem = 224 * 1024;   // dynamic; static use stays below 3 KB
constexpr int kPlaneMaxThreads = 1024;
// nodes a thread of the shifted-plane sweep takes per step (band <= this x
// threads): the node loop is unrolled over them, which costs registers where
// the compiler overlaps them (FP32 with more than two slots: two nodes)
__host__ __device__ constexpr int plane_max_pass(int np, bool fp64) {
    return fp64 || np <= 2 ? 4 : 2;
}
bool plane_np_supported(int np);
size_t plane_smem_bytes(int prec, int np, int rows, int nx);
cudaError_t launch_plane_sweep_f64(const PlaneArgs<double> &a, const SweepShape &s,
                                   cudaStream_t st);
cudaError_t launch_plane_sweep_f32(const PlaneArgs<float> &a, const SweepShape &s,
                                   cudaStream_t st);
cudaError_t launch_plane_async_f64(const PlaneArgs<double> &a, const SweepShape &s,
                                   cudaStream_t st);
cudaError_t launch_plane_async_f32(const PlaneArgs<float> &a, const SweepShape &s,
                                   cudaStream_t st);
cudaError_t plane_async_clusters_f64(const SweepShape &s, int nx, int *n);
cudaError_t plane_async_clusters_f32(const SweepShape &s, int nx, int *n);
cudaError_t plane_active_clusters(int prec, const SweepShape &s, int nx, int *n);

// Sweep variants: linear upwind interpolation, Hermite, moving atmosphere,
// partial redistribution.
constexpr int kSweepLinear = 0, kSweepHermite = 1, kSweepMoving = 2, kSweepPrd = 3;

// Arguments of the sweep kernel.  T is the formal-solution precision.
template <typename T>
struct SweepArgs {
    int nx, ny, nz, nfreq;
    int ng, ngroups, rows;
    unsigned up_mask;        // bit r set when ray r points up
    const T *chi0;           // [nvox] line opacity at unit profile
    const T *S;              // [nvox] line source function
    const T *bbot;           // [nx*ny] intensity entering at the bottom
    const StepGeom *geom;    // [kRays][nz], entry t = 1..nz-1 used
    const T *phi;            // [nfreq] profile
    const T *inv_phi;        // [nfreq] 1/profile
    const T *wphi;           // [nfreq] ray weight x frequency weight x profile
    T *pj, *pu;              // [kRays*ngroups][nvox] partial Jeff and U
    const double *exp_tab;   // [kExpTab] 2^{j/kExpTab} for the FP64 exp (FP64 sweeps only)
    double exp_l1, exp_l2;   // two-part ln2/kExpTab
    const T *dchi0, *dS;     // [nvox] x-slopes of chi0 and S (Hermite sweeps only)
    // moving atmospheres only: per ray and node the projected velocity and
    // the profile normalisation [kRays][nvox]; per frequency (natural order)
    // the offset x_f and the quadrature weight w_f [nfreq]
    const T *uproj, *vnorm, *xf, *wq;
    // partial redistribution only: rho S and rho per frequency in natural
    // order [nfreq][nvox], the natural index of each table position
    // [nfreq], and the per-ray slots of the new mean intensity
    // [kRays][nfreq][nvox] (w_r I; every element written by the sweep)
    const T *rhoS, *rho;
    const int *fidx;
    T *jnu;
};

// Table and reduction constants of the FP64 e^{-x} of the sweep.
void exp_neg_constants(double *tab, double *l1, double *l2);  // tab: kExpTab entries
cudaError_t launch_exp_check(int n, const double *x, double *out, const double *tab, double l1,
                             double l2, cudaStream_t st);

size_t sweep_smem_bytes(int prec, const SweepShape &s, int nx);
// Projected velocities and profile normalisations of a level ([kRays][nvox]
// each) from mu [kRays][3], the velocity [3][nvox] and the frequency offsets
// and weights [nfreq].
cudaError_t launch_vel_prep(int prec, long nvox, int nfreq, const double *mu, const double *vel,
                            const double *xf, const double *wq, void *uproj, void *vnorm,
                            cudaStream_t st);
// Partial redistribution (two-level atom): per node rho_f and rho_f S from
// the lagged mean intensity jnu [nfreq][nvox] (natural frequency order), the
// populations n [2][nvox] and the collisional rates; kmat [nfreq][nfreq] =
// w_f' R(f', f) / phi_f and wphi [nfreq] (normalised) in natural order.
cudaError_t launch_prd_source(int prec, long nvox, int nfreq, double gamma, double g_ratio,
                              double a_ul, const double *kmat, const double *wphi,
                              const double *n, const double *c_lu, const void *jnu, void *rho,
                              void *rhoS, cudaStream_t st);
// jnu [len] = the sum of slots [kRays][len] over rays, in ray order.
cudaError_t launch_prd_collect(int prec, long len, const void *slots, void *jnu,
                               cudaStream_t st);
// Monotone x-slopes (one cell units, periodic rows of nx) of a and b.
cudaError_t launch_xslopes(int prec, int nx, long nvox, const void *a, const void *b, void *da,
                           void *db, cudaStream_t st);

// One cluster of a batched sweep: problem index, ray (two-level) or
// hemisphere (multi-level), frequency group (two-level) or frequency.
struct BatchItem {
    int member, ray, group;
};
cudaError_t launch_sweep_batch(int prec, const void *args, const BatchItem *items, int n_items,
                               int bands, int threads, size_t smem, cudaStream_t st);

// Kernel launchers; each returns the launch error.
cudaError_t launch_opacity(int prec, long nvox, double g_ratio, double kappa,
                           const double *n, void *chi0, void *S, cudaStream_t st);
cudaError_t launch_planck_bottom(int prec, long nplane, double theta, const double *T,
                                 void *bbot, cudaStream_t st);
// How many clusters of shape s the GPU can hold at once (0: it cannot run).
cudaError_t sweep_active_clusters(int prec, const SweepShape &s, int nx, int *n);
cudaError_t launch_sweep_f64(const SweepArgs<double> &a, const SweepShape &s, cudaStream_t st);
cudaError_t launch_sweep_f32(const SweepArgs<float> &a, const SweepShape &s, cudaStream_t st);

// Rate kernel modes.
enum RateMode {
    kRateSolve = 0,      // n <- solution of Gamma(Jeff, U) n = f; C, counts
    kRateResidual = 1,   // out <- f - Gamma(Jeff, U) n
    kRateAddW = 2,       // out <- out + Gamma(Jeff, U) n
    kRateReduce = 3,     // out[0] <- Jeff, out[1] <- U
};

struct RateArgs {
    long nvox;
    int nslots;
    int prec;                  // type of pj/pu
    const void *pj, *pu;       // [nslots][nvox]
    int zero_radiation;        // Jeff = 0, U = 1 instead of the partials
    double a_ul, g_ratio;
    const double *c_ul, *c_lu, *n_tot;
    const double *f;           // [2][nvox] or nullptr for (n_tot, 0)
    double *n;                 // [2][nvox]
    double *out;               // [2][nvox]
    int mode;
    unsigned long long *scal;  // [0] max rel change bits, [1] negatives, [2] non-finite,
                               // [3] populations reset by the 10 % rule
};
cudaError_t launch_rates(const RateArgs &a, cudaStream_t st);

cudaError_t launch_collisions_up(long nvox, double g_ratio, double theta, const double *T,
                                 const double *c_ul, double *c_lu, cudaStream_t st);
// mode: 0 full weighting, 1 half weighting, 2 injection
cudaError_t launch_restrict(int ncomp, int nxf, int nyf, int nzf, const double *fine,
                            double *coarse, cudaStream_t st, int mode = 0);
// The same operators (full weighting; trilinear or Hermite) on arrays of
// the formal-solution precision (prec 0 FP64, 1 FP32), accumulated in FP64.
cudaError_t launch_restrict_prec(int prec, int ncomp, int nxf, int nyf, int nzf,
                                 const void *fine, void *coarse, cudaStream_t st);
// Interpolation onto the fine grid (Sec. 4.5): interp 0 trilinear (tz: the
// fine grid's upper-plane weights), 1 monotone cubic Hermite (zf: the fine
// grid's heights).
cudaError_t launch_prolong_prec(int interp, int prec, int ncomp, int nxc, int nyc, int nzc,
                                const double *tz, const double *zf, const void *coarse,
                                void *fine, cudaStream_t st);
cudaError_t launch_prolong(int interp, int ncomp, int nxc, int nyc, int nzc, const double *tz,
                           const double *zf, const double *coarse, double *fine,
                           cudaStream_t st);
// Eqs. 10-11 with the 10 % rule; the Hermite variant first overwrites
// n_before with the relative correction.
cudaError_t launch_prolong_correct(int interp, int ncomp, int nxc, int nyc, int nzc,
                                   const double *tz, const double *zf, const double *n_after,
                                   double *n_before, double *n_fine, unsigned long long *scal,
                                   cudaStream_t st);
cudaError_t launch_max_rel_change(long len, const double *n_new, const double *n_old,
                                  unsigned long long *scal, cudaStream_t st);

// ---------------------------------------------------------------- multi-level

constexpr int kMaxLevels = 8;

// One frequency point of a multi-level atom; each belongs to one transition.
struct FreqInfo {
    int kind;       // 0 line, 1 bound-free continuum
    int lo, up;     // lower and upper level
    double xy;      // line: offset in reference Doppler widths; continuum: nu/nu_threshold
    double w;       // trapezoid weight in x or y
    double rho;     // line: nu/nu_ref; continuum: threshold nu/nu_ref
    double kappa;   // opacity coefficient
    double gr;      // line: g_u/g_l (unused for continua)
    double adamp;   // line: Voigt damping parameter at t_ref (0: Doppler profile)
};

// One transition: its frequencies are [f_begin, f_end) of the table.
struct TransInfo {
    int kind, lo, up, f_begin, f_end;
    double rho;     // as in FreqInfo
    double coef;    // line: A_ul; continuum: beta
    double gr;      // line: g_u/g_l
};

template <typename T>
struct MlSweepArgs {
    int nx, ny, nz, nfreq, rows;
    const T *chi, *S, *sc, *oc;   // [nfreq][nvox]
    const T *ib;                  // [nfreq][nx*ny] intensity entering at the bottom
    const StepGeom *geom;         // [kRays][nz]
    const double *exp_tab;
    double exp_l1, exp_l2;
    T *jx, *ux;                   // [2 * 12 / rpb slots][nfreq][nvox]
    int rpb;                      // rays per block: 12, 6, 4, 3, 2 or 1 of a hemisphere
    T *jm;                        // mean intensity sum_r w_r I per slot, or null
    const T *dchi, *dS;           // [nfreq][nvox] x-slopes of chi and S (herm only)
    int herm;                     // 1: monotone cubic Hermite upwind interpolation
    // moving atmospheres (moving = 1): chi, S, sc, oc hold the parts the
    // opacity kernel writes in moving mode; per global frequency f0 + f the
    // line offset, quadrature weight and line index (-1: continuum); per
    // line, ray and node the inverse profile sum [nlines][kRays][nvox]; per
    // ray and node the projected velocity [kRays][nvox]; per node 1/d [nvox]
    int moving, f0;
    const T *vx, *vwq;
    const int *vline;
    const T *vnorm, *uproj, *dinv;
};

// Arguments of the multi-level shifted-plane sweep (ml_plane.cuh), one chunk
// of nfreq frequencies.
template <typename T>
struct MlPlaneArgs {
    int nx, ny, nz, nfreq, rows, bands, rpb;
    unsigned long long rmagic, xmagic;   // band_magic(rows), band_magic(nx)
    const T *chi, *S, *sc, *oc;          // [nfreq][nvox]
    const T *ib;                         // [nfreq][nx*ny] intensity entering at the bottom
    const PlaneStep<T> *steps;           // [kRays][nz]
    T *jx, *ux, *jm;                     // [2 * 12 / rpb slots][nfreq][nvox]; jm nullable
    const double *exp_tab;
    double exp_l1, exp_l2;
};

// Frequencies per block the multi-level shifted-plane sweep is built for,
// and the nodes a thread takes per step (band <= this x threads).
constexpr int kMlPlaneNf[] = {1, 2, 4};
// dynamic shared memory limit of the multi-level shifted-plane sweep: its
// static part (the FP64 exp table and the rays' step constants, 3.2 KB) and
// this stay within the 227 KB a block may take
constexpr size_t kMlPlaneMaxSmem = 220 * 1024;
constexpr int kMlPlaneNfCount = 3;
__host__ __device__ constexpr int ml_plane_max_pass(int nf) { return nf <= 2 ? 4 : 2; }
size_t ml_plane_smem_bytes(int prec, int nf, int rows, int nx, int rpb);
cudaError_t launch_ml_plane_f64(const MlPlaneArgs<double> &a, int nf_block, int threads,
                                cudaStream_t st);
cudaError_t launch_ml_plane_f32(const MlPlaneArgs<float> &a, int nf_block, int threads,
                                cudaStream_t st);
cudaError_t ml_plane_active_clusters(int prec, int nf_block, int bands, int rows, int nx,
                                     int rpb, int nfreq, int threads, int *n);

// Partial redistribution of one line of a multi-level atom: its frequencies
// [f_begin, f_end) of the frequency table, their positions pf0 .. pf0+nf-1
// among all PRD line frequencies (the rows of the scaling and rho arrays),
// and `ord` (entries ord0 .. ord0+nf-1 of the order table): the line's
// frequencies (table indices) sorted by |x| with mirror offsets adjacent,
// grouped by equal |x| (grp: entries grp0 .. grp0+ngrp of the group-start
// table, positions within the sorted list).
constexpr int kMaxPrdLineFreq = 128;   // frequencies of one PRD line of a multi-level atom
struct PrdLine {
    int lo, up, f_begin, f_end, pf0, nf, ord0, grp0, ngrp;
    double gamma;   // coherence fraction
    double gr;      // g_u / g_l
    double b_ul;    // A_ul / rho^3
};

// Rates of the lagged field and partial-redistribution ratios per node (see
// launch_ml_prd_rho).
struct MlPrdArgs {
    long nvox;
    int n_levels, n_trans, n_prd;
    const FreqInfo *fi;
    const TransInfo *ti;
    const PrdLine *pl;
    const int *ord, *grp;
    double theta_ref, t_ref;
    const double *n, *T, *c, *saha;  // populations [N][nvox], T, collisions [N][N][nvox], saha
    const void *jbg;                 // lagged mean intensity [n_freq][nvox] (FS precision)
    int prec;
    const double *scale;             // [n_prd_freq][nvox] symmetric scaling of R
    double *rho;                     // [n_prd_freq][nvox] out
    const double *exp_tab;
    double exp_l1, exp_l2;
    const double *chi_c, *sigma_c;   // background opacity [nvox] and scattering (nullable)
    double *oc;                      // [n_prd_freq][nvox] out: 1 - rho chi_t/chi
};

// Opacity of the chunk of frequencies f0 .. f0+nfreq-1, written at the
// chunk-local index [f - f0][nvox].
struct MlOpacityArgs {
    long nvox;
    int nfreq, n_levels, prec;
    const FreqInfo *fi;
    double theta_ref, t_ref;
    const double *n, *T, *chi_c, *saha;
    void *chi, *S, *sc, *oc;       // sc = S - rho eta_t/chi, oc = 1 - chi_t/chi (0 for a
                                   // PRD frequency: its 1 - rho chi_t/chi goes in FP64
                                   // to the radiative sums, MlAccumArgs::prd_oc)
    int f0;
    const double *exp_tab;         // FP64 exp table of the sweep
    double exp_l1, exp_l2;
    const double *sigma_c;         // background scattering [nvox], or null
    const void *jbg;               // background field [n_freq][nvox] (FS precision)
    int moving;                    // 1: write the ray-independent parts instead (a
                                   // moving atmosphere): chi <- the transition's opacity
                                   // at unit profile, S <- its emissivity at unit profile
                                   // (continua: their own), oc <- background opacity,
                                   // sc <- background emissivity
    const int *prd_index;          // [n_freq] row of rho for a PRD line frequency, else -1
                                   // (null: no partial redistribution)
    const double *prd_rho;         // [n_prd_freq][nvox] emission-profile ratio psi/phi
    const VoigtTable *voigt;       // coefficients of the Voigt function (damped lines), or null
};

// Radiative sums per transition and node, [n_trans][3][nvox] in FP64:
//   line:       sum w phi, sum w phi J, sum w phi U   (phi at the node's T)
//   continuum:  sum qa J, sum qa E J, sum qa E (rho y)^3 U
// accumulated chunk by chunk from the per-frequency angle sums Jx, Ux.
constexpr int kAccTerms = 3;

struct MlAccumArgs {
    long nvox;
    int f0, nfreq, n_trans, prec;  // chunk f0 .. f0+nfreq-1
    const FreqInfo *fi;
    const TransInfo *ti;
    double theta_ref, t_ref;
    const double *T;
    const void *jx, *ux;           // [nslots][nfreq][nvox] of the chunk
    int nslots;                    // ray groups of both hemispheres
    int zero_radiation;            // 1: J = 0, U = 1 (jx, ux unused)
    double *acc;
    const double *exp_tab;         // FP64 exp table of the sweep
    double exp_l1, exp_l2;
    const void *jm;                // mean intensity per slot [nslots][nfreq][nvox], or null
    void *jbg;                     // background field [n_freq][nvox] written from jm
    int moving;                    // 1: line sums already carry their per-ray profile
                                   // weights (sum 1 over a line), so they add as they are
    const int *prd_index;          // [n_freq] PRD row of a frequency, else -1 (null: none)
    const double *prd_oc;          // [n_prd_freq][nvox] 1 - rho chi_t/chi in FP64: U of a
                                   // PRD frequency is oc + (1 - oc) sum_r w_r u_r
    const VoigtTable *voigt;       // coefficients of the Voigt function (damped lines), or null
};

struct MlRateArgs {
    long nvox;
    int n_levels, n_trans;
    const TransInfo *ti;
    const double *acc;            // [n_trans][kAccTerms][nvox]
    const double *T, *c, *saha, *n_tot;   // c [N][N][nvox], saha [N][nvox]
    const double *f;              // [N][nvox] or nullptr for (n_tot, 0, ...)
    double *n, *out;              // [N][nvox]
    int mode;                     // RateMode (kRateReduce not used)
    unsigned long long *scal;
};

size_t ml_sweep_smem_bytes(int prec, int rows, int nx, int rpb, int herm = 0,
                           int moving = 0);
// Moving multi-level atmospheres: uproj [kRays][nvox], dinv [nvox] and vnorm
// [nlines][kRays][nvox] of a level (see MlSweepArgs).
cudaError_t launch_ml_vel_prep(int prec, long nvox, int ntrans, const TransInfo *ti,
                               const FreqInfo *fi, const double *mu, const double *vel,
                               const double *T, double t_ref, void *uproj, void *dinv,
                               void *vnorm, cudaStream_t st);
cudaError_t launch_ml_opacity(const MlOpacityArgs &a, cudaStream_t st);
// Per node and PRD line: the symmetric scaling c of R_I-A at the node's
// Doppler width, the fixed point of c <- sqrt(c phi / (R0^T (wq c))) after
// 200 steps from c = 1 (R = diag(c) R0 diag(c) then has marginals phi).
cudaError_t launch_ml_prd_scale(long nvox, int n_prd, const PrdLine *pl, const FreqInfo *fi,
                                const int *ord, const int *grp, double t_ref, const double *T,
                                double *scale, cudaStream_t st);
// Per node and PRD line frequency: rho = 1 + gamma f_rad (sum_f' wq R(f', f)
// J_f' / (phi_f Jbar) - 1) from the lagged mean intensity.
cudaError_t launch_ml_prd_rho(const MlPrdArgs &a, cudaStream_t st);
cudaError_t launch_ml_bottom(int prec, long nplane, int nfreq, const FreqInfo *fi,
                             double theta_ref, const double *T, void *ib, cudaStream_t st);
cudaError_t launch_ml_sweep_f64(const MlSweepArgs<double> &a, int bands, int threads,
                                cudaStream_t st);
cudaError_t launch_ml_sweep_f32(const MlSweepArgs<float> &a, int bands, int threads,
                                cudaStream_t st);
cudaError_t launch_ml_accum(const MlAccumArgs &a, cudaStream_t st);
cudaError_t launch_ml_rates(const MlRateArgs &a, cudaStream_t st);
cudaError_t launch_ml_sweep_batch(int prec, const void *args, const BatchItem *items,
                                  int n_items, int bands, int threads, size_t smem,
                                  cudaStream_t st);

}  // namespace mg3d
