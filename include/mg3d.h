/*
 * mg3d.h -- C ABI of a GB300 (sm_103a) library for non-LTE 3D radiative
 * transfer with a non-linear multigrid method (Bjorgen & Leenaarts 2017).
 *
 * The problem (Sec. 2.1): find atomic level populations n on a Cartesian grid
 * such that the transfer equation dI/dtau = S(n) - I (Eq. 1) and statistical
 * equilibrium (Eq. 2), with the first rate equation replaced by particle
 * conservation (Eq. 3), hold everywhere: W(n) = f with f = (n_tot, 0) per node
 * (Eq. 4).  The library solves it with MALI (Jacobi iteration with the
 * diagonal approximate operator), FAS V-cycles (Sec. 2.2, Eqs. 5-11) and full
 * multigrid (Sec. 2.3) on one GPU.
 *
 * Models supported: a static two-level atom in complete redistribution with a
 * Doppler line profile sampled at n_freq points and no background continuum
 * (mg3d_create, the fast path), and multi-level atoms with lines, bound-free
 * continua and a grey background continuum (mg3d_create_ml).
 *
 * Conventions for every entry point:
 *  - returns MG3D_OK (0) or a negative MG3D_E_* code; no exception crosses the
 *    ABI; mg3d_last_error() then gives a message (per calling thread);
 *  - arrays are C-ordered: a field is [nz][ny][nx] (x fastest) and a set of
 *    populations is [n_levels][nz][ny][nx] (two-level atom: index 0 the lower
 *    and 1 the upper level); z[0] is the bottom boundary plane;
 *  - pointers named *_host are host memory owned by the caller; the library
 *    reads them during the call (or writes them before returning) and keeps
 *    no reference.  All other state lives in device memory that the handle
 *    owns and frees in mg3d_destroy;
 *  - "level" numbers grids as the paper does: 1 is the coarsest and
 *    n_grids the finest;
 *  - work is ordered on the handle's CUDA stream; calls that return host data
 *    or a convergence measure synchronise that stream; a handle must not be
 *    used from two threads at once.
 */
#ifndef MG3D_H
#define MG3D_H

#ifdef __cplusplus
extern "C" {
#endif

#define MG3D_OK 0
#define MG3D_E_ARG (-1)       /* bad argument (null pointer, out of range) */
#define MG3D_E_GRID (-2)      /* grid does not coarsen n_grids - 1 times */
#define MG3D_E_CUDA (-3)      /* a CUDA call failed */
#define MG3D_E_OOM (-4)       /* device or host allocation failed */
#define MG3D_E_DIVERGED (-5)  /* a solve produced non-finite populations */
#define MG3D_E_MAXITER (-6)   /* iteration or cycle cap reached before tol */
#define MG3D_E_STATE (-8)     /* call not valid in the handle's current state */

#define MG3D_MAX_GRIDS 8

/* Precision of the formal solution (interpolation, opacities, intensities).
 * Rate equations, residuals and grid transfer are always FP64. */
#define MG3D_PREC_F64 0
#define MG3D_PREC_F32 1

typedef struct mg3d_handle mg3d_handle;

/* Input atmosphere on the finest grid (Sec. 3.1, 4.1-4.2). */
typedef struct {
    int nx, ny, nz;        /* nodes; x, y periodic, z bounded (nz odd) */
    double dx, dy;         /* constant horizontal spacing */
    const double *z;       /* [nz] node heights, strictly increasing */
    const double *T;       /* [nz][ny][nx] gas temperature, K */
    const double *n_tot;   /* [nz][ny][nx] total number density of the atom */
    const double *c_ul;    /* [nz][ny][nx] collisional de-excitation rate */
    const double *vel;     /* nullable: [3][nz][ny][nx] velocity (x, y, z components)
                              in Doppler widths.  A moving atmosphere (the paper's
                              Bifrost snapshots move): along ray r the CRD profile
                              at a node is phi(x - mu_r . vel), and the frequency
                              weights w phi are renormalised per node and ray to sum
                              to 1; coarse grids full-weight the field.  Takes the
                              linear upwind interpolation, no batches; the mirror
                              frequency sharing of the static sweep does not apply. */
} mg3d_atmosphere;

/* Two-level model atom (Sec. 3.2).  Intensities are in units of
 * 2 h nu0^3 / c^2, so B_ul = A_ul and B_lu = g_ratio A_ul.  The line opacity
 * at normalised offset x is kappa (n_l g_ratio - n_u) exp(-x^2)/sqrt(pi) and
 * the source function n_u / (n_l g_ratio - n_u).  The frequency grid is
 * n_freq equidistant offsets in [-x_max, x_max] with trapezoid weights,
 * renormalised so that the weighted profile sums to one. */
typedef struct {
    double a_ul;     /* Einstein A_ul, the rate unit */
    double g_ratio;  /* g_u / g_l */
    double theta;    /* h nu0 / k in K; B(T) = 1/(exp(theta/T) - 1) */
    double kappa;    /* line opacity constant */
    int n_freq;      /* frequency points across the line, >= 1 */
    double x_max;    /* half width of the grid in Doppler widths */
    double gamma_prd; /* coherence fraction of partial redistribution in [0, 1];
                         0: complete redistribution (the paper's runs).  Reading
                         of the next step the paper names: angle-averaged Doppler
                         redistribution R(x', x) = erfc(max(|x|, |x'|))/2 on the
                         grid (scaled symmetrically so that both marginals are
                         the profile), mixed with CRD by gamma; the line source
                         function of frequency f is rho_f S with
                         rho_f = 1 + gamma f_rad (sum_f' w_f' R(f', f) J_f' /
                         (phi_f Jbar) - 1), f_rad = B_lu Jbar/(B_lu Jbar + C_lu),
                         from the mean intensity of the previous formal solution on
                         the grid (lagged like a background field: restricted and
                         Lambda-iterated once on a coarse-grid entry, then fixed on
                         that grid; prolonged in FMG); MALI preconditions with
                         U = sum w phi (1 - w0 rho).  Static atmospheres, linear
                         upwind interpolation, no batches. */
    double a_damp;    /* damping parameter in Doppler widths, >= 0: the line
                         profile is the Voigt profile H(a, x)/sqrt(pi) (0: the
                         Doppler profile), and partial redistribution uses
                         Hummer's angle-averaged R_II (the average over the
                         scattering angle g, weight sin g/2, of exp(-[(x - x')/(2
                         sin(g/2))]^2) H(a/cos(g/2), (x + x')/(2 cos(g/2)))/(pi
                         sin g)); both are tabulated on the host at creation,
                         H by adaptive Gauss-Kronrod quadrature, R_II-A by the
                         same quadrature over g with H from Weideman's rational
                         expansion (mg3d_check_voigt).  Static atmospheres only
                         (MG3D_E_ARG with a velocity field). */
} mg3d_atom;

/* Angle quadrature: the 24-direction A4 set of Carlson (Sec. 3): per octant
 * the permutations of (a, a, b), b = sqrt(1 - 2a^2), weights 1/24.
 * a <= 0 selects a = sqrt((4 - sqrt(6.4))/12) = 0.3500212..., which
 * integrates mu^4 exactly. */
typedef struct {
    double a;
} mg3d_quadrature;

/* Multigrid schedule (Sec. 2.2-2.3, 4.12, Table 1). */
typedef struct {
    int n_grids;   /* number of grids l, 1..MG3D_MAX_GRIDS */
    int nu_fmg;    /* MALI iterations on the coarsest grid in FMG */
    int nu0;       /* pre-smoothing on the finest grid in the first V-cycle */
    int nu1;       /* pre-smoothing iterations */
    int nu2;       /* post-smoothing iterations */
    int nu3;       /* iterations on the coarsest grid */
    int fs_prec;   /* MG3D_PREC_F64 or MG3D_PREC_F32 */
    int restriction; /* of populations and residuals (Sec. 4.4):
                        MG3D_RESTRICT_FULL (the paper's choice), _HALF, _INJECT;
                        the atmosphere is always full-weighted (Sec. 4.7) */
    int ml_chunk;  /* multi-level handles: frequencies per chunk of the formal
                      solution, 0 for the automatic choice (mg3d_set_ml_chunk);
                      ignored by two-level handles */
    int interpolation; /* interpolation operator (Sec. 4.5) of the V-cycle
                          correction, the FMG transfer and mg3d_prolong:
                          MG3D_INTERP_LINEAR (trilinear, the paper's choice)
                          or MG3D_INTERP_HERMITE (monotone cubic Hermite) */
    int sc_interp; /* upwind interpolation of the formal solution (Sec. 3):
                      MG3D_INTERP_LINEAR (bilinear) or MG3D_INTERP_HERMITE */
} mg3d_params;

/* Monotone cubic Hermite (Auer 2003) means successive 1D passes along x and
 * y (periodic) and, for the prolongation, z (physical heights): on each
 * interval the cubic through its two nodes with slopes from their
 * neighbours, the harmonic mean of the adjacent secants where they have the
 * same sign and 0 otherwise (Fritsch & Butland 1984; shape-preserving
 * three-point slopes at the z ends).  Values stay between the two nodes of
 * every interval, so positive data give positive results. */
#define MG3D_INTERP_LINEAR 0
#define MG3D_INTERP_HERMITE 1

#define MG3D_RESTRICT_FULL 0    /* 27-node full weighting */
#define MG3D_RESTRICT_HALF 1    /* centre 1/2, six axis neighbours 1/12 */
#define MG3D_RESTRICT_INJECT 2  /* coarse node takes the fine node's value */

/* Outcome of a solve. */
typedef struct {
    int iterations;              /* MALI sweeps (mali) or V-cycles (fas, fmg) */
    int sweeps[MG3D_MAX_GRIDS + 1];            /* MALI sweeps per level */
    int formal_solutions[MG3D_MAX_GRIDS + 1];  /* formal solutions per level */
    double last_change;          /* C of the last iteration or cycle */
    long long negatives;         /* populations reset by the 10 % rule */
    double seconds;              /* wall time of the solve */
    double fine_fs_equivalents;  /* sum over levels of FS count x 8^(k - l) */
} mg3d_stats;

/* Counters of the handle since creation (or the last reset).  The level_*
 * arrays split the sweep counters by grid level (index = level). */
typedef struct {
    long long kernel_launches;   /* launches of this library's kernels */
    long long fs_launches;       /* formal-solution sweep launches */
    double fs_units;             /* nodes x rays x frequencies swept */
    double fs_kernel_ms;         /* summed device time of the sweep kernel,
                                    valid only while timing is enabled */
    long long fs_timed_launches; /* sweeps included in fs_kernel_ms */
    long long level_fs_launches[MG3D_MAX_GRIDS + 1];
    double level_fs_units[MG3D_MAX_GRIDS + 1];
    double level_fs_kernel_ms[MG3D_MAX_GRIDS + 1];
    long long level_fs_timed_launches[MG3D_MAX_GRIDS + 1];
} mg3d_counters;

/* Message of the last failed call on this thread ("" if none).
 * No counterpart in the paper (error reporting). */
const char *mg3d_last_error(void);

/* Create a solver: validates the grid (Sec. 4.2; MG3D_E_GRID unless every
 * coarsening keeps nz odd and nx, ny even, i.e. nz = A 2^(l-1) + 1 and
 * nx, ny = B 2^(l-1) with A, B >= 1 for l = n_grids; nx, ny below 65536,
 * else MG3D_E_ARG), checks dx, dy > 0 and z
 * increasing (MG3D_E_ARG), copies the atmosphere to device memory, builds the
 * coarser grids by
 * dropping every second node and full-weighting T, n_tot and c_ul (Sec. 4.1,
 * 4.7), and precomputes the per-plane upwind geometry of every ray.
 * Populations start at zero-radiation equilibrium (Sec. 4.11) on every grid.
 * On success *out holds the handle; on failure *out is NULL. */
int mg3d_create(const mg3d_atmosphere *atm, const mg3d_atom *atom,
                const mg3d_quadrature *quad, const mg3d_params *params,
                mg3d_handle **out);

/* Free every device and host resource of the handle (NULL is accepted).
 * No counterpart in the paper (resource management). */
int mg3d_destroy(mg3d_handle *h);

/* Order the handle's work on an existing CUDA stream (a cudaStream_t passed
 * as void*; NULL restores the handle's own stream).  The caller keeps
 * ownership of the stream and must keep it alive while the handle uses it.
 * No counterpart in the paper (launch control). */
int mg3d_set_stream(mg3d_handle *h, void *cuda_stream);

/* Shape of a level's grid.
 * The levels are the grids of Sec. 2.2, coarsened as in Sec. 4.3. */
int mg3d_level_shape(const mg3d_handle *h, int level, int *nx, int *ny, int *nz);

/* Copy a level's populations [n_levels][nz][ny][nx] out to, or in from, host
 * memory.  The populations are the whole state of a CRD handle, so a new
 * handle given them resumes bit for bit.  The lagged fields of background
 * scattering (sigma_c) and of partial redistribution (gamma_prd) are not
 * part of them: a resumed handle restarts those from the state its creation
 * left (the zero-radiation field), and its next iterates differ from the
 * uninterrupted run until the fields have been recomputed.
 * n is the unknown of Eq. 4; checkpoint and resume have no counterpart in
 * the paper. */
int mg3d_get_populations(mg3d_handle *h, int level, double *n_host);
int mg3d_set_populations(mg3d_handle *h, int level, const double *n_host);

/* Reset a level's populations to the zero-radiation solution of statistical
 * equilibrium (all radiative rates from J = 0; Sec. 4.11) and its right-hand
 * side to f = (n_tot, 0). */
int mg3d_init_zero_radiation(mg3d_handle *h, int level);

/* One formal solution on a level with its current populations (Sec. 3:
 * short characteristics, linear interpolation, A4 rays, CRD).  Optional host
 * outputs [nz][ny][nx]: Jeff = Jbar - Lambda* S (the profile-averaged mean
 * intensity minus its local part) and U = 1 - Lambda* (Lambda* the diagonal
 * of the Lambda operator).  Either pointer may be NULL. */
int mg3d_formal_solve(mg3d_handle *h, int level, double *jeff_host, double *u_host);

/* The same formal solution (Sec. 2.1: Jeff and U = 1 - Lambda* are what the
 * MALI update of Eqs. 2-4 takes from it) in a chosen precision prec
 * (MG3D_PREC_F64 or MG3D_PREC_F32) instead of the handle's fs_prec.  In the
 * handle's own precision it is mg3d_formal_solve.  In the other precision
 * (two-level atoms, static, complete redistribution, linear upwind
 * interpolation; MG3D_E_ARG otherwise) the first call on a level allocates
 * that precision's opacity, source, bottom-intensity and step buffers for the
 * level and the handle's partial sums and frequency tables in it, which the
 * handle keeps until mg3d_destroy; populations, rates and outputs stay FP64.
 * MG3D_E_STATE for multi-level handles. */
int mg3d_formal_solve_ex(mg3d_handle *h, int level, int prec, double *jeff_host,
                         double *u_host);

/* Device-pointer variants for callers whose buffers live on the GPU (for
 * example PyTorch tensors' data_ptr()), ordered on the caller's CUDA stream
 * cuda_stream (NULL: the legacy default stream): the work waits for what was
 * enqueued on that stream before the call, and work enqueued on it after the
 * call waits for the results.  They return once the work is enqueued and do
 * not synchronise.  Device buffers are owned by the caller and must stay
 * valid until the stream reaches the call's work.
 * mg3d_formal_solve_dev: as mg3d_formal_solve_ex (Sec. 2.1), outputs
 *   jeff_dev, u_dev [nz][ny][nx] FP64 (either may be NULL);
 * mg3d_get_populations_dev / mg3d_set_populations_dev: as
 *   mg3d_get/set_populations, n_dev [n_levels][nz][ny][nx] FP64 (n of Eq. 4;
 *   checkpoints have no counterpart in the paper). */
int mg3d_formal_solve_dev(mg3d_handle *h, int level, int prec, double *jeff_dev, double *u_dev,
                          void *cuda_stream);
int mg3d_get_populations_dev(mg3d_handle *h, int level, double *n_dev, void *cuda_stream);
int mg3d_set_populations_dev(mg3d_handle *h, int level, const double *n_dev,
                             void *cuda_stream);

/* n_sweeps MALI iterations on a level solving W(n) = f for that level's f
 * (f = (n_tot, 0) on the finest grid, the tau-corrected f of Eq. 9 on a
 * coarser one).  *max_rel_change (nullable) receives C of the last sweep:
 * max |n_new - n_old| / |n_new| over levels and nodes (Sec. 3.3). */
int mg3d_mali_sweep(mg3d_handle *h, int level, int n_sweeps, double *max_rel_change);

/* Residual r = f - W_*(n) of a level (Eq. 5), with an extra formal solution
 * for the current populations; r_host is [n_levels][nz][ny][nx]. */
int mg3d_residual(mg3d_handle *h, int level, double *r_host);

/* One FAS V-cycle from the finest grid (Sec. 2.2).  is_first selects nu0
 * instead of nu1 for the finest-grid pre-smoothing (Sec. 4.12).
 * *max_rel_change (nullable) receives C over the whole cycle. */
int mg3d_fas_vcycle(mg3d_handle *h, int is_first, double *max_rel_change);

/* Plain MALI on the finest grid from the zero-radiation start until C < tol
 * (MG3D_E_MAXITER after max_sweeps).  stats is nullable.
 * Follows Sec. 2.1 and Sec. 3 (MALI), Sec. 4.11 (the start) and Sec. 3.3 (C). */
int mg3d_mali_solve(mg3d_handle *h, double tol, int max_sweeps, mg3d_stats *stats);

/* FAS V-cycles from the zero-radiation start until C(cycle) < tol.
 * Follows Sec. 2.2 (the V-cycle, Eqs. 5-11) and Sec. 3.3 (C). */
int mg3d_fas_solve(mg3d_handle *h, double tol, int max_cycles, mg3d_stats *stats);

/* Full multigrid (Sec. 2.3): nu_fmg MALI iterations on grid 1 from the
 * zero-radiation start, trilinear interpolation of the full approximation to
 * each finer grid with one V-cycle there, then V-cycles on the finest grid
 * until C(cycle) < tol. */
int mg3d_fmg_solve(mg3d_handle *h, double tol, int max_cycles, mg3d_stats *stats);

/* One stage of full multigrid (Sec. 2.3, Fig. 1), for callers that inspect
 * each grid's solution as FMG builds it: stage 1 starts grid 1 from the
 * zero-radiation populations and runs nu_fmg MALI sweeps on it; stage k =
 * 2..n_grids interpolates the full approximation from grid k-1 to grid k
 * (Sec. 4.5) and, below the finest grid, runs one V-cycle on grid k.  After
 * stage k, mg3d_get_populations(h, k) reads grid k's approximation.  Stages
 * run in order (MG3D_E_STATE otherwise; stage 1 restarts);
 * mg3d_fmg_solve is stages 1..n_grids followed by V-cycles on the finest grid
 * (mg3d_fas_vcycle, the first with is_first = 1) until C < tol.  Synchronises
 * the handle's stream. */
int mg3d_fmg_stage(mg3d_handle *h, int stage);

/* ------------------------------------------------------------------------
 * Multi-level atoms (Sec. 3.2: the paper's 3- and 6-level Ca II and H I atoms;
 * here any atom of 2..8 levels with lines and bound-free continua).
 *
 * Each frequency point belongs to one transition.  With a grey LTE background
 * continuum chi_c (source function B_nu), the opacity and source function at
 * a frequency of transition t (lower l, upper u) are
 *   chi = chi_t + chi_c,   S = (eta_t + chi_c B_nu) / chi,
 * line:        chi_t = kappa (n_l g_u/g_l - n_u) phi,  eta_t = kappa rho^3 n_u phi,
 *              phi = exp(-(x/d)^2)/(sqrt(pi) d), d = sqrt(T/t_ref) (thermal
 *              Doppler width relative to t_ref), B_nu taken at line centre;
 * bound-free:  chi_t = kappa y^-3 (n_l - n_u G E),  eta_t = kappa y^-3 n_u G E (rho y)^3,
 *              y = nu/nu_threshold, G = (n_l/n_u) in LTE (saha input), E = exp(-theta_ref rho y/T).
 * Intensities are in units of 2 h nu_ref^3/c^2; B_nu = (nu/nu_ref)^3 /
 * (exp(theta_ref (nu/nu_ref)/T) - 1).  MALI uses the diagonal-operator
 * preconditioning of Rybicki & Hummer (1992): the transition's own share of
 * S and of chi enters the local operator; rates for a line are
 * P_lu = B_lu Jbar + C_lu, P_ul = A_ul Ubar + B_ul Jbar + C_ul (B_ul = A_ul/rho^3,
 * B_lu = g_u/g_l B_ul), for a continuum (qa = beta w_y y^-4)
 * P_lc = sum qa Jx + C_lc, P_cl = G sum qa E ((rho y)^3 Ux + Jx) + C_cl.
 * The N x N system with row 0 replaced by conservation is solved by Gaussian
 * elimination with partial pivoting.  The frequency grid of a line is n_freq
 * equidistant offsets in [-x_max, x_max] (reference Doppler widths), of a
 * continuum n_freq equidistant y in [1, y_max]; both with trapezoid weights,
 * the line profile weights renormalised per node. */
typedef struct {
    int lower, upper;   /* level indices, lower < upper */
    double rho;         /* nu / nu_ref */
    double a_ul;        /* Einstein A (rate units) */
    double kappa;       /* opacity coefficient at unit profile */
    int n_freq;
    double x_max;
    double a_damp;      /* Voigt damping parameter at t_ref in [0, 1000) (0:
                           Doppler profile).  The damping width does not scale
                           with temperature while the Doppler width d =
                           sqrt(T/t_ref) does, so a node's profile is
                           H(a/d, x/d)/(sqrt(pi) d), from the rational Voigt
                           function (mg3d_check_voigt) in FP64 per node and
                           frequency, rounded once to the formal-solution
                           precision.  MG3D_E_ARG with a velocity field, in an
                           atom with partial-redistribution lines, or in a
                           batch */
    double gamma_prd;   /* coherence fraction of partial redistribution in
                           [0, 1] (0: CRD).  The next step Sec. 6 names, read as
                           for the two-level atom: the line emits with the
                           profile rho_f phi_f, rho_f = 1 + gamma_prd f_rad
                           (sum_f' wq_f' R(f', f) J_f' / (phi_f Jbar) - 1), R the
                           angle-averaged Doppler redistribution R_I-A at each
                           node's Doppler width d, erfc(max(|x|, |x'|)/d)/(2 d^2),
                           scaled symmetrically so that its marginals over the
                           line's normalised weights wq are the node's profile
                           (200 steps of the fixed point, once per grid), J the
                           lagged mean intensity of the previous formal solution
                           on the grid (shared with background scattering:
                           cleared at the zero-radiation start, restricted and
                           Lambda-iterated on a coarse-grid entry, prolonged in
                           FMG), f_rad = n_l B_lu Jbar over the inflow into the
                           upper level with the lagged field's plain rates;
                           rho = 1 where Jbar = 0.  The line's emissivity and
                           the transition's shares of S and chi in MALI scale by
                           rho.  At most 128 frequencies per PRD line; static
                           atmospheres with linear upwind interpolation, no
                           batches (MG3D_E_ARG otherwise) */
} mg3d_line;

typedef struct {
    int lower;          /* bound level; the upper level is the last level */
    double rho;         /* threshold nu / nu_ref */
    double beta;        /* photoionisation rate per unit J at threshold */
    double kappa;       /* opacity per unit population at threshold */
    int n_freq;
    double y_max;       /* frequencies nu/nu_threshold in [1, y_max] */
} mg3d_continuum;

typedef struct {
    int n_levels;                 /* 2..8; bound-free continua end on the last */
    const double *g;              /* [n_levels] statistical weights */
    const double *theta;          /* [n_levels] level energies / k (K), informative */
    double theta_ref;             /* h nu_ref / k (K) */
    double t_ref;                 /* temperature of the reference Doppler width */
    int n_lines;
    const mg3d_line *lines;
    int n_continua;
    const mg3d_continuum *continua;
} mg3d_ml_atom;

typedef struct {
    int nx, ny, nz;
    double dx, dy;
    const double *z;        /* [nz] */
    const double *T;        /* [nz][ny][nx] */
    const double *n_tot;    /* [nz][ny][nx] */
    const double *chi_c;    /* [nz][ny][nx] grey background absorption (source B_nu) */
    const double *c;        /* [N][N][nz][ny][nx] collisional rate from i to j (i != j) */
    const double *saha;     /* [N][nz][ny][nx] LTE ratio (n_i/n_c) to the last level */
    const double *sigma_c;  /* [nz][ny][nx] grey background coherent scattering, or NULL
                               (Sec. 4.8): chi = chi_t + chi_c + sigma_c and
                               S = (eta_t + chi_c B_nu + sigma_c J_nu)/chi, with J_nu the
                               mean intensity of the previous formal solution on the same
                               grid (a Lambda-iteration of the background; the MALI
                               preconditioning treats only the transition's own emission
                               as new).  The zero-radiation start clears the field and
                               runs one Lambda-iteration; a V-cycle entering a coarser
                               grid full-weights it; FMG prolongs it with the
                               populations.  Not supported in batches. */
    const double *vel;      /* [3][nz][ny][nx] velocity in Doppler widths at t_ref, or
                               NULL: a moving atmosphere.  Along ray r a line's profile
                               at a node is phi((x - mu_r . vel)/d)/(d sqrt(pi)), d the
                               node's Doppler width in units of the one at t_ref,
                               renormalised over the line's frequencies per node and
                               ray; continua and the background do not shift.  The
                               per-frequency angle sums of mg3d_formal_solve_ml then
                               carry each ray's normalised profile weight of a line
                               inside the ray sum.  Linear upwind interpolation only;
                               not supported in batches. */
} mg3d_ml_atmosphere;

/* Create a solver for a multi-level atom; everything else as mg3d_create.
 * Populations are [n_levels][nz][ny][nx] in every entry point.
 * The atom, its opacities and rates follow Eqs. 1-4 and Sec. 3.2. */
int mg3d_create_ml(const mg3d_ml_atmosphere *atm, const mg3d_ml_atom *atom,
                   const mg3d_quadrature *quad, const mg3d_params *params,
                   mg3d_handle **out);

/* Levels of the handle's atom and its number of frequency points.
 * No counterpart in the paper. */
int mg3d_n_levels(const mg3d_handle *h, int *n_levels, int *n_freq);

/* One multi-level formal solution: per frequency and node the angle sums
 * Jx = sum_r w_r (I - w0 S_t) and Ux = sum_r w_r (1 - w0 chi_t/chi), with S_t
 * the transition's part of the source function (for a partial-redistribution
 * line S_t = rho eta_t/chi and Ux = sum_r w_r (1 - w0 rho chi_t/chi), with
 * rho from the grid's lagged mean intensity); host outputs
 * [n_freq][nz][ny][nx] (nullable).  MG3D_E_STATE on a two-level handle.
 * The formal solution of Sec. 3 at every frequency of every transition. */
int mg3d_formal_solve_ml(mg3d_handle *h, int level, double *jx_host, double *ux_host);

/* Frequencies per chunk of the multi-level formal solution.  The opacity,
 * the sweep and the reduction of the angle sums to the per-transition sums
 * the rate equations use run chunk by chunk, so device memory for the
 * per-frequency arrays scales with the chunk, not with n_freq (the rates and
 * the populations are the same for every chunk size, up to rounding).  At
 * creation the library takes all frequencies when their arrays fit in 60 % of
 * the free device memory, else the largest chunk that does.  freq_per_chunk =
 * 0 means all frequencies.  Reallocates the chunk buffers (MG3D_E_OOM if they
 * do not fit); MG3D_E_STATE on a two-level handle.  Batch members need all
 * frequencies in one chunk.
 * No counterpart in the paper (memory layout). */
int mg3d_set_ml_chunk(mg3d_handle *h, int freq_per_chunk);
int mg3d_get_ml_chunk(const mg3d_handle *h, int *freq_per_chunk);

/* Launch shape of a level's multi-level sweep: bands = thread blocks (one
 * cluster, 1..8) sharing each plane, rays_per_block = rays of a hemisphere
 * each block carries (a divisor of 12; fewer rays need less shared memory,
 * 2 x rays x rows x nx values, and give more blocks), threads per block (a
 * multiple of 32 up to 512).  The library picks one at creation (all 12 rays
 * where some band count fits); MG3D_E_ARG for shapes that do not fit.
 * No counterpart in the paper (launch control). */
int mg3d_set_ml_shape(mg3d_handle *h, int level, int bands, int rays_per_block, int threads);
int mg3d_get_ml_shape(const mg3d_handle *h, int level, int *bands, int *rays_per_block,
                      int *threads);

/* Multi-level sweep shape with its kind: kind 0 as mg3d_set_ml_shape (any
 * atmosphere; freq_per_block 1); kind 1 the shifted-plane form (static
 * atmospheres with the linear upwind interpolation, Sec. 3 and Sec. 4.2):
 * each ray's finished plane is stored shifted by the offset of the step that
 * reads it, so every node finds its upwind corners at fixed offsets, and the
 * opacity and source function of freq_per_block (1, 2 or 4; FP64: 1)
 * frequencies ride along with the intensities; bands 1..16 (above 8 a
 * non-portable cluster size), threads 32..512 covering the band in at most 4
 * nodes per thread (2 with 4 frequencies per block).  MG3D_E_ARG for shapes
 * that do not fit in shared memory or cannot be scheduled; the autotuner
 * times both kinds.  No counterpart in the paper (launch control). */
int mg3d_set_ml_shape_ex(mg3d_handle *h, int level, int bands, int rays_per_block, int threads,
                         int kind, int freq_per_block);
int mg3d_get_ml_shape_ex(const mg3d_handle *h, int level, int *bands, int *rays_per_block,
                         int *threads, int *kind, int *freq_per_block);

/* ------------------------------------------------------------------------
 * Batches: many independent atmospheres of uneven size (two-level and
 * multi-level atoms mixed) iterated in lockstep.  Every formal solution of
 * the batch is one launch per atom kind whose thread-block clusters each
 * take one (member, ray or hemisphere, frequency group) of a shared work
 * table; the other per-node kernels run per member; a whole batched V-cycle
 * is captured once into a CUDA graph and replayed.  Members must share
 * n_grids, the formal-solution precision and the multigrid schedule; creating
 * the batch moves them onto the batch's stream and fixes their sweep shapes
 * (a common number of bands per level), so they should not be autotuned or
 * used alone while the batch exists.  The batch does not own its members. */
typedef struct mg3d_batch mg3d_batch;
int mg3d_batch_create(int n, mg3d_handle *const *members, mg3d_batch **out);
int mg3d_batch_destroy(mg3d_batch *b);
/* One lockstep V-cycle; max_rel_change (nullable) receives C of each member
 * ([n] doubles).
 * The V-cycle of Sec. 2.2 per member; batching has no counterpart in the
 * paper. */
int mg3d_batch_fas_vcycle(mg3d_batch *b, int is_first, double *max_rel_change);
/* FAS from the zero-radiation start, or full multigrid, until every member's
 * change over a cycle is below tol; stats (nullable) is [n] (iterations: the
 * cycle at which each member first met tol).
 * FAS and FMG of Sec. 2.2-2.3 per member; batching has no counterpart in the
 * paper. */
int mg3d_batch_fas_solve(mg3d_batch *b, double tol, int max_cycles, mg3d_stats *stats);
int mg3d_batch_fmg_solve(mg3d_batch *b, double tol, int max_cycles, mg3d_stats *stats);
/* Kernel launches and formal-solution units (nodes x rays x frequencies)
 * of the batch so far.
 * No counterpart in the paper (instrumentation). */
int mg3d_batch_counters(const mg3d_batch *b, long long *kernel_launches, double *fs_units);

/* Grid-transfer operators on host arrays of ncomp fields, for checking.
 * mg3d_restrict: the handle's restriction (Sec. 4.4) from level_fine to level_fine-1,
 * fine_host [ncomp][fine nodes] -> coarse_host [ncomp][coarse nodes].
 * mg3d_prolong: trilinear interpolation (Sec. 4.5) from level_fine-1 to
 * level_fine.  1 <= ncomp <= 4. */
int mg3d_restrict(mg3d_handle *h, int level_fine, int ncomp, const double *fine_host,
                  double *coarse_host);
int mg3d_prolong(mg3d_handle *h, int level_fine, int ncomp, const double *coarse_host,
                 double *fine_host);

/* Sweep launch shape of a level (two-level handles): freq_per_block
 * frequencies per thread block, bands = thread blocks (one cluster) sharing
 * each horizontal plane (1..16; above 8 a non-portable cluster size that not
 * every shape can be scheduled with), threads per block (32..512, a multiple
 * of 32), the register budget of the kernel variant (lean = 0 full, 1
 * compiled for 1024 resident threads per SM, i.e. 64 registers per thread, 2
 * for three blocks of at most 256 threads per SM, 85 registers), and the
 * sweep kind `stage`:
 *   0, 1  band sweep: 1 copies each step's rows of chi0 and S into shared
 *         memory one step ahead (0: reads them from global memory where used,
 *         which frees that shared memory for more resident blocks);
 *   2, 3  shifted-plane sweep (static atmospheres in complete redistribution
 *         with linear upwind interpolation): each finished plane is stored
 *         shifted by the next step's upwind offset; freq_per_block = n_freq
 *         (at most 16) or 2, 4, 6, 10, 16; up to 1024 threads in FP32 with 2
 *         or 4 frequencies per block; lean 0, or 1 in FP32.  2 orders the
 *         planes with one cluster barrier per step, 3 with stores into other
 *         blocks that count their bytes on an mbarrier of the receiving block
 *         (a wait that runs past 2 s makes the next call that reads results
 *         return MG3D_E_CUDA).
 * The library picks a shape at creation (the shifted-plane sweep with
 * cluster barriers where it applies, at most 8 bands); this overrides it.
 * Returns MG3D_E_ARG if the shape does not fit in shared memory or the GPU
 * cannot hold one of its clusters.
 * No counterpart in the paper (launch control). */
int mg3d_set_fs_config(mg3d_handle *h, int level, int freq_per_block, int bands,
                       int threads, int lean, int stage);
int mg3d_get_fs_config(const mg3d_handle *h, int level, int *freq_per_block, int *bands,
                       int *threads, int *lean, int *stage);

/* Occupancy of a candidate shape (same arguments as mg3d_set_fs_config) on
 * this GPU without applying it: *max_clusters = clusters of the shape the GPU
 * can hold at once (0: it cannot run; a sweep launches 24 x ceil(n_freq /
 * freq_per_block) clusters, so fewer than that means several waves), and
 * *smem_bytes = its dynamic shared memory per block.  Either output may be
 * NULL.  MG3D_E_ARG for shapes mg3d_set_fs_config would reject as invalid.
 * No counterpart in the paper (launch control). */
int mg3d_get_fs_occupancy(mg3d_handle *h, int level, int freq_per_block, int bands,
                          int threads, int lean, int stage, int *max_clusters,
                          long long *smem_bytes);

/* Autotuner: times candidate sweep shapes on this GPU with the level's current
 * populations and keeps the fastest per level (level = 0: every level).
 * Multi-level handles: every band count (1-8), 12/6/4/3/2 rays per block (1
 * where none of those fits) and 128/256/512 threads that fit, and for static
 * atmospheres with the linear upwind interpolation the shifted-plane shapes
 * (1, 2 or 4 frequencies per block, 1-16 bands, 12..1 rays per block), timed
 * on the first 32 frequencies; the chunk
 * buffers are then resized for the chosen shapes (keeping a requested chunk
 * size).  Two-level handles taking the shifted-plane sweep: groupings of up
 * to 8 groups, 1-16 bands, 32-1024 threads in powers of two and the block
 * sizes that cover a band in equal passes, both register budgets in FP32 and
 * both completion schemes (stages 2 and 3) with more than one band; other
 * two-level handles (band sweep): every number of frequency groups up to 64, 1-16 bands,
 * 32-512 threads in powers of two and the block sizes that cover a band in
 * 1-4 equal passes, the three register budgets, staged or not; where the shape fits and
 * can be scheduled; one launch each,
 * then the best eight three more times.  Overwrites the partial sums (not the populations).
 * *evaluated and *seconds (nullable) report the candidates and wall time.
 * No counterpart in the paper (launch control). */
int mg3d_autotune(mg3d_handle *h, int level, int *evaluated, double *seconds);

/* Check of the FP64 exponential the sweep uses: for each x_host[i] >= 0 the
 * GPU writes out_host[2i] = the sweep's e^{-x} and out_host[2i+1] = CUDA's
 * exp(-x), so callers can bound the difference.  Allocates temporary device
 * memory; out_host holds 2n doubles.
 * A test of a building block; no counterpart in the paper. */
int mg3d_check_exp(int n, const double *x_host, double *out_host);

/* Check of the host-built line tables of a damped two-level atom (no GPU):
 * for each i, out_host[2i] = the Voigt function H(a, x_host[i]) (profile
 * times sqrt(pi)) and out_host[2i+1] = the angle-averaged redistribution
 * R_II-A(x_host[i], xp_host[i]) (R_I-A for a = 0), as the frequency table and
 * the partial-redistribution matrix use them.  a >= 0; out_host holds 2n
 * doubles.
 * A test of a building block; no counterpart in the paper. */
int mg3d_check_profiles(int n, double a, const double *x_host, const double *xp_host,
                        double *out_host);

/* Check of the rational Voigt function (no GPU): Weideman's 40-term
 * expansion of the Faddeeva function, plain arithmetic that host and device
 * code can both evaluate; R_II-A's angle integrand uses it.  For each i,
 * out_host[i] = H(a_host[i], x_host[i]) with a_host[i] > 0; relative error
 * below 5e-14 + 2e-14/a (rounding, in the cancellation of the expansion's
 * two terms as a -> 0).  MG3D_E_ARG for n < 1, null pointers or a
 * non-positive (or non-finite) a; out_host holds n doubles.
 * A test of a building block; no counterpart in the paper. */
int mg3d_check_voigt(int n, const double *a_host, const double *x_host, double *out_host);

/* Replay V-cycles from CUDA graphs (default on).  The first V-cycle of each
 * kind (first cycle / later cycles) is captured on the handle's stream and
 * later ones replay the graph; graphs are rebuilt after a change of stream or
 * sweep shapes or of the timing switch; with timing on, the graphs carry
 * the event records and each replay's sweep times are read back.
 * No counterpart in the paper (launch control). */
int mg3d_set_graphs(mg3d_handle *h, int enable);

/* Per-launch device timing of the sweep kernel (CUDA events on the handle's
 * stream) on or off, counters and their reset.
 * No counterpart in the paper (instrumentation). */
int mg3d_set_timing(mg3d_handle *h, int enable);
int mg3d_get_counters(mg3d_handle *h, mg3d_counters *out);
int mg3d_reset_counters(mg3d_handle *h);

/* Peak rates of the arithmetic the formal solution runs on, measured on the
 * current device: out_host[0] FP32 fused multiply-adds, out_host[1] ex2 and
 * out_host[2] rcp approximations (the FP32 e^-x and 1/x), out_host[3] FP64
 * fused multiply-adds, each in thread operations per second.  Each kernel
 * runs eight independent chains per thread on 8 blocks of 256 threads per SM;
 * one warm-up launch, then the fastest of `reps` (1..100) launches timed with
 * CUDA events on the legacy default stream (the call synchronises).
 * Allocates a small device buffer.  The sweep kernels are bound by these
 * pipes rather than by memory; the rates are the denominators of their
 * roofline.  Changes no clock or other device setting.
 * No counterpart in the paper (measurement aid). */
int mg3d_probe_alu_peaks(int reps, double *out_host);

/* Allocation-free formal solution.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at the moment
 * they need a formal solution -- code running under another framework's
 * memory pool that forbids foreign cudaMalloc calls, allocation-free sections
 * of a real-time pipeline, or a process whose device memory is all held by a
 * caching allocator.  It allocates nothing: the caller passes device inputs
 * and outputs, and the scratch of the sweep (partial sums per ray, upwind
 * geometry, frequency tables) lives in one fixed array in the library's
 * device image, about 26 MB, which every GPU that loads the library holds
 * until the process exits.
 *
 * It computes what mg3d_formal_solve computes on one grid, always in FP64:
 *   z_dev    [nz] node heights (device), strictly increasing;
 *   chi0_dev [nz][ny][nx] line opacity at unit profile, kappa (n_l g_u/g_l - n_u);
 *   S_dev    [nz][ny][nx] line source function n_u / (n_l g_u/g_l - n_u);
 *   bbot_dev [ny][nx] intensity entering through the bottom plane;
 *   jeff_dev, u_dev [nz][ny][nx] outputs Jeff and U = 1 - Lambda*;
 *   atom gives n_freq and x_max (Doppler profile, CRD: gamma_prd and a_damp
 *   must be 0, else MG3D_E_ARG); quad_a selects the A4 set as in
 *   mg3d_quadrature; cuda_stream orders the work (NULL: the legacy default
 *   stream).  The call returns once the work is enqueued.
 * Limits: at most MG3D_NOALLOC_MAX_NODES nodes, MG3D_NOALLOC_MAX_NZ planes and
 * MG3D_NOALLOC_MAX_FREQ frequencies; larger inputs return MG3D_E_ARG with a
 * message naming the limit.  Within them, the sweep keeps every frequency's
 * intensities of a row band in shared memory, in at most 8 bands of 200 KB:
 * about 16 (n_freq + 4) nx ceil(ny/8) bytes per band must fit (a 64 x 64
 * plane takes at most 20 frequencies); a larger plane returns MG3D_E_ARG.
 * quad_a as in mg3d_quadrature (MG3D_E_ARG unless finite and below
 * 1/sqrt(2)).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) while that device is current and writes its
 * constant table; with CUDA's lazy module loading this is also when the
 * device reserves the array, so make that first call at start-up, before the
 * caller's allocator takes the device's memory (otherwise it can fail with
 * MG3D_E_OOM) and before any stream capture.  All calls share the one array,
 * and each call rewrites all of it that it reads apart from that table:
 * calls whose work overlaps on the GPU race, so order them on one stream or
 * synchronise between them. */
#define MG3D_NOALLOC_MAX_NODES 65536
#define MG3D_NOALLOC_MAX_NZ 1024
#define MG3D_NOALLOC_MAX_FREQ 64
int mg3d_formal_solve_noalloc(int nx, int ny, int nz, double dx, double dy,
                              const double *z_dev, const mg3d_atom *atom, double quad_a,
                              const double *chi0_dev, const double *S_dev,
                              const double *bbot_dev, double *jeff_dev, double *u_dev,
                              void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MG3D_H */
