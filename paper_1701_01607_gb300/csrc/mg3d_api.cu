// C ABI and host driver: handle, grid hierarchy, MALI, FAS V-cycle and FMG.
//
// The driver follows Sec. 2.2-2.3 of Bjorgen & Leenaarts (2017):
//   V-cycle(k):  nu1 MALI sweeps (nu0 on the finest grid in the first cycle)
//                r^k = f^k - W^k_*(n^k)                     (Eq. 5, extra FS)
//                n^{k-1} = R n^k,  n_before = n^{k-1}
//                f^{k-1} = R r^k + W^{k-1}_*(R n^k)         (Eq. 9, extra FS)
//                k-1 == 1 ? nu3 MALI sweeps : V-cycle(k-1)
//                e = (n_after - n_before)/n_before           (Eq. 10)
//                n^k <- n^k (1 + I e), <= 0 -> 0.1 n^k       (Eq. 11, Sec. 4.10)
//                nu2 MALI sweeps
//   FMG:         nu_fmg sweeps on grid 1, then for k = 2..l: n^k = I n^{k-1}
//                and one V-cycle on grid k (k < l); V-cycles on grid l until
//                the change over a cycle falls below the tolerance.
// Every step runs in the library's kernels on the handle's stream; the host
// only sequences launches and reads one scalar at convergence checks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mg3d.h"
#include "profiles.h"
#include "mg3d_internal.h"
#include "sc_step.cuh"

using namespace mg3d;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

// On failure the runtime's last-error state is cleared as well, so that a
// later launch check does not report this error again.
#define MG_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            (void)cudaGetLastError();                                                  \
            return fail(MG3D_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                              \
    } while (0)

#define MG_TRY(call)             \
    do {                                 \
        int rc_ = (call);                \
        if (rc_ != MG3D_OK) return rc_;  \
    } while (0)

struct Level {
    int nx = 0, ny = 0, nz = 0;
    long nplane = 0, nvox = 0;
    double dx = 0, dy = 0;
    std::vector<double> z;
    double *T = nullptr, *n_tot = nullptr, *c_ul = nullptr, *c_lu = nullptr;
    double *tz = nullptr;        // [nz] prolongation weight of the upper coarse plane
    double *zf = nullptr;        // [nz] heights (Hermite prolongation onto this grid)
    double *n = nullptr;         // [2][nvox]
    double *f = nullptr;         // [2][nvox]
    bool f_default = true;       // f = (n_tot, 0)
    double *n_before = nullptr;  // [2][nvox]
    double *r = nullptr;         // [2][nvox] residual / scratch
    void *chi0 = nullptr, *S = nullptr, *bbot = nullptr;
    void *dchi0 = nullptr, *dS = nullptr;  // x-slopes of chi0, S (Hermite upwind interpolation)
    double *vel = nullptr;       // [3][nvox] velocity in Doppler widths (moving atmosphere)
    void *uproj = nullptr, *vnorm = nullptr;  // [kRays][nvox] projected velocity, 1/sum w phi
                                              // (multi-level: vnorm [nlines][kRays][nvox])
    void *dinv = nullptr;        // multi-level, moving: 1/d per node [nvox]
    // partial redistribution (two-level): the lagged mean intensity, rho and
    // rho S [nf][nvox] (natural order); per-ray slots of the new mean
    // intensity [kRays][nf][nvox]
    void *jnu = nullptr, *jnu_new = nullptr, *rho = nullptr, *rhoS = nullptr;
    StepGeom *geom = nullptr;    // [kRays][nz]
    void *psteps = nullptr;      // [kRays][nz] PlaneStep<T> of the shifted-plane sweep
    SweepShape shape{};
    // formal solutions in the precision other than the handle's (built on the
    // first request, two-level static CRD handles): chi0, S, the bottom
    // intensity, the plane-sweep step table, and the shape
    void *o_chi0 = nullptr, *o_S = nullptr, *o_bbot = nullptr, *o_psteps = nullptr;
    SweepShape o_shape{};
    // multi-level atom only
    double *chi_c = nullptr;     // [nvox] background opacity
    double *cmat = nullptr;      // [N][N][nvox] collisional rates
    double *saha = nullptr;      // [N][nvox] LTE ratios to the continuum
    void *mchi = nullptr, *mS = nullptr, *msc = nullptr, *moc = nullptr;  // [nf][nvox]
    void *mdchi = nullptr, *mdS = nullptr;  // [nf][nvox] x-slopes of mchi, mS (Hermite)
    void *mib = nullptr;         // [nf][nplane] bottom intensity
    double *sigma_c = nullptr;   // background coherent scattering [nvox] (FP64)
    void *jbg = nullptr;         // background radiation field [nf][nvox] (FS precision)
    double *prd_c = nullptr;     // partial redistribution of multi-level lines: scaling
    double *prd_rho = nullptr;   // of R and emission-profile ratio [n_prd_freq][nvox],
    double *prd_oc = nullptr;    // and 1 - rho chi_t/chi in FP64 [n_prd_freq][nvox]
    int ml_bands = 0, ml_rows = 0, ml_threads = 0;
    int ml_rpb = 12;             // rays of a hemisphere per block of the multi-level sweep
    int ml_plane = 0;            // 1: the shifted-plane form (ml_plane.cuh), ml_nf
    int ml_nf = 1;               //    frequencies per block
};

struct TimedLaunch {
    cudaEvent_t a, b;
    int level;
};

}  // namespace

// Index of the sweep status word in mg3d_handle::scal (after the eight
// scalars that reset_scalars clears).
constexpr int kScalStatus = 8;

struct mg3d_handle {
    int L = 0;
    int prec = 0;
    int kind = 0;                // 0: two-level atom, 1: multi-level atom
    int N = 2;                   // levels of the atom
    // multi-level atom
    double theta_ref = 0, t_ref = 0;
    int nfreq_ml = 0, ntrans = 0;
    std::vector<FreqInfo> fi;
    std::vector<TransInfo> ti;
    FreqInfo *d_fi = nullptr;
    TransInfo *d_ti = nullptr;
    // multi-level formal solution, in chunks of ml_chunk frequencies:
    // angle sums of the chunk [2 hemispheres][ml_chunk][nvox] and the
    // radiative sums per transition [ntrans][kAccTerms][finest nvox] (FP64)
    int ml_chunk = 0;
    int ml_chunk_req = 0;        // chunk asked for (0: automatic), kept across retuning
    bool scatter = false;        // background coherent scattering present
    // partial redistribution of multi-level lines: the PRD lines, the
    // |x|-sorted frequency order and its groups, and each frequency's row of
    // the rho arrays (-1: not a PRD line frequency)
    bool ml_prd = false;
    int n_prd = 0, n_prd_freq = 0;
    PrdLine *d_prd = nullptr;
    int *d_prd_ord = nullptr, *d_prd_grp = nullptr, *d_prd_index = nullptr;
    std::vector<int> prd_index;  // host copy of d_prd_index
    VoigtTable *d_voigt = nullptr;   // Voigt coefficients when a multi-level line is damped
    int fmg_next = 1;            // the FMG stage mg3d_fmg_stage may run next (1 restarts)
    int top = 0;                 // grid being solved (0: the finest); only its formal
                                 // solutions update its background field
    bool force_bg = false;       // the current formal solution is a Lambda-iteration
    void *ml_jm = nullptr;       // mean intensity per slot [slots][chunk][nvox] (scatter)
    int ml_slots = 2;            // most ray-group slots of any level (2 x 12 / ml_rpb)
    void *ml_jx = nullptr, *ml_ux = nullptr;
    double *ml_acc = nullptr;
    mg3d_atom atom{};
    mg3d_params params{};
    double mu[kRays][3];
    double wray[kRays];
    unsigned up_mask = 0;
    Level lev[MG3D_MAX_GRIDS + 1];
    std::vector<double> phi, wphi;
    // frequency tables of the sweep, [order][phi, 1/phi, w phi / 24][n_freq]
    // in the formal-solution precision (see freq_tables)
    void *d_ftab = nullptr;
    // slot tables of the shifted-plane sweep, one per slot count kPlaneNp[i]:
    // [ceil(n_freq / (2 np))][np] PlaneSlot<T>
    void *d_pslot[kPlaneNpCount] = {};
    // the other precision's slot tables and partial sums (see Level::o_chi0)
    int o_prec = -1;
    void *o_pslot[kPlaneNpCount] = {};
    void *o_pj = nullptr, *o_pu = nullptr;
    size_t partial_elems_o = 0;
    void *d_vtab = nullptr;      // moving atmospheres: [nf] offsets x, [nf] weights w
    int *d_vline = nullptr;      // multi-level, moving: line index of each frequency or -1
    bool prd = false;            // two-level partial redistribution
    double *d_kmat = nullptr;    // [nf][nf] w_f' R(f', f) / phi_f
    double *d_wphin = nullptr;   // [nf] normalised w phi, natural order
    int *d_fidx = nullptr;       // [2][nf] natural frequency of each table position
    bool moving = false;         // the atmosphere has a velocity field
    double *d_exp_tab = nullptr;         // [64] table of the FP64 exp in the sweep
    double exp_l1 = 0, exp_l2 = 0;
    void *pj = nullptr, *pu = nullptr;
    size_t partial_elems = 0;
    unsigned long long *scal = nullptr;  // [0] C bits, [1] negative after a sweep,
                                         // [2] non-finite, [3] reset by the 10 % rule,
                                         // [4] cycle C bits, [6] cycle non-finite;
                                         // [kScalStatus] sweep status bits, kept
                                         // until read
    double *scratch = nullptr;           // [4][finest nvox]
    cudaStream_t own_stream = nullptr, stream = nullptr;
    // counters
    long long launches = 0, fs_launches = 0;
    double fs_units = 0;
    long long level_launches[MG3D_MAX_GRIDS + 1] = {};
    double level_units[MG3D_MAX_GRIDS + 1] = {};
    bool timing = false;
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    // CUDA graphs of the V-cycle (index: first cycle or not)
    bool use_graphs = true;
    cudaGraphExec_t cycle_exec[2] = {nullptr, nullptr};
    cudaStream_t graph_stream = nullptr;     // stream the graphs were captured on
    std::vector<TimedLaunch> cycle_timed[2]; // event pairs recorded by each graph
    double acc_ms[MG3D_MAX_GRIDS + 1] = {};  // sweep time read back from graph replays
    long long acc_n[MG3D_MAX_GRIDS + 1] = {};
    struct CycleDelta {
        long long launches = 0, fs_launches = 0;
        double fs_units = 0;
        long long level_launches[MG3D_MAX_GRIDS + 1] = {};
        double level_units[MG3D_MAX_GRIDS + 1] = {};
        int sweeps[MG3D_MAX_GRIDS + 1] = {};
        int fss[MG3D_MAX_GRIDS + 1] = {};
    } cycle_delta[2];
    // per-solve statistics
    int sweeps[MG3D_MAX_GRIDS + 1] = {};
    int fss[MG3D_MAX_GRIDS + 1] = {};
    long long negatives = 0;
};

namespace {

size_t elem_size(int prec) { return prec == MG3D_PREC_F64 ? sizeof(double) : sizeof(float); }

// A4 set (Sec. 3): per octant the permutations of (a, a, b), weights 1/24;
// rays 0-11 point up.
void build_quadrature(mg3d_handle *h, double a) {
    if (!(a > 0.0)) a = std::sqrt((4.0 - std::sqrt(6.4)) / 12.0);
    const double b = std::sqrt(1.0 - 2.0 * a * a);
    const double perm[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
    int r = 0;
    for (int oz = 0; oz < 2; ++oz)
        for (int oy = 0; oy < 2; ++oy)
            for (int ox = 0; ox < 2; ++ox)
                for (int p = 0; p < 3; ++p) {
                    h->mu[r][0] = (ox ? -1.0 : 1.0) * perm[p][0];
                    h->mu[r][1] = (oy ? -1.0 : 1.0) * perm[p][1];
                    h->mu[r][2] = (oz ? -1.0 : 1.0) * perm[p][2];
                    h->wray[r] = 1.0 / kRays;
                    if (h->mu[r][2] > 0) h->up_mask |= 1u << r;
                    ++r;
                }
}

// Doppler profile phi(x) = exp(-x^2)/sqrt(pi) on equidistant x in
// [-x_max, x_max], trapezoid weights, renormalised to sum(w phi) = 1.
void build_frequencies(mg3d_handle *h) {
    const int nf = h->atom.n_freq;
    h->phi.assign(nf, 0.0);
    h->wphi.assign(nf, 0.0);
    double sum = 0.0;
    for (int i = 0; i < nf; ++i) {
        // x_i = -x_{nf-1-i} exactly, so mirror frequencies get equal phi
        double x = nf == 1 ? 0.0 : h->atom.x_max * (2 * i - (nf - 1)) / (nf - 1);
        double w = nf == 1 ? 1.0 : 2.0 * h->atom.x_max / (nf - 1);
        if (nf > 1 && (i == 0 || i == nf - 1)) w *= 0.5;
        // Doppler, or Voigt with damping (even in x: mirror offsets stay equal)
        h->phi[i] = voigt_H(h->atom.a_damp, x) / std::sqrt(M_PI);
        h->wphi[i] = w * h->phi[i];
        sum += h->wphi[i];
    }
    for (int i = 0; i < nf; ++i) h->wphi[i] /= sum;
}

// Frequency index i at table position j.  Order 0 pairs the mirror
// frequencies with the centre last (x_0, x_{nf-1}, x_1, x_{nf-2}, ..., centre),
// order 1 puts the centre (odd nf) first and then the pairs.
int mirror_order(int nf, int order, int j) {
    if (order == 1 && nf % 2 == 1) {
        if (j == 0) return nf / 2;
        --j;
    }
    return j % 2 == 0 ? j / 2 : nf - 1 - j / 2;
}

// Frequency tables for a sweep whose blocks take ng frequencies each.  Blocks
// of an even number of frequencies take order 0 (each group whole pairs, the
// centre alone at the end); blocks of an odd number take order 1 (the first
// group is the centre and pairs, and for two groups the second is pairs
// only), so that mirror pairs share a block, and so their weights, wherever
// the group size allows.
template <typename T>
void freq_tables(const mg3d_handle *h, int ng, const T **phi, const T **inv_phi,
                 const T **wphi) {
    const int nf = h->atom.n_freq;
    const T *base = static_cast<const T *>(h->d_ftab) + (ng % 2 == 1 ? 3 * (size_t)nf : 0);
    *phi = base;
    *inv_phi = base + nf;
    *wphi = base + 2 * (size_t)nf;
}

// Launch arguments of the sweep of level L with shape s.
template <typename T>
SweepArgs<T> sweep_args(const mg3d_handle *h, const Level &L, const SweepShape &s) {
    const T *phi, *inv_phi, *wphi;
    freq_tables<T>(h, s.ng, &phi, &inv_phi, &wphi);
    return SweepArgs<T>{L.nx, L.ny, L.nz, h->atom.n_freq, s.ng, s.ngroups, s.rows,
                        h->up_mask, (const T *)L.chi0, (const T *)L.S, (const T *)L.bbot,
                        L.geom, phi, inv_phi, wphi, (T *)h->pj, (T *)h->pu, h->d_exp_tab,
                        h->exp_l1, h->exp_l2, (const T *)L.dchi0, (const T *)L.dS,
                        (const T *)L.uproj, (const T *)L.vnorm,
                        h->moving ? (const T *)h->d_vtab : nullptr,
                        h->moving ? (const T *)h->d_vtab + h->atom.n_freq : nullptr,
                        (const T *)L.rhoS, (const T *)L.rho,
                        h->prd ? h->d_fidx + (s.ng % 2 == 1 ? h->atom.n_freq : 0) : nullptr,
                        (T *)L.jnu_new};
}

// Upwind crossing of every (ray, sweep step): for step t the plane is
// k = t (up) or nz-1-t (down), the upwind plane kp = k-1 or k+1, the path
// s = |z_k - z_kp| / |mu_z|, and the crossing lies at x - s mu_x/dx cells.
void build_geometry(const mg3d_handle *h, const Level &L, std::vector<StepGeom> &g) {
    g.assign((size_t)kRays * L.nz, StepGeom{0, 0, 0.0, 0.0, 0.0});
    for (int r = 0; r < kRays; ++r) {
        const bool up = h->mu[r][2] > 0;
        for (int t = 1; t < L.nz; ++t) {
            const int k = up ? t : L.nz - 1 - t;
            const int kp = up ? k - 1 : k + 1;
            const double s = std::fabs(L.z[k] - L.z[kp]) / std::fabs(h->mu[r][2]);
            const double sx = -s * h->mu[r][0] / L.dx;
            const double sy = -s * h->mu[r][1] / L.dy;
            const double fx = std::floor(sx), fy = std::floor(sy);
            long ix = (long)fx % L.nx, iy = (long)fy % L.ny;
            if (ix < 0) ix += L.nx;
            if (iy < 0) iy += L.ny;
            StepGeom &e = g[(size_t)r * L.nz + t];
            e.ix0 = (int)ix;
            e.iy0 = (int)iy;
            e.tx = sx - fx;
            e.ty = sy - fy;
            e.s = s;
        }
    }
}

// Per-step constants of the shifted-plane sweep from the upwind geometry:
// the bilinear weights and half path of step t, and the corner offsets of
// step t+1 as the shift of the plane written at step t.
template <typename T>
std::vector<PlaneStep<T>> plane_steps(const Level &L, const std::vector<StepGeom> &g) {
    std::vector<PlaneStep<T>> out((size_t)kRays * L.nz);
    for (int r = 0; r < kRays; ++r)
        for (int t = 0; t < L.nz; ++t) {
            const StepGeom &e = g[(size_t)r * L.nz + t];
            PlaneStep<T> &p = out[(size_t)r * L.nz + t];
            p.w00 = (T)((1.0 - e.tx) * (1.0 - e.ty));
            p.w10 = (T)(e.tx * (1.0 - e.ty));
            p.w01 = (T)((1.0 - e.tx) * e.ty);
            p.w11 = (T)(e.tx * e.ty);
            p.half_s = (T)(0.5 * e.s);
            const bool last = t + 1 >= L.nz;
            p.sx = last ? 0 : g[(size_t)r * L.nz + t + 1].ix0;
            p.sy = last ? 0 : g[(size_t)r * L.nz + t + 1].iy0;
        }
    return out;
}

int plane_np_index(int np) {
    for (int i = 0; i < kPlaneNpCount; ++i)
        if (kPlaneNp[i] == np) return i;
    return -1;
}

// Launch arguments of the shifted-plane sweep of level L with shape s.
template <typename T>
PlaneArgs<T> plane_args(const mg3d_handle *h, const Level &L, const SweepShape &s,
                        bool other = false) {
    const int nf = h->atom.n_freq;
    const int last = nf - (s.ngroups - 1) * 2 * s.np;   // frequencies of the last group
    PlaneArgs<T> a{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.rows = s.rows;
    a.bands = s.bands;
    a.ngroups = s.ngroups;
    a.nslot_last = (last + 1) / 2;
    a.up_mask = h->up_mask;
    a.rmagic = band_magic(s.rows);
    a.xmagic = band_magic(L.nx);
    a.chi0 = (const T *)(other ? L.o_chi0 : L.chi0);
    a.S = (const T *)(other ? L.o_S : L.S);
    a.bbot = (const T *)(other ? L.o_bbot : L.bbot);
    a.steps = (const PlaneStep<T> *)(other ? L.o_psteps : L.psteps);
    a.slots = (const PlaneSlot<T> *)(other ? h->o_pslot : h->d_pslot)[plane_np_index(s.np)];
    a.pj = (T *)(other ? h->o_pj : h->pj);
    a.pu = (T *)(other ? h->o_pu : h->pu);
    a.exp_tab = h->d_exp_tab;
    a.exp_l1 = h->exp_l1;
    a.exp_l2 = h->exp_l2;
    a.status = reinterpret_cast<unsigned *>(h->scal + kScalStatus);
    return a;
}

int dev_alloc(void **p, size_t bytes);

// Slot tables of the shifted-plane sweep for every supported slot count:
// group g takes the table positions [2 np g, 2 np (g + 1)) of mirror order 0
// (x_0, x_{nf-1}, x_1, x_{nf-2}, ..., centre last), slot p of the group the
// positions 2p and 2p + 1, so mirror pairs share a slot.
template <typename T>
int build_plane_slots(mg3d_handle *h, void **out) {
    const int nf = h->atom.n_freq;
    for (int i = 0; i < kPlaneNpCount; ++i) {
        const int np = kPlaneNp[i];
        const int ngroups = (nf + 2 * np - 1) / (2 * np);
        std::vector<PlaneSlot<T>> tab((size_t)ngroups * np);
        for (int g = 0; g < ngroups; ++g)
            for (int p = 0; p < np; ++p) {
                PlaneSlot<T> &e = tab[(size_t)g * np + p];
                e = PlaneSlot<T>{};
                const int ja = 2 * np * g + 2 * p, jb = ja + 1;
                if (ja >= nf) continue;   // inactive slot of the last group
                const int ia = mirror_order(nf, 0, ja);
                e.phi_a = (T)h->phi[ia];
                e.iphi_a = (T)(1.0 / h->phi[ia]);
                e.wphi_a = (T)(h->wphi[ia] / kRays);
                e.wu_a = e.wphi_a;
                if (jb < nf) {
                    const int ib = mirror_order(nf, 0, jb);
                    e.flags = plane::kHasB;
                    e.phi_b = (T)h->phi[ib];
                    e.iphi_b = (T)(1.0 / h->phi[ib]);
                    e.wphi_b = (T)(h->wphi[ib] / kRays);
                    e.wu_b = e.wphi_b;
                    if (h->phi[ib] == h->phi[ia]) {
                        e.flags |= plane::kShared;
                        e.wu_a = (T)((h->wphi[ia] + h->wphi[ib]) / kRays);
                    }
                }
            }
        MG_TRY(dev_alloc(&out[i], tab.size() * sizeof(PlaneSlot<T>)));
        MG_CUDA(cudaMemcpy(out[i], tab.data(), tab.size() * sizeof(PlaneSlot<T>),
                           cudaMemcpyHostToDevice));
    }
    return MG3D_OK;
}

// Threads per block for a band of `band` nodes: as few passes of at most
// kMaxSweepThreads threads as possible, split evenly, rounded to warps.
int threads_for_band(int band) {
    const int passes = (band + kMaxSweepThreads - 1) / kMaxSweepThreads;
    int th = (band + passes - 1) / passes;
    th = ((th + 31) / 32) * 32;
    return th < 32 ? 32 : (th > kMaxSweepThreads ? kMaxSweepThreads : th);
}

// Default sweep shape before any autotuning: three frequencies per block and
// the number of bands that brings the grid closest to two blocks per SM (the
// shapes measured fastest on the 64x64 planes of the bench workload, in both
// precisions, were of this kind); mg3d_autotune replaces it by measurement.
// Slot count of the shifted-plane sweep that takes all n_freq frequencies in
// one group (0 when more than 16 frequencies need several groups).
int plane_np_for(int nfreq) {
    for (int i = 0; i < kPlaneNpCount; ++i)
        if (2 * kPlaneNp[i] >= nfreq) return kPlaneNp[i];
    return 0;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
    }
    return n;
}

// How many clusters of shape s the GPU holds at once (plain launches: blocks).
int shape_capacity(int prec, const SweepShape &s, int nx) {
    int n = 0;
    const cudaError_t e = s.plane ? plane_active_clusters(prec, s, nx, &n)
                                  : sweep_active_clusters(prec, s, nx, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return s.bands == 1 ? n * sm_count() : n;
}

// Default shifted-plane shape: the largest slot count that takes all
// frequencies in one group (or groups of 16 beyond 16 frequencies), and the
// most bands (up to 8) whose 24 x groups clusters the GPU holds in one wave.
// Planes too large for that take fewer slots per group and up to 16 bands,
// the first shape that fits.  mg3d_autotune replaces it by measurement.
SweepShape choose_plane_shape(int prec, int nx, int ny, int nfreq) {
    int np0 = plane_np_for(nfreq);
    if (np0 == 0) np0 = kPlaneNp[kPlaneNpCount - 1];
    SweepShape fallback{};
    for (int i = kPlaneNpCount - 1; i >= 0; --i) {
        const int np = kPlaneNp[i];
        if (np > np0) continue;
        const int ngroups = (nfreq + 2 * np - 1) / (2 * np);
        SweepShape best{};
        for (int bands = 1; bands <= kMaxBands && bands <= ny; ++bands) {
            const int rows = (ny + bands - 1) / bands;
            if ((long)(bands - 1) * rows >= ny) continue;
            if (plane_smem_bytes(prec, np, rows, nx) > kMaxPlaneSmem) continue;
            // one thread per node up to 512 (1024 for FP32 with one or two slots)
            const int cap = prec == MG3D_PREC_F32 && np <= 2 ? kPlaneMaxThreads : 512;
            const int th = std::max(32, std::min(cap, ((rows * nx + 31) / 32) * 32));
            if ((long)rows * nx > (long)plane_max_pass(np, prec == MG3D_PREC_F64) * th) continue;
            SweepShape s{2 * np, ngroups, bands, rows, th};
            s.stage = 0;
            s.plane = 1;
            s.np = np;
            const int held = shape_capacity(prec, s, nx);
            if (held < 1) continue;
            if (fallback.ng == 0) fallback = s;
            if (bands <= kPortableBands && held >= kRays * ngroups) best = s;
        }
        if (best.ng) return best;
    }
    return fallback;
}

// Grids the shifted-plane sweep's 32-bit node indices cover.
bool plane_grid_ok(int nx, int ny, int nz) {
    return (long)nx * ny * nx < (1L << 32) && (long)nx * ny * nz < (1L << 31);
}

SweepShape choose_shape(int prec, int nx, int ny, int nz, int nfreq, int herm, int vel,
                        int prd) {
    if (!herm && !vel && !prd && plane_grid_ok(nx, ny, nz)) {
        const SweepShape s = choose_plane_shape(prec, nx, ny, nfreq);
        if (s.ng) return s;
    }
    const int ng = nfreq < 3 ? nfreq : 3;
    const int ngroups = (nfreq + ng - 1) / ng;
    SweepShape best{};
    auto with_mode = [&](SweepShape s) {
        s.herm = herm;
        s.vel = vel;
        s.prd = prd;
        s.stage = herm || vel || prd ? 0 : 1;
        return s;
    };
    long best_gap = 1L << 40;
    for (int bands = 1; bands <= kPortableBands && bands <= ny; ++bands) {
        const int rows = (ny + bands - 1) / bands;
        if ((long)(bands - 1) * rows >= ny) continue;
        const SweepShape s = with_mode(SweepShape{ng, ngroups, bands, rows, 256});
        if (sweep_smem_bytes(prec, s, nx) > kMaxSweepSmem) continue;
        const long blocks = (long)kRays * ngroups * bands;
        const long gap = blocks > 304 ? blocks - 304 : 304 - blocks;
        if (gap < best_gap) {
            best_gap = gap;
            best = s;
        }
    }
    if (best.ng == 0) {
        // planes too large for three frequencies: one frequency, most bands
        for (int bands = kPortableBands; bands >= 1; --bands) {
            if (bands > ny) continue;
            const int rows = (ny + bands - 1) / bands;
            if ((long)(bands - 1) * rows >= ny) continue;
            const SweepShape s = with_mode(SweepShape{1, nfreq, bands, rows, 256});
            if (sweep_smem_bytes(prec, s, nx) <= kMaxSweepSmem) {
                best = s;
                break;
            }
        }
    }
    int th = threads_for_band(best.rows * nx);
    best.threads = th > 256 ? 256 : th;
    return best;
}

int dev_alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(MG3D_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return MG3D_OK;
}

template <typename P>
int dalloc(P **p, size_t count) {
    return dev_alloc((void **)p, count * sizeof(P));
}

void free_level(Level &L) {
    void *ptrs[] = {L.T,     L.n_tot, L.c_ul, L.c_lu, L.tz,   L.zf,   L.n,    L.f,   L.n_before,
                    L.r,     L.chi0,  L.S,    L.bbot, L.geom, L.chi_c, L.cmat, L.saha,
                    L.mchi,  L.mS,    L.msc,  L.moc,  L.mib,  L.sigma_c, L.jbg,
                    L.dchi0, L.dS,   L.mdchi, L.mdS,  L.vel,  L.uproj, L.vnorm, L.dinv,
                    L.jnu,   L.jnu_new, L.rho, L.rhoS, L.psteps, L.o_chi0, L.o_S, L.o_bbot,
                    L.o_psteps, L.prd_c, L.prd_rho, L.prd_oc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    L = Level{};
}

int check_level(const mg3d_handle *h, int level) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (level < 1 || level > h->L) return fail(MG3D_E_ARG, "level out of range");
    return MG3D_OK;
}

int launched(mg3d_handle *h, cudaError_t e, const char *what) {
    ++h->launches;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(MG3D_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return MG3D_OK;
}

// Record an event on the handle's stream; inside a stream capture it becomes
// an event-record node of the graph, so that replays can be timed.
cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(st, &cs);
    if (r != cudaSuccess) return r;
    if (cs == cudaStreamCaptureStatusActive)
        return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    return cudaEventRecord(e, st);
}

cudaEvent_t pool_event(mg3d_handle *h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// ------------------------------------------------------------- operations

// Multi-level formal solution on level k: per-frequency angle sums per
// hemisphere into ml_jx/ml_ux.
// The multi-level shifted-plane sweep of level L over the chunk's nc
// frequencies (opacity already formed; ib: the chunk's bottom intensities).
cudaError_t launch_ml_level_plane(const mg3d_handle *h, const Level &L, int nc, const void *ib,
                                  int bands, int rpb, int nf, int threads) {
    const int rows = (L.ny + bands - 1) / bands;
    if (h->prec == MG3D_PREC_F64) {
        MlPlaneArgs<double> a{L.nx, L.ny, L.nz, nc, rows, bands, rpb, band_magic(rows),
                              band_magic(L.nx), (const double *)L.mchi, (const double *)L.mS,
                              (const double *)L.msc, (const double *)L.moc, (const double *)ib,
                              (const PlaneStep<double> *)L.psteps, (double *)h->ml_jx,
                              (double *)h->ml_ux, (double *)h->ml_jm, h->d_exp_tab, h->exp_l1,
                              h->exp_l2};
        return launch_ml_plane_f64(a, nf, threads, h->stream);
    }
    MlPlaneArgs<float> a{L.nx, L.ny, L.nz, nc, rows, bands, rpb, band_magic(rows),
                         band_magic(L.nx), (const float *)L.mchi, (const float *)L.mS,
                         (const float *)L.msc, (const float *)L.moc, (const float *)ib,
                         (const PlaneStep<float> *)L.psteps, (float *)h->ml_jx,
                         (float *)h->ml_ux, (float *)h->ml_jm, h->d_exp_tab, h->exp_l1,
                         h->exp_l2};
    return launch_ml_plane_f32(a, nf, threads, h->stream);
}

// Opacity and sweep of the chunk of frequencies f0 .. f0+nc-1 on level k:
// per-frequency angle sums of both hemispheres into ml_jx/ml_ux.
int ml_chunk_fs(mg3d_handle *h, int k, int f0, int nc) {
    Level &L = h->lev[k];
    MlOpacityArgs oa{L.nvox, nc, h->N, h->prec, h->d_fi, h->theta_ref, h->t_ref,
                     L.n, L.T, L.chi_c, L.saha, L.mchi, L.mS, L.msc, L.moc, f0,
                     h->d_exp_tab, h->exp_l1, h->exp_l2,
                     h->scatter ? L.sigma_c : nullptr, h->scatter ? L.jbg : nullptr,
                     h->moving ? 1 : 0, h->ml_prd ? h->d_prd_index : nullptr,
                     h->ml_prd ? L.prd_rho : nullptr, h->d_voigt};
    MG_TRY(launched(h, launch_ml_opacity(oa, h->stream), "multi-level opacity"));
    if (h->params.sc_interp)
        MG_TRY(launched(h, launch_xslopes(h->prec, L.nx, (long)nc * L.nvox, L.mchi, L.mS, L.mdchi,
                                          L.mdS, h->stream),
                        "x-slopes"));
    TimedLaunch tl{nullptr, nullptr, k};
    if (h->timing) {
        tl.a = pool_event(h);
        tl.b = pool_event(h);
        MG_CUDA(record_event(tl.a, h->stream));
    }
    const size_t es = elem_size(h->prec);
    const void *ib = static_cast<const unsigned char *>(L.mib) + (size_t)f0 * L.nplane * es;
    cudaError_t e;
    if (L.ml_plane) {
        e = launch_ml_level_plane(h, L, nc, ib, L.ml_bands, L.ml_rpb, L.ml_nf, L.ml_threads);
    } else if (h->prec == MG3D_PREC_F64) {
        MlSweepArgs<double> a{L.nx, L.ny, L.nz, nc, L.ml_rows,
                              (const double *)L.mchi, (const double *)L.mS,
                              (const double *)L.msc, (const double *)L.moc,
                              (const double *)ib, L.geom, h->d_exp_tab, h->exp_l1, h->exp_l2,
                              (double *)h->ml_jx, (double *)h->ml_ux, L.ml_rpb,
                              (double *)h->ml_jm, (const double *)L.mdchi, (const double *)L.mdS,
                              h->params.sc_interp, h->moving ? 1 : 0, f0,
                              (const double *)h->d_vtab, (const double *)h->d_vtab + h->nfreq_ml,
                              h->d_vline, (const double *)L.vnorm, (const double *)L.uproj,
                              (const double *)L.dinv};
        e = launch_ml_sweep_f64(a, L.ml_bands, L.ml_threads, h->stream);
    } else {
        MlSweepArgs<float> a{L.nx, L.ny, L.nz, nc, L.ml_rows,
                             (const float *)L.mchi, (const float *)L.mS,
                             (const float *)L.msc, (const float *)L.moc,
                             (const float *)ib, L.geom, h->d_exp_tab, h->exp_l1, h->exp_l2,
                             (float *)h->ml_jx, (float *)h->ml_ux, L.ml_rpb,
                             (float *)h->ml_jm, (const float *)L.mdchi, (const float *)L.mdS,
                             h->params.sc_interp, h->moving ? 1 : 0, f0,
                             (const float *)h->d_vtab, (const float *)h->d_vtab + h->nfreq_ml,
                             h->d_vline, (const float *)L.vnorm, (const float *)L.uproj,
                             (const float *)L.dinv};
        e = launch_ml_sweep_f32(a, L.ml_bands, L.ml_threads, h->stream);
    }
    MG_TRY(launched(h, e, "multi-level sweep"));
    if (h->timing) {
        MG_CUDA(record_event(tl.b, h->stream));
        h->timed.push_back(tl);
    }
    return MG3D_OK;
}

// Whether a formal solution of grid k replaces the grid's background field
// by its mean intensity (Sec. 4.8): always on the grid being solved (the
// finest of a V-cycle, the current grid of an FMG stage or of MALI); on a
// coarser grid only in the Lambda-iteration that starts it, so that the
// coarse operator stays the same from the tau-correction of Eq. 9 to the
// correction of Eq. 10.
bool updates_background(const mg3d_handle *h, int k) {
    return (h->scatter || h->prd || h->ml_prd) && (h->force_bg || k == (h->top ? h->top : h->L));
}

// Multi-level handles with a lagged per-frequency field (jbg): background
// scattering reads it in its source term, partial redistribution forms its
// emission-profile ratios from it.
bool ml_lagged(const mg3d_handle *h) { return h->kind == 1 && (h->scatter || h->ml_prd); }

// Partial redistribution before a multi-level formal solution of grid k:
// rho of every PRD line frequency from the grid's lagged field.
int ml_prd_prepare(mg3d_handle *h, int k) {
    if (!h->ml_prd) return MG3D_OK;
    Level &L = h->lev[k];
    MlPrdArgs a{L.nvox, h->N, h->ntrans, h->n_prd, h->d_fi, h->d_ti, h->d_prd, h->d_prd_ord,
                h->d_prd_grp, h->theta_ref, h->t_ref, L.n, L.T, L.cmat, L.saha, L.jbg, h->prec,
                L.prd_c, L.prd_rho, h->d_exp_tab, h->exp_l1, h->exp_l2, L.chi_c, L.sigma_c,
                L.prd_oc};
    return launched(h, launch_ml_prd_rho(a, h->stream), "partial redistribution ratios");
}

int formal_solution(mg3d_handle *h, int k);

// One Lambda-iteration of the lagged field of grid k (background field, or
// the mean intensity of partial redistribution): a formal solution with the
// populations held whose mean intensity becomes the field.
int lambda_iteration(mg3d_handle *h, int k) {
    h->force_bg = true;
    const int rc = formal_solution(h, k);
    h->force_bg = false;
    return rc;
}

// Radiative sums of level k from the chunk's angle sums (zero_rad: J = 0,
// U = 1 for all frequencies, no formal solution).
int ml_accumulate(mg3d_handle *h, int k, int f0, int nc, bool zero_rad) {
    Level &L = h->lev[k];
    const bool bg = !zero_rad && updates_background(h, k);   // the mean intensity becomes the field
    MlAccumArgs a{L.nvox, f0, nc, h->ntrans, h->prec, h->d_fi, h->d_ti, h->theta_ref,
                  h->t_ref, L.T, h->ml_jx, h->ml_ux, 2 * (12 / L.ml_rpb), zero_rad ? 1 : 0,
                  h->ml_acc, h->d_exp_tab, h->exp_l1, h->exp_l2, bg ? h->ml_jm : nullptr,
                  bg ? L.jbg : nullptr, h->moving ? 1 : 0,
                  h->ml_prd ? h->d_prd_index : nullptr, h->ml_prd ? L.prd_oc : nullptr,
                  h->d_voigt};
    return launched(h, launch_ml_accum(a, h->stream), "radiative sums");
}

int ml_clear_acc(mg3d_handle *h, int k) {
    MG_CUDA(cudaMemsetAsync(h->ml_acc, 0,
                            (size_t)h->ntrans * kAccTerms * h->lev[k].nvox * sizeof(double),
                            h->stream));
    return MG3D_OK;
}

// Formal solution of level k, chunk by chunk, reduced to the radiative sums
// the rate equations use.
int ml_formal_solution(mg3d_handle *h, int k) {
    Level &L = h->lev[k];
    MG_TRY(ml_prd_prepare(h, k));
    MG_TRY(ml_clear_acc(h, k));
    for (int f0 = 0; f0 < h->nfreq_ml; f0 += h->ml_chunk) {
        const int nc = std::min(h->ml_chunk, h->nfreq_ml - f0);
        MG_TRY(ml_chunk_fs(h, k, f0, nc));
        MG_TRY(ml_accumulate(h, k, f0, nc, false));
    }
    const double units = (double)L.nvox * kRays * h->nfreq_ml;
    ++h->fs_launches;
    h->fs_units += units;
    ++h->level_launches[k];
    h->level_units[k] += units;
    ++h->fss[k];
    return MG3D_OK;
}

MlRateArgs ml_rate_args(mg3d_handle *h, int k, int mode) {
    Level &L = h->lev[k];
    MlRateArgs a{};
    a.nvox = L.nvox;
    a.n_levels = h->N;
    a.n_trans = h->ntrans;
    a.ti = h->d_ti;
    a.acc = h->ml_acc;
    a.T = L.T;
    a.c = L.cmat;
    a.saha = L.saha;
    a.n_tot = L.n_tot;
    a.f = L.f_default ? nullptr : L.f;
    a.n = L.n;
    a.out = nullptr;
    a.mode = mode;
    a.scal = h->scal;
    return a;
}

// Partial redistribution before a sweep of level k: rho and rho S from the
// lagged field (the sweep writes every slot of the new mean intensity).
int prd_prepare(mg3d_handle *h, int k) {
    Level &L = h->lev[k];
    MG_TRY(launched(h, launch_prd_source(h->prec, L.nvox, h->atom.n_freq, h->atom.gamma_prd,
                                         h->atom.g_ratio, h->atom.a_ul, h->d_kmat, h->d_wphin,
                                         L.n, L.c_lu, L.jnu, L.rho, L.rhoS, h->stream),
                    "partial redistribution"));
    return MG3D_OK;
}

// The sweep launch of level L with shape s (shifted-plane or band sweep).
cudaError_t launch_level_sweep(const mg3d_handle *h, const Level &L, const SweepShape &s) {
    if (s.plane) {
        if (h->prec == MG3D_PREC_F64)
            return launch_plane_sweep_f64(plane_args<double>(h, L, s), s, h->stream);
        return launch_plane_sweep_f32(plane_args<float>(h, L, s), s, h->stream);
    }
    if (h->prec == MG3D_PREC_F64)
        return launch_sweep_f64(sweep_args<double>(h, L, s), s, h->stream);
    return launch_sweep_f32(sweep_args<float>(h, L, s), s, h->stream);
}

// Formal solution on level k with its populations: partial sums into pj/pu.
int formal_solution(mg3d_handle *h, int k) {
    if (h->kind == 1) return ml_formal_solution(h, k);
    Level &L = h->lev[k];
    MG_TRY(launched(h, launch_opacity(h->prec, L.nvox, h->atom.g_ratio, h->atom.kappa, L.n,
                                      L.chi0, L.S, h->stream),
                    "opacity"));
    if (h->params.sc_interp)
        MG_TRY(launched(h, launch_xslopes(h->prec, L.nx, L.nvox, L.chi0, L.S, L.dchi0, L.dS,
                                          h->stream),
                        "x-slopes"));
    if (h->prd) MG_TRY(prd_prepare(h, k));
    TimedLaunch tl{nullptr, nullptr, k};
    if (h->timing) {
        tl.a = pool_event(h);
        tl.b = pool_event(h);
        MG_CUDA(record_event(tl.a, h->stream));
    }
    MG_TRY(launched(h, launch_level_sweep(h, L, L.shape), "sweep"));
    if (h->timing) {
        MG_CUDA(record_event(tl.b, h->stream));
        h->timed.push_back(tl);
    }
    if (h->prd && updates_background(h, k))   // the new mean intensity becomes the field
        MG_TRY(launched(h, launch_prd_collect(h->prec, (long)h->atom.n_freq * L.nvox, L.jnu_new,
                                              L.jnu, h->stream),
                        "mean intensity"));
    ++h->fs_launches;
    h->fs_units += (double)L.nvox * kRays * h->atom.n_freq;
    ++h->level_launches[k];
    h->level_units[k] += (double)L.nvox * kRays * h->atom.n_freq;
    ++h->fss[k];
    return MG3D_OK;
}

// Formal solutions of level k in the precision other than the handle's (a
// per-call precision, two-level static CRD handles): on the first request
// the level's chi0/S/bottom-intensity buffers, step table and shape in that
// precision, and the handle's slot tables and partial sums, are built; then
// opacity, shifted-plane sweep and reduction run like the handle's own, with
// those buffers.  Output: Jeff and U in h->scratch [2][nvox].
int other_prec_fs(mg3d_handle *h, int k, int prec) {
    Level &L = h->lev[k];
    if (h->kind != 0 || h->moving || h->prd || h->params.sc_interp)
        return fail(MG3D_E_ARG, "a formal solution in another precision than the handle's is "
                                "built for static two-level atoms in complete redistribution "
                                "with linear upwind interpolation");
    if (!plane_grid_ok(L.nx, L.ny, L.nz))
        return fail(MG3D_E_ARG, "grid too large for the shifted-plane sweep");
    const size_t es = elem_size(prec);
    if (h->o_prec != prec) {
        if (h->o_prec >= 0) return fail(MG3D_E_STATE, "other-precision state mismatch");
        if (prec == MG3D_PREC_F64) MG_TRY(build_plane_slots<double>(h, h->o_pslot));
        else MG_TRY(build_plane_slots<float>(h, h->o_pslot));
        h->o_prec = prec;
    }
    if (!L.o_chi0) {
        MG_TRY(dev_alloc(&L.o_chi0, L.nvox * es));
        MG_TRY(dev_alloc(&L.o_S, L.nvox * es));
        MG_TRY(dev_alloc(&L.o_bbot, L.nplane * es));
        std::vector<StepGeom> g;
        build_geometry(h, L, g);
        if (prec == MG3D_PREC_F64) {
            const auto ps = plane_steps<double>(L, g);
            MG_TRY(dev_alloc(&L.o_psteps, ps.size() * sizeof(ps[0])));
            MG_CUDA(cudaMemcpy(L.o_psteps, ps.data(), ps.size() * sizeof(ps[0]),
                               cudaMemcpyHostToDevice));
        } else {
            const auto ps = plane_steps<float>(L, g);
            MG_TRY(dev_alloc(&L.o_psteps, ps.size() * sizeof(ps[0])));
            MG_CUDA(cudaMemcpy(L.o_psteps, ps.data(), ps.size() * sizeof(ps[0]),
                               cudaMemcpyHostToDevice));
        }
        L.o_shape = choose_plane_shape(prec, L.nx, L.ny, h->atom.n_freq);
        if (L.o_shape.ng == 0) return fail(MG3D_E_ARG, "no sweep shape fits in shared memory");
        MG_TRY(launched(h, launch_planck_bottom(prec, L.nplane, h->atom.theta, L.T, L.o_bbot,
                                                h->stream),
                        "planck"));
    }
    size_t need = 0;
    for (int j = 1; j <= h->L; ++j)
        if (h->lev[j].o_chi0)
            need = std::max(need, (size_t)kRays * h->lev[j].o_shape.ngroups *
                                      (size_t)h->lev[j].nvox);
    static_assert(sizeof(size_t) == 8, "64-bit sizes");
    if (!h->o_pj || need > h->partial_elems_o) {
        MG_CUDA(cudaStreamSynchronize(h->stream));
        if (h->o_pj) cudaFree(h->o_pj);
        if (h->o_pu) cudaFree(h->o_pu);
        h->o_pj = h->o_pu = nullptr;
        h->partial_elems_o = 0;
        MG_TRY(dev_alloc(&h->o_pj, need * es));
        MG_TRY(dev_alloc(&h->o_pu, need * es));
        h->partial_elems_o = need;
    }
    MG_TRY(launched(h, launch_opacity(prec, L.nvox, h->atom.g_ratio, h->atom.kappa, L.n,
                                      L.o_chi0, L.o_S, h->stream),
                    "opacity"));
    const cudaError_t e =
        prec == MG3D_PREC_F64
            ? launch_plane_sweep_f64(plane_args<double>(h, L, L.o_shape, true), L.o_shape,
                                     h->stream)
            : launch_plane_sweep_f32(plane_args<float>(h, L, L.o_shape, true), L.o_shape,
                                     h->stream);
    MG_TRY(launched(h, e, "sweep"));
    ++h->fs_launches;
    h->fs_units += (double)L.nvox * kRays * h->atom.n_freq;
    ++h->level_launches[k];
    h->level_units[k] += (double)L.nvox * kRays * h->atom.n_freq;
    RateArgs a{};
    a.nvox = L.nvox;
    a.nslots = kRays * L.o_shape.ngroups;
    a.prec = prec;
    a.pj = h->o_pj;
    a.pu = h->o_pu;
    a.a_ul = h->atom.a_ul;
    a.g_ratio = h->atom.g_ratio;
    a.c_ul = L.c_ul;
    a.c_lu = L.c_lu;
    a.n_tot = L.n_tot;
    a.n = L.n;
    a.out = h->scratch;
    a.mode = kRateReduce;
    MG_TRY(launched(h, launch_rates(a, h->stream), "reduce"));
    return MG3D_OK;
}

RateArgs rate_args(mg3d_handle *h, int k, int mode) {
    Level &L = h->lev[k];
    RateArgs a{};
    a.nvox = L.nvox;
    a.nslots = kRays * L.shape.ngroups;
    a.prec = h->prec;
    a.pj = h->pj;
    a.pu = h->pu;
    a.zero_radiation = 0;
    a.a_ul = h->atom.a_ul;
    a.g_ratio = h->atom.g_ratio;
    a.c_ul = L.c_ul;
    a.c_lu = L.c_lu;
    a.n_tot = L.n_tot;
    a.f = L.f_default ? nullptr : L.f;
    a.n = L.n;
    a.out = nullptr;
    a.mode = mode;
    a.scal = h->scal;
    return a;
}

int sweep(mg3d_handle *h, int k) {
    MG_TRY(formal_solution(h, k));
    if (h->kind == 1) {
        MlRateArgs a = ml_rate_args(h, k, kRateSolve);
        MG_TRY(launched(h, launch_ml_rates(a, h->stream), "multi-level rates"));
    } else {
        RateArgs a = rate_args(h, k, kRateSolve);
        MG_TRY(launched(h, launch_rates(a, h->stream), "rates"));
    }
    ++h->sweeps[k];
    return MG3D_OK;
}

int reset_scalars(mg3d_handle *h) {
    MG_CUDA(cudaMemsetAsync(h->scal, 0, 8 * sizeof(unsigned long long), h->stream));
    return MG3D_OK;
}

// MG3D_E_CUDA (and the word cleared) when the sweep status word read back
// from the device holds a bit: a shifted-plane sweep's bounded wait for the
// data of a plane ran out, so its formal solution is not valid.
int sweep_status(mg3d_handle *h, unsigned long long word) {
    if (!word) return MG3D_OK;
    cudaMemsetAsync(h->scal + kScalStatus, 0, sizeof(unsigned long long), h->stream);
    return fail(MG3D_E_CUDA, "a formal-solution sweep gave up waiting for the data of a plane "
                             "(shifted-plane sweep, transaction-counted stores)");
}

// Reads the status word after the work enqueued so far.
int take_sweep_status(mg3d_handle *h) {
    unsigned long long w = 0;
    MG_CUDA(cudaMemcpyAsync(&w, h->scal + kScalStatus, sizeof(w), cudaMemcpyDeviceToHost,
                            h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return sweep_status(h, w);
}

int read_scalars(mg3d_handle *h, double *C, long long *neg, long long *bad) {
    unsigned long long s[kScalStatus + 1];
    MG_CUDA(cudaMemcpyAsync(s, h->scal, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    MG_TRY(sweep_status(h, s[kScalStatus]));
    double c;
    std::memcpy(&c, &s[0], sizeof(c));
    if (C) *C = c;
    if (neg) *neg = (long long)s[3];
    if (bad) *bad = (long long)s[2];
    return MG3D_OK;
}

int zero_radiation(mg3d_handle *h, int k) {
    Level &L = h->lev[k];
    L.f_default = true;
    if (h->kind == 1) {
        MG_TRY(ml_clear_acc(h, k));
        MG_TRY(ml_accumulate(h, k, 0, h->nfreq_ml, true));
        MlRateArgs a = ml_rate_args(h, k, kRateSolve);
        a.scal = nullptr;
        MG_TRY(launched(h, launch_ml_rates(a, h->stream), "zero radiation"));
        if (ml_lagged(h)) {
            // the lagged field from nothing: cleared (rho = 1 for partial
            // redistribution); with background scattering one Lambda-iteration
            // (a formal solution with the populations held, Sec. 4.8)
            Level &L = h->lev[k];
            MG_CUDA(cudaMemsetAsync(L.jbg, 0,
                                    (size_t)h->nfreq_ml * L.nvox * elem_size(h->prec),
                                    h->stream));
            if (h->scatter) MG_TRY(lambda_iteration(h, k));
        }
        return MG3D_OK;
    }
    RateArgs a = rate_args(h, k, kRateSolve);
    a.zero_radiation = 1;
    a.scal = nullptr;
    MG_TRY(launched(h, launch_rates(a, h->stream), "zero radiation"));
    if (h->prd)   // the lagged field starts at zero: the first formal solution sees CRD
        MG_CUDA(cudaMemsetAsync(h->lev[k].jnu, 0,
                                (size_t)h->atom.n_freq * h->lev[k].nvox * elem_size(h->prec),
                                h->stream));
    return MG3D_OK;
}

// out <- f - W(n) (mode residual) or out += W(n) (mode add), one extra FS.
int apply_W(mg3d_handle *h, int k, int mode, double *out) {
    MG_TRY(formal_solution(h, k));
    if (h->kind == 1) {
        MlRateArgs a = ml_rate_args(h, k, mode);
        a.out = out;
        a.scal = nullptr;
        MG_TRY(launched(h, launch_ml_rates(a, h->stream), "multi-level residual"));
        return MG3D_OK;
    }
    RateArgs a = rate_args(h, k, mode);
    a.out = out;
    a.scal = nullptr;
    MG_TRY(launched(h, launch_rates(a, h->stream), "residual"));
    return MG3D_OK;
}

int vcycle(mg3d_handle *h, int k, bool first) {
    Level &F = h->lev[k];
    Level &C = h->lev[k - 1];
    const int nu_pre = (first && k == h->L) ? h->params.nu0 : h->params.nu1;
    for (int i = 0; i < nu_pre; ++i) MG_TRY(sweep(h, k));
    // residual with an extra formal solution (Eq. 5)
    MG_TRY(apply_W(h, k, kRateResidual, F.r));
    // coarse-grid equation (Eq. 9)
    MG_TRY(launched(h, launch_restrict(h->N, F.nx, F.ny, F.nz, F.n, C.n, h->stream,
                                       h->params.restriction),
                    "restrict n"));
    MG_CUDA(cudaMemcpyAsync(C.n_before, C.n, (size_t)h->N * C.nvox * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream));
    if (ml_lagged(h)) {
        // background field (and the lagged field of partial redistribution):
        // full-weighted, then one Lambda-iteration with the restricted
        // populations; fixed on this grid until the cycle leaves it (Sec. 4.8)
        MG_TRY(launched(h, launch_restrict_prec(h->prec, h->nfreq_ml, F.nx, F.ny, F.nz, F.jbg,
                                                C.jbg, h->stream),
                        "restrict background field"));
        MG_TRY(lambda_iteration(h, k - 1));
    }
    if (h->kind == 0 && h->prd) {
        // the lagged mean intensity of partial redistribution, like the
        // background field: full-weighted, one Lambda-iteration, then fixed
        MG_TRY(launched(h, launch_restrict_prec(h->prec, h->atom.n_freq, F.nx, F.ny, F.nz, F.jnu,
                                                C.jnu, h->stream),
                        "restrict mean intensity"));
        MG_TRY(lambda_iteration(h, k - 1));
    }
    MG_TRY(launched(h, launch_restrict(h->N, F.nx, F.ny, F.nz, F.r, C.f, h->stream,
                                       h->params.restriction),
                    "restrict r"));
    C.f_default = false;
    MG_TRY(apply_W(h, k - 1, kRateAddW, C.f));
    if (k - 1 == 1) {
        for (int i = 0; i < h->params.nu3; ++i) MG_TRY(sweep(h, 1));
    } else {
        MG_TRY(vcycle(h, k - 1, false));
    }
    // relative correction, interpolated (Eqs. 10-11), 10 % rule (Sec. 4.10)
    MG_TRY(launched(h, launch_prolong_correct(h->params.interpolation, h->N, C.nx, C.ny, C.nz,
                                              F.tz, F.zf, C.n, C.n_before, F.n, h->scal,
                                              h->stream),
                    "prolong correction"));
    if (h->params.interpolation) ++h->launches;  // the Hermite correction is two kernels
    for (int i = 0; i < h->params.nu2; ++i) MG_TRY(sweep(h, k));
    return MG3D_OK;
}

// One V-cycle from the finest grid; C over the cycle into *C.
// The work of one V-cycle from the finest grid, with no host synchronisation:
// copy of the starting populations, the cycle, and C over the cycle into
// scal[4] (non-finite count into scal[6]); the 10 % rule counts into scal[3].
int cycle_work(mg3d_handle *h, bool first) {
    Level &F = h->lev[h->L];
    MG_CUDA(cudaMemcpyAsync(h->scratch, F.n, (size_t)h->N * F.nvox * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream));
    F.f_default = true;
    MG_TRY(reset_scalars(h));
    MG_TRY(vcycle(h, h->L, first));
    MG_TRY(launched(h, launch_max_rel_change((long)h->N * F.nvox, F.n, h->scratch, h->scal + 4,
                                             h->stream),
                    "max rel change"));
    return MG3D_OK;
}

void drop_graphs(mg3d_handle *h) {
    for (int i = 0; i < 2; ++i) {
        if (h->cycle_exec[i]) {
            cudaGraphExecDestroy(h->cycle_exec[i]);
            h->cycle_exec[i] = nullptr;
        }
        for (auto &t : h->cycle_timed[i]) {
            h->event_pool.push_back(t.a);
            h->event_pool.push_back(t.b);
        }
        h->cycle_timed[i].clear();
    }
}

// Capture the cycle into a graph (once per variant), then replay it; the
// library's counters advance by what the captured cycle launched.
int graph_cycle(mg3d_handle *h, bool first) {
    const int idx = first ? 1 : 0;
    if (h->graph_stream != h->stream) {
        drop_graphs(h);
        h->graph_stream = h->stream;
    }
    if (!h->cycle_exec[idx]) {
        mg3d_handle::CycleDelta before;
        before.launches = h->launches;
        before.fs_launches = h->fs_launches;
        before.fs_units = h->fs_units;
        std::memcpy(before.level_launches, h->level_launches, sizeof(before.level_launches));
        std::memcpy(before.level_units, h->level_units, sizeof(before.level_units));
        std::memcpy(before.sweeps, h->sweeps, sizeof(before.sweeps));
        std::memcpy(before.fss, h->fss, sizeof(before.fss));
        const size_t timed_before = h->timed.size();
        MG_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
        int rc = cycle_work(h, first);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (rc != MG3D_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(MG3D_E_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->cycle_exec[idx], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return fail(MG3D_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        // event pairs recorded inside the graph are read after every replay
        h->cycle_timed[idx].assign(h->timed.begin() + timed_before, h->timed.end());
        h->timed.resize(timed_before);
        // what one replay adds to the counters; capturing itself ran nothing
        mg3d_handle::CycleDelta &d = h->cycle_delta[idx];
        d.launches = h->launches - before.launches;
        d.fs_launches = h->fs_launches - before.fs_launches;
        d.fs_units = h->fs_units - before.fs_units;
        for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) {
            d.level_launches[k] = h->level_launches[k] - before.level_launches[k];
            d.level_units[k] = h->level_units[k] - before.level_units[k];
            d.sweeps[k] = h->sweeps[k] - before.sweeps[k];
            d.fss[k] = h->fss[k] - before.fss[k];
        }
        h->launches = before.launches;
        h->fs_launches = before.fs_launches;
        h->fs_units = before.fs_units;
        std::memcpy(h->level_launches, before.level_launches, sizeof(before.level_launches));
        std::memcpy(h->level_units, before.level_units, sizeof(before.level_units));
        std::memcpy(h->sweeps, before.sweeps, sizeof(before.sweeps));
        std::memcpy(h->fss, before.fss, sizeof(before.fss));
    }
    MG_CUDA(cudaGraphLaunch(h->cycle_exec[idx], h->stream));
    const mg3d_handle::CycleDelta &d = h->cycle_delta[idx];
    h->launches += d.launches;
    h->fs_launches += d.fs_launches;
    h->fs_units += d.fs_units;
    for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) {
        h->level_launches[k] += d.level_launches[k];
        h->level_units[k] += d.level_units[k];
        h->sweeps[k] += d.sweeps[k];
        h->fss[k] += d.fss[k];
    }
    return MG3D_OK;
}

// One V-cycle from the finest grid; C over the cycle into *C.  Replayed from
// a CUDA graph unless graphs are off or per-launch timing is on.
int fas_cycle(mg3d_handle *h, bool first, double *C, long long *neg) {
    if (h->L < 2) return fail(MG3D_E_STATE, "a V-cycle needs n_grids >= 2");
    h->top = h->L;
    const bool graphs = h->use_graphs;
    if (graphs) {
        MG_TRY(graph_cycle(h, first));
    } else {
        MG_TRY(cycle_work(h, first));
    }
    unsigned long long sc[kScalStatus + 1];
    MG_CUDA(cudaMemcpyAsync(sc, h->scal, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    MG_TRY(sweep_status(h, sc[kScalStatus]));
    if (graphs) {
        for (auto &t : h->cycle_timed[first ? 1 : 0]) {
            float ms = 0.f;
            MG_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
            h->acc_ms[t.level] += ms;
            ++h->acc_n[t.level];
        }
    }
    if (C) std::memcpy(C, &sc[4], sizeof(double));
    if (neg) *neg = (long long)sc[3];
    if (sc[6]) return fail(MG3D_E_DIVERGED, "non-finite populations after a V-cycle");
    return MG3D_OK;
}

void begin_stats(mg3d_handle *h) {
    std::memset(h->sweeps, 0, sizeof(h->sweeps));
    std::memset(h->fss, 0, sizeof(h->fss));
    h->negatives = 0;
}

void end_stats(mg3d_handle *h, mg3d_stats *st, int iters, double C, double secs) {
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    st->iterations = iters;
    st->last_change = C;
    st->negatives = h->negatives;
    st->seconds = secs;
    double eq = 0;
    for (int k = 1; k <= h->L; ++k) {
        st->sweeps[k] = h->sweeps[k];
        st->formal_solutions[k] = h->fss[k];
        eq += h->fss[k] * std::pow(0.125, h->L - k);
    }
    st->fine_fs_equivalents = eq;
}

int host_to_level(mg3d_handle *h, double *dst, const double *src, size_t count) {
    MG_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return MG3D_OK;
}

int level_to_host(mg3d_handle *h, double *dst, const double *src, size_t count) {
    MG_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return MG3D_OK;
}

int make_shape(const mg3d_handle *h, int k, int ng, int bands, int threads, SweepShape *out) {
    const Level &L = h->lev[k];
    const int nf = h->atom.n_freq;
    if (ng < 1 || ng > nf || bands < 1 || bands > kMaxBands || bands > L.ny || threads < 32 ||
        threads > kMaxSweepThreads || threads % 32)
        return fail(MG3D_E_ARG, "bad sweep shape");
    SweepShape s{ng, (nf + ng - 1) / ng, bands, (L.ny + bands - 1) / bands, threads};
    if ((long)(bands - 1) * s.rows >= L.ny) return fail(MG3D_E_ARG, "empty band");
    s.herm = h->params.sc_interp;
    s.vel = h->moving ? 1 : 0;
    s.prd = h->prd ? 1 : 0;
    s.stage = s.herm || s.vel || s.prd ? 0 : 1;
    *out = s;
    return MG3D_OK;
}

// Shifted-plane shape (stage 2) of the given launch parameters: freq_per_block
// >= n_freq takes all frequencies in one group (at most 16), else it must be
// twice a supported slot count (2, 4, 6, 10 or 16).
static int plane_shape_from_args(const mg3d_handle *h, int level, int freq_per_block, int bands,
                                 int threads, int lean, SweepShape *out, int kind = 1) {
    const Level &L = h->lev[level];
    const int nf = h->atom.n_freq;
    if (h->params.sc_interp || h->moving || h->prd)
        return fail(MG3D_E_ARG, "the shifted-plane sweep (stage 2) takes static atmospheres in "
                                "complete redistribution with linear upwind interpolation");
    if (!plane_grid_ok(L.nx, L.ny, L.nz))
        return fail(MG3D_E_ARG, "grid too large for the shifted-plane sweep");
    int np = 0;
    if (freq_per_block >= nf) {
        np = plane_np_for(nf);
        if (np == 0)
            return fail(MG3D_E_ARG, "more than 16 frequencies: the shifted-plane sweep takes "
                                    "2, 4, 6, 10 or 16 frequencies per block");
    } else if (freq_per_block >= 1 && freq_per_block % 2 == 0 &&
               plane_np_supported(freq_per_block / 2)) {
        np = freq_per_block / 2;
    } else {
        return fail(MG3D_E_ARG, "the shifted-plane sweep takes all frequencies or 2, 4, 6, 10 "
                                "or 16 per block");
    }
    if (bands < 1 || bands > kMaxBands || bands > L.ny || threads < 32 ||
        threads > kPlaneMaxThreads || threads % 32)
        return fail(MG3D_E_ARG, "bad sweep shape");
    if (lean < 0 || lean > 1 || (lean == 1 && h->prec == MG3D_PREC_F64))
        return fail(MG3D_E_ARG, "the shifted-plane sweep takes lean 0, or 1 in FP32");
    if (threads > 512 && (h->prec == MG3D_PREC_F64 || lean != 0 || np > 2))
        return fail(MG3D_E_ARG, "blocks above 512 threads: FP32, lean 0, at most 4 frequencies "
                                "per block");
    SweepShape s{2 * np, (nf + 2 * np - 1) / (2 * np), bands, (L.ny + bands - 1) / bands, threads};
    if ((long)(bands - 1) * s.rows >= L.ny) return fail(MG3D_E_ARG, "empty band");
    if ((long)s.rows * L.nx > (long)plane_max_pass(np, h->prec == MG3D_PREC_F64) * threads)
        return fail(MG3D_E_ARG, "too few threads for the band (the shifted-plane sweep takes at "
                                "most " + std::to_string(plane_max_pass(np, h->prec == MG3D_PREC_F64)) +
                                " nodes per thread)");
    s.lean = lean;
    s.stage = 0;
    s.plane = kind;
    s.np = np;
    if (plane_smem_bytes(h->prec, np, s.rows, L.nx) > kMaxPlaneSmem)
        return fail(MG3D_E_ARG, "sweep shape exceeds shared memory");
    *out = s;
    return MG3D_OK;
}

// Shape of the given launch parameters on a level, validated except for
// whether the GPU can schedule it.
static int shape_from_args(const mg3d_handle *h, int level, int freq_per_block, int bands,
                           int threads, int lean, int stage, SweepShape *out) {
    MG_TRY(check_level(h, level));
    if (h->kind != 0) return fail(MG3D_E_STATE, "sweep shapes apply to two-level handles");
    if (stage == 2 || stage == 3)
        return plane_shape_from_args(h, level, freq_per_block, bands, threads, lean, out,
                                     stage - 1);
    if (lean < 0 || lean > 2 || (lean == 2 && threads > 256))
        return fail(MG3D_E_ARG, "lean must be 0, 1 or (up to 256 threads) 2");
    if (stage != 0 && stage != 1) return fail(MG3D_E_ARG, "stage must be 0, 1, 2 or 3");
    if (stage && h->params.sc_interp)
        return fail(MG3D_E_ARG, "Hermite upwind interpolation runs unstaged (stage 0)");
    if (stage && h->moving) return fail(MG3D_E_ARG, "moving atmospheres run unstaged (stage 0)");
    if (stage && h->prd)
        return fail(MG3D_E_ARG, "partial redistribution runs unstaged (stage 0)");
    SweepShape s;
    MG_TRY(make_shape(h, level, freq_per_block, bands, threads, &s));
    s.lean = lean;
    s.stage = stage;
    if (sweep_smem_bytes(h->prec, s, h->lev[level].nx) > kMaxSweepSmem)
        return fail(MG3D_E_ARG, "sweep shape exceeds shared memory");
    *out = s;
    return MG3D_OK;
}

// MG3D_E_ARG unless the GPU can hold at least one cluster of shape s on level
// k (clusters of more than 8 blocks are not guaranteed to fit).
int check_schedulable(const mg3d_handle *h, int k, const SweepShape &s) {
    int n = 0;
    const cudaError_t e = s.plane ? plane_active_clusters(h->prec, s, h->lev[k].nx, &n)
                                  : sweep_active_clusters(h->prec, s, h->lev[k].nx, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MG3D_E_ARG,
                    std::string("sweep shape cannot be scheduled: ") + cudaGetErrorString(e));
    }
    if (n < 1) return fail(MG3D_E_ARG, "sweep shape cannot be scheduled: cluster does not fit");
    return MG3D_OK;
}

void drop_graphs(mg3d_handle *h);

// Partial-sum buffers of at least `need` elements (contents not kept).
int ensure_partials(mg3d_handle *h, size_t need) {
    if (need <= h->partial_elems) return MG3D_OK;
    const size_t es = elem_size(h->prec);
    MG_CUDA(cudaStreamSynchronize(h->stream));
    cudaFree(h->pj);
    cudaFree(h->pu);
    h->pj = h->pu = nullptr;
    h->partial_elems = 0;
    MG_TRY(dev_alloc(&h->pj, need * es));
    MG_TRY(dev_alloc(&h->pu, need * es));
    h->partial_elems = need;
    drop_graphs(h);
    return MG3D_OK;
}

// Shrink the partial buffers to what the current shapes of all levels need.
int shrink_partials(mg3d_handle *h) {
    size_t need = 0;
    for (int k = 1; k <= h->L; ++k)
        need = std::max(need, (size_t)kRays * h->lev[k].shape.ngroups * (size_t)h->lev[k].nvox);
    if (need >= h->partial_elems) return MG3D_OK;
    h->partial_elems = 0;
    return ensure_partials(h, need);
}

// Device time of `reps` sweep launches of level k with shape s (ms each).
int time_shape(mg3d_handle *h, int k, const SweepShape &s, int reps, float *ms) {
    Level &L = h->lev[k];
    const SweepShape saved = L.shape;
    L.shape = s;
    cudaEvent_t a = pool_event(h), b = pool_event(h);
    int rc = MG3D_OK;
    cudaError_t e = cudaEventRecord(a, h->stream);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        e = launch_level_sweep(h, L, s);
        ++h->launches;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e != cudaSuccess) rc = fail(MG3D_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    else *ms /= (float)reps;
    h->event_pool.push_back(a);
    h->event_pool.push_back(b);
    L.shape = saved;
    return rc;
}

// Time candidate sweep shapes of level k with its current populations and
// keep the fastest: every (frequencies per block, bands, threads) that fits,
// one launch each, then the best eight again three times each.
// Shifted-plane candidates of level k: one group (the fewest slots that take
// every frequency) and every smaller supported slot count with at most 8
// groups; 1-16 bands; 32-512 threads in powers of two and the block sizes
// that cover a band in 1-4 equal passes; in FP32 both register budgets.
void plane_candidates(mg3d_handle *h, int k, std::vector<SweepShape> &cands) {
    const Level &L = h->lev[k];
    const int nf = h->atom.n_freq;
    for (int i = 0; i < kPlaneNpCount; ++i) {
        const int np = kPlaneNp[i];
        const int groups = (nf + 2 * np - 1) / (2 * np);
        if (groups > 8) continue;
        if (groups == 1 && np != plane_np_for(nf)) continue;   // one-group: fewest slots
        const int fpb = groups == 1 ? nf : 2 * np;
        for (int bands = 1; bands <= kMaxBands && bands <= L.ny; ++bands) {
            const int band = ((L.ny + bands - 1) / bands) * L.nx;
            std::vector<int> ths = {32, 64, 128, 256, 512, 1024};
            for (int passes = 1; passes <= plane_max_pass(np, h->prec == MG3D_PREC_F64); ++passes) {
                const int th = ((band + passes - 1) / passes + 31) / 32 * 32;
                if (th <= kPlaneMaxThreads && std::find(ths.begin(), ths.end(), th) == ths.end())
                    ths.push_back(th);
            }
            for (int th : ths)
                for (int lean = 0; lean < (h->prec == MG3D_PREC_F64 ? 1 : 2); ++lean)
                    // both completion schemes where blocks exchange rows
                    for (int kind = 1; kind <= (bands > 1 ? 2 : 1); ++kind) {
                        if (th > 32 && th / 2 >= band) continue;  // a smaller block covers it
                        SweepShape s;
                        if (plane_shape_from_args(h, k, fpb, bands, th, lean, &s, kind) !=
                            MG3D_OK)
                            continue;
                        if (check_schedulable(h, k, s) != MG3D_OK) continue;
                        cands.push_back(s);
                    }
        }
    }
}

int autotune_level(mg3d_handle *h, int k, int *evaluated) {
    Level &L = h->lev[k];
    const int nf = h->atom.n_freq;
    const bool plane_ok = !h->params.sc_interp && !h->moving && !h->prd &&
                          plane_grid_ok(L.nx, L.ny, L.nz);
    // band-sweep frequency groupings (variants the shifted-plane sweep does not take)
    std::vector<int> ngs;
    for (int ng = 1; ng <= nf && !plane_ok; ++ng) {
        const int groups = (nf + ng - 1) / ng;
        if (groups > 64) continue;
        // one ng per distinct group count, the smallest that gives it
        if (!ngs.empty() && (nf + ngs.back() - 1) / ngs.back() == groups) continue;
        ngs.push_back(ng);
    }
    std::vector<SweepShape> cands;
    if (plane_ok) plane_candidates(h, k, cands);
    for (int ng : ngs)
        for (int bands = 1; bands <= kMaxBands && bands <= L.ny; ++bands) {
            // 32 to 512 threads in powers of two and the block sizes that
            // cover a band in 1-4 equal passes
            const int band = ((L.ny + bands - 1) / bands) * L.nx;
            std::vector<int> ths = {32, 64, 128, 256, 512};
            for (int passes = 1; passes <= 4; ++passes) {
                const int th = ((band + passes - 1) / passes + 31) / 32 * 32;
                if (th <= kMaxSweepThreads && std::find(ths.begin(), ths.end(), th) == ths.end())
                    ths.push_back(th);
            }
            for (int th : ths)
                for (int lean = 0; lean < 3; ++lean)
                    for (int stage = 1; stage >= 0; --stage) {
                        if (lean == 2 && th > 256) continue;  // same as lean 0 above 256
                        if (th > 32 && th / 2 >= band) continue;  // a smaller block covers it
                        SweepShape s;
                        if (shape_from_args(h, k, ng, bands, th, lean, stage, &s) != MG3D_OK)
                            continue;
                        if (check_schedulable(h, k, s) != MG3D_OK) continue;
                        cands.push_back(s);
                    }
        }
    g_last_error.clear();
    if (cands.empty()) return fail(MG3D_E_ARG, "no sweep shape fits");
    (void)0;
    size_t need = 0;
    for (auto &s : cands) need = std::max(need, (size_t)kRays * s.ngroups * (size_t)L.nvox);
    MG_TRY(ensure_partials(h, need));
    MG_TRY(launched(h, launch_opacity(h->prec, L.nvox, h->atom.g_ratio, h->atom.kappa, L.n,
                                      L.chi0, L.S, h->stream),
                    "opacity"));
    if (h->params.sc_interp)
        MG_TRY(launched(h, launch_xslopes(h->prec, L.nx, L.nvox, L.chi0, L.S, L.dchi0, L.dS,
                                          h->stream),
                        "x-slopes"));
    if (h->prd) MG_TRY(prd_prepare(h, k));
    float warm = 0.f;
    MG_TRY(time_shape(h, k, L.shape, 1, &warm));
    std::vector<std::pair<float, size_t>> t1;
    for (size_t i = 0; i < cands.size(); ++i) {
        float ms = 0.f;
        MG_TRY(time_shape(h, k, cands[i], 1, &ms));
        t1.push_back({ms, i});
    }
    std::sort(t1.begin(), t1.end());
    const size_t keep = std::min<size_t>(8, t1.size());
    float best_ms = 1e30f;
    size_t best = t1[0].second;
    for (size_t j = 0; j < keep; ++j) {
        float ms = 0.f;
        MG_TRY(time_shape(h, k, cands[t1[j].second], 3, &ms));
        if (ms < best_ms) {
            best_ms = ms;
            best = t1[j].second;
        }
    }
    L.shape = cands[best];
    if (evaluated) *evaluated = (int)cands.size();
    return MG3D_OK;
}

// Velocity field of a moving atmosphere: the fine field, full-weighted onto
// every coarser grid like the other atmosphere fields; per level and ray the
// projected velocity and the profile normalisation; the frequency offsets
// and quadrature weights in natural order.
int setup_velocity(mg3d_handle *h, const double *vel_host) {
    const int nf = h->atom.n_freq;
    const size_t es = elem_size(h->prec);
    std::vector<double> xw(2 * (size_t)nf);
    for (int i = 0; i < nf; ++i) {
        xw[i] = nf == 1 ? 0.0 : h->atom.x_max * (2 * i - (nf - 1)) / (nf - 1);
        double w = nf == 1 ? 1.0 : 2.0 * h->atom.x_max / (nf - 1);
        if (nf > 1 && (i == 0 || i == nf - 1)) w *= 0.5;
        xw[nf + i] = w;
    }
    MG_TRY(dev_alloc(&h->d_vtab, 2 * (size_t)nf * es));
    if (h->prec == MG3D_PREC_F64) {
        MG_CUDA(cudaMemcpy(h->d_vtab, xw.data(), xw.size() * es, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f32(xw.begin(), xw.end());
        MG_CUDA(cudaMemcpy(h->d_vtab, f32.data(), f32.size() * es, cudaMemcpyHostToDevice));
    }
    for (int k = 1; k <= h->L; ++k) MG_TRY(dalloc(&h->lev[k].vel, 3 * (size_t)h->lev[k].nvox));
    Level &F = h->lev[h->L];
    MG_CUDA(cudaMemcpy(F.vel, vel_host, 3 * (size_t)F.nvox * sizeof(double),
                       cudaMemcpyHostToDevice));
    for (int k = h->L; k >= 2; --k) {
        Level &Fk = h->lev[k];
        MG_TRY(launched(h, launch_restrict(3, Fk.nx, Fk.ny, Fk.nz, Fk.vel, h->lev[k - 1].vel,
                                           h->stream),
                        "restrict velocity"));
    }
    double *dmu = nullptr, *dxw = nullptr;
    MG_TRY(dalloc(&dmu, 3 * (size_t)kRays));
    int rc = dalloc(&dxw, xw.size());
    if (rc == MG3D_OK && (cudaMemcpy(dmu, h->mu, 3 * kRays * sizeof(double),
                                     cudaMemcpyHostToDevice) != cudaSuccess ||
                          cudaMemcpy(dxw, xw.data(), xw.size() * sizeof(double),
                                     cudaMemcpyHostToDevice) != cudaSuccess))
        rc = fail(MG3D_E_CUDA, "velocity tables");
    for (int k = 1; k <= h->L && rc == MG3D_OK; ++k) {
        Level &L = h->lev[k];
        rc = dev_alloc(&L.uproj, (size_t)kRays * L.nvox * es);
        if (rc == MG3D_OK) rc = dev_alloc(&L.vnorm, (size_t)kRays * L.nvox * es);
        if (rc == MG3D_OK)
            rc = launched(h, launch_vel_prep(h->prec, L.nvox, nf, dmu, L.vel, dxw, dxw + nf,
                                             L.uproj, L.vnorm, h->stream),
                          "velocity projection");
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && rc == MG3D_OK)
        rc = fail(MG3D_E_CUDA, "velocity set-up");
    cudaFree(dmu);
    if (dxw) cudaFree(dxw);
    return rc;
}

// Partial redistribution tables: the discrete redistribution matrix
// R = diag(c) R0 diag(c), R0(x', x) = erfc(max(|x|, |x'|))/2, with c from the
// fixed-point iteration c <- sqrt(c phi / (R0^T (wq c))) so that both
// marginals sum_f' wq_f' R(f', f) are phi_f (wq: the quadrature weights
// normalised so that sum wq phi = 1); uploaded as kmat[f'][f] = wq_f' R(f', f)
// / phi_f with the normalised w phi and the table-order to natural-order map.
int setup_prd(mg3d_handle *h) {
    const int nf = h->atom.n_freq;
    std::vector<double> x(nf), wq(nf);
    for (int i = 0; i < nf; ++i) {
        x[i] = nf == 1 ? 0.0 : h->atom.x_max * (2 * i - (nf - 1)) / (nf - 1);
        wq[i] = h->wphi[i] / h->phi[i];
    }
    std::vector<double> R0((size_t)nf * nf), c(nf, 1.0), t(nf);
    for (int a = 0; a < nf; ++a)
        for (int b = a; b < nf; ++b)   // R_I-A, or R_II-A with damping; symmetric
            R0[(size_t)a * nf + b] = R0[(size_t)b * nf + a] =
                redistribution_r2a(x[a], x[b], h->atom.a_damp);
    for (int it = 0; it < 200; ++it) {
        for (int b = 0; b < nf; ++b) {
            double s = 0.0;
            for (int a = 0; a < nf; ++a) s += R0[(size_t)a * nf + b] * wq[a] * c[a];
            t[b] = s;
        }
        for (int b = 0; b < nf; ++b) c[b] = std::sqrt(c[b] * h->phi[b] / t[b]);
    }
    std::vector<double> kmat((size_t)nf * nf);
    for (int a = 0; a < nf; ++a)
        for (int b = 0; b < nf; ++b)
            kmat[(size_t)a * nf + b] = wq[a] * c[a] * R0[(size_t)a * nf + b] * c[b] / h->phi[b];
    std::vector<int> fidx(2 * (size_t)nf);
    for (int order = 0; order < 2; ++order)
        for (int j = 0; j < nf; ++j) fidx[(size_t)order * nf + j] = mirror_order(nf, order, j);
    MG_TRY(dalloc(&h->d_kmat, kmat.size()));
    MG_TRY(dalloc(&h->d_wphin, (size_t)nf));
    MG_TRY(dev_alloc((void **)&h->d_fidx, fidx.size() * sizeof(int)));
    MG_CUDA(cudaMemcpy(h->d_kmat, kmat.data(), kmat.size() * sizeof(double),
                       cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(h->d_wphin, h->wphi.data(), (size_t)nf * sizeof(double),
                       cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(h->d_fidx, fidx.data(), fidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    return MG3D_OK;
}

int create_impl(const mg3d_atmosphere *atm, const mg3d_atom *atom, const mg3d_quadrature *quad,
                const mg3d_params *params, mg3d_handle *h) {
    h->L = params->n_grids;
    h->prec = params->fs_prec;
    h->atom = *atom;
    h->params = *params;
    h->moving = atm->vel != nullptr;
    h->prd = atom->gamma_prd > 0.0;
    build_quadrature(h, quad ? quad->a : 0.0);
    build_frequencies(h);
    MG_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    const size_t es = elem_size(h->prec);

    // grid hierarchy
    for (int k = h->L; k >= 1; --k) {
        Level &L = h->lev[k];
        if (k == h->L) {
            L.nx = atm->nx;
            L.ny = atm->ny;
            L.nz = atm->nz;
            L.dx = atm->dx;
            L.dy = atm->dy;
            L.z.assign(atm->z, atm->z + atm->nz);
        } else {
            const Level &Fn = h->lev[k + 1];
            L.nx = Fn.nx / 2;
            L.ny = Fn.ny / 2;
            L.nz = (Fn.nz + 1) / 2;
            L.dx = 2 * Fn.dx;
            L.dy = 2 * Fn.dy;
            L.z.clear();
            for (int i = 0; i < Fn.nz; i += 2) L.z.push_back(Fn.z[i]);
        }
        L.nplane = (long)L.nx * L.ny;
        L.nvox = L.nplane * L.nz;
        MG_TRY(dalloc(&L.T, L.nvox));
        MG_TRY(dalloc(&L.n_tot, L.nvox));
        MG_TRY(dalloc(&L.c_ul, L.nvox));
        MG_TRY(dalloc(&L.c_lu, L.nvox));
        MG_TRY(dalloc(&L.tz, L.nz));
        MG_TRY(dalloc(&L.n, 2 * L.nvox));
        MG_TRY(dalloc(&L.f, 2 * L.nvox));
        MG_TRY(dalloc(&L.n_before, 2 * L.nvox));
        MG_TRY(dalloc(&L.r, 2 * L.nvox));
        MG_TRY(dev_alloc(&L.chi0, L.nvox * es));
        MG_TRY(dev_alloc(&L.S, L.nvox * es));
        MG_TRY(dev_alloc(&L.bbot, L.nplane * es));
        MG_TRY(dalloc(&L.geom, (size_t)kRays * L.nz));
        std::vector<double> tz(L.nz, 0.0);
        for (int i = 1; i + 1 < L.nz; i += 2) tz[i] = (L.z[i] - L.z[i - 1]) / (L.z[i + 1] - L.z[i - 1]);
        MG_CUDA(cudaMemcpy(L.tz, tz.data(), L.nz * sizeof(double), cudaMemcpyHostToDevice));
        MG_TRY(dalloc(&L.zf, L.nz));
        MG_CUDA(cudaMemcpy(L.zf, L.z.data(), L.nz * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<StepGeom> g;
        build_geometry(h, L, g);
        MG_CUDA(cudaMemcpy(L.geom, g.data(), g.size() * sizeof(StepGeom), cudaMemcpyHostToDevice));
        if (h->prec == MG3D_PREC_F64) {
            const auto ps = plane_steps<double>(L, g);
            MG_TRY(dev_alloc(&L.psteps, ps.size() * sizeof(ps[0])));
            MG_CUDA(cudaMemcpy(L.psteps, ps.data(), ps.size() * sizeof(ps[0]),
                               cudaMemcpyHostToDevice));
        } else {
            const auto ps = plane_steps<float>(L, g);
            MG_TRY(dev_alloc(&L.psteps, ps.size() * sizeof(ps[0])));
            MG_CUDA(cudaMemcpy(L.psteps, ps.data(), ps.size() * sizeof(ps[0]),
                               cudaMemcpyHostToDevice));
        }
        L.shape = choose_shape(h->prec, L.nx, L.ny, L.nz, atom->n_freq, params->sc_interp,
                               atm->vel ? 1 : 0, atom->gamma_prd > 0.0 ? 1 : 0);
        if (atom->gamma_prd > 0.0) {
            void **bufs[3] = {&L.jnu, &L.rho, &L.rhoS};
            for (void **p : bufs) MG_TRY(dev_alloc(p, (size_t)atom->n_freq * L.nvox * es));
            MG_TRY(dev_alloc(&L.jnu_new, (size_t)kRays * atom->n_freq * L.nvox * es));
            MG_CUDA(cudaMemset(L.jnu, 0, (size_t)atom->n_freq * L.nvox * es));
        }
        if (params->sc_interp) {
            MG_TRY(dev_alloc(&L.dchi0, L.nvox * es));
            MG_TRY(dev_alloc(&L.dS, L.nvox * es));
        }
        if (L.shape.ng == 0) return fail(MG3D_E_ARG, "no sweep shape fits in shared memory");
        h->partial_elems = std::max(h->partial_elems,
                                    (size_t)kRays * L.shape.ngroups * (size_t)L.nvox);
    }
    // atmosphere on the finest grid, then full weighting downward (Sec. 4.7)
    Level &F = h->lev[h->L];
    MG_CUDA(cudaMemcpy(F.T, atm->T, F.nvox * sizeof(double), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(F.n_tot, atm->n_tot, F.nvox * sizeof(double), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(F.c_ul, atm->c_ul, F.nvox * sizeof(double), cudaMemcpyHostToDevice));
    MG_TRY(dalloc(&h->scratch, 4 * F.nvox));
    for (int k = h->L; k >= 2; --k) {
        Level &Fk = h->lev[k];
        Level &Ck = h->lev[k - 1];
        // pack T, n_tot, c_ul into scratch, restrict, unpack
        MG_CUDA(cudaMemcpyAsync(h->scratch, Fk.T, Fk.nvox * 8, cudaMemcpyDeviceToDevice, h->stream));
        MG_CUDA(cudaMemcpyAsync(h->scratch + Fk.nvox, Fk.n_tot, Fk.nvox * 8,
                                cudaMemcpyDeviceToDevice, h->stream));
        MG_CUDA(cudaMemcpyAsync(h->scratch + 2 * Fk.nvox, Fk.c_ul, Fk.nvox * 8,
                                cudaMemcpyDeviceToDevice, h->stream));
        double *coarse = h->scratch + 3 * Fk.nvox;  // 3 coarse fields fit in nvox
        MG_TRY(launched(h, launch_restrict(3, Fk.nx, Fk.ny, Fk.nz, h->scratch, coarse, h->stream),
                        "restrict atmosphere"));
        MG_CUDA(cudaMemcpyAsync(Ck.T, coarse, Ck.nvox * 8, cudaMemcpyDeviceToDevice, h->stream));
        MG_CUDA(cudaMemcpyAsync(Ck.n_tot, coarse + Ck.nvox, Ck.nvox * 8,
                                cudaMemcpyDeviceToDevice, h->stream));
        MG_CUDA(cudaMemcpyAsync(Ck.c_ul, coarse + 2 * Ck.nvox, Ck.nvox * 8,
                                cudaMemcpyDeviceToDevice, h->stream));
    }
    if (h->moving) MG_TRY(setup_velocity(h, atm->vel));
    for (int k = 1; k <= h->L; ++k) {
        Level &L = h->lev[k];
        MG_TRY(launched(h, launch_collisions_up(L.nvox, atom->g_ratio, atom->theta, L.T, L.c_ul,
                                                L.c_lu, h->stream),
                        "collisions"));
        MG_TRY(launched(h, launch_planck_bottom(h->prec, L.nplane, atom->theta, L.T, L.bbot,
                                                h->stream),
                        "planck"));
    }
    // frequency tables in the formal-solution precision, in two orders: the
    // sweep sums over frequencies, so their order is internal to it, and a
    // frequency whose phi equals its predecessor's in the table reuses that
    // one's short-characteristics weights (see freq_tables)
    const int nf = atom->n_freq;
    MG_TRY(dev_alloc(&h->d_ftab, 6 * (size_t)nf * es));
    std::vector<double> tabs(6 * (size_t)nf);
    for (int order = 0; order < 2; ++order)
        for (int j = 0; j < nf; ++j) {
            const int i = mirror_order(nf, order, j);
            double *t = tabs.data() + (size_t)order * 3 * nf;
            t[j] = h->phi[i];
            t[nf + j] = 1.0 / h->phi[i];
            t[2 * nf + j] = h->wphi[i] / kRays;
        }
    if (h->prec == MG3D_PREC_F64) {
        MG_CUDA(cudaMemcpy(h->d_ftab, tabs.data(), tabs.size() * es, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> t32(tabs.begin(), tabs.end());
        MG_CUDA(cudaMemcpy(h->d_ftab, t32.data(), t32.size() * es, cudaMemcpyHostToDevice));
    }
    if (h->prd) MG_TRY(setup_prd(h));
    if (h->prec == MG3D_PREC_F64) MG_TRY(build_plane_slots<double>(h, h->d_pslot));
    else MG_TRY(build_plane_slots<float>(h, h->d_pslot));
    {
        double tab[kExpTab];
        exp_neg_constants(tab, &h->exp_l1, &h->exp_l2);
        MG_TRY(dalloc(&h->d_exp_tab, kExpTab));
        MG_CUDA(cudaMemcpy(h->d_exp_tab, tab, sizeof(tab), cudaMemcpyHostToDevice));
    }
    MG_TRY(dev_alloc(&h->pj, h->partial_elems * es));
    MG_TRY(dev_alloc(&h->pu, h->partial_elems * es));
    MG_TRY(dalloc(&h->scal, kScalStatus + 1));
    MG_CUDA(cudaMemset(h->scal, 0, (kScalStatus + 1) * sizeof(unsigned long long)));
    for (int k = 1; k <= h->L; ++k) MG_TRY(zero_radiation(h, k));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return MG3D_OK;
}

// Equidistant points on [a, b] (the last one exactly b) and trapezoid weights.
void trapezoid_grid(double a, double b, int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, a);
    w.assign(n, n == 1 ? 1.0 : 0.0);
    if (n == 1) return;
    const double step = (b - a) / (n - 1);
    for (int i = 0; i < n; ++i) x[i] = i == n - 1 ? b : a + i * step;
    for (int i = 0; i + 1 < n; ++i) {
        const double d = x[i + 1] - x[i];
        w[i] += 0.5 * d;
        w[i + 1] += 0.5 * d;
    }
}

// Bytes the multi-level formal solution needs per frequency of a chunk:
// opacity, source function and their two transition shares on every level,
// and the angle sums of every ray-group slot on the finest.
size_t ml_bytes_per_freq(const mg3d_handle *h) {
    const size_t es = elem_size(h->prec);
    size_t b = (ml_lagged(h) ? 3 : 2) * (size_t)h->ml_slots * h->lev[h->L].nvox * es;
    const size_t per_level = h->params.sc_interp ? 6 : 4;  // Hermite: slopes of chi, S
    for (int k = 1; k <= h->L; ++k) b += per_level * (size_t)h->lev[k].nvox * es;
    return b;
}

// All frequencies in one chunk when their buffers take at most 60 % of the
// free device memory, else the largest chunk that does.
int default_ml_chunk(const mg3d_handle *h) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return h->nfreq_ml;
    }
    const size_t fit = (size_t)(0.6 * (double)free_b) / ml_bytes_per_freq(h);
    return (int)std::max<size_t>(1, std::min<size_t>(fit, (size_t)h->nfreq_ml));
}

// (Re)allocates the per-chunk buffers of a multi-level handle for `chunk`
// frequencies per chunk.
int alloc_ml_chunks(mg3d_handle *h, int chunk) {
    const size_t es = elem_size(h->prec);
    for (int k = 1; k <= h->L; ++k) {
        Level &L = h->lev[k];
        void **bufs[6] = {&L.mchi, &L.mS, &L.msc, &L.moc, &L.mdchi, &L.mdS};
        for (void **p : bufs) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
    }
    if (h->ml_jx) cudaFree(h->ml_jx);
    if (h->ml_ux) cudaFree(h->ml_ux);
    if (h->ml_jm) cudaFree(h->ml_jm);
    h->ml_jx = h->ml_ux = h->ml_jm = nullptr;
    h->ml_chunk = 0;
    for (int k = 1; k <= h->L; ++k) {
        Level &L = h->lev[k];
        void **bufs[6] = {&L.mchi, &L.mS, &L.msc, &L.moc, &L.mdchi, &L.mdS};
        const int nbufs = h->params.sc_interp ? 6 : 4;
        for (int i = 0; i < nbufs; ++i) MG_TRY(dev_alloc(bufs[i], (size_t)chunk * L.nvox * es));
    }
    const size_t nv = h->lev[h->L].nvox;
    MG_TRY(dev_alloc(&h->ml_jx, (size_t)h->ml_slots * chunk * nv * es));
    MG_TRY(dev_alloc(&h->ml_ux, (size_t)h->ml_slots * chunk * nv * es));
    if (ml_lagged(h)) MG_TRY(dev_alloc(&h->ml_jm, (size_t)h->ml_slots * chunk * nv * es));
    h->ml_chunk = chunk;
    return MG3D_OK;
}

// Device time (ms per launch) of `reps` multi-level sweeps of level k's first
// nc frequencies with shape (bands, rpb, threads); the opacity of those
// frequencies must be in place and the angle-sum buffers hold 2 x 12 / rpb
// slots.
// Checks a shifted-plane shape of the multi-level sweep on level k.
int ml_plane_shape_check(const mg3d_handle *h, int k, int bands, int rpb, int threads, int nf) {
    const Level &L = h->lev[k];
    if (h->moving || h->params.sc_interp || !L.psteps)
        return fail(MG3D_E_ARG, "the shifted-plane multi-level sweep takes static atmospheres "
                                "and the linear upwind interpolation");
    if (!plane_grid_ok(L.nx, L.ny, L.nz))
        return fail(MG3D_E_ARG, "grid too large for the shifted-plane multi-level sweep");
    if (bands < 1 || bands > kMaxBands || bands > L.ny)
        return fail(MG3D_E_ARG, "bands must be 1..16 and at most ny");
    const int rows = (L.ny + bands - 1) / bands;
    if ((long)(bands - 1) * rows >= L.ny) return fail(MG3D_E_ARG, "empty band");
    if (rpb < 1 || 12 % rpb) return fail(MG3D_E_ARG, "rays_per_block must divide 12");
    if (threads < 32 || threads > 512 || threads % 32)
        return fail(MG3D_E_ARG, "threads must be a multiple of 32 up to 512");
    if (nf != 1 && nf != 2 && nf != 4)
        return fail(MG3D_E_ARG, "freq_per_block must be 1, 2 or 4");
    if (nf > 1 && h->prec == MG3D_PREC_F64)
        return fail(MG3D_E_ARG, "the FP64 shifted-plane multi-level sweep takes one frequency "
                                "per block");
    if ((long)rows * L.nx > (long)ml_plane_max_pass(nf) * threads)
        return fail(MG3D_E_ARG, "too few threads for the band (at most " +
                                    std::to_string(ml_plane_max_pass(nf)) + " nodes per thread)");
    if (ml_plane_smem_bytes(h->prec, nf, rows, L.nx, rpb) > kMlPlaneMaxSmem)
        return fail(MG3D_E_ARG, "multi-level sweep shape exceeds shared memory");
    int n = 0;
    const cudaError_t e = ml_plane_active_clusters(h->prec, nf, bands, rows, L.nx, rpb,
                                                   std::min(h->ml_chunk, h->nfreq_ml), threads,
                                                   &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MG3D_E_ARG, std::string("multi-level sweep shape cannot be scheduled: ") +
                                    cudaGetErrorString(e));
    }
    if (n < 1) return fail(MG3D_E_ARG, "multi-level sweep shape cannot be scheduled");
    return MG3D_OK;
}

int time_ml_shape(mg3d_handle *h, int k, int bands, int rpb, int threads, int nc, int reps,
                  float *ms, int plane = 0, int nf = 1) {
    Level &L = h->lev[k];
    const int sb = L.ml_bands, sr = L.ml_rows, sp = L.ml_rpb, sth = L.ml_threads;
    L.ml_bands = bands;
    L.ml_rows = (L.ny + bands - 1) / bands;
    L.ml_rpb = rpb;
    L.ml_threads = threads;
    cudaEvent_t a = pool_event(h), b = pool_event(h);
    int rc = MG3D_OK;
    cudaError_t e = cudaEventRecord(a, h->stream);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        if (plane) {
            e = launch_ml_level_plane(h, L, nc, L.mib, bands, rpb, nf, threads);
        } else if (h->prec == MG3D_PREC_F64) {
            MlSweepArgs<double> sa{L.nx, L.ny, L.nz, nc, L.ml_rows,
                                   (const double *)L.mchi, (const double *)L.mS,
                                   (const double *)L.msc, (const double *)L.moc,
                                   (const double *)L.mib, L.geom, h->d_exp_tab, h->exp_l1,
                                   h->exp_l2, (double *)h->ml_jx, (double *)h->ml_ux, rpb,
                                   nullptr, (const double *)L.mdchi, (const double *)L.mdS,
                                   h->params.sc_interp, h->moving ? 1 : 0, 0,
                                   (const double *)h->d_vtab,
                                   (const double *)h->d_vtab + h->nfreq_ml, h->d_vline,
                                   (const double *)L.vnorm, (const double *)L.uproj,
                                   (const double *)L.dinv};
            e = launch_ml_sweep_f64(sa, bands, threads, h->stream);
        } else {
            MlSweepArgs<float> sa{L.nx, L.ny, L.nz, nc, L.ml_rows,
                                  (const float *)L.mchi, (const float *)L.mS,
                                  (const float *)L.msc, (const float *)L.moc,
                                  (const float *)L.mib, L.geom, h->d_exp_tab, h->exp_l1,
                                  h->exp_l2, (float *)h->ml_jx, (float *)h->ml_ux, rpb,
                                  nullptr, (const float *)L.mdchi, (const float *)L.mdS,
                                  h->params.sc_interp, h->moving ? 1 : 0, 0,
                                  (const float *)h->d_vtab,
                                  (const float *)h->d_vtab + h->nfreq_ml, h->d_vline,
                                  (const float *)L.vnorm, (const float *)L.uproj,
                                  (const float *)L.dinv};
            e = launch_ml_sweep_f32(sa, bands, threads, h->stream);
        }
        ++h->launches;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e != cudaSuccess)
        rc = fail(MG3D_E_CUDA, std::string("multi-level autotune: ") + cudaGetErrorString(e));
    else
        *ms /= (float)reps;
    h->event_pool.push_back(a);
    h->event_pool.push_back(b);
    L.ml_bands = sb;
    L.ml_rows = sr;
    L.ml_rpb = sp;
    L.ml_threads = sth;
    return rc;
}

// True when no multi-level sweep shape with two or more rays per block fits
// level k's plane in shared memory (a 256-wide FP64 plane): its candidates
// then take one ray per block, 24 ray-group slots.
bool ml_single_ray_only(const mg3d_handle *h, int k) {
    const Level &L = h->lev[k];
    for (int rpb : {12, 6, 4, 3, 2})
        for (int bands = 1; bands <= kPortableBands && bands <= L.ny; ++bands) {
            const int rows = (L.ny + bands - 1) / bands;
            if ((long)(bands - 1) * rows >= L.ny) continue;
            if (ml_sweep_smem_bytes(h->prec, rows, L.nx, rpb, h->params.sc_interp,
                                    h->moving ? 1 : 0) <= kMaxSweepSmem)
                return false;
        }
    return true;
}

// Times the multi-level sweep shapes of level k on its first nc frequencies
// (every band count, rays per block 12, 6, 4, 3 or 2, else 1, and 128/256/512 threads
// that fit; once each, the best six three more times) and keeps the fastest.
int autotune_ml_level(mg3d_handle *h, int k, int nc, int *evaluated) {
    Level &L = h->lev[k];
    MlOpacityArgs oa{L.nvox, nc, h->N, h->prec, h->d_fi, h->theta_ref, h->t_ref,
                     L.n, L.T, L.chi_c, L.saha, L.mchi, L.mS, L.msc, L.moc, 0,
                     h->d_exp_tab, h->exp_l1, h->exp_l2, nullptr, nullptr, h->moving ? 1 : 0,
                     nullptr, nullptr, h->d_voigt};
    MG_TRY(launched(h, launch_ml_opacity(oa, h->stream), "multi-level opacity"));
    if (h->params.sc_interp)
        MG_TRY(launched(h, launch_xslopes(h->prec, L.nx, (long)nc * L.nvox, L.mchi, L.mS, L.mdchi,
                                          L.mdS, h->stream),
                        "x-slopes"));
    struct Cand {
        int bands, rpb, threads, plane = 0, nf = 1;
    };
    std::vector<Cand> cands;
    // rays per block 1 only where no larger group fits (a 256-wide FP64 plane)
    for (int rpb : {12, 6, 4, 3, 2, 1})
        for (int bands = 1; bands <= kPortableBands && bands <= L.ny; ++bands) {
            const int rows = (L.ny + bands - 1) / bands;
            if ((long)(bands - 1) * rows >= L.ny) continue;
            if (rpb == 1 && !cands.empty()) break;
            if (ml_sweep_smem_bytes(h->prec, rows, L.nx, rpb, h->params.sc_interp,
                                    h->moving ? 1 : 0) > kMaxSweepSmem)
                continue;
            for (int th : {128, 256, 512}) {
                if (th > 128 && th / 2 >= rows * L.nx) continue;  // a smaller block covers it
                cands.push_back(Cand{bands, rpb, th});
            }
        }
    // shifted-plane shapes (static atmospheres, linear upwind interpolation)
    // whose ray-group slots the tuning buffers hold
    if (!h->moving && !h->params.sc_interp && L.psteps)
        for (int nf : {1, 2, 4})
            for (int rpb : {12, 6, 4, 3, 2, 1}) {
                if (2 * (12 / rpb) > h->ml_slots) continue;
                for (int bands = 1; bands <= kMaxBands && bands <= L.ny; ++bands) {
                    const int rows = (L.ny + bands - 1) / bands;
                    if ((long)(bands - 1) * rows >= L.ny) continue;
                    for (int th : {128, 256, 512}) {
                        if (th > 128 && th / 2 >= rows * L.nx) continue;
                        if (ml_plane_shape_check(h, k, bands, rpb, th, nf) != MG3D_OK) continue;
                        Cand c{bands, rpb, th};
                        c.plane = 1;
                        c.nf = nf;
                        cands.push_back(c);
                    }
                }
            }
    g_last_error.clear();
    if (cands.empty()) return fail(MG3D_E_ARG, "no multi-level sweep shape fits");
    float warm = 0.f;
    if (2 * (12 / L.ml_rpb) <= h->ml_slots)
        MG_TRY(time_ml_shape(h, k, L.ml_bands, L.ml_rpb, L.ml_threads, nc, 1, &warm, L.ml_plane,
                             L.ml_nf));
    std::vector<std::pair<float, size_t>> t1;
    for (size_t i = 0; i < cands.size(); ++i) {
        float ms = 0.f;
        MG_TRY(time_ml_shape(h, k, cands[i].bands, cands[i].rpb, cands[i].threads, nc, 1, &ms,
                             cands[i].plane, cands[i].nf));
        t1.push_back({ms, i});
    }
    std::sort(t1.begin(), t1.end());
    float best_ms = 1e30f;
    size_t best = t1[0].second;
    for (size_t j = 0; j < std::min<size_t>(6, t1.size()); ++j) {
        const Cand &c = cands[t1[j].second];
        float ms = 0.f;
        MG_TRY(time_ml_shape(h, k, c.bands, c.rpb, c.threads, nc, 3, &ms, c.plane, c.nf));
        if (ms < best_ms) {
            best_ms = ms;
            best = t1[j].second;
        }
    }
    L.ml_bands = cands[best].bands;
    L.ml_rows = (L.ny + L.ml_bands - 1) / L.ml_bands;
    L.ml_rpb = cands[best].rpb;
    L.ml_threads = cands[best].threads;
    L.ml_plane = cands[best].plane;
    L.ml_nf = cands[best].nf;
    if (evaluated) *evaluated = (int)cands.size();
    return MG3D_OK;
}

// Autotunes every level (or `level`) of a multi-level handle, then sizes the
// chunk buffers for the chosen shapes (the requested chunk, else the
// automatic one).
int autotune_ml(mg3d_handle *h, int level, int *evaluated) {
    MG_CUDA(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    // tuning buffers: the slots of the candidates (12 for two rays per block,
    // 24 where a level fits only one, or where the shifted-plane form applies:
    // wide planes take it with one ray per block), at most 32 frequencies
    // that fit
    h->ml_slots = 12;
    for (int k = 1; k <= h->L; ++k)
        if ((level == 0 || k == level) &&
            (ml_single_ray_only(h, k) || (!h->moving && !h->params.sc_interp && h->lev[k].psteps)))
            h->ml_slots = 24;
    MG_TRY(alloc_ml_chunks(h, 1));
    const int nc = std::min(32, default_ml_chunk(h));
    MG_TRY(alloc_ml_chunks(h, nc));
    int count = 0;
    for (int k = 1; k <= h->L; ++k) {
        if (level != 0 && k != level) continue;
        int c = 0;
        MG_TRY(autotune_ml_level(h, k, nc, &c));
        count += c;
    }
    h->ml_slots = 2;
    for (int k = 1; k <= h->L; ++k) h->ml_slots = std::max(h->ml_slots, 2 * (12 / h->lev[k].ml_rpb));
    MG_TRY(alloc_ml_chunks(h, 1));
    const int chunk = h->ml_chunk_req > 0 ? std::min(h->ml_chunk_req, h->nfreq_ml)
                                          : default_ml_chunk(h);
    MG_TRY(alloc_ml_chunks(h, chunk));
    if (evaluated) *evaluated = count;
    return MG3D_OK;
}

// Velocity field of a moving multi-level atmosphere: per frequency the line
// offset, weight and line index (lines numbered in transition order); the
// field on every grid (full weighting downward); per grid the projected
// velocities, 1/d and the inverse profile sums of every line and ray.
int setup_velocity_ml(mg3d_handle *h, const double *vel_host) {
    const int nf = h->nfreq_ml;
    const size_t es = elem_size(h->prec);
    std::vector<double> xw(2 * (size_t)nf, 0.0);
    std::vector<int> line(nf, -1);
    int nlines = 0;
    for (const TransInfo &t : h->ti) {
        if (t.kind != 0) continue;
        for (int f = t.f_begin; f < t.f_end; ++f) {
            xw[f] = h->fi[f].xy;
            xw[nf + f] = h->fi[f].w;
            line[f] = nlines;
        }
        ++nlines;
    }
    MG_TRY(dev_alloc(&h->d_vtab, 2 * (size_t)nf * es));
    if (h->prec == MG3D_PREC_F64) {
        MG_CUDA(cudaMemcpy(h->d_vtab, xw.data(), xw.size() * es, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f32(xw.begin(), xw.end());
        MG_CUDA(cudaMemcpy(h->d_vtab, f32.data(), f32.size() * es, cudaMemcpyHostToDevice));
    }
    MG_TRY(dev_alloc((void **)&h->d_vline, (size_t)nf * sizeof(int)));
    MG_CUDA(cudaMemcpy(h->d_vline, line.data(), (size_t)nf * sizeof(int), cudaMemcpyHostToDevice));
    for (int k = 1; k <= h->L; ++k) MG_TRY(dalloc(&h->lev[k].vel, 3 * (size_t)h->lev[k].nvox));
    Level &F = h->lev[h->L];
    MG_CUDA(cudaMemcpy(F.vel, vel_host, 3 * (size_t)F.nvox * sizeof(double),
                       cudaMemcpyHostToDevice));
    for (int k = h->L; k >= 2; --k) {
        Level &Fk = h->lev[k];
        MG_TRY(launched(h, launch_restrict(3, Fk.nx, Fk.ny, Fk.nz, Fk.vel, h->lev[k - 1].vel,
                                           h->stream),
                        "restrict velocity"));
    }
    double *dmu = nullptr;
    MG_TRY(dalloc(&dmu, 3 * (size_t)kRays));
    int rc = MG3D_OK;
    if (cudaMemcpy(dmu, h->mu, 3 * kRays * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(MG3D_E_CUDA, "velocity tables");
    for (int k = 1; k <= h->L && rc == MG3D_OK; ++k) {
        Level &L = h->lev[k];
        rc = dev_alloc(&L.uproj, (size_t)kRays * L.nvox * es);
        if (rc == MG3D_OK) rc = dev_alloc(&L.dinv, (size_t)L.nvox * es);
        if (rc == MG3D_OK)
            rc = dev_alloc(&L.vnorm, (size_t)std::max(1, nlines) * kRays * L.nvox * es);
        if (rc == MG3D_OK)
            rc = launched(h, launch_ml_vel_prep(h->prec, L.nvox, h->ntrans, h->d_ti, h->d_fi, dmu,
                                                L.vel, L.T, h->t_ref, L.uproj, L.dinv, L.vnorm,
                                                h->stream),
                          "velocity projection");
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && rc == MG3D_OK)
        rc = fail(MG3D_E_CUDA, "velocity set-up");
    cudaFree(dmu);
    return rc;
}

// Partial redistribution of multi-level lines: the PRD line table (each
// line's frequencies sorted by |x|, mirror offsets adjacent, grouped by equal
// |x|), each frequency's row of the rho arrays, and per grid the symmetric
// scaling of R at every node's Doppler width (fixed for the handle: it
// depends on the temperature only) and rho = 1 until the first formal
// solution.
int setup_ml_prd(mg3d_handle *h, const mg3d_ml_atom *atom) {
    std::vector<PrdLine> pl;
    std::vector<int> ord, grp, index(h->nfreq_ml, -1);
    int pf = 0;
    for (int t = 0; t < atom->n_lines; ++t) {
        const mg3d_line &ln = atom->lines[t];
        if (!(ln.gamma_prd > 0.0)) continue;
        const TransInfo &tr = h->ti[t];
        PrdLine L{};
        L.lo = ln.lower;
        L.up = ln.upper;
        L.f_begin = tr.f_begin;
        L.f_end = tr.f_end;
        L.pf0 = pf;
        L.nf = tr.f_end - tr.f_begin;
        L.ord0 = (int)ord.size();
        L.grp0 = (int)grp.size();
        L.gamma = ln.gamma_prd;
        L.gr = tr.gr;
        L.b_ul = tr.coef / (tr.rho * tr.rho * tr.rho);
        std::vector<int> fs;
        for (int f = tr.f_begin; f < tr.f_end; ++f) {
            fs.push_back(f);
            index[f] = pf + (f - tr.f_begin);
        }
        std::stable_sort(fs.begin(), fs.end(), [&](int a, int b) {
            return std::fabs(h->fi[a].xy) < std::fabs(h->fi[b].xy);
        });
        for (int i = 0; i < L.nf; ++i) {
            if (i == 0 || std::fabs(h->fi[fs[i]].xy) != std::fabs(h->fi[fs[i - 1]].xy))
                grp.push_back(i);
            ord.push_back(fs[i]);
        }
        L.ngrp = (int)grp.size() - L.grp0;
        grp.push_back(L.nf);   // end of the last group
        pl.push_back(L);
        pf += L.nf;
    }
    h->n_prd = (int)pl.size();
    h->n_prd_freq = pf;
    MG_TRY(dev_alloc((void **)&h->d_prd, pl.size() * sizeof(PrdLine)));
    MG_TRY(dev_alloc((void **)&h->d_prd_ord, ord.size() * sizeof(int)));
    MG_TRY(dev_alloc((void **)&h->d_prd_grp, grp.size() * sizeof(int)));
    MG_TRY(dev_alloc((void **)&h->d_prd_index, index.size() * sizeof(int)));
    MG_CUDA(cudaMemcpy(h->d_prd, pl.data(), pl.size() * sizeof(PrdLine), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(h->d_prd_ord, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(h->d_prd_grp, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(h->d_prd_index, index.data(), index.size() * sizeof(int),
                       cudaMemcpyHostToDevice));
    h->prd_index = index;
    std::vector<double> ones;
    for (int k = 1; k <= h->L; ++k) {
        Level &L = h->lev[k];
        MG_TRY(dalloc(&L.prd_c, (size_t)pf * L.nvox));
        MG_TRY(dalloc(&L.prd_rho, (size_t)pf * L.nvox));
        MG_TRY(dalloc(&L.prd_oc, (size_t)pf * L.nvox));
        MG_CUDA(cudaMemset(L.prd_oc, 0, (size_t)pf * L.nvox * sizeof(double)));
        ones.assign((size_t)pf * L.nvox, 1.0);
        MG_CUDA(cudaMemcpy(L.prd_rho, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice));
        MG_TRY(launched(h, launch_ml_prd_scale(L.nvox, h->n_prd, h->d_prd, h->d_fi, h->d_prd_ord,
                                               h->d_prd_grp, h->t_ref, L.T, L.prd_c, h->stream),
                        "partial redistribution scaling"));
    }
    return MG3D_OK;
}

int create_ml_impl(const mg3d_ml_atmosphere *atm, const mg3d_ml_atom *atom,
                   const mg3d_quadrature *quad, const mg3d_params *params, mg3d_handle *h) {
    h->kind = 1;
    h->N = atom->n_levels;
    h->L = params->n_grids;
    h->prec = params->fs_prec;
    h->params = *params;
    h->moving = atm->vel != nullptr;
    h->theta_ref = atom->theta_ref;
    h->t_ref = atom->t_ref;
    for (int t = 0; t < atom->n_lines; ++t) h->ml_prd = h->ml_prd || atom->lines[t].gamma_prd > 0.0;
    for (int t = 0; t < atom->n_lines; ++t)
        if (atom->lines[t].a_damp > 0.0 && !h->d_voigt) {
            // damped lines: the opacity step and the radiative sums evaluate
            // the Voigt function per node and frequency
            MG_TRY(dev_alloc((void **)&h->d_voigt, sizeof(VoigtTable)));
            MG_CUDA(cudaMemcpy(h->d_voigt, &voigt_coefficients(), sizeof(VoigtTable),
                               cudaMemcpyHostToDevice));
        }
    build_quadrature(h, quad ? quad->a : 0.0);
    const int N = h->N;
    // frequency table: lines, then continua, each transition contiguous
    for (int t = 0; t < atom->n_lines; ++t) {
        const mg3d_line &ln = atom->lines[t];
        std::vector<double> x, w;
        trapezoid_grid(-ln.x_max, ln.x_max, ln.n_freq, x, w);
        if (ln.n_freq == 1) x[0] = 0.0;
        TransInfo tr{0, ln.lower, ln.upper, (int)h->fi.size(), 0, ln.rho, ln.a_ul,
                     atom->g[ln.upper] / atom->g[ln.lower]};
        for (int i = 0; i < ln.n_freq; ++i)
            h->fi.push_back(
                FreqInfo{0, ln.lower, ln.upper, x[i], w[i], ln.rho, ln.kappa, tr.gr, ln.a_damp});
        tr.f_end = (int)h->fi.size();
        h->ti.push_back(tr);
    }
    for (int t = 0; t < atom->n_continua; ++t) {
        const mg3d_continuum &ct = atom->continua[t];
        std::vector<double> y, w;
        trapezoid_grid(1.0, ct.y_max, ct.n_freq, y, w);
        if (ct.n_freq == 1) y[0] = 1.0;
        TransInfo tr{1, ct.lower, N - 1, (int)h->fi.size(), 0, ct.rho, ct.beta, 1.0};
        for (int i = 0; i < ct.n_freq; ++i)
            h->fi.push_back(FreqInfo{1, ct.lower, N - 1, y[i], w[i], ct.rho, ct.kappa, 1.0});
        tr.f_end = (int)h->fi.size();
        h->ti.push_back(tr);
    }
    h->nfreq_ml = (int)h->fi.size();
    h->ntrans = (int)h->ti.size();
    MG_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    const size_t es = elem_size(h->prec);
    const int nf = h->nfreq_ml;
    for (int k = h->L; k >= 1; --k) {
        Level &L = h->lev[k];
        if (k == h->L) {
            L.nx = atm->nx;
            L.ny = atm->ny;
            L.nz = atm->nz;
            L.dx = atm->dx;
            L.dy = atm->dy;
            L.z.assign(atm->z, atm->z + atm->nz);
        } else {
            const Level &Fn = h->lev[k + 1];
            L.nx = Fn.nx / 2;
            L.ny = Fn.ny / 2;
            L.nz = (Fn.nz + 1) / 2;
            L.dx = 2 * Fn.dx;
            L.dy = 2 * Fn.dy;
            L.z.clear();
            for (int i = 0; i < Fn.nz; i += 2) L.z.push_back(Fn.z[i]);
        }
        L.nplane = (long)L.nx * L.ny;
        L.nvox = L.nplane * L.nz;
        MG_TRY(dalloc(&L.T, L.nvox));
        MG_TRY(dalloc(&L.n_tot, L.nvox));
        MG_TRY(dalloc(&L.chi_c, L.nvox));
        MG_TRY(dalloc(&L.cmat, (size_t)N * N * L.nvox));
        MG_TRY(dalloc(&L.saha, (size_t)N * L.nvox));
        MG_TRY(dalloc(&L.tz, L.nz));
        MG_TRY(dalloc(&L.n, (size_t)N * L.nvox));
        MG_TRY(dalloc(&L.f, (size_t)N * L.nvox));
        MG_TRY(dalloc(&L.n_before, (size_t)N * L.nvox));
        MG_TRY(dalloc(&L.r, (size_t)N * L.nvox));
        MG_TRY(dev_alloc(&L.mib, (size_t)nf * L.nplane * es));
        MG_TRY(dalloc(&L.geom, (size_t)kRays * L.nz));
        std::vector<double> tz(L.nz, 0.0);
        for (int i = 1; i + 1 < L.nz; i += 2) tz[i] = (L.z[i] - L.z[i - 1]) / (L.z[i + 1] - L.z[i - 1]);
        MG_CUDA(cudaMemcpy(L.tz, tz.data(), L.nz * sizeof(double), cudaMemcpyHostToDevice));
        MG_TRY(dalloc(&L.zf, L.nz));
        MG_CUDA(cudaMemcpy(L.zf, L.z.data(), L.nz * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<StepGeom> g;
        build_geometry(h, L, g);
        MG_CUDA(cudaMemcpy(L.geom, g.data(), g.size() * sizeof(StepGeom), cudaMemcpyHostToDevice));
        // per-step constants of the shifted-plane form (static, linear upwind)
        if (!atm->vel && !params->sc_interp) {
            if (h->prec == MG3D_PREC_F64) {
                const auto ps = plane_steps<double>(L, g);
                MG_TRY(dev_alloc(&L.psteps, ps.size() * sizeof(ps[0])));
                MG_CUDA(cudaMemcpy(L.psteps, ps.data(), ps.size() * sizeof(ps[0]),
                                   cudaMemcpyHostToDevice));
            } else {
                const auto ps = plane_steps<float>(L, g);
                MG_TRY(dev_alloc(&L.psteps, ps.size() * sizeof(ps[0])));
                MG_CUDA(cudaMemcpy(L.psteps, ps.data(), ps.size() * sizeof(ps[0]),
                                   cudaMemcpyHostToDevice));
            }
        }
        // rays per block: all 12 of a hemisphere if some band count fits in
        // shared memory, else the largest divisor of 12 that does; bands: the
        // fewest that fit and give >= 300 blocks, else the most that fit
        int pick = 0;
        for (int rpb : {12, 6, 4, 3, 2, 1}) {
            for (int b = 1; b <= kPortableBands && b <= L.ny; ++b) {
                const int rows = (L.ny + b - 1) / b;
                if ((long)(b - 1) * rows >= L.ny) continue;
                if (ml_sweep_smem_bytes(h->prec, rows, L.nx, rpb, params->sc_interp,
                                        atm->vel ? 1 : 0) > kMaxSweepSmem)
                    continue;
                pick = b;
                if (2L * (12 / rpb) * nf * b >= 300) break;
            }
            if (pick) {
                L.ml_rpb = rpb;
                h->ml_slots = std::max(h->ml_slots, 2 * (12 / rpb));
                break;
            }
        }
        if (pick == 0) return fail(MG3D_E_ARG, "plane too large for the multi-level sweep");
        L.ml_bands = pick;
        L.ml_rows = (L.ny + pick - 1) / pick;
        const int th = threads_for_band(L.ml_rows * L.nx);
        L.ml_threads = th > 256 ? 256 : th;
    }
    Level &F = h->lev[h->L];
    const size_t nfld = 3 + (size_t)N * N + N;   // T, n_tot, chi_c, c, saha
    MG_CUDA(cudaMemcpy(F.T, atm->T, F.nvox * 8, cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(F.n_tot, atm->n_tot, F.nvox * 8, cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(F.chi_c, atm->chi_c, F.nvox * 8, cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(F.cmat, atm->c, (size_t)N * N * F.nvox * 8, cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(F.saha, atm->saha, (size_t)N * F.nvox * 8, cudaMemcpyHostToDevice));
    const size_t scratch_fields = std::max<size_t>(4, (size_t)N + 2);
    MG_TRY(dalloc(&h->scratch, scratch_fields * F.nvox));
    if (h->L > 1) {
        // full weighting of every atmospheric field, grid by grid (Sec. 4.7)
        double *pack = nullptr;
        MG_TRY(dalloc(&pack, nfld * (F.nvox + h->lev[h->L - 1].nvox)));
        int rc = MG3D_OK;
        for (int k = h->L; k >= 2 && rc == MG3D_OK; --k) {
            Level &Fk = h->lev[k];
            Level &Ck = h->lev[k - 1];
            double *fine = pack, *coarse = pack + nfld * Fk.nvox;
            const double *src[3] = {Fk.T, Fk.n_tot, Fk.chi_c};
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                e = cudaMemcpyAsync(fine + i * Fk.nvox, src[i], Fk.nvox * 8,
                                    cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(fine + 3 * Fk.nvox, Fk.cmat, (size_t)N * N * Fk.nvox * 8,
                                    cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(fine + (3 + (size_t)N * N) * Fk.nvox, Fk.saha,
                                    (size_t)N * Fk.nvox * 8, cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess) {
                rc = launched(h, launch_restrict((int)nfld, Fk.nx, Fk.ny, Fk.nz, fine, coarse,
                                                 h->stream),
                              "restrict atmosphere");
                if (rc != MG3D_OK) break;
            }
            double *dst[3] = {Ck.T, Ck.n_tot, Ck.chi_c};
            for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                e = cudaMemcpyAsync(dst[i], coarse + i * Ck.nvox, Ck.nvox * 8,
                                    cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(Ck.cmat, coarse + 3 * Ck.nvox, (size_t)N * N * Ck.nvox * 8,
                                    cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(Ck.saha, coarse + (3 + (size_t)N * N) * Ck.nvox,
                                    (size_t)N * Ck.nvox * 8, cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) rc = fail(MG3D_E_CUDA, std::string("coarsening: ") +
                                                             cudaGetErrorString(e));
        }
        cudaFree(pack);
        if (rc != MG3D_OK) return rc;
    }
    MG_TRY(dev_alloc((void **)&h->d_fi, h->fi.size() * sizeof(FreqInfo)));
    MG_TRY(dev_alloc((void **)&h->d_ti, h->ti.size() * sizeof(TransInfo)));
    MG_CUDA(cudaMemcpy(h->d_fi, h->fi.data(), h->fi.size() * sizeof(FreqInfo),
                       cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(h->d_ti, h->ti.data(), h->ti.size() * sizeof(TransInfo),
                       cudaMemcpyHostToDevice));
    for (int k = 1; k <= h->L; ++k) {
        Level &L = h->lev[k];
        MG_TRY(launched(h, launch_ml_bottom(h->prec, L.nplane, nf, h->d_fi, h->theta_ref, L.T,
                                            L.mib, h->stream),
                        "bottom intensity"));
    }
    {
        double tab[kExpTab];
        exp_neg_constants(tab, &h->exp_l1, &h->exp_l2);
        MG_TRY(dalloc(&h->d_exp_tab, kExpTab));
        MG_CUDA(cudaMemcpy(h->d_exp_tab, tab, sizeof(tab), cudaMemcpyHostToDevice));
    }
    if (atm->sigma_c) {
        for (long i = 0; i < F.nvox && !h->scatter; ++i) h->scatter = atm->sigma_c[i] > 0.0;
        for (long i = 0; i < F.nvox; ++i)
            if (!(atm->sigma_c[i] >= 0.0)) return fail(MG3D_E_ARG, "negative sigma_c");
    }
    if (h->ml_prd && !h->scatter)
        for (int k = 1; k <= h->L; ++k) {
            Level &L = h->lev[k];
            MG_TRY(dev_alloc(&L.jbg, (size_t)nf * L.nvox * elem_size(h->prec)));
            MG_CUDA(cudaMemset(L.jbg, 0, (size_t)nf * L.nvox * elem_size(h->prec)));
        }
    if (h->ml_prd) MG_TRY(setup_ml_prd(h, atom));
    if (h->scatter) {
        for (int k = 1; k <= h->L; ++k) {
            Level &L = h->lev[k];
            MG_TRY(dalloc(&L.sigma_c, L.nvox));
            MG_TRY(dev_alloc(&L.jbg, (size_t)nf * L.nvox * elem_size(h->prec)));
            MG_CUDA(cudaMemset(L.jbg, 0, (size_t)nf * L.nvox * elem_size(h->prec)));
        }
        MG_CUDA(cudaMemcpy(F.sigma_c, atm->sigma_c, F.nvox * 8, cudaMemcpyHostToDevice));
        for (int k = h->L; k >= 2; --k)   // full weighting, like the atmosphere (Sec. 4.7)
            MG_TRY(launched(h, launch_restrict(1, h->lev[k].nx, h->lev[k].ny, h->lev[k].nz,
                                               h->lev[k].sigma_c, h->lev[k - 1].sigma_c,
                                               h->stream),
                            "restrict scattering"));
    }
    if (h->moving) MG_TRY(setup_velocity_ml(h, atm->vel));
    MG_TRY(dalloc(&h->ml_acc, (size_t)h->ntrans * kAccTerms * F.nvox));
    if (params && params->ml_chunk < 0) return fail(MG3D_E_ARG, "negative ml_chunk");
    h->ml_chunk_req = params ? params->ml_chunk : 0;
    MG_TRY(alloc_ml_chunks(h, params && params->ml_chunk > 0
                                  ? std::min(params->ml_chunk, h->nfreq_ml)
                                  : default_ml_chunk(h)));
    MG_TRY(dalloc(&h->scal, kScalStatus + 1));
    MG_CUDA(cudaMemset(h->scal, 0, (kScalStatus + 1) * sizeof(unsigned long long)));
    for (int k = 1; k <= h->L; ++k) MG_TRY(zero_radiation(h, k));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return MG3D_OK;
}

// ------------------------------------------------------------------- batches

}  // namespace

struct mg3d_batch {
    int n = 0, L = 0, prec = 0;
    mg3d_params params{};
    std::vector<mg3d_handle *> m;
    cudaStream_t stream = nullptr;
    struct KindLevel {
        std::vector<int> members;          // batch indices of this kind
        int n_items = 0, bands = 0, threads = 0;
        size_t smem = 0;
        BatchItem *d_items = nullptr;
        void *d_args = nullptr;
    } two[MG3D_MAX_GRIDS + 1], ml[MG3D_MAX_GRIDS + 1];
    // multi-level members: one sweep table per chunk index c, covering the
    // members that have a chunk c (each member's own chunk size)
    std::vector<KindLevel> mlc[MG3D_MAX_GRIDS + 1];
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long long launches = 0, delta_launches[2] = {0, 0};
    double fs_units = 0, delta_units[2] = {0, 0};
    // per member and level: sweeps and formal solutions one replay performs
    std::vector<std::vector<int>> delta_sweeps[2], delta_fss[2];
};

namespace {

int batch_launched(mg3d_batch *b, cudaError_t e, const char *what) {
    ++b->launches;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(MG3D_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return MG3D_OK;
}

// Radiative sums of a multi-level member on level k: the chunk f0 .. f0+nc-1
// of its angle sums added (clear: start from zero), or, for zero radiation,
// all frequencies with J = 0 and U = 1.
int batch_ml_sums(mg3d_batch *b, mg3d_handle *h, int k, int f0, int nc, bool zero_rad,
                  bool clear) {
    const Level &L = h->lev[k];
    if (clear)
        MG_CUDA(cudaMemsetAsync(h->ml_acc, 0,
                                (size_t)h->ntrans * kAccTerms * L.nvox * sizeof(double),
                                b->stream));
    MlAccumArgs a{L.nvox, f0, nc, h->ntrans, h->prec, h->d_fi, h->d_ti, h->theta_ref,
                  h->t_ref, L.T, h->ml_jx, h->ml_ux, 2 * (12 / L.ml_rpb), zero_rad ? 1 : 0,
                  h->ml_acc, h->d_exp_tab, h->exp_l1, h->exp_l2};
    return batch_launched(b, launch_ml_accum(a, b->stream), "batch radiative sums");
}

int ml_chunks(const mg3d_handle *h) { return (h->nfreq_ml + h->ml_chunk - 1) / h->ml_chunk; }

// Formal solution of level k for every member: per-member opacity, then one
// batched sweep launch per atom kind (per frequency chunk for multi-level
// members, each chunk followed by the members' radiative sums).
int batch_fs(mg3d_batch *b, int k) {
    for (mg3d_handle *h : b->m) {
        Level &L = h->lev[k];
        if (h->kind == 1) {
            b->fs_units += (double)L.nvox * kRays * h->nfreq_ml;
        } else {
            MG_TRY(batch_launched(b, launch_opacity(h->prec, L.nvox, h->atom.g_ratio,
                                                    h->atom.kappa, L.n, L.chi0, L.S, b->stream),
                                  "batch opacity"));
            b->fs_units += (double)L.nvox * kRays * h->atom.n_freq;
        }
        ++h->fss[k];
    }
    mg3d_batch::KindLevel &t = b->two[k];
    if (t.n_items)
        MG_TRY(batch_launched(b, launch_sweep_batch(b->prec, t.d_args, t.d_items, t.n_items,
                                                    t.bands, t.threads, t.smem, b->stream),
                              "batched sweep"));
    for (size_t c = 0; c < b->mlc[k].size(); ++c) {
        for (int i : b->ml[k].members) {
            mg3d_handle *h = b->m[i];
            if ((int)c >= ml_chunks(h)) continue;
            Level &L = h->lev[k];
            const int f0 = (int)c * h->ml_chunk, nc = std::min(h->ml_chunk, h->nfreq_ml - f0);
            MlOpacityArgs oa{L.nvox, nc, h->N, h->prec, h->d_fi, h->theta_ref, h->t_ref,
                             L.n, L.T, L.chi_c, L.saha, L.mchi, L.mS, L.msc, L.moc, f0,
                             h->d_exp_tab, h->exp_l1, h->exp_l2};
            MG_TRY(batch_launched(b, launch_ml_opacity(oa, b->stream), "batch opacity"));
        }
        mg3d_batch::KindLevel &q = b->mlc[k][c];
        if (q.n_items)
            MG_TRY(batch_launched(b, launch_ml_sweep_batch(b->prec, q.d_args, q.d_items,
                                                           q.n_items, q.bands, q.threads, q.smem,
                                                           b->stream),
                                  "batched multi-level sweep"));
        for (int i : b->ml[k].members) {
            mg3d_handle *h = b->m[i];
            if ((int)c >= ml_chunks(h)) continue;
            const int f0 = (int)c * h->ml_chunk, nc = std::min(h->ml_chunk, h->nfreq_ml - f0);
            MG_TRY(batch_ml_sums(b, h, k, f0, nc, false, c == 0));
        }
    }
    return MG3D_OK;
}

int member_rates(mg3d_batch *b, mg3d_handle *h, int k, int mode, double *out, bool zero_rad,
                 unsigned long long *scal) {
    if (h->kind == 1) {
        if (zero_rad) MG_TRY(batch_ml_sums(b, h, k, 0, h->nfreq_ml, true, true));
        MlRateArgs a = ml_rate_args(h, k, mode);
        a.out = out;
        a.scal = scal;
        return batch_launched(b, launch_ml_rates(a, b->stream), "batch rates");
    }
    RateArgs a = rate_args(h, k, mode);
    a.out = out;
    a.zero_radiation = zero_rad;
    a.scal = scal;
    return batch_launched(b, launch_rates(a, b->stream), "batch rates");
}

int batch_sweep(mg3d_batch *b, int k) {
    MG_TRY(batch_fs(b, k));
    for (mg3d_handle *h : b->m) {
        MG_TRY(member_rates(b, h, k, kRateSolve, nullptr, false, h->scal));
        ++h->sweeps[k];
    }
    return MG3D_OK;
}

int batch_vcycle(mg3d_batch *b, int k, bool first) {
    const int nu_pre = (first && k == b->L) ? b->params.nu0 : b->params.nu1;
    for (int i = 0; i < nu_pre; ++i) MG_TRY(batch_sweep(b, k));
    MG_TRY(batch_fs(b, k));
    for (mg3d_handle *h : b->m)
        MG_TRY(member_rates(b, h, k, kRateResidual, h->lev[k].r, false, nullptr));
    for (mg3d_handle *h : b->m) {
        Level &F = h->lev[k];
        Level &C = h->lev[k - 1];
        MG_TRY(batch_launched(b, launch_restrict(h->N, F.nx, F.ny, F.nz, F.n, C.n, b->stream,
                                                 h->params.restriction),
                              "restrict n"));
        MG_CUDA(cudaMemcpyAsync(C.n_before, C.n, (size_t)h->N * C.nvox * sizeof(double),
                                cudaMemcpyDeviceToDevice, b->stream));
        MG_TRY(batch_launched(b, launch_restrict(h->N, F.nx, F.ny, F.nz, F.r, C.f, b->stream,
                                                 h->params.restriction),
                              "restrict r"));
        C.f_default = false;
    }
    MG_TRY(batch_fs(b, k - 1));
    for (mg3d_handle *h : b->m)
        MG_TRY(member_rates(b, h, k - 1, kRateAddW, h->lev[k - 1].f, false, nullptr));
    if (k - 1 == 1) {
        for (int i = 0; i < b->params.nu3; ++i) MG_TRY(batch_sweep(b, 1));
    } else {
        MG_TRY(batch_vcycle(b, k - 1, false));
    }
    for (mg3d_handle *h : b->m) {
        Level &F = h->lev[k];
        Level &C = h->lev[k - 1];
        MG_TRY(batch_launched(b, launch_prolong_correct(h->params.interpolation, h->N, C.nx, C.ny,
                                                        C.nz, F.tz, F.zf, C.n, C.n_before, F.n,
                                                        h->scal, b->stream),
                              "prolong correction"));
        if (h->params.interpolation) ++b->launches;
    }
    for (int i = 0; i < b->params.nu2; ++i) MG_TRY(batch_sweep(b, k));
    return MG3D_OK;
}

int batch_cycle_work(mg3d_batch *b, bool first) {
    for (mg3d_handle *h : b->m) {
        Level &F = h->lev[h->L];
        MG_CUDA(cudaMemcpyAsync(h->scratch, F.n, (size_t)h->N * F.nvox * sizeof(double),
                                cudaMemcpyDeviceToDevice, b->stream));
        F.f_default = true;
        MG_CUDA(cudaMemsetAsync(h->scal, 0, 8 * sizeof(unsigned long long), b->stream));
    }
    MG_TRY(batch_vcycle(b, b->L, first));
    for (mg3d_handle *h : b->m) {
        Level &F = h->lev[h->L];
        MG_TRY(batch_launched(b, launch_max_rel_change((long)h->N * F.nvox, F.n, h->scratch,
                                                       h->scal + 4, b->stream),
                              "max rel change"));
    }
    return MG3D_OK;
}

void batch_drop_graphs(mg3d_batch *b) {
    for (auto &g : b->exec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// One batched V-cycle (captured once per variant, then replayed); C per
// member into C[i] and the 10 % rule counts into neg[i].
int batch_cycle(mg3d_batch *b, bool first, double *C, long long *neg) {
    const int idx = first ? 1 : 0;
    if (!b->exec[idx]) {
        const long long l0 = b->launches;
        const double u0 = b->fs_units;
        std::vector<std::vector<int>> sw0(b->n), fs0(b->n);
        for (int i = 0; i < b->n; ++i) {
            sw0[i].assign(b->m[i]->sweeps, b->m[i]->sweeps + MG3D_MAX_GRIDS + 1);
            fs0[i].assign(b->m[i]->fss, b->m[i]->fss + MG3D_MAX_GRIDS + 1);
        }
        MG_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        int rc = batch_cycle_work(b, first);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (rc != MG3D_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(MG3D_E_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec[idx], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return fail(MG3D_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->delta_launches[idx] = b->launches - l0;
        b->delta_units[idx] = b->fs_units - u0;
        b->launches = l0;
        b->fs_units = u0;
        b->delta_sweeps[idx].assign(b->n, std::vector<int>(MG3D_MAX_GRIDS + 1, 0));
        b->delta_fss[idx].assign(b->n, std::vector<int>(MG3D_MAX_GRIDS + 1, 0));
        for (int i = 0; i < b->n; ++i)
            for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) {
                b->delta_sweeps[idx][i][k] = b->m[i]->sweeps[k] - sw0[i][k];
                b->delta_fss[idx][i][k] = b->m[i]->fss[k] - fs0[i][k];
                b->m[i]->sweeps[k] = sw0[i][k];
                b->m[i]->fss[k] = fs0[i][k];
            }
    }
    MG_CUDA(cudaGraphLaunch(b->exec[idx], b->stream));
    b->launches += b->delta_launches[idx];
    b->fs_units += b->delta_units[idx];
    for (int i = 0; i < b->n; ++i)
        for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) {
            b->m[i]->sweeps[k] += b->delta_sweeps[idx][i][k];
            b->m[i]->fss[k] += b->delta_fss[idx][i][k];
        }
    MG_CUDA(cudaStreamSynchronize(b->stream));
    bool bad = false;
    for (int i = 0; i < b->n; ++i) {
        unsigned long long sc[8];
        MG_CUDA(cudaMemcpy(sc, b->m[i]->scal, sizeof(sc), cudaMemcpyDeviceToHost));
        if (C) std::memcpy(&C[i], &sc[4], sizeof(double));
        if (neg) neg[i] = (long long)sc[3];
        if (sc[6]) bad = true;
    }
    if (bad) return fail(MG3D_E_DIVERGED, "non-finite populations after a batched V-cycle");
    return MG3D_OK;
}

// Launch tables of level k: common bands and block size per kind, each
// member's frequency grouping chosen to fit.
int batch_build_level(mg3d_batch *b, int k) {
    // two-level members
    {
        mg3d_batch::KindLevel &t = b->two[k];
        int bands = kPortableBands;
        for (int i : t.members) {
            const Level &L = b->m[i]->lev[k];
            int bmax = 0;
            for (int bb = 1; bb <= kPortableBands && bb <= L.ny; ++bb) {
                const int rows = (L.ny + bb - 1) / bb;
                if ((long)(bb - 1) * rows < L.ny) bmax = bb;
            }
            bands = std::min(bands, bmax);
        }
        std::vector<BatchItem> items;
        std::vector<unsigned char> args;
        const size_t asz = b->prec == MG3D_PREC_F64 ? sizeof(SweepArgs<double>)
                                                    : sizeof(SweepArgs<float>);
        int threads = 32;
        size_t smem = 0;
        for (size_t j = 0; j < t.members.size(); ++j) {
            mg3d_handle *h = b->m[t.members[j]];
            Level &L = h->lev[k];
            const int nf = h->atom.n_freq;
            SweepShape s{};
            for (int ng = std::min(nf, 3); ng >= 1; --ng) {
                SweepShape c{ng, (nf + ng - 1) / ng, bands, (L.ny + bands - 1) / bands, 0};
                if (sweep_smem_bytes(h->prec, c, L.nx) <= kMaxSweepSmem) {
                    s = c;
                    break;
                }
            }
            if (s.ng == 0) return fail(MG3D_E_ARG, "batch member plane too large for the sweep");
            s.threads = std::min(256, threads_for_band(s.rows * L.nx));
            threads = std::max(threads, s.threads);
            smem = std::max(smem, sweep_smem_bytes(h->prec, s, L.nx));
            // partial buffers were sized for every level's shape before any
            // table was built (see mg3d_batch_create)
            if ((size_t)kRays * s.ngroups * (size_t)L.nvox > h->partial_elems)
                return fail(MG3D_E_STATE, "batch member partial buffers too small");
            L.shape = s;
            drop_graphs(h);
            for (int r = 0; r < kRays; ++r)
                for (int g = 0; g < s.ngroups; ++g) items.push_back(BatchItem{(int)j, r, g});
            args.resize(args.size() + asz);
            unsigned char *dst = args.data() + args.size() - asz;
            if (b->prec == MG3D_PREC_F64) {
                const SweepArgs<double> a = sweep_args<double>(h, L, s);
                std::memcpy(dst, &a, asz);
            } else {
                const SweepArgs<float> a = sweep_args<float>(h, L, s);
                std::memcpy(dst, &a, asz);
            }
        }
        if (items.size() > 65535) return fail(MG3D_E_ARG, "batch too large for one launch");
        t.n_items = (int)items.size();
        t.bands = bands;
        t.threads = threads;
        t.smem = smem;
        if (t.n_items) {
            MG_TRY(dev_alloc((void **)&t.d_items, items.size() * sizeof(BatchItem)));
            MG_TRY(dev_alloc(&t.d_args, args.size()));
            MG_CUDA(cudaMemcpy(t.d_items, items.data(), items.size() * sizeof(BatchItem),
                               cudaMemcpyHostToDevice));
            MG_CUDA(cudaMemcpy(t.d_args, args.data(), args.size(), cudaMemcpyHostToDevice));
        }
    }
    // multi-level members
    {
        mg3d_batch::KindLevel &q = b->ml[k];
        int bands = 0;
        for (int bb = kPortableBands; bb >= 1 && !bands && !q.members.empty(); --bb) {
            bool ok = true;
            for (int i : q.members) {
                const Level &L = b->m[i]->lev[k];
                const int rows = (L.ny + bb - 1) / bb;
                if (bb > L.ny || (long)(bb - 1) * rows >= L.ny ||
                    ml_sweep_smem_bytes(b->prec, rows, L.nx, L.ml_rpb) > kMaxSweepSmem)
                    ok = false;
            }
            if (ok) bands = bb;
        }
        if (!q.members.empty() && !bands)
            return fail(MG3D_E_ARG, "multi-level batch members need a common band count");
        const size_t asz = b->prec == MG3D_PREC_F64 ? sizeof(MlSweepArgs<double>)
                                                    : sizeof(MlSweepArgs<float>);
        int threads = 32, chunks = 0;
        size_t smem = 0;
        for (int i : q.members) {
            mg3d_handle *h = b->m[i];
            Level &L = h->lev[k];
            const int rows = (L.ny + bands - 1) / bands;
            L.ml_bands = bands;
            L.ml_rows = rows;
            L.ml_threads = std::min(256, threads_for_band(rows * L.nx));
            threads = std::max(threads, L.ml_threads);
            smem = std::max(smem, ml_sweep_smem_bytes(h->prec, rows, L.nx, L.ml_rpb));
            chunks = std::max(chunks, ml_chunks(h));
            drop_graphs(h);
        }
        b->mlc[k].assign(chunks, mg3d_batch::KindLevel{});
        for (int c = 0; c < chunks; ++c) {
            std::vector<BatchItem> items;
            std::vector<unsigned char> args;
            int j = 0;
            for (int i : q.members) {
                mg3d_handle *h = b->m[i];
                if (c >= ml_chunks(h)) continue;
                Level &L = h->lev[k];
                const int f0 = c * h->ml_chunk, nc = std::min(h->ml_chunk, h->nfreq_ml - f0);
                for (int slot = 0; slot < 2 * (12 / L.ml_rpb); ++slot)
                    for (int f = 0; f < nc; ++f) items.push_back(BatchItem{j, slot, f});
                ++j;
                args.resize(args.size() + asz);
                unsigned char *dst = args.data() + args.size() - asz;
                const size_t es = elem_size(h->prec);
                const void *ib =
                    static_cast<const unsigned char *>(L.mib) + (size_t)f0 * L.nplane * es;
                if (b->prec == MG3D_PREC_F64) {
                    MlSweepArgs<double> a{L.nx, L.ny, L.nz, nc, L.ml_rows,
                                          (const double *)L.mchi, (const double *)L.mS,
                                          (const double *)L.msc, (const double *)L.moc,
                                          (const double *)ib, L.geom, h->d_exp_tab, h->exp_l1,
                                          h->exp_l2, (double *)h->ml_jx, (double *)h->ml_ux,
                                          L.ml_rpb};
                    std::memcpy(dst, &a, asz);
                } else {
                    MlSweepArgs<float> a{L.nx, L.ny, L.nz, nc, L.ml_rows,
                                         (const float *)L.mchi, (const float *)L.mS,
                                         (const float *)L.msc, (const float *)L.moc,
                                         (const float *)ib, L.geom, h->d_exp_tab, h->exp_l1,
                                         h->exp_l2, (float *)h->ml_jx, (float *)h->ml_ux,
                                         L.ml_rpb};
                    std::memcpy(dst, &a, asz);
                }
            }
            if (items.size() > 65535)
                return fail(MG3D_E_ARG, "batch chunk too large for one launch (use smaller chunks)");
            mg3d_batch::KindLevel &t = b->mlc[k][c];
            t.n_items = (int)items.size();
            t.bands = bands;
            t.threads = threads;
            t.smem = smem;
            if (t.n_items) {
                MG_TRY(dev_alloc((void **)&t.d_items, items.size() * sizeof(BatchItem)));
                MG_TRY(dev_alloc(&t.d_args, args.size()));
                MG_CUDA(cudaMemcpy(t.d_items, items.data(), items.size() * sizeof(BatchItem),
                                   cudaMemcpyHostToDevice));
                MG_CUDA(cudaMemcpy(t.d_args, args.data(), args.size(), cudaMemcpyHostToDevice));
            }
        }
    }
    return MG3D_OK;
}

}  // namespace

namespace mg3d {
// Lets other translation units report through mg3d_last_error().
void record_error(const std::string &msg) { g_last_error = msg; }
}  // namespace mg3d

// ======================================================================= ABI

extern "C" {

const char *mg3d_last_error(void) { return g_last_error.c_str(); }

// The A4 parameter a must leave b = sqrt(1 - 2a^2) real and positive: a <= 0
// (the default set) or 0 < a < 1/sqrt(2); non-finite values are refused.
static int check_quadrature(const mg3d_quadrature *quad) {
    if (!quad) return MG3D_OK;
    const double a = quad->a;
    if (!std::isfinite(a) || (a > 0.0 && 2.0 * a * a >= 1.0))
        return fail(MG3D_E_ARG, "quadrature parameter a must be finite and below 1/sqrt(2) "
                                "(a <= 0 selects the default A4 set)");
    return MG3D_OK;
}

int mg3d_create(const mg3d_atmosphere *atm, const mg3d_atom *atom, const mg3d_quadrature *quad,
                const mg3d_params *params, mg3d_handle **out) {
    if (!out) return fail(MG3D_E_ARG, "null output pointer");
    *out = nullptr;
    if (!atm || !atom || !params) return fail(MG3D_E_ARG, "null argument");
    MG_TRY(check_quadrature(quad));
    if (!atm->z || !atm->T || !atm->n_tot || !atm->c_ul) return fail(MG3D_E_ARG, "null array");
    if (params->n_grids < 1 || params->n_grids > MG3D_MAX_GRIDS)
        return fail(MG3D_E_ARG, "n_grids out of range");
    if (params->fs_prec != MG3D_PREC_F64 && params->fs_prec != MG3D_PREC_F32)
        return fail(MG3D_E_ARG, "fs_prec must be MG3D_PREC_F64 or MG3D_PREC_F32");
    if (params->nu_fmg < 0 || params->nu0 < 0 || params->nu1 < 0 || params->nu2 < 0 ||
        params->nu3 < 0)
        return fail(MG3D_E_ARG, "negative iteration count");
    if (params->restriction < 0 || params->restriction > 2)
        return fail(MG3D_E_ARG, "restriction must be 0, 1 or 2");
    if (params->interpolation < 0 || params->interpolation > 1)
        return fail(MG3D_E_ARG, "interpolation must be 0 or 1");
    if (params->sc_interp < 0 || params->sc_interp > 1)
        return fail(MG3D_E_ARG, "sc_interp must be 0 or 1");
    if (atm->vel && params->sc_interp)
        return fail(MG3D_E_ARG, "moving atmospheres take the linear upwind interpolation");
    if (!(atom->gamma_prd >= 0.0 && atom->gamma_prd <= 1.0))
        return fail(MG3D_E_ARG, "gamma_prd must lie in [0, 1]");
    if (!(atom->a_damp >= 0.0 && atom->a_damp < 1e3))
        return fail(MG3D_E_ARG, "a_damp must lie in [0, 1000)");
    if (atom->a_damp > 0.0 && atm->vel)
        return fail(MG3D_E_ARG, "moving atmospheres take Doppler profiles (a_damp 0)");
    if (atom->gamma_prd > 0.0 && (atm->vel || params->sc_interp))
        return fail(MG3D_E_ARG,
                    "partial redistribution takes a static atmosphere and linear interpolation");
    if (atom->n_freq < 1 || atom->n_freq > 4096 || !(atom->x_max >= 0.0) ||
        !(atom->a_ul > 0.0) || !(atom->g_ratio > 0.0) || !(atom->theta > 0.0) ||
        !(atom->kappa > 0.0))
        return fail(MG3D_E_ARG, "bad atom parameters");
    if (atm->nx < 1 || atm->ny < 1 || atm->nz < 2) return fail(MG3D_E_ARG, "grid too small");
    if (atm->nx >= 65536 || atm->ny >= 65536)
        return fail(MG3D_E_ARG, "nx and ny must be below 65536");
    if (!(atm->dx > 0.0) || !(atm->dy > 0.0)) return fail(MG3D_E_ARG, "dx, dy must be > 0");
    for (int k = 1; k < atm->nz; ++k)
        if (!(atm->z[k] > atm->z[k - 1])) return fail(MG3D_E_ARG, "z must increase");
    const long step = 1L << (params->n_grids - 1);
    if ((atm->nz - 1) % step != 0 || atm->nx % step != 0 || atm->ny % step != 0 ||
        (atm->nz - 1) / step < 1)
        return fail(MG3D_E_GRID, "grid does not coarsen n_grids - 1 times "
                                 "(need nz = A 2^(l-1) + 1, nx, ny = B 2^(l-1))");
    mg3d_handle *h = new (std::nothrow) mg3d_handle();
    if (!h) return fail(MG3D_E_OOM, "host allocation failed");
    int rc = create_impl(atm, atom, quad, params, h);
    if (rc != MG3D_OK) {
        std::string msg = g_last_error;
        mg3d_destroy(h);
        g_last_error = msg;
        return rc;
    }
    *out = h;
    g_last_error.clear();
    return MG3D_OK;
}

int mg3d_create_ml(const mg3d_ml_atmosphere *atm, const mg3d_ml_atom *atom,
                   const mg3d_quadrature *quad, const mg3d_params *params, mg3d_handle **out) {
    if (!out) return fail(MG3D_E_ARG, "null output pointer");
    *out = nullptr;
    if (!atm || !atom || !params) return fail(MG3D_E_ARG, "null argument");
    MG_TRY(check_quadrature(quad));
    if (!atm->z || !atm->T || !atm->n_tot || !atm->chi_c || !atm->c || !atm->saha)
        return fail(MG3D_E_ARG, "null atmosphere array");
    const int N = atom->n_levels;
    if (N < 2 || N > kMaxLevels || !atom->g || !atom->theta)
        return fail(MG3D_E_ARG, "n_levels must be 2..8 with g and theta given");
    if (!(atom->theta_ref > 0.0) || !(atom->t_ref > 0.0))
        return fail(MG3D_E_ARG, "theta_ref and t_ref must be > 0");
    if (atom->n_lines < 0 || atom->n_continua < 0 || atom->n_lines + atom->n_continua < 1 ||
        (atom->n_lines && !atom->lines) || (atom->n_continua && !atom->continua))
        return fail(MG3D_E_ARG, "no transitions");
    long nf = 0;
    for (int t = 0; t < atom->n_lines; ++t) {
        const mg3d_line &ln = atom->lines[t];
        if (ln.lower < 0 || ln.upper >= N || ln.lower >= ln.upper || ln.n_freq < 1 ||
            !(ln.rho > 0) || !(ln.a_ul > 0) || !(ln.kappa >= 0) || !(ln.x_max >= 0))
            return fail(MG3D_E_ARG, "bad line " + std::to_string(t));
        if (!(ln.a_damp >= 0.0 && ln.a_damp < 1e3))
            return fail(MG3D_E_ARG, "line " + std::to_string(t) + ": a_damp must lie in [0, 1000)");
        if (ln.a_damp > 0.0 && atm->vel)
            return fail(MG3D_E_ARG, "line " + std::to_string(t) +
                                        ": damped lines take a static atmosphere");
        if (!(ln.gamma_prd >= 0.0 && ln.gamma_prd <= 1.0))
            return fail(MG3D_E_ARG, "line " + std::to_string(t) + ": gamma_prd must lie in [0, 1]");
        if (ln.gamma_prd > 0.0 && (atm->vel || params->sc_interp))
            return fail(MG3D_E_ARG, "line " + std::to_string(t) +
                                        ": partial redistribution of multi-level lines takes a "
                                        "static atmosphere and linear upwind interpolation");
        if (ln.gamma_prd > 0.0 && ln.n_freq > kMaxPrdLineFreq)
            return fail(MG3D_E_ARG, "line " + std::to_string(t) + ": partial redistribution takes "
                                        "at most " + std::to_string(kMaxPrdLineFreq) +
                                        " frequencies per line");
        nf += ln.n_freq;
    }
    {
        bool damped = false, prd = false;
        for (int t = 0; t < atom->n_lines; ++t) {
            damped = damped || atom->lines[t].a_damp > 0.0;
            prd = prd || atom->lines[t].gamma_prd > 0.0;
        }
        if (damped && prd)
            return fail(MG3D_E_ARG, "damped lines and partial redistribution in one multi-level "
                                    "atom are not built (the ratios' plain rates take Doppler "
                                    "profiles)");
    }
    for (int t = 0; t < atom->n_continua; ++t) {
        const mg3d_continuum &ct = atom->continua[t];
        if (ct.lower < 0 || ct.lower >= N - 1 || ct.n_freq < 1 || !(ct.rho > 0) ||
            !(ct.beta >= 0) || !(ct.kappa >= 0) || !(ct.y_max >= 1.0))
            return fail(MG3D_E_ARG, "bad continuum " + std::to_string(t));
        nf += ct.n_freq;
    }
    if (nf > 65535) return fail(MG3D_E_ARG, "too many frequencies");
    if (params->n_grids < 1 || params->n_grids > MG3D_MAX_GRIDS)
        return fail(MG3D_E_ARG, "n_grids out of range");
    if (params->fs_prec != MG3D_PREC_F64 && params->fs_prec != MG3D_PREC_F32)
        return fail(MG3D_E_ARG, "fs_prec must be MG3D_PREC_F64 or MG3D_PREC_F32");
    if (params->nu_fmg < 0 || params->nu0 < 0 || params->nu1 < 0 || params->nu2 < 0 ||
        params->nu3 < 0)
        return fail(MG3D_E_ARG, "negative iteration count");
    if (params->restriction < 0 || params->restriction > 2)
        return fail(MG3D_E_ARG, "restriction must be 0, 1 or 2");
    if (params->interpolation < 0 || params->interpolation > 1)
        return fail(MG3D_E_ARG, "interpolation must be 0 or 1");
    if (params->sc_interp < 0 || params->sc_interp > 1)
        return fail(MG3D_E_ARG, "sc_interp must be 0 or 1");
    if (atm->vel && params->sc_interp)
        return fail(MG3D_E_ARG, "moving atmospheres take the linear upwind interpolation");
    if (atm->nx < 1 || atm->ny < 1 || atm->nz < 2) return fail(MG3D_E_ARG, "grid too small");
    if (atm->nx >= 65536 || atm->ny >= 65536)
        return fail(MG3D_E_ARG, "nx and ny must be below 65536");
    if (!(atm->dx > 0.0) || !(atm->dy > 0.0)) return fail(MG3D_E_ARG, "dx, dy must be > 0");
    for (int k = 1; k < atm->nz; ++k)
        if (!(atm->z[k] > atm->z[k - 1])) return fail(MG3D_E_ARG, "z must increase");
    const long step = 1L << (params->n_grids - 1);
    if ((atm->nz - 1) % step != 0 || atm->nx % step != 0 || atm->ny % step != 0)
        return fail(MG3D_E_GRID, "grid does not coarsen n_grids - 1 times "
                                 "(need nz = A 2^(l-1) + 1, nx, ny = B 2^(l-1))");
    mg3d_handle *h = new (std::nothrow) mg3d_handle();
    if (!h) return fail(MG3D_E_OOM, "host allocation failed");
    int rc = create_ml_impl(atm, atom, quad, params, h);
    if (rc != MG3D_OK) {
        std::string msg = g_last_error;
        mg3d_destroy(h);
        g_last_error = msg;
        return rc;
    }
    *out = h;
    g_last_error.clear();
    return MG3D_OK;
}

int mg3d_n_levels(const mg3d_handle *h, int *n_levels, int *n_freq) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (n_levels) *n_levels = h->N;
    if (n_freq) *n_freq = h->kind == 1 ? h->nfreq_ml : h->atom.n_freq;
    return MG3D_OK;
}

int mg3d_formal_solve_ml(mg3d_handle *h, int level, double *jx_host, double *ux_host) {
    MG_TRY(check_level(h, level));
    if (h->kind != 1) return fail(MG3D_E_STATE, "not a multi-level handle");
    Level &L = h->lev[level];
    const size_t es = elem_size(h->prec);
    const size_t nv = (size_t)L.nvox;
    std::vector<unsigned char> hj, hu;
    MG_TRY(ml_prd_prepare(h, level));
    // a PRD frequency's sweep sums u alone; its U adds the local term in FP64
    // (1 - rho chi_t/chi of the ratios kernel), as the radiative sums do
    std::vector<double> prd_oc;
    if (h->ml_prd) {
        prd_oc.resize((size_t)h->n_prd_freq * nv);
        MG_CUDA(cudaMemcpyAsync(prd_oc.data(), L.prd_oc, prd_oc.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, h->stream));
    }
    for (int f0 = 0; f0 < h->nfreq_ml; f0 += h->ml_chunk) {
        const int nc = std::min(h->ml_chunk, h->nfreq_ml - f0);
        MG_TRY(ml_chunk_fs(h, level, f0, nc));
        if (ml_lagged(h)) {   // the lagged field takes the new mean intensity
            h->force_bg = true;
            const int rc = ml_accumulate(h, level, f0, nc, false);
            h->force_bg = false;
            MG_TRY(rc);
        }
        MG_CUDA(cudaStreamSynchronize(h->stream));
        // the chunk's per-frequency sums of every ray-group slot, added on the
        // host in slot order
        const size_t cnt = (size_t)nc * nv;
        const int slots = 2 * (12 / L.ml_rpb);
        hj.resize(slots * cnt * es);
        hu.resize(slots * cnt * es);
        MG_CUDA(cudaMemcpy(hj.data(), h->ml_jx, slots * cnt * es, cudaMemcpyDeviceToHost));
        MG_CUDA(cudaMemcpy(hu.data(), h->ml_ux, slots * cnt * es, cudaMemcpyDeviceToHost));
        auto at = [&](const std::vector<unsigned char> &v, size_t i) {
            return h->prec == MG3D_PREC_F64 ? ((const double *)v.data())[i]
                                            : (double)((const float *)v.data())[i];
        };
        for (size_t i = 0; i < cnt; ++i) {
            double J = at(hj, i), U = at(hu, i);
            for (int sl = 1; sl < slots; ++sl) {
                J += at(hj, sl * cnt + i);
                U += at(hu, sl * cnt + i);
            }
            const size_t o = (size_t)f0 * nv + i;
            if (h->ml_prd) {
                const int pr = h->prd_index[f0 + i / nv];
                if (pr >= 0) {
                    const double oc = prd_oc[(size_t)pr * nv + i % nv];
                    U = oc + (1.0 - oc) * U;
                }
            }
            if (jx_host) jx_host[o] = J;
            if (ux_host) ux_host[o] = U;
        }
    }
    const double units = (double)L.nvox * kRays * h->nfreq_ml;
    ++h->fs_launches;
    h->fs_units += units;
    ++h->level_launches[level];
    h->level_units[level] += units;
    return MG3D_OK;
}

int mg3d_set_ml_chunk(mg3d_handle *h, int freq_per_chunk) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (h->kind != 1) return fail(MG3D_E_STATE, "not a multi-level handle");
    if (freq_per_chunk < 0) return fail(MG3D_E_ARG, "negative chunk size");
    const int c = freq_per_chunk == 0 ? h->nfreq_ml : std::min(freq_per_chunk, h->nfreq_ml);
    h->ml_chunk_req = c;
    MG_CUDA(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    return alloc_ml_chunks(h, c);
}

int mg3d_set_ml_shape(mg3d_handle *h, int level, int bands, int rays_per_block, int threads) {
    MG_TRY(check_level(h, level));
    if (h->kind != 1) return fail(MG3D_E_STATE, "not a multi-level handle");
    Level &L = h->lev[level];
    if (bands < 1 || bands > kPortableBands || bands > L.ny)
        return fail(MG3D_E_ARG, "bands must be 1..8 and at most ny");
    const int rows = (L.ny + bands - 1) / bands;
    if ((long)(bands - 1) * rows >= L.ny) return fail(MG3D_E_ARG, "empty band");
    if (rays_per_block < 1 || 12 % rays_per_block)
        return fail(MG3D_E_ARG, "rays_per_block must divide 12");
    if (threads < 32 || threads > kMaxSweepThreads || threads % 32)
        return fail(MG3D_E_ARG, "threads must be a multiple of 32 up to 512");
    if (ml_sweep_smem_bytes(h->prec, rows, L.nx, rays_per_block, h->params.sc_interp,
                            h->moving ? 1 : 0) > kMaxSweepSmem)
        return fail(MG3D_E_ARG, "multi-level sweep shape exceeds shared memory");
    MG_CUDA(cudaStreamSynchronize(h->stream));
    L.ml_bands = bands;
    L.ml_rows = rows;
    L.ml_rpb = rays_per_block;
    L.ml_threads = threads;
    L.ml_plane = 0;
    L.ml_nf = 1;
    drop_graphs(h);
    const int slots = 2 * (12 / rays_per_block);
    if (slots > h->ml_slots) {
        h->ml_slots = slots;
        MG_TRY(alloc_ml_chunks(h, h->ml_chunk));
    }
    return MG3D_OK;
}

int mg3d_set_ml_shape_ex(mg3d_handle *h, int level, int bands, int rays_per_block, int threads,
                         int kind, int freq_per_block) {
    MG_TRY(check_level(h, level));
    if (h->kind != 1) return fail(MG3D_E_STATE, "not a multi-level handle");
    if (kind == 0) {
        if (freq_per_block != 1) return fail(MG3D_E_ARG, "kind 0 takes freq_per_block 1");
        MG_TRY(mg3d_set_ml_shape(h, level, bands, rays_per_block, threads));
        h->lev[level].ml_plane = 0;
        h->lev[level].ml_nf = 1;
        return MG3D_OK;
    }
    if (kind != 1) return fail(MG3D_E_ARG, "kind must be 0 or 1");
    MG_TRY(ml_plane_shape_check(h, level, bands, rays_per_block, threads, freq_per_block));
    Level &L = h->lev[level];
    MG_CUDA(cudaStreamSynchronize(h->stream));
    L.ml_bands = bands;
    L.ml_rows = (L.ny + bands - 1) / bands;
    L.ml_rpb = rays_per_block;
    L.ml_threads = threads;
    L.ml_plane = 1;
    L.ml_nf = freq_per_block;
    drop_graphs(h);
    const int slots = 2 * (12 / rays_per_block);
    if (slots > h->ml_slots) {
        h->ml_slots = slots;
        MG_TRY(alloc_ml_chunks(h, h->ml_chunk));
    }
    return MG3D_OK;
}

int mg3d_get_ml_shape_ex(const mg3d_handle *h, int level, int *bands, int *rays_per_block,
                         int *threads, int *kind, int *freq_per_block) {
    MG_TRY(mg3d_get_ml_shape(h, level, bands, rays_per_block, threads));
    if (kind) *kind = h->lev[level].ml_plane;
    if (freq_per_block) *freq_per_block = h->lev[level].ml_nf;
    return MG3D_OK;
}

int mg3d_get_ml_shape(const mg3d_handle *h, int level, int *bands, int *rays_per_block,
                      int *threads) {
    MG_TRY(check_level(h, level));
    if (h->kind != 1) return fail(MG3D_E_STATE, "not a multi-level handle");
    const Level &L = h->lev[level];
    if (bands) *bands = L.ml_bands;
    if (rays_per_block) *rays_per_block = L.ml_rpb;
    if (threads) *threads = L.ml_threads;
    return MG3D_OK;
}

int mg3d_get_ml_chunk(const mg3d_handle *h, int *freq_per_chunk) {
    if (!h || !freq_per_chunk) return fail(MG3D_E_ARG, "null argument");
    if (h->kind != 1) return fail(MG3D_E_STATE, "not a multi-level handle");
    *freq_per_chunk = h->ml_chunk;
    return MG3D_OK;
}

int mg3d_batch_create(int n, mg3d_handle *const *members, mg3d_batch **out) {
    if (!out) return fail(MG3D_E_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || !members) return fail(MG3D_E_ARG, "empty batch");
    for (int i = 0; i < n; ++i) {
        if (!members[i]) return fail(MG3D_E_ARG, "null member");
        if (members[i]->scatter)
            return fail(MG3D_E_ARG, "batches do not take background scattering");
        if (members[i]->d_voigt)
            return fail(MG3D_E_ARG, "batches do not take damped multi-level lines");
        if (members[i]->ml_prd)
            return fail(MG3D_E_ARG, "batches do not take partial redistribution");
        if (members[i]->params.sc_interp)
            return fail(MG3D_E_ARG, "batches do not take Hermite upwind interpolation");
        if (members[i]->moving)
            return fail(MG3D_E_ARG, "batches do not take moving atmospheres");
        if (members[i]->prd)
            return fail(MG3D_E_ARG, "batches do not take partial redistribution");
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return fail(MG3D_E_ARG, "member listed twice");
    }
    const mg3d_handle *h0 = members[0];
    for (int i = 1; i < n; ++i) {
        const mg3d_handle *h = members[i];
        const mg3d_params &p = h->params, &q = h0->params;
        if (h->L != h0->L || h->prec != h0->prec || p.nu0 != q.nu0 || p.nu1 != q.nu1 ||
            p.nu2 != q.nu2 || p.nu3 != q.nu3 || p.nu_fmg != q.nu_fmg ||
            p.restriction != q.restriction || p.interpolation != q.interpolation ||
            p.sc_interp != q.sc_interp)
            return fail(MG3D_E_ARG, "batch members need equal n_grids, precision and schedule");
    }

    mg3d_batch *b = new (std::nothrow) mg3d_batch();
    if (!b) return fail(MG3D_E_OOM, "host allocation failed");
    b->n = n;
    b->L = h0->L;
    b->prec = h0->prec;
    b->params = h0->params;
    b->m.assign(members, members + n);
    int rc = MG3D_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = fail(MG3D_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    for (int i = 0; i < n && rc == MG3D_OK; ++i) {
        rc = mg3d_set_stream(b->m[i], b->stream);
        for (int k = 1; k <= b->L; ++k)
            (b->m[i]->kind == 1 ? b->ml[k] : b->two[k]).members.push_back(i);
    }
    // the largest partial buffer any level of a two-level member can need
    // with at most three frequencies per block, allocated before any table
    for (int i = 0; i < n && rc == MG3D_OK; ++i) {
        mg3d_handle *h = b->m[i];
        if (h->kind != 0) continue;
        size_t need = 0;
        for (int k = 1; k <= b->L; ++k)
            need = std::max(need, (size_t)kRays * (size_t)h->atom.n_freq * (size_t)h->lev[k].nvox);
        rc = ensure_partials(h, need);
    }
    for (int k = 1; k <= b->L && rc == MG3D_OK; ++k) rc = batch_build_level(b, k);
    if (rc != MG3D_OK) {
        std::string msg = g_last_error;
        mg3d_batch_destroy(b);
        g_last_error = msg;
        return rc;
    }
    *out = b;
    return MG3D_OK;
}

int mg3d_batch_destroy(mg3d_batch *b) {
    if (!b) return MG3D_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (int k = 0; k <= MG3D_MAX_GRIDS; ++k)
    {
        for (auto *t : {&b->two[k], &b->ml[k]}) {
            if (t->d_items) cudaFree(t->d_items);
            if (t->d_args) cudaFree(t->d_args);
        }
        for (auto &t : b->mlc[k]) {
            if (t.d_items) cudaFree(t.d_items);
            if (t.d_args) cudaFree(t.d_args);
        }
    }
    for (mg3d_handle *h : b->m) mg3d_set_stream(h, nullptr);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return MG3D_OK;
}

int mg3d_batch_fas_vcycle(mg3d_batch *b, int is_first, double *max_rel_change) {
    if (!b) return fail(MG3D_E_ARG, "null batch");
    if (b->L < 2) return fail(MG3D_E_STATE, "a V-cycle needs n_grids >= 2");
    std::vector<long long> neg(b->n);
    MG_TRY(batch_cycle(b, is_first != 0, max_rel_change, neg.data()));
    for (int i = 0; i < b->n; ++i) b->m[i]->negatives += neg[i];
    return MG3D_OK;
}

int mg3d_batch_fas_solve(mg3d_batch *b, double tol, int max_cycles, mg3d_stats *stats) {
    if (!b) return fail(MG3D_E_ARG, "null batch");
    if (b->L < 2) return fail(MG3D_E_STATE, "a V-cycle needs n_grids >= 2");
    if (!(tol > 0.0) || max_cycles < 1) return fail(MG3D_E_ARG, "bad tol or max_cycles");
    auto t0 = std::chrono::steady_clock::now();
    for (mg3d_handle *h : b->m) {
        begin_stats(h);
        MG_TRY(zero_radiation(h, h->L));
    }
    std::vector<double> C(b->n, 1.0);
    std::vector<int> done_at(b->n, 0);
    int cyc = 0;
    while (cyc < max_cycles) {
        std::vector<long long> neg(b->n);
        MG_TRY(batch_cycle(b, cyc == 0, C.data(), neg.data()));
        ++cyc;
        bool all = true;
        for (int i = 0; i < b->n; ++i) {
            b->m[i]->negatives += neg[i];
            if (!done_at[i] && C[i] < tol) done_at[i] = cyc;
            all = all && done_at[i];
        }
        if (all) break;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int i = 0; i < b->n; ++i) {
        if (stats) end_stats(b->m[i], &stats[i], done_at[i] ? done_at[i] : cyc, C[i], secs);
        all = all && done_at[i];
    }
    if (!all) return fail(MG3D_E_MAXITER, "not every member reached tol");
    return MG3D_OK;
}

int mg3d_batch_fmg_solve(mg3d_batch *b, double tol, int max_cycles, mg3d_stats *stats) {
    if (!b) return fail(MG3D_E_ARG, "null batch");
    if (b->L < 2) return fail(MG3D_E_STATE, "FMG needs n_grids >= 2");
    if (!(tol > 0.0) || max_cycles < 1) return fail(MG3D_E_ARG, "bad tol or max_cycles");
    auto t0 = std::chrono::steady_clock::now();
    for (mg3d_handle *h : b->m) {
        begin_stats(h);
        MG_TRY(zero_radiation(h, 1));
    }
    for (int i = 0; i < b->params.nu_fmg; ++i) MG_TRY(batch_sweep(b, 1));
    for (int k = 2; k <= b->L; ++k) {
        for (mg3d_handle *h : b->m) {
            Level &Fk = h->lev[k];
            Level &Ck = h->lev[k - 1];
            MG_TRY(batch_launched(b, launch_prolong(h->params.interpolation, h->N, Ck.nx, Ck.ny,
                                                    Ck.nz, Fk.tz, Fk.zf, Ck.n, Fk.n, b->stream),
                                  "prolong full approximation"));
            Fk.f_default = true;
        }
        if (k < b->L) MG_TRY(batch_vcycle(b, k, false));
    }
    std::vector<double> C(b->n, 1.0);
    std::vector<int> done_at(b->n, 0);
    int cyc = 0;
    while (cyc < max_cycles) {
        std::vector<long long> neg(b->n);
        MG_TRY(batch_cycle(b, cyc == 0, C.data(), neg.data()));
        ++cyc;
        bool all = true;
        for (int i = 0; i < b->n; ++i) {
            b->m[i]->negatives += neg[i];
            if (!done_at[i] && C[i] < tol) done_at[i] = cyc;
            all = all && done_at[i];
        }
        if (all) break;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int i = 0; i < b->n; ++i) {
        if (stats) end_stats(b->m[i], &stats[i], done_at[i] ? done_at[i] : cyc, C[i], secs);
        all = all && done_at[i];
    }
    if (!all) return fail(MG3D_E_MAXITER, "not every member reached tol");
    return MG3D_OK;
}

int mg3d_batch_counters(const mg3d_batch *b, long long *kernel_launches, double *fs_units) {
    if (!b) return fail(MG3D_E_ARG, "null batch");
    if (kernel_launches) *kernel_launches = b->launches;
    if (fs_units) *fs_units = b->fs_units;
    return MG3D_OK;
}

int mg3d_destroy(mg3d_handle *h) {
    if (!h) return MG3D_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) free_level(h->lev[k]);
    for (void *p : h->d_pslot)
        if (p) cudaFree(p);
    for (void *p : h->o_pslot)
        if (p) cudaFree(p);
    for (void *p : {(void *)h->d_prd, (void *)h->d_prd_ord, (void *)h->d_prd_grp,
                    (void *)h->d_prd_index, (void *)h->d_voigt})
        if (p) cudaFree(p);
    if (h->o_pj) cudaFree(h->o_pj);
    if (h->o_pu) cudaFree(h->o_pu);
    void *ptrs[] = {h->d_ftab, h->d_vtab, h->d_vline, h->d_kmat, h->d_wphin, h->d_fidx,
                    h->d_exp_tab, h->pj, h->pu, h->scal,
                    h->scratch, h->d_fi, h->d_ti, h->ml_jx, h->ml_ux, h->ml_acc,
                    h->ml_jm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &t : h->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return MG3D_OK;
}

int mg3d_set_stream(mg3d_handle *h, void *cuda_stream) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    MG_CUDA(cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
    return MG3D_OK;
}

int mg3d_level_shape(const mg3d_handle *h, int level, int *nx, int *ny, int *nz) {
    MG_TRY(check_level(h, level));
    const Level &L = h->lev[level];
    if (nx) *nx = L.nx;
    if (ny) *ny = L.ny;
    if (nz) *nz = L.nz;
    return MG3D_OK;
}

int mg3d_get_populations(mg3d_handle *h, int level, double *n_host) {
    MG_TRY(check_level(h, level));
    if (!n_host) return fail(MG3D_E_ARG, "null buffer");
    Level &L = h->lev[level];
    return level_to_host(h, n_host, L.n, (size_t)h->N * L.nvox);
}

int mg3d_set_populations(mg3d_handle *h, int level, const double *n_host) {
    MG_TRY(check_level(h, level));
    if (!n_host) return fail(MG3D_E_ARG, "null buffer");
    Level &L = h->lev[level];
    return host_to_level(h, L.n, n_host, (size_t)h->N * L.nvox);
}

int mg3d_init_zero_radiation(mg3d_handle *h, int level) {
    MG_TRY(check_level(h, level));
    MG_TRY(zero_radiation(h, level));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return MG3D_OK;
}

int mg3d_formal_solve(mg3d_handle *h, int level, double *jeff_host, double *u_host) {
    MG_TRY(check_level(h, level));
    if (h->kind != 0) return fail(MG3D_E_STATE, "multi-level handle: use mg3d_formal_solve_ml");
    Level &L = h->lev[level];
    MG_TRY(formal_solution(h, level));
    RateArgs a = rate_args(h, level, kRateReduce);
    a.out = h->scratch;
    a.scal = nullptr;
    MG_TRY(launched(h, launch_rates(a, h->stream), "reduce"));
    if (jeff_host) MG_CUDA(cudaMemcpyAsync(jeff_host, h->scratch, L.nvox * 8,
                                           cudaMemcpyDeviceToHost, h->stream));
    if (u_host) MG_CUDA(cudaMemcpyAsync(u_host, h->scratch + L.nvox, L.nvox * 8,
                                        cudaMemcpyDeviceToHost, h->stream));
    return take_sweep_status(h);
}

// Orders stream `to` after the work enqueued so far on stream `from`.
static int order_after(mg3d_handle *h, cudaStream_t from, cudaStream_t to) {
    if (from == to) return MG3D_OK;
    cudaEvent_t e = pool_event(h);
    const cudaError_t r1 = cudaEventRecord(e, from);
    const cudaError_t r2 = r1 == cudaSuccess ? cudaStreamWaitEvent(to, e, 0) : r1;
    h->event_pool.push_back(e);   // the wait holds the recorded state: reusable
    MG_CUDA(r2);
    return MG3D_OK;
}

// Formal solution of a two-level handle's level in precision prec into
// h->scratch [2][nvox] (Jeff, U), on the handle's stream.
static int formal_solution_into_scratch(mg3d_handle *h, int level, int prec) {
    if (prec != h->prec) return other_prec_fs(h, level, prec);
    MG_TRY(formal_solution(h, level));
    RateArgs a = rate_args(h, level, kRateReduce);
    a.out = h->scratch;
    a.scal = nullptr;
    MG_TRY(launched(h, launch_rates(a, h->stream), "reduce"));
    return MG3D_OK;
}

static int check_fs_call(const mg3d_handle *h, int level, int prec) {
    MG_TRY(check_level(h, level));
    if (h->kind != 0) return fail(MG3D_E_STATE, "multi-level handle: use mg3d_formal_solve_ml");
    if (prec != MG3D_PREC_F64 && prec != MG3D_PREC_F32)
        return fail(MG3D_E_ARG, "prec must be MG3D_PREC_F64 or MG3D_PREC_F32");
    return MG3D_OK;
}

int mg3d_formal_solve_ex(mg3d_handle *h, int level, int prec, double *jeff_host,
                         double *u_host) {
    MG_TRY(check_fs_call(h, level, prec));
    const Level &L = h->lev[level];
    MG_TRY(formal_solution_into_scratch(h, level, prec));
    if (jeff_host) MG_CUDA(cudaMemcpyAsync(jeff_host, h->scratch, L.nvox * 8,
                                           cudaMemcpyDeviceToHost, h->stream));
    if (u_host) MG_CUDA(cudaMemcpyAsync(u_host, h->scratch + L.nvox, L.nvox * 8,
                                        cudaMemcpyDeviceToHost, h->stream));
    return take_sweep_status(h);
}

int mg3d_formal_solve_dev(mg3d_handle *h, int level, int prec, double *jeff_dev, double *u_dev,
                          void *cuda_stream) {
    MG_TRY(check_fs_call(h, level, prec));
    const Level &L = h->lev[level];
    const cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    MG_TRY(order_after(h, cs, h->stream));
    MG_TRY(formal_solution_into_scratch(h, level, prec));
    if (jeff_dev) MG_CUDA(cudaMemcpyAsync(jeff_dev, h->scratch, L.nvox * 8,
                                          cudaMemcpyDeviceToDevice, h->stream));
    if (u_dev) MG_CUDA(cudaMemcpyAsync(u_dev, h->scratch + L.nvox, L.nvox * 8,
                                       cudaMemcpyDeviceToDevice, h->stream));
    return order_after(h, h->stream, cs);
}

int mg3d_get_populations_dev(mg3d_handle *h, int level, double *n_dev, void *cuda_stream) {
    MG_TRY(check_level(h, level));
    if (!n_dev) return fail(MG3D_E_ARG, "null buffer");
    const Level &L = h->lev[level];
    const cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    MG_TRY(order_after(h, cs, h->stream));
    MG_CUDA(cudaMemcpyAsync(n_dev, L.n, (size_t)h->N * L.nvox * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream));
    return order_after(h, h->stream, cs);
}

int mg3d_set_populations_dev(mg3d_handle *h, int level, const double *n_dev,
                             void *cuda_stream) {
    MG_TRY(check_level(h, level));
    if (!n_dev) return fail(MG3D_E_ARG, "null buffer");
    const Level &L = h->lev[level];
    const cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    MG_TRY(order_after(h, cs, h->stream));
    MG_CUDA(cudaMemcpyAsync(L.n, n_dev, (size_t)h->N * L.nvox * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream));
    return order_after(h, h->stream, cs);
}

int mg3d_mali_sweep(mg3d_handle *h, int level, int n_sweeps, double *max_rel_change) {
    MG_TRY(check_level(h, level));
    if (n_sweeps < 0) return fail(MG3D_E_ARG, "negative sweep count");
    h->top = level;
    double C = 0.0;
    long long bad = 0;
    for (int i = 0; i < n_sweeps; ++i) {
        if (i == n_sweeps - 1) MG_TRY(reset_scalars(h));
        MG_TRY(sweep(h, level));
    }
    if (n_sweeps > 0) MG_TRY(read_scalars(h, &C, nullptr, &bad));
    if (max_rel_change) *max_rel_change = C;
    if (bad) return fail(MG3D_E_DIVERGED, "non-finite populations");
    return MG3D_OK;
}

int mg3d_residual(mg3d_handle *h, int level, double *r_host) {
    MG_TRY(check_level(h, level));
    if (!r_host) return fail(MG3D_E_ARG, "null buffer");
    Level &L = h->lev[level];
    MG_TRY(apply_W(h, level, kRateResidual, L.r));
    return level_to_host(h, r_host, L.r, (size_t)h->N * L.nvox);
}

int mg3d_fas_vcycle(mg3d_handle *h, int is_first, double *max_rel_change) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    long long neg = 0;
    MG_TRY(fas_cycle(h, is_first != 0, max_rel_change, &neg));
    h->negatives += neg;
    return MG3D_OK;
}

int mg3d_mali_solve(mg3d_handle *h, double tol, int max_sweeps, mg3d_stats *stats) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(MG3D_E_ARG, "bad tol or max_sweeps");
    auto t0 = std::chrono::steady_clock::now();
    begin_stats(h);
    h->top = h->L;
    MG_TRY(zero_radiation(h, h->L));
    double C = 1.0;
    int it = 0;
    while (it < max_sweeps) {
        MG_TRY(reset_scalars(h));
        MG_TRY(sweep(h, h->L));
        ++it;
        long long bad = 0;
        MG_TRY(read_scalars(h, &C, nullptr, &bad));
        if (bad) return fail(MG3D_E_DIVERGED, "non-finite populations");
        if (C < tol) break;
    }
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    end_stats(h, stats, it, C, secs);
    if (!(C < tol)) return fail(MG3D_E_MAXITER, "MALI did not reach tol");
    return MG3D_OK;
}

int mg3d_fas_solve(mg3d_handle *h, double tol, int max_cycles, mg3d_stats *stats) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (!(tol > 0.0) || max_cycles < 1) return fail(MG3D_E_ARG, "bad tol or max_cycles");
    auto t0 = std::chrono::steady_clock::now();
    begin_stats(h);
    MG_TRY(zero_radiation(h, h->L));
    double C = 1.0;
    int cyc = 0;
    while (cyc < max_cycles) {
        long long neg = 0;
        MG_TRY(fas_cycle(h, cyc == 0, &C, &neg));
        h->negatives += neg;
        ++cyc;
        if (C < tol) break;
    }
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    end_stats(h, stats, cyc, C, secs);
    if (!(C < tol)) return fail(MG3D_E_MAXITER, "FAS did not reach tol");
    return MG3D_OK;
}

// Stage k of full multigrid (Sec. 2.3, Fig. 1): k = 1 starts grid 1 from the
// zero-radiation populations and runs nu_fmg MALI sweeps on it; k >= 2
// interpolates the full approximation (and the lagged fields) from grid k-1
// to grid k and, below the finest grid, runs one V-cycle on grid k.
int fmg_stage(mg3d_handle *h, int k) {
    h->top = k;  // each stage solves on its own grid
    if (k == 1) {
        MG_TRY(zero_radiation(h, 1));
        for (int i = 0; i < h->params.nu_fmg; ++i) MG_TRY(sweep(h, 1));
        return MG3D_OK;
    }
    Level &Fk = h->lev[k];
    Level &Ck = h->lev[k - 1];
    MG_TRY(launched(h, launch_prolong(h->params.interpolation, h->N, Ck.nx, Ck.ny, Ck.nz,
                                      Fk.tz, Fk.zf, Ck.n, Fk.n, h->stream),
                    "prolong full approximation"));
    if (ml_lagged(h))
        MG_TRY(launched(h, launch_prolong_prec(h->params.interpolation, h->prec, h->nfreq_ml,
                                               Ck.nx, Ck.ny, Ck.nz, Fk.tz, Fk.zf, Ck.jbg,
                                               Fk.jbg, h->stream),
                        "prolong background field"));
    if (h->kind == 0 && h->prd)
        MG_TRY(launched(h, launch_prolong_prec(h->params.interpolation, h->prec,
                                               h->atom.n_freq, Ck.nx, Ck.ny, Ck.nz, Fk.tz,
                                               Fk.zf, Ck.jnu, Fk.jnu, h->stream),
                        "prolong mean intensity"));
    Fk.f_default = true;
    if (k < h->L) {
        MG_TRY(reset_scalars(h));
        MG_TRY(vcycle(h, k, false));
        long long neg = 0;
        MG_TRY(read_scalars(h, nullptr, &neg, nullptr));
        h->negatives += neg;
    }
    return MG3D_OK;
}

int mg3d_fmg_stage(mg3d_handle *h, int stage) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (h->L < 2) return fail(MG3D_E_STATE, "FMG needs n_grids >= 2");
    if (stage < 1 || stage > h->L) return fail(MG3D_E_ARG, "stage must be 1..n_grids");
    if (stage != 1 && stage != h->fmg_next)
        return fail(MG3D_E_STATE, "FMG stages run in order, starting at 1");
    MG_TRY(fmg_stage(h, stage));
    h->fmg_next = stage + 1;
    MG_CUDA(cudaStreamSynchronize(h->stream));
    return MG3D_OK;
}

int mg3d_fmg_solve(mg3d_handle *h, double tol, int max_cycles, mg3d_stats *stats) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (!(tol > 0.0) || max_cycles < 1) return fail(MG3D_E_ARG, "bad tol or max_cycles");
    if (h->L < 2) return fail(MG3D_E_STATE, "FMG needs n_grids >= 2");
    auto t0 = std::chrono::steady_clock::now();
    begin_stats(h);
    for (int k = 1; k <= h->L; ++k) MG_TRY(fmg_stage(h, k));
    h->fmg_next = h->L + 1;
    double C = 1.0;
    int cyc = 0;
    while (cyc < max_cycles) {
        long long neg = 0;
        MG_TRY(fas_cycle(h, cyc == 0, &C, &neg));
        h->negatives += neg;
        ++cyc;
        if (C < tol) break;
    }
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    end_stats(h, stats, cyc, C, secs);
    if (!(C < tol)) return fail(MG3D_E_MAXITER, "FMG did not reach tol");
    return MG3D_OK;
}

int mg3d_restrict(mg3d_handle *h, int level_fine, int ncomp, const double *fine_host,
                  double *coarse_host) {
    MG_TRY(check_level(h, level_fine));
    if (level_fine < 2) return fail(MG3D_E_ARG, "level_fine must be >= 2");
    if (ncomp < 1 || ncomp > 4 || !fine_host || !coarse_host) return fail(MG3D_E_ARG, "bad args");
    Level &F = h->lev[level_fine];
    Level &C = h->lev[level_fine - 1];
    double *dfine = nullptr, *dcoarse = nullptr;
    MG_TRY(dalloc(&dfine, (size_t)ncomp * F.nvox));
    int rc = dalloc(&dcoarse, (size_t)ncomp * C.nvox);
    if (rc == MG3D_OK) rc = host_to_level(h, dfine, fine_host, (size_t)ncomp * F.nvox);
    if (rc == MG3D_OK)
        rc = launched(h, launch_restrict(ncomp, F.nx, F.ny, F.nz, dfine, dcoarse, h->stream,
                                         h->params.restriction),
                      "restrict");
    if (rc == MG3D_OK) rc = level_to_host(h, coarse_host, dcoarse, (size_t)ncomp * C.nvox);
    cudaFree(dfine);
    if (dcoarse) cudaFree(dcoarse);
    return rc;
}

int mg3d_prolong(mg3d_handle *h, int level_fine, int ncomp, const double *coarse_host,
                 double *fine_host) {
    MG_TRY(check_level(h, level_fine));
    if (level_fine < 2) return fail(MG3D_E_ARG, "level_fine must be >= 2");
    if (ncomp < 1 || ncomp > 4 || !fine_host || !coarse_host) return fail(MG3D_E_ARG, "bad args");
    Level &F = h->lev[level_fine];
    Level &C = h->lev[level_fine - 1];
    double *dfine = nullptr, *dcoarse = nullptr;
    MG_TRY(dalloc(&dcoarse, (size_t)ncomp * C.nvox));
    int rc = dalloc(&dfine, (size_t)ncomp * F.nvox);
    if (rc == MG3D_OK) rc = host_to_level(h, dcoarse, coarse_host, (size_t)ncomp * C.nvox);
    if (rc == MG3D_OK)
        rc = launched(h, launch_prolong(h->params.interpolation, ncomp, C.nx, C.ny, C.nz, F.tz,
                                        F.zf, dcoarse, dfine, h->stream),
                      "prolong");
    if (rc == MG3D_OK) rc = level_to_host(h, fine_host, dfine, (size_t)ncomp * F.nvox);
    cudaFree(dcoarse);
    if (dfine) cudaFree(dfine);
    return rc;
}

int mg3d_set_fs_config(mg3d_handle *h, int level, int freq_per_block, int bands, int threads,
                       int lean, int stage) {
    SweepShape s;
    MG_TRY(shape_from_args(h, level, freq_per_block, bands, threads, lean, stage, &s));
    MG_TRY(check_schedulable(h, level, s));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    MG_TRY(ensure_partials(h, (size_t)kRays * s.ngroups * (size_t)h->lev[level].nvox));
    h->lev[level].shape = s;
    drop_graphs(h);
    return MG3D_OK;
}

int mg3d_get_fs_occupancy(mg3d_handle *h, int level, int freq_per_block, int bands,
                          int threads, int lean, int stage, int *max_clusters,
                          long long *smem_bytes) {
    SweepShape s;
    MG_TRY(shape_from_args(h, level, freq_per_block, bands, threads, lean, stage, &s));
    int n = 0;
    const cudaError_t e = s.plane ? plane_active_clusters(h->prec, s, h->lev[level].nx, &n)
                                  : sweep_active_clusters(h->prec, s, h->lev[level].nx, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MG3D_E_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    }
    if (max_clusters) *max_clusters = n;
    if (smem_bytes)
        *smem_bytes = (long long)(s.plane ? plane_smem_bytes(h->prec, s.np, s.rows,
                                                             h->lev[level].nx)
                                          : sweep_smem_bytes(h->prec, s, h->lev[level].nx));
    return MG3D_OK;
}

int mg3d_autotune(mg3d_handle *h, int level, int *evaluated, double *seconds) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    if (level != 0) MG_TRY(check_level(h, level));
    auto t0 = std::chrono::steady_clock::now();
    int count = 0;
    if (h->kind == 1) {
        MG_TRY(autotune_ml(h, level, &count));
        if (evaluated) *evaluated = count;
        if (seconds)
            *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return MG3D_OK;
    }
    for (int k = 1; k <= h->L; ++k) {
        if (level != 0 && k != level) continue;
        int c = 0;
        MG_TRY(autotune_level(h, k, &c));
        count += c;
    }
    MG_TRY(shrink_partials(h));
    drop_graphs(h);
    if (evaluated) *evaluated = count;
    if (seconds)
        *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return MG3D_OK;
}

int mg3d_get_fs_config(const mg3d_handle *h, int level, int *freq_per_block, int *bands,
                       int *threads, int *lean, int *stage) {
    MG_TRY(check_level(h, level));
    const Level &L = h->lev[level];
    if (freq_per_block)
        *freq_per_block = L.shape.plane && L.shape.ngroups == 1 ? h->atom.n_freq : L.shape.ng;
    if (bands) *bands = L.shape.bands;
    if (threads) *threads = L.shape.threads;
    if (lean) *lean = L.shape.lean;
    if (stage) *stage = L.shape.plane ? 1 + L.shape.plane : L.shape.stage;
    return MG3D_OK;
}

int mg3d_check_profiles(int n, double a, const double *x_host, const double *xp_host,
                        double *out_host) {
    if (n < 1 || !x_host || !xp_host || !out_host || !(a >= 0.0 && a < 1e3))
        return fail(MG3D_E_ARG, "bad arguments");
    for (int i = 0; i < n; ++i) {
        out_host[2 * i] = voigt_H(a, x_host[i]);
        out_host[2 * i + 1] = redistribution_r2a(x_host[i], xp_host[i], a);
    }
    return MG3D_OK;
}

int mg3d_check_voigt(int n, const double *a_host, const double *x_host, double *out_host) {
    if (n < 1 || !a_host || !x_host || !out_host) return fail(MG3D_E_ARG, "bad arguments");
    for (int i = 0; i < n; ++i)
        if (!(a_host[i] > 0.0 && a_host[i] < INFINITY) || !std::isfinite(x_host[i]))
            return fail(MG3D_E_ARG, "a must be positive and finite, x finite");
    const VoigtTable &tab = voigt_coefficients();
    for (int i = 0; i < n; ++i) out_host[i] = voigt_H_rational(tab, a_host[i], x_host[i]);
    return MG3D_OK;
}

int mg3d_check_exp(int n, const double *x_host, double *out_host) {
    if (n < 1 || !x_host || !out_host) return fail(MG3D_E_ARG, "bad arguments");
    double tab[kExpTab], l1, l2;
    exp_neg_constants(tab, &l1, &l2);
    double *d = nullptr;
    MG_TRY(dalloc(&d, kExpTab + 3 * (size_t)n));
    int rc = MG3D_OK;
    double *dx = d + kExpTab, *dout = dx + n;
    cudaError_t e = cudaMemcpy(d, tab, sizeof(tab), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x_host, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_exp_check(n, dx, dout, d, l1, l2, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out_host, dout, 2 * n * sizeof(double),
                                         cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = fail(MG3D_E_CUDA, std::string("exp check: ") + cudaGetErrorString(e));
    cudaFree(d);
    return rc;
}

int mg3d_set_graphs(mg3d_handle *h, int enable) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    MG_CUDA(cudaStreamSynchronize(h->stream));
    h->use_graphs = enable != 0;
    if (!h->use_graphs) drop_graphs(h);
    return MG3D_OK;
}

int mg3d_set_timing(mg3d_handle *h, int enable) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    MG_CUDA(cudaStreamSynchronize(h->stream));
    if ((enable != 0) != h->timing) drop_graphs(h);
    h->timing = enable != 0;
    return MG3D_OK;
}

int mg3d_get_counters(mg3d_handle *h, mg3d_counters *out) {
    if (!h || !out) return fail(MG3D_E_ARG, "null argument");
    MG_CUDA(cudaStreamSynchronize(h->stream));
    std::memset(out, 0, sizeof(*out));
    for (auto &t : h->timed) {
        float ms = 0.f;
        MG_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
        out->fs_kernel_ms += ms;
        ++out->fs_timed_launches;
        out->level_fs_kernel_ms[t.level] += ms;
        ++out->level_fs_timed_launches[t.level];
    }
    for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) {
        out->fs_kernel_ms += h->acc_ms[k];
        out->fs_timed_launches += h->acc_n[k];
        out->level_fs_kernel_ms[k] += h->acc_ms[k];
        out->level_fs_timed_launches[k] += h->acc_n[k];
    }
    out->kernel_launches = h->launches;
    out->fs_launches = h->fs_launches;
    out->fs_units = h->fs_units;
    for (int k = 0; k <= MG3D_MAX_GRIDS; ++k) {
        out->level_fs_launches[k] = h->level_launches[k];
        out->level_fs_units[k] = h->level_units[k];
    }
    return MG3D_OK;
}

int mg3d_reset_counters(mg3d_handle *h) {
    if (!h) return fail(MG3D_E_ARG, "null handle");
    MG_CUDA(cudaStreamSynchronize(h->stream));
    for (auto &t : h->timed) {
        h->event_pool.push_back(t.a);
        h->event_pool.push_back(t.b);
    }
    h->timed.clear();
    h->launches = 0;
    h->fs_launches = 0;
    h->fs_units = 0;
    std::memset(h->level_launches, 0, sizeof(h->level_launches));
    std::memset(h->level_units, 0, sizeof(h->level_units));
    std::memset(h->acc_ms, 0, sizeof(h->acc_ms));
    std::memset(h->acc_n, 0, sizeof(h->acc_n));
    return MG3D_OK;
}

}  // extern "C"
