// Formal solution: opacity/source kernel and the plane-sweep kernel.
//
// The transfer equation (Eq. 1) is solved with short characteristics and
// linear interpolation (Sec. 3, Kunasz & Auer 1988) for the 24 rays of the A4
// set.  For a ray going up, plane k depends only on plane k-1: the short
// characteristic of each node crosses plane k-1 at the same horizontal offset
// for all nodes of the plane (periodic in x and y, Sec. 4.2), so a whole plane
// is one parallel step and the sweep is a chain of nz dependent steps.
//
// GPU layout: one thread-block cluster per (ray, frequency group).  The
// cluster holds the intensity planes of that ray and group in shared memory,
// split in horizontal bands of rows, one band per block, double buffered
// (plane k-1 is read while plane k is written).  A block reads the upwind
// intensities of rows owned by another block of its cluster through
// distributed shared memory.  One cluster barrier per plane orders the steps;
// no global synchronisation is needed, and the intensities never leave the
// chip.  Opacity and source function of the two planes involved come from
// global memory (L2-resident at these sizes); their upwind interpolation is
// shared by all frequencies of the group, because for the two-level atom the
// opacity factorises as chi0(node) phi(nu) and S does not depend on nu.
//
// With the Hermite-spline option (Sec. 3) the upwind values come from a 4 x 4
// stencil instead: monotone cubic Hermite along x on the four rows around the
// crossing, then along y.  Each finished intensity plane gets its per-node
// x-slopes next to it in shared memory (one pass over the band after a block
// barrier), so that an upwind row costs four values and four products; chi0
// and S take their x-slopes from global memory, computed after the opacity.
//
// Each block accumulates, per node, the frequency sum of its group for
//   Jeff = sum w phi (I - w0 S)    and    U = sum w phi (1 - w0)
// and stores it into a partial slot (ray, group); the rate kernel adds the
// slots in a fixed order, so results are deterministic.
#include <cooperative_groups.h>
#include <cuda_pipeline.h>

#include <cmath>

#include "mg3d_internal.h"
#include "sc_step.cuh"

namespace cg = cooperative_groups;

namespace mg3d {

template <typename T>
__global__ void opacity_kernel(long nvox, double g_ratio, double kappa,
                               const double *__restrict__ n, T *__restrict__ chi0,
                               T *__restrict__ S) {
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x) {
        double nl = n[v], nu = n[nvox + v];
        double diff = nl * g_ratio - nu;
        chi0[v] = (T)(kappa * diff);
        S[v] = (T)(nu / diff);
    }
}

template <typename T>
__global__ void planck_bottom_kernel(long nplane, double theta, const double *__restrict__ Tgas,
                                     T *__restrict__ bbot) {
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < nplane;
         p += (long)gridDim.x * blockDim.x)
        bbot[p] = (T)(1.0 / expm1(theta / Tgas[p]));
}

// Shared-memory layout of one block (elements of T):
//   I planes      [2][ng][rows][nx]           plane k-1 read, plane k written
//   slope planes  [2][ng][rows][nx]           Hermite sweeps only: x-slopes of
//                                             the I planes
//   staging       [2][2][2 rows + 1][nx]      per step: chi0 and S of the
//                 upwind window (rows + 1 rows of plane k-1, shifted by the
//                 step's row offset) then of the block's own rows of plane k
//   tables        [4][ng]                     phi, 1/phi, w phi of the group, and
//                                             the w phi summed over frequencies
//                                             sharing weights (for U)
// Staging for step t+1 is copied asynchronously while step t computes.
__host__ __device__ inline long sweep_stage_elems(int rows, int nx) {
    return 2L * (2 * rows + 1) * nx;
}

template <typename T>
__device__ __forceinline__ void stage_rows(const SweepArgs<T> &a, T *dst, long arr_stride,
                                           int plane, int row0, int nrows, bool wrap,
                                           bool vec16) {
    // rows row0 .. row0+nrows-1 of `plane` (mod ny when wrap) of chi0 into
    // dst and of S into dst + arr_stride
    const int nx = a.nx, ny = a.ny;
    const long nplane = (long)nx * ny;
    const int per_row = vec16 ? (int)(nx * sizeof(T) / 16) : nx;
    const int total = 2 * nrows * per_row;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int arr = i / (nrows * per_row);
        const int rem = i - arr * nrows * per_row;
        const int j = rem / per_row, c = rem - j * per_row;
        int row = row0 + j;
        if (wrap && row >= ny) row -= ny;
        const T *src = (arr == 0 ? a.chi0 : a.S) + (long)plane * nplane + (long)row * nx;
        T *d = dst + arr * arr_stride + (long)j * nx;
        if (vec16)
            __pipeline_memcpy_async(d + c * (16 / sizeof(T)), src + c * (16 / sizeof(T)), 16);
        else
            __pipeline_memcpy_async(d + c, src + c, sizeof(T));
    }
}

// One sweep step (plane k from upwind plane kp) of a block's band with
// monotone cubic Hermite upwind interpolation: for each node the rows
// ya-1, ya, ya+1, ya+2 (periodic) of plane kp are interpolated along x at
// tx (values and slopes at xa and xa+1), then the four results along y at
// ty.  chi0 and S come from global memory with their x-slopes; I and its
// slopes from the block's or a peer block's shared memory.  Weights,
// accumulation and the mirror-frequency sharing are those of the linear
// step.
template <typename T, typename Fresh>
__device__ __forceinline__ void hermite_step(
    const SweepArgs<T> &a, int rank, unsigned long long rmagic, cg::cluster_group &cluster,
    const T *prev, const T *dprev, T *cur, T *__restrict__ pj, T *__restrict__ pu, int k, int kp,
    const StepGeom &o, T half_s, int nf, const T *phi, const T *inv_phi, const T *wphi,
    const T *wu, const ExpNegTable &et, const Fresh &is_fresh) {
    const int nx = a.nx, ny = a.ny, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = max(0, min(rows, ny - y0));
    const int band = myrows * nx;
    const long nplane = (long)nx * ny;
    const HermiteBasis<T> bx((T)o.tx), by((T)o.ty);
    for (int q = threadIdx.x; q < band; q += blockDim.x) {
        const int yl = q / nx, x = q - yl * nx;
        const int y = y0 + yl;
        int xa = x + o.ix0;
        if (xa >= nx) xa -= nx;
        const int xb = (xa + 1 == nx) ? 0 : xa + 1;
        int ya = y + o.iy0;
        if (ya >= ny) ya -= ny;
        int yr[4];
        yr[1] = ya;
        yr[0] = ya == 0 ? ny - 1 : ya - 1;
        yr[2] = ya + 1 == ny ? 0 : ya + 1;
        yr[3] = yr[2] + 1 == ny ? 0 : yr[2] + 1;
        const long pp = (long)kp * nplane, pk = (long)k * nplane + (long)y * nx;
        auto up2d = [&](const T *v, const T *d) {
            T gq[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const long ro = (long)yr[m] * nx;
                gq[m] = bx.at(v[ro + xa], d[ro + xa], v[ro + xb], d[ro + xb]);
            }
            return by.through4(gq[0], gq[1], gq[2], gq[3]);
        };
        const T chi_up = up2d(a.chi0 + pp, a.dchi0 + pp);
        const T S_up = up2d(a.S + pp, a.dS + pp);
        const T chi_loc = a.chi0[pk + x];
        const T S_loc = a.S[pk + x];
        const T dtau0 = (chi_up + chi_loc) * half_s;
        const T inv_dtau0 = sc_rcp(dtau0);
        // the four upwind rows of the intensity and slope planes
        const T *P[4], *D[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int b = band_of(yr[m], rmagic);
            const long ro = (long)(yr[m] - b * rows) * nx;
            P[m] = (b == rank ? prev : cluster.map_shared_rank(prev, b)) + ro;
            D[m] = (b == rank ? dprev : cluster.map_shared_rank(dprev, b)) + ro;
        }
        T cj = 0, cu = 0;
        auto step = [&](int f, T ex, T w0, T wup) {
            const long off = (long)f * rows * nx;
            T gq[4];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                gq[m] = bx.at(P[m][off + xa], D[m][off + xa], P[m][off + xb], D[m][off + xb]);
            const T I_up = by.through4(gq[0], gq[1], gq[2], gq[3]);
            const T part = I_up * ex + wup * S_up;
            cur[((long)f * rows + yl) * nx + x] = part + w0 * S_loc;
            cj += wphi[f] * part;
        };
        for (int f = 0; f < nf;) {
            const bool a2 = f + 1 < nf && !is_fresh(f + 1);
            T ex, w0, wup, u;
            ScWeights<T>::eval(dtau0 * phi[f], inv_dtau0 * inv_phi[f], et, ex, w0, wup, u);
            cu += wu[f] * u;
            step(f, ex, w0, wup);
            if (a2) step(f + 1, ex, w0, wup);
            f += a2 ? 2 : 1;
        }
        const long v = (long)k * nplane + (long)y * nx + x;
        pj[v] = cj;
        pu[v] = cu;
    }
}

// Doppler profile exp(-d2)/sqrt(pi) in the formal-solution precision.
__device__ __forceinline__ double doppler_profile(double d2, const ExpNegTable &et) {
    return 0.56418958354775628 * exp_neg(d2, et);
}
__device__ __forceinline__ float doppler_profile(float d2, const ExpNegTable &) {
    return 0.564189584f * __expf(-d2);
}

// One sweep step of a band in a moving atmosphere (CRD).  Along ray r the
// profile of frequency x_f at a node is phi(x_f - u) with u the velocity
// projected on the ray (in Doppler widths), so the line opacity chi0 phi
// depends on node, ray and frequency: it is formed at the node, used for
// the node's half of the optical depth and kept in the opacity plane next to
// the intensity plane, where the next step interpolates its upwind value
// like the intensity's.  The frequency weights are w_f phi(x_f - u) times
// the node's and ray's normalisation, so that they sum to 1 over all
// frequencies.  Mirror frequencies no longer share weights.
template <typename T>
__device__ __forceinline__ void moving_step(
    const SweepArgs<T> &a, int r, int rank, unsigned long long rmagic, cg::cluster_group &cluster,
    const T *prev, const T *cprev, T *cur, T *ccur, T *__restrict__ pj, T *__restrict__ pu, int k,
    int kp, const StepGeom &o, T half_s, int f0, int nf, const ExpNegTable &et) {
    const int nx = a.nx, ny = a.ny, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = max(0, min(rows, ny - y0));
    const int band = myrows * nx;
    const long nplane = (long)nx * ny;
    const long nvox = nplane * a.nz;
    const T tx = (T)o.tx, ty = (T)o.ty;
    const T w00 = (T(1) - tx) * (T(1) - ty), w10 = tx * (T(1) - ty);
    const T w01 = (T(1) - tx) * ty, w11 = tx * ty;
    const long pp = (long)kp * nplane;
    for (int q = threadIdx.x; q < band; q += blockDim.x) {
        const int yl = q / nx, x = q - yl * nx;
        const int y = y0 + yl;
        int xa = x + o.ix0;
        if (xa >= nx) xa -= nx;
        const int xb = (xa + 1 == nx) ? 0 : xa + 1;
        int ya = y + o.iy0;
        if (ya >= ny) ya -= ny;
        const int yb = (ya + 1 == ny) ? 0 : ya + 1;
        const T *sa = a.S + pp + (long)ya * nx, *sb = a.S + pp + (long)yb * nx;
        const T S_up = w00 * sa[xa] + w10 * sa[xb] + w01 * sb[xa] + w11 * sb[xb];
        const long v = (long)k * nplane + (long)y * nx + x;
        const T S_loc = a.S[v], c0 = a.chi0[v];
        const T u = a.uproj[(long)r * nvox + v], nrm = a.vnorm[(long)r * nvox + v];
        const int ba = band_of(ya, rmagic), bb = band_of(yb, rmagic);
        const long ra = (long)(ya - ba * rows) * nx, rb = (long)(yb - bb * rows) * nx;
        const T *Pa = (ba == rank ? prev : cluster.map_shared_rank(prev, ba)) + ra;
        const T *Pb = (bb == rank ? prev : cluster.map_shared_rank(prev, bb)) + rb;
        const T *Ca = (ba == rank ? cprev : cluster.map_shared_rank(cprev, ba)) + ra;
        const T *Cb = (bb == rank ? cprev : cluster.map_shared_rank(cprev, bb)) + rb;
        T cj = 0, cu = 0;
        for (int f = 0; f < nf; ++f) {
            const long off = (long)f * rows * nx;
            const T d = a.xf[f0 + f] - u;
            const T prof = doppler_profile(d * d, et);
            const T chi_loc = c0 * prof;
            const T chi_up = w00 * Ca[off + xa] + w10 * Ca[off + xb] + w01 * Cb[off + xa] +
                             w11 * Cb[off + xb];
            const T I_up = w00 * Pa[off + xa] + w10 * Pa[off + xb] + w01 * Pb[off + xa] +
                           w11 * Pb[off + xb];
            const T dtau = (chi_up + chi_loc) * half_s;
            T ex, w0, wup, uu;
            ScWeights<T>::eval(dtau, sc_rcp(dtau), et, ex, w0, wup, uu);
            const T part = I_up * ex + wup * S_up;
            const long i = off + (long)yl * nx + x;
            cur[i] = part + w0 * S_loc;
            ccur[i] = chi_loc;
            const T w = a.wq[f0 + f] * prof * nrm;
            cj += w * part;
            cu += w * uu;
        }
        pj[v] = cj;
        pu[v] = cu;
    }
}

// One sweep step of a band with partial redistribution (two-level atom):
// the opacity is the static chi0 phi_f, so mirror frequencies share their
// step weights, but the source function rho_f S depends on the frequency.
// Its upwind value is interpolated per frequency from global memory; U takes
// w phi (1 - w0 rho_f); every new intensity, with the ray weight, is stored
// in the ray's slot of the new mean intensity (each (ray, frequency, node)
// has one writer; the slots are added in ray order afterwards, so the sum
// does not depend on scheduling).
template <typename T>
__device__ __forceinline__ void prd_step(
    const SweepArgs<T> &a, int r, int rank, unsigned long long rmagic, cg::cluster_group &cluster,
    const T *prev, T *cur, T *__restrict__ pj, T *__restrict__ pu, int k, int kp,
    const StepGeom &o, T half_s, int f0, int nf, const T *phi, const T *inv_phi, const T *wphi,
    const ExpNegTable &et) {
    const int nx = a.nx, ny = a.ny, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = max(0, min(rows, ny - y0));
    const int band = myrows * nx;
    const long nplane = (long)nx * ny;
    const long nvox = nplane * a.nz;
    const T tx = (T)o.tx, ty = (T)o.ty;
    const T w00 = (T(1) - tx) * (T(1) - ty), w10 = tx * (T(1) - ty);
    const T w01 = (T(1) - tx) * ty, w11 = tx * ty;
    const long pp = (long)kp * nplane;
    const T wr = T(1.0 / kRays);
    for (int q = threadIdx.x; q < band; q += blockDim.x) {
        const int yl = q / nx, x = q - yl * nx;
        const int y = y0 + yl;
        int xa = x + o.ix0;
        if (xa >= nx) xa -= nx;
        const int xb = (xa + 1 == nx) ? 0 : xa + 1;
        int ya = y + o.iy0;
        if (ya >= ny) ya -= ny;
        const int yb = (ya + 1 == ny) ? 0 : ya + 1;
        const T *ca = a.chi0 + pp + (long)ya * nx, *cb = a.chi0 + pp + (long)yb * nx;
        const T chi_up = w00 * ca[xa] + w10 * ca[xb] + w01 * cb[xa] + w11 * cb[xb];
        const long v = (long)k * nplane + (long)y * nx + x;
        const T dtau0 = (chi_up + a.chi0[v]) * half_s;
        const T inv_dtau0 = sc_rcp(dtau0);
        const int ba = band_of(ya, rmagic), bb = band_of(yb, rmagic);
        const T *Pa = (ba == rank ? prev : cluster.map_shared_rank(prev, ba)) +
                      (long)(ya - ba * rows) * nx;
        const T *Pb = (bb == rank ? prev : cluster.map_shared_rank(prev, bb)) +
                      (long)(yb - bb * rows) * nx;
        T cj = 0, cu = 0;
        for (int f = 0; f < nf; ++f) {
            const long fo = (long)a.fidx[f0 + f] * nvox;
            const T *sa = a.rhoS + fo + pp + (long)ya * nx;
            const T *sb = a.rhoS + fo + pp + (long)yb * nx;
            const T S_up = w00 * sa[xa] + w10 * sa[xb] + w01 * sb[xa] + w11 * sb[xb];
            const T S_loc = a.rhoS[fo + v], rho_loc = a.rho[fo + v];
            T ex, w0, wup, uu;
            ScWeights<T>::eval(dtau0 * phi[f], inv_dtau0 * inv_phi[f], et, ex, w0, wup, uu);
            const long off = (long)f * rows * nx;
            const T I_up = w00 * Pa[off + xa] + w10 * Pa[off + xb] + w01 * Pb[off + xa] +
                           w11 * Pb[off + xb];
            const T part = I_up * ex + wup * S_up;
            const T I = part + w0 * S_loc;
            cur[off + (long)yl * nx + x] = I;
            cj += wphi[f] * part;
            cu += wphi[f] * (T(1) - w0 * rho_loc);
            a.jnu[(long)r * a.nfreq * nvox + fo + v] = wr * I;
        }
        pj[v] = cj;
        pu[v] = cu;
    }
}

// Body of the sweep for ray r and frequency group g of one problem.  STAGE:
// chi0 and S rows of each step are copied to shared memory one step ahead;
// without it they are read from global memory (L1/L2) where used.  HERM:
// monotone cubic Hermite upwind interpolation (unstaged).  MODE: kSweepLinear,
// kSweepHermite (Hermite upwind interpolation) or kSweepMoving (a velocity
// field; unstaged).
template <typename T, bool STAGE, int MODE>
__device__ __forceinline__ void sweep_body(const SweepArgs<T> &a, int g, int r) {
    constexpr bool HERM = MODE == kSweepHermite, VEL = MODE == kSweepMoving;
    constexpr bool PRD = MODE == kSweepPrd;
    static_assert(!(STAGE && MODE != kSweepLinear), "Hermite and moving sweeps run unstaged");
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int nx = a.nx, ny = a.ny, nz = a.nz, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = max(0, min(rows, ny - y0));
    const int band = myrows * nx;
    const int f0 = g * a.ng;
    const int nf = min(a.ng, a.nfreq - f0);
    const bool up = (a.up_mask >> r) & 1u;
    const long nplane = (long)nx * ny;
    const long nvox = nplane * nz;
    const long slot = (long)r * a.ngroups + g;
    T *__restrict__ pj = a.pj + slot * nvox;
    T *__restrict__ pu = a.pu + slot * nvox;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const long bufstride = (long)a.ng * rows * nx;
    T *dbuf = buf + 2 * bufstride;  // slope planes (HERM) or opacity planes (VEL)
    // Hermite and moving sweeps keep a second plane pair (sweep_smem_bytes)
    T *stage = buf + ((HERM || VEL) ? 4 : 2) * bufstride;
    const long stagestride = STAGE ? sweep_stage_elems(rows, nx) : 0;
    T *tabs = stage + 2 * stagestride;
    T *phi = tabs, *inv_phi = tabs + a.ng, *wphi = tabs + 2 * a.ng, *wu = tabs + 3 * a.ng;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        phi[i] = a.phi[f0 + i];
        inv_phi[i] = a.inv_phi[f0 + i];
        wphi[i] = a.wphi[f0 + i];
    }
    __shared__ double exp_tab[kExpTab];
    if (sizeof(T) == 8)
        for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) exp_tab[i] = a.exp_tab[i];
    __syncthreads();
    const ExpNegTable et{exp_tab, a.exp_l1, a.exp_l2};
    const bool vec16 = (nx * sizeof(T)) % 16 == 0;
    const unsigned long long rmagic = band_magic(rows);
    // bit f set: frequency f needs its own weights; clear: its phi equals
    // that of frequency f-1 (mirror halves of the profile stored next to
    // each other), so the weights of f-1, still in registers, are its own
    unsigned long long fresh = ~0ull;
    for (int f = 1; f < nf && f < 64; ++f)
        if (phi[f] == phi[f - 1]) fresh &= ~(1ull << f);
    auto is_fresh = [&](int f) { return f >= 64 || ((fresh >> f) & 1ull); };
    // frequencies that share weights share u: U gets their summed w phi once
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        T w = 0;
        if (is_fresh(f)) {
            w = wphi[f];
            for (int h = f + 1; h < nf && !is_fresh(h); ++h) w += wphi[h];
        }
        wu[f] = w;
    }
    __syncthreads();

    // stage the window and band of step t into staging buffer t & 1
    auto stage_step = [&](int t) {
        const int k = up ? t : nz - 1 - t;
        const int kp = up ? k - 1 : k + 1;
        const StepGeom o = a.geom[(long)r * nz + t];
        T *dst = stage + (t & 1) * stagestride;
        int w0 = y0 + o.iy0;
        if (w0 >= ny) w0 -= ny;
        stage_rows<T>(a, dst, (long)(rows + 1) * nx, kp, w0, myrows + 1, true, vec16);
        stage_rows<T>(a, dst + 2L * (rows + 1) * nx, (long)rows * nx, k, y0, myrows, false,
                      vec16);
        __pipeline_commit();
    };
    if (STAGE && nz > 1) stage_step(1);

    for (int t = 0; t < nz; ++t) {
        const int k = up ? t : nz - 1 - t;
        T *cur = buf + (t & 1) * bufstride;
        if (t == 0 && VEL) {
            // entering boundary of a moving atmosphere: I prescribed, w0 = 0;
            // the opacity plane gets the shifted profile for the next step
            T *ccur = dbuf + (t & 1) * bufstride;
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                const long v = (long)k * nplane + (long)y * nx + x;
                const T Ib = up ? a.bbot[(long)y * nx + x] : T(0);
                const T u = a.uproj[(long)r * nvox + v], nrm = a.vnorm[(long)r * nvox + v];
                const T c0 = a.chi0[v];
                T cj = 0, cu = 0;
                for (int f = 0; f < nf; ++f) {
                    const T d = a.xf[f0 + f] - u;
                    const T prof = doppler_profile(d * d, et);
                    const long i = ((long)f * rows + yl) * nx + x;
                    cur[i] = Ib;
                    ccur[i] = c0 * prof;
                    const T w = a.wq[f0 + f] * prof * nrm;
                    cj += w * Ib;
                    cu += w;
                }
                pj[v] = cj;
                pu[v] = cu;
            }
        } else if (t == 0 && PRD) {
            // entering boundary with partial redistribution: as below, and
            // the intensity enters the new mean intensity of its frequency
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                const long v = (long)k * nplane + (long)y * nx + x;
                const T Ib = up ? a.bbot[(long)y * nx + x] : T(0);
                T cj = 0, cu = 0;
                for (int f = 0; f < nf; ++f) {
                    cur[((long)f * rows + yl) * nx + x] = Ib;
                    cj += wphi[f] * Ib;
                    cu += wphi[f];
                    a.jnu[((long)r * a.nfreq + a.fidx[f0 + f]) * nvox + v] = Ib * T(1.0 / kRays);
                }
                pj[v] = cj;
                pu[v] = cu;
            }
        } else if (t == 0) {
            // entering boundary: I prescribed (bottom: Planck at the local
            // temperature; top: zero), so w0 = 0 and 1 - w0 = 1
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                const T Ib = up ? a.bbot[(long)y * nx + x] : T(0);
                T cj = 0, cu = 0;
                for (int f = 0; f < nf; ++f) {
                    cur[((long)f * rows + yl) * nx + x] = Ib;
                    const T w = wphi[f];
                    cj += w * Ib;
                    cu += w;
                }
                const long v = (long)k * nplane + (long)y * nx + x;
                pj[v] = cj;
                pu[v] = cu;
            }
        } else {
            if constexpr (STAGE) {
                __pipeline_wait_prior(0);
                __syncthreads();
                if (t + 1 < nz) stage_step(t + 1);
            }
            const T *st = stage + (t & 1) * stagestride;
            const T *chiW = st, *SW = st + (long)(rows + 1) * nx;
            const T *chiB = st + 2L * (rows + 1) * nx, *SB = chiB + (long)rows * nx;
            const int kp = up ? k - 1 : k + 1;
            const T *prev = buf + ((t - 1) & 1) * bufstride;
            const StepGeom o = a.geom[(long)r * nz + t];
            const T tx = (T)o.tx, ty = (T)o.ty;
            const T half_s = (T)(0.5 * o.s);
            const T w00 = (T(1) - tx) * (T(1) - ty), w10 = tx * (T(1) - ty);
            const T w01 = (T(1) - tx) * ty, w11 = tx * ty;
            if constexpr (HERM) {
                hermite_step(a, rank, rmagic, cluster, prev, dbuf + ((t - 1) & 1) * bufstride,
                             cur, pj, pu, k, kp, o, half_s, nf, phi, inv_phi, wphi, wu, et,
                             is_fresh);
            } else if constexpr (VEL) {
                moving_step(a, r, rank, rmagic, cluster, prev, dbuf + ((t - 1) & 1) * bufstride,
                            cur, dbuf + (t & 1) * bufstride, pj, pu, k, kp, o, half_s, f0, nf,
                            et);
            } else if constexpr (PRD) {
                prd_step(a, r, rank, rmagic, cluster, prev, cur, pj, pu, k, kp, o, half_s, f0, nf,
                         phi, inv_phi, wphi, et);
            } else
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int y = y0 + yl;
                int xa = x + o.ix0;
                if (xa >= nx) xa -= nx;
                const int xb = (xa + 1 == nx) ? 0 : xa + 1;
                int ya = y + o.iy0;
                if (ya >= ny) ya -= ny;
                const int yb = (ya + 1 == ny) ? 0 : ya + 1;
                // rows ya, yb of chi0 and S on plane kp, row y on plane k:
                // staged (window row yl holds ya, row yl + 1 holds yb) or in
                // global memory
                const T *ca, *cb, *sa, *sb, *cl, *sl;
                if constexpr (STAGE) {
                    ca = chiW + (long)yl * nx;
                    cb = ca + nx;
                    sa = SW + (long)yl * nx;
                    sb = sa + nx;
                    cl = chiB + (long)yl * nx;
                    sl = SB + (long)yl * nx;
                } else {
                    const long pp = (long)kp * nplane, pk = (long)k * nplane + (long)y * nx;
                    ca = a.chi0 + pp + (long)ya * nx;
                    cb = a.chi0 + pp + (long)yb * nx;
                    sa = a.S + pp + (long)ya * nx;
                    sb = a.S + pp + (long)yb * nx;
                    cl = a.chi0 + pk;
                    sl = a.S + pk;
                }
                const T chi_up = w00 * ca[xa] + w10 * ca[xb] + w01 * cb[xa] + w11 * cb[xb];
                const T S_up = w00 * sa[xa] + w10 * sa[xb] + w01 * sb[xa] + w11 * sb[xb];
                const T chi_loc = cl[x];
                const T S_loc = sl[x];
                const T dtau0 = (chi_up + chi_loc) * half_s;
                // 1/dtau0 is only used where dtau0 phi >= the series threshold,
                // so dtau0 > 0 there
                const T inv_dtau0 = sc_rcp(dtau0);
                // upwind rows of the intensity planes: local or in a peer block
                const int ba = band_of(ya, rmagic), bb = band_of(yb, rmagic);
                const T *Pa = (ba == rank) ? prev : cluster.map_shared_rank(prev, ba);
                const T *Pb = (bb == rank) ? prev : cluster.map_shared_rank(prev, bb);
                Pa += (long)(ya - ba * rows) * nx;
                Pb += (long)(yb - bb * rows) * nx;
                T cj = 0, cu = 0;
                // new intensity of frequency f from its step weights
                auto step = [&](int f, T ex, T w0, T wup) {
                    const long off = (long)f * rows * nx;
                    const T I_up = w00 * Pa[off + xa] + w10 * Pa[off + xb] +
                                   w01 * Pb[off + xa] + w11 * Pb[off + xb];
                    const T part = I_up * ex + wup * S_up;
                    cur[((long)f * rows + yl) * nx + x] = part + w0 * S_loc;
                    cj += wphi[f] * part;
                };
                // weight slots: a frequency and, when its mirror follows, the
                // mirror.  FP32 takes two slots per pass, so that their
                // independent weight evaluations overlap (its pipes wait on
                // latency); FP64 is bound by the FP64 pipe's throughput, where
                // the extra registers of two slots cost more than they hide.
                constexpr bool kTwoSlots = sizeof(T) == 4;
                for (int f = 0; f < nf;) {
                    const bool a2 = f + 1 < nf && !is_fresh(f + 1);
                    const int fb = f + (a2 ? 2 : 1);
                    if (kTwoSlots && fb < nf) {
                        const bool b2 = fb + 1 < nf && !is_fresh(fb + 1);
                        const T xa_ = dtau0 * phi[f], xb_ = dtau0 * phi[fb];
                        T exa, w0a, wupa, ua, exb, w0b, wupb, ub;
                        ScWeights<T>::closed(xa_, inv_dtau0 * inv_phi[f], et, exa, w0a, wupa, ua);
                        ScWeights<T>::closed(xb_, inv_dtau0 * inv_phi[fb], et, exb, w0b, wupb,
                                             ub);
                        if (ScWeights<T>::small(xa_)) ScWeights<T>::series(xa_, w0a, wupa, ua);
                        if (ScWeights<T>::small(xb_)) ScWeights<T>::series(xb_, w0b, wupb, ub);
                        cu += wu[f] * ua;
                        cu += wu[fb] * ub;
                        step(f, exa, w0a, wupa);
                        if (a2) step(f + 1, exa, w0a, wupa);
                        step(fb, exb, w0b, wupb);
                        if (b2) step(fb + 1, exb, w0b, wupb);
                        f = fb + (b2 ? 2 : 1);
                    } else {
                        T ex, w0, wup, u;
                        ScWeights<T>::eval(dtau0 * phi[f], inv_dtau0 * inv_phi[f], et, ex, w0,
                                           wup, u);
                        cu += wu[f] * u;
                        step(f, ex, w0, wup);
                        if (a2) step(f + 1, ex, w0, wup);
                        f = fb;
                    }
                }
                const long v = (long)k * nplane + (long)y * nx + x;
                pj[v] = cj;
                pu[v] = cu;
            }
        }
        if constexpr (HERM) {
            // x-slopes of the new plane; a band holds whole rows
            __syncthreads();
            T *dcur = dbuf + (t & 1) * bufstride;
            for (int q = threadIdx.x; q < band; q += blockDim.x) {
                const int yl = q / nx, x = q - yl * nx;
                const int xm = x == 0 ? nx - 1 : x - 1, xp = x + 1 == nx ? 0 : x + 1;
                for (int f = 0; f < nf; ++f) {
                    const long row = ((long)f * rows + yl) * nx;
                    dcur[row + x] =
                        mono_slope(cur[row + x] - cur[row + xm], cur[row + xp] - cur[row + x]);
                }
            }
        }
        // plane t complete in every block before any block reads it, and no
        // block overwrites plane t-1 (written again at t+1) while it is read
        cluster.sync();
    }
}

// MAXT: the block size bound the kernel is compiled for (256 or 512); MINB:
// blocks per SM it must fit, which sets the register budget (MINB = 1: up to
// 255 registers; 1024/MAXT: 64 registers, 32 resident warps per SM; 3 blocks
// of 256: 85 registers).
template <typename T, int MAXT, int MINB, bool STAGE, int MODE>
__global__ void __launch_bounds__(MAXT, MINB) sweep_kernel(const SweepArgs<T> a) {
    sweep_body<T, STAGE, MODE>(a, blockIdx.y, blockIdx.z);
}

// Batched sweep: cluster y of the grid runs work item items[y] = (problem,
// ray, group) of problems args[]; every problem uses the launch's number of
// bands.
template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, 1024 / MAXT) sweep_batch_kernel(
    const SweepArgs<T> *__restrict__ args, const BatchItem *__restrict__ items) {
    const BatchItem it = items[blockIdx.y];
    const SweepArgs<T> a = args[it.member];
    sweep_body<T, true, kSweepLinear>(a, it.group, it.ray);
}

__global__ void exp_check_kernel(int n, const double *__restrict__ x, double *__restrict__ out,
                                 const double *__restrict__ tab, double l1, double l2) {
    const ExpNegTable et{tab, l1, l2};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[2 * i] = exp_neg(x[i], et);
        out[2 * i + 1] = exp(-x[i]);
    }
}

cudaError_t launch_exp_check(int n, const double *x, double *out, const double *tab, double l1,
                             double l2, cudaStream_t st) {
    exp_check_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, x, out, tab, l1, l2);
    return cudaGetLastError();
}

void exp_neg_constants(double *tab, double *l1, double *l2) {
    // 2^{j/256} correctly rounded through the wider long double
    for (int j = 0; j < kExpTab; ++j)
        tab[j] = (double)exp2l((long double)j / (long double)kExpTab);
    // ln2 = LN2_HI + LN2_LO to about 1e-33
    const double ln2_hi = 0.6931471805599453094172321;
    const double ln2_lo = 2.3190468138462996e-17;
    const double c = ln2_hi / kExpTab;                // exact: division by a power of two
    // high part: c truncated to 34 significant bits (c is in [2^-9, 2^-8))
    const double hi = std::ldexp(std::floor(std::ldexp(c, 34 + 8)), -(34 + 8));
    *l1 = hi;
    *l2 = (c - hi) + ln2_lo / kExpTab;
}

size_t sweep_smem_bytes(int prec, const SweepShape &s, int nx) {
    size_t elem = prec == 0 ? sizeof(double) : sizeof(float);
    return ((s.herm || s.vel ? 4ull : 2ull) * s.ng * s.rows * nx +
            (s.stage ? 2ull * sweep_stage_elems(s.rows, nx) : 0ull) + 4ull * s.ng) *
           elem;
}

// Kernel attributes for shape s (dynamic shared memory; clusters of more
// than 8 blocks are a non-portable size the kernel must opt into) and the
// launch configuration; a is null for an occupancy query.
template <typename T, int MAXT, int MINB, bool STAGE, int MODE>
static cudaError_t sweep_config(const SweepShape &s, int nx, cudaStream_t st,
                                cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr) {
    const size_t smem = sweep_smem_bytes(sizeof(T) == 8 ? 0 : 1, s, nx);
    // the limit is the same for every launch: a CUDA graph that captured a
    // launch needing more than a later launch of the same kernel must still
    // find the attribute large enough when it replays
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<T, MAXT, MINB, STAGE, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSweepSmem);
    if (e == cudaSuccess && s.bands > kPortableBands)
        e = cudaFuncSetAttribute(sweep_kernel<T, MAXT, MINB, STAGE, MODE>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(s.bands, s.ngroups, kRays);
    cfg->blockDim = dim3(s.threads, 1, 1);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s.bands;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    // one band: a plain launch (its implicit one-block cluster)
    cfg->numAttrs = s.bands > 1 ? 1 : 0;
    return cudaSuccess;
}

template <typename T, int MAXT, int MINB, bool STAGE, int MODE>
static cudaError_t launch_sweep_t(const SweepArgs<T> &a, const SweepShape &s,
                                  cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = sweep_config<T, MAXT, MINB, STAGE, MODE>(s, a.nx, st, &cfg, attr);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, sweep_kernel<T, MAXT, MINB, STAGE, MODE>, a);
}

template <typename T, int MAXT, int MINB, bool STAGE, int MODE>
static cudaError_t clusters_t(const SweepShape &s, int nx, int *n) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = sweep_config<T, MAXT, MINB, STAGE, MODE>(s, nx, 0, &cfg, attr);
    if (e != cudaSuccess) return e;
    if (s.bands == 1)  // plain launch: resident blocks per SM
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n,
                                                             sweep_kernel<T, MAXT, MINB, STAGE, MODE>,
                                                             s.threads, cfg.dynamicSmemBytes);
    return cudaOccupancyMaxActiveClusters(n, sweep_kernel<T, MAXT, MINB, STAGE, MODE>, &cfg);
}

template <typename T, bool STAGE, int MODE>
static cudaError_t launch_sweep_st(const SweepArgs<T> &a, const SweepShape &s, cudaStream_t st) {
    if (s.threads <= 256) {
        if (s.lean == 1) return launch_sweep_t<T, 256, 4, STAGE, MODE>(a, s, st);
        if (s.lean == 2) return launch_sweep_t<T, 256, 3, STAGE, MODE>(a, s, st);
        return launch_sweep_t<T, 256, 1, STAGE, MODE>(a, s, st);
    }
    return s.lean == 1 ? launch_sweep_t<T, 512, 2, STAGE, MODE>(a, s, st)
                       : launch_sweep_t<T, 512, 1, STAGE, MODE>(a, s, st);
}

template <typename T>
static cudaError_t launch_sweep_any(const SweepArgs<T> &a, const SweepShape &s,
                                    cudaStream_t st) {
    if (s.herm && s.vel) return cudaErrorInvalidValue;
    if (s.herm) {
        if (s.stage || !a.dchi0 || !a.dS) return cudaErrorInvalidValue;
        return launch_sweep_st<T, false, kSweepHermite>(a, s, st);
    }
    if (s.vel) {
        if (s.stage || !a.uproj || !a.vnorm || !a.xf || !a.wq) return cudaErrorInvalidValue;
        return launch_sweep_st<T, false, kSweepMoving>(a, s, st);
    }
    if (s.prd) {
        if (s.stage || !a.rhoS || !a.rho || !a.fidx || !a.jnu) return cudaErrorInvalidValue;
        return launch_sweep_st<T, false, kSweepPrd>(a, s, st);
    }
    return s.stage ? launch_sweep_st<T, true, kSweepLinear>(a, s, st)
                   : launch_sweep_st<T, false, kSweepLinear>(a, s, st);
}

template <typename T, bool STAGE, int MODE>
static cudaError_t clusters_st(const SweepShape &s, int nx, int *n) {
    if (s.threads <= 256) {
        if (s.lean == 1) return clusters_t<T, 256, 4, STAGE, MODE>(s, nx, n);
        if (s.lean == 2) return clusters_t<T, 256, 3, STAGE, MODE>(s, nx, n);
        return clusters_t<T, 256, 1, STAGE, MODE>(s, nx, n);
    }
    return s.lean == 1 ? clusters_t<T, 512, 2, STAGE, MODE>(s, nx, n)
                       : clusters_t<T, 512, 1, STAGE, MODE>(s, nx, n);
}

template <typename T>
static cudaError_t clusters_any(const SweepShape &s, int nx, int *n) {
    if ((s.herm || s.vel || s.prd) && s.stage) return cudaErrorInvalidValue;
    if (s.herm) return clusters_st<T, false, kSweepHermite>(s, nx, n);
    if (s.vel) return clusters_st<T, false, kSweepMoving>(s, nx, n);
    if (s.prd) return clusters_st<T, false, kSweepPrd>(s, nx, n);
    return s.stage ? clusters_st<T, true, kSweepLinear>(s, nx, n)
                   : clusters_st<T, false, kSweepLinear>(s, nx, n);
}

cudaError_t sweep_active_clusters(int prec, const SweepShape &s, int nx, int *n) {
    *n = 0;
    return prec == 0 ? clusters_any<double>(s, nx, n) : clusters_any<float>(s, nx, n);
}

template <typename T, int MAXT>
static cudaError_t launch_sweep_batch_t(const SweepArgs<T> *args, const BatchItem *items,
                                        int n_items, int bands, int threads, size_t smem,
                                        cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweep_batch_kernel<T, MAXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSweepSmem);  // fixed, as for sweep_kernel
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
    return cudaLaunchKernelEx(&cfg, sweep_batch_kernel<T, MAXT>, args, items);
}

cudaError_t launch_sweep_batch(int prec, const void *args, const BatchItem *items, int n_items,
                               int bands, int threads, size_t smem, cudaStream_t st) {
    if (prec == 0)
        return threads <= 256
                   ? launch_sweep_batch_t<double, 256>((const SweepArgs<double> *)args, items,
                                                       n_items, bands, threads, smem, st)
                   : launch_sweep_batch_t<double, 512>((const SweepArgs<double> *)args, items,
                                                       n_items, bands, threads, smem, st);
    return threads <= 256
               ? launch_sweep_batch_t<float, 256>((const SweepArgs<float> *)args, items, n_items,
                                                  bands, threads, smem, st)
               : launch_sweep_batch_t<float, 512>((const SweepArgs<float> *)args, items, n_items,
                                                  bands, threads, smem, st);
}

cudaError_t launch_sweep_f64(const SweepArgs<double> &a, const SweepShape &s, cudaStream_t st) {
    return launch_sweep_any<double>(a, s, st);
}

cudaError_t launch_sweep_f32(const SweepArgs<float> &a, const SweepShape &s, cudaStream_t st) {
    return launch_sweep_any<float>(a, s, st);
}

static int grid_for(long n, int threads) {
    long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152L * 32) b = 152L * 32;
    return (int)b;
}

cudaError_t launch_opacity(int prec, long nvox, double g_ratio, double kappa,
                           const double *n, void *chi0, void *S, cudaStream_t st) {
    const int th = 256;
    if (prec == 0)
        opacity_kernel<double><<<grid_for(nvox, th), th, 0, st>>>(
            nvox, g_ratio, kappa, n, (double *)chi0, (double *)S);
    else
        opacity_kernel<float><<<grid_for(nvox, th), th, 0, st>>>(
            nvox, g_ratio, kappa, n, (float *)chi0, (float *)S);
    return cudaGetLastError();
}

template <typename T>
__global__ void xslope_kernel(int nx, long nvox, const T *__restrict__ a, const T *__restrict__ b,
                              T *__restrict__ da, T *__restrict__ db) {
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx);
        const long vm = v + ((x == 0 ? nx - 1 : x - 1) - x);
        const long vp = v + ((x + 1 == nx ? 0 : x + 1) - x);
        da[v] = mono_slope(a[v] - a[vm], a[vp] - a[v]);
        db[v] = mono_slope(b[v] - b[vm], b[vp] - b[v]);
    }
}

cudaError_t launch_xslopes(int prec, int nx, long nvox, const void *a, const void *b, void *da,
                           void *db, cudaStream_t st) {
    const int th = 256;
    if (prec == 0)
        xslope_kernel<double><<<grid_for(nvox, th), th, 0, st>>>(
            nx, nvox, (const double *)a, (const double *)b, (double *)da, (double *)db);
    else
        xslope_kernel<float><<<grid_for(nvox, th), th, 0, st>>>(
            nx, nvox, (const float *)a, (const float *)b, (float *)da, (float *)db);
    return cudaGetLastError();
}

// Projected velocity u_r = mu_r . v and the inverse of kRays sum_f w_f
// phi(x_f - u_r) at every node, per ray (the velocity field of a level does
// not change), so that the weights w_f phi vnorm of a node and ray sum to the
// ray weight 1/kRays.
template <typename T>
__global__ void vel_prep_kernel(long nvox, int nfreq, const double *__restrict__ mu,
                                const double *__restrict__ vel, const double *__restrict__ xf,
                                const double *__restrict__ wq, T *__restrict__ uproj,
                                T *__restrict__ vnorm) {
    const long total = (long)kRays * nvox;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / nvox);
        const long v = i - (long)r * nvox;
        const double u = mu[3 * r] * vel[v] + mu[3 * r + 1] * vel[nvox + v] +
                         mu[3 * r + 2] * vel[2 * nvox + v];
        double sum = 0.0;
        for (int f = 0; f < nfreq; ++f) {
            const double d = xf[f] - u;
            sum += wq[f] * 0.56418958354775628 * exp(-d * d);
        }
        uproj[i] = (T)u;
        vnorm[i] = (T)(1.0 / (kRays * sum));  // with the ray weight 1/kRays
    }
}

cudaError_t launch_vel_prep(int prec, long nvox, int nfreq, const double *mu, const double *vel,
                            const double *xf, const double *wq, void *uproj, void *vnorm,
                            cudaStream_t st) {
    const int th = 256;
    const long total = (long)kRays * nvox;
    if (prec == 0)
        vel_prep_kernel<double><<<grid_for(total, th), th, 0, st>>>(
            nvox, nfreq, mu, vel, xf, wq, (double *)uproj, (double *)vnorm);
    else
        vel_prep_kernel<float><<<grid_for(total, th), th, 0, st>>>(
            nvox, nfreq, mu, vel, xf, wq, (float *)uproj, (float *)vnorm);
    return cudaGetLastError();
}

// Per node: Jbar = sum wphi_f J_f, f_rad = B_lu Jbar/(B_lu Jbar + C_lu),
// rho_f = 1 + gamma f_rad (sum_f' kmat[f'][f] J_f' / Jbar - 1) (1 where
// Jbar = 0), and rho_f S with S = n_u/(n_l g - n_u); sums in FP64.
template <typename T>
__global__ void prd_source_kernel(long nvox, int nfreq, double gamma, double g_ratio, double a_ul,
                                  const double *__restrict__ kmat,
                                  const double *__restrict__ wphi, const double *__restrict__ n,
                                  const double *__restrict__ c_lu, const T *__restrict__ jnu,
                                  T *__restrict__ rho, T *__restrict__ rhoS) {
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x) {
        double jbar = 0.0;
        for (int f = 0; f < nfreq; ++f) jbar += wphi[f] * (double)jnu[(long)f * nvox + v];
        const double blu = g_ratio * a_ul;
        const double frad = jbar > 0.0 ? blu * jbar / (blu * jbar + c_lu[v]) : 0.0;
        const double nl = n[v], nu = n[nvox + v];
        const double S = nu / (nl * g_ratio - nu);
        for (int f = 0; f < nfreq; ++f) {
            double r = 1.0;
            if (jbar > 0.0) {
                double acc = 0.0;
                for (int fp = 0; fp < nfreq; ++fp)
                    acc += kmat[(long)fp * nfreq + f] * (double)jnu[(long)fp * nvox + v];
                r = 1.0 + gamma * frad * (acc / jbar - 1.0);
            }
            rho[(long)f * nvox + v] = (T)r;
            rhoS[(long)f * nvox + v] = (T)(r * S);
        }
    }
}

cudaError_t launch_prd_source(int prec, long nvox, int nfreq, double gamma, double g_ratio,
                              double a_ul, const double *kmat, const double *wphi,
                              const double *n, const double *c_lu, const void *jnu, void *rho,
                              void *rhoS, cudaStream_t st) {
    const int th = 256;
    if (prec == 0)
        prd_source_kernel<double><<<grid_for(nvox, th), th, 0, st>>>(
            nvox, nfreq, gamma, g_ratio, a_ul, kmat, wphi, n, c_lu, (const double *)jnu,
            (double *)rho, (double *)rhoS);
    else
        prd_source_kernel<float><<<grid_for(nvox, th), th, 0, st>>>(
            nvox, nfreq, gamma, g_ratio, a_ul, kmat, wphi, n, c_lu, (const float *)jnu,
            (float *)rho, (float *)rhoS);
    return cudaGetLastError();
}

// jnu[f][v] = sum over rays r, in order, of slots[r][f][v].
template <typename T>
__global__ void prd_collect_kernel(long len, const T *__restrict__ slots, T *__restrict__ jnu) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < len;
         i += (long)gridDim.x * blockDim.x) {
        T s = slots[i];
        for (int r = 1; r < kRays; ++r) s += slots[(long)r * len + i];
        jnu[i] = s;
    }
}

cudaError_t launch_prd_collect(int prec, long len, const void *slots, void *jnu,
                               cudaStream_t st) {
    const int th = 256;
    if (prec == 0)
        prd_collect_kernel<double><<<grid_for(len, th), th, 0, st>>>(len, (const double *)slots,
                                                                     (double *)jnu);
    else
        prd_collect_kernel<float><<<grid_for(len, th), th, 0, st>>>(len, (const float *)slots,
                                                                    (float *)jnu);
    return cudaGetLastError();
}

cudaError_t launch_planck_bottom(int prec, long nplane, double theta, const double *T,
                                 void *bbot, cudaStream_t st) {
    const int th = 256;
    if (prec == 0)
        planck_bottom_kernel<double><<<grid_for(nplane, th), th, 0, st>>>(nplane, theta, T,
                                                                          (double *)bbot);
    else
        planck_bottom_kernel<float><<<grid_for(nplane, th), th, 0, st>>>(nplane, theta, T,
                                                                         (float *)bbot);
    return cudaGetLastError();
}

}  // namespace mg3d
