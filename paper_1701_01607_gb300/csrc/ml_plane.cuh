// Multi-level formal solution with shifted plane storage: the linear
// short-characteristics sweep (Sec. 3) of a static atmosphere, laid out as
// the two-level shifted-plane sweep (plane_sweep.cuh) is.
//
// The upwind crossing of a (ray, step) lies at the same horizontal offset from
// every node of the plane (periodic boundaries, Sec. 4.2), so each ray's
// finished plane is stored shifted by the offset of the step that reads it and
// a node finds its four upwind corners at fixed offsets (x, y), (x+1, y),
// (x, y+1), (x+1, y+1) of its ray's stored frame.  In the multi-level atom the
// opacity and source function differ from frequency to frequency, so they ride
// along as channels beside the intensity: per node, ray and frequency (I, chi,
// S), NF frequencies per block, padded to whole 16-byte vectors with an odd
// node stride (conflict-free 16-byte loads).
//
// One thread-block cluster per (group of NF frequencies of the chunk, group of
// rays of one hemisphere); its blocks split the stored frames in bands of
// rows, each with a halo row and a pad column, and a block holds one frame per
// ray of its group (double buffered).  A thread owns its nodes for the whole
// sweep and walks the group's rays at each of them, so the angle sums over the
// group are complete in registers and written once per (slot, frequency,
// node), the slot layout of the other multi-level sweep:
//   Jx = sum (I - w0 S) + sc sum w0,   Ux = sum u + oc sum w0,   Jm = sum I
// (times the ray weight; sc, oc: the parts of S and the opacity share the
// transition does not set), all sums of non-negative terms.  Writes go to the
// block owning the shifted row (distributed shared memory) with copies into
// the pad column and the halo row; one cluster barrier per plane orders them.
#pragma once

#include "plane_sweep.cuh"

namespace mg3d {

namespace mlplane {

template <typename T>
__host__ __device__ constexpr int channels(int nf) {
    return (3 * nf + plane::vec_width<T>() - 1) / plane::vec_width<T>() * plane::vec_width<T>();
}
template <typename T>
__host__ __device__ constexpr int node_stride(int nf) {
    return ((channels<T>(nf) / plane::vec_width<T>()) | 1) * plane::vec_width<T>();
}

}  // namespace mlplane

template <typename T, int NF>
__device__ __forceinline__ void ml_plane_body(const MlPlaneArgs<T> &a) {
    using namespace plane;
    constexpr int VW = vec_width<T>();
    constexpr int NCH = mlplane::channels<T>(NF);
    constexpr int NV = NCH / VW;
    constexpr int CS = mlplane::node_stride<T>(NF);
    constexpr int MAXP = ml_plane_max_pass(NF);

    const int g = blockIdx.y, slot = blockIdx.z;
    const int rpb = a.rpb, groups = 12 / rpb;
    const int hemi = slot / groups;
    const int r0 = hemi * 12 + (slot - hemi * groups) * rpb;   // rays 0-11 point up
    const bool up = hemi == 0;
    const int f0 = g * NF;
    const int nfl = min(NF, a.nfreq - f0);   // active frequencies of the group
    const int nb = a.bands;
    const bool cl = nb > 1;
    const int rank = (int)cluster_rank();
    const int nx = a.nx, ny = a.ny, nz = a.nz, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = min(rows, ny - y0);
    const int lastrows = ny - (nb - 1) * rows;
    const int pitch = (nx + 1) * CS;          // one stored row, elements
    const int ray_el = (rows + 1) * pitch;    // one ray's stored frame
    const int plane_el = rpb * ray_el;        // all rays of one buffer
    const int nplane = nx * ny;
    const long nvox = (long)nplane * nz;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const unsigned buf_addr = smem_addr(buf);
    __shared__ double exp_tab[kExpTab];
    __shared__ PlaneStep<T> sstep[2][12];   // the rays' constants of step t in [t & 1]
    if (sizeof(T) == 8)
        for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) exp_tab[i] = a.exp_tab[i];
    if (threadIdx.x < rpb) {
        sstep[0][threadIdx.x] = a.steps[(long)(r0 + threadIdx.x) * nz];
        if (nz > 1) sstep[1][threadIdx.x] = a.steps[(long)(r0 + threadIdx.x) * nz + 1];
    }
    __syncthreads();
    const ExpNegTable et{exp_tab, a.exp_l1, a.exp_l2};
    const T wray = T(1.0 / kRays);

    // the thread's nodes, the same at every step
    const int band = myrows * nx;
    const int nth = blockDim.x;
    bool valid[MAXP];
    int xq[MAXP], yq[MAXP], nodeq[MAXP], corq[MAXP];
#pragma unroll
    for (int i = 0; i < MAXP; ++i) {
        const int q = threadIdx.x + i * nth;
        valid[i] = q < band;
        const int yl = band_of(valid[i] ? q : 0, a.xmagic);
        xq[i] = (valid[i] ? q : 0) - yl * nx;
        yq[i] = y0 + yl;
        nodeq[i] = yq[i] * nx + xq[i];
        corq[i] = yl * pitch + xq[i] * CS;
    }

    // channels of node (x, y) for ray j into buffer `par`, shifted by (sx, sy),
    // with the pad and halo copies
    auto store_node = [&](const T *ch, int x, int y, int sx, int sy, int par, int j) {
        int xs = x - sx;
        xs += xs < 0 ? nx : 0;
        int ys = y - sy;
        ys += ys < 0 ? ny : 0;
        const int ob = band_of(ys, a.rmagic);
        const int lr = ys - ob * rows;
        const int hb = ob == 0 ? nb - 1 : ob - 1;
        const int hr = hb == nb - 1 ? lastrows : rows;
        const unsigned col = (unsigned)((par * plane_el + j * ray_el + xs * CS) * (int)sizeof(T));
        const unsigned base = cluster_addr(buf_addr, (unsigned)ob) + col +
                              (unsigned)(lr * pitch * (int)sizeof(T));
        const unsigned hbase = cluster_addr(buf_addr, (unsigned)hb) + col +
                               (unsigned)(hr * pitch * (int)sizeof(T));
        const unsigned padoff = (unsigned)(nx * CS * (int)sizeof(T));
        const bool pad = xs == 0, halo = lr == 0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            st16(base + v * 16, ch + v * VW);
            st16_if(pad, base + padoff + v * 16, ch + v * VW);
            st16_if(halo, hbase + v * 16, ch + v * VW);
            st16_if(halo && pad, hbase + padoff + v * 16, ch + v * VW);
        }
    };

    // chi and S of the thread's nodes on the next plane, one step ahead
    T nchi[MAXP][NF], nS[MAXP][NF];
    auto prefetch = [&](int t) {
        const long kp = (long)(up ? t : nz - 1 - t) * nplane;
#pragma unroll
        for (int i = 0; i < MAXP; ++i)
#pragma unroll
            for (int k = 0; k < NF; ++k)
                if (valid[i] && k < nfl) {
                    const long o = (long)(f0 + k) * nvox + kp + nodeq[i];
                    nchi[i][k] = a.chi[o];
                    nS[i][k] = a.S[o];
                } else {
                    nchi[i][k] = T(0);
                    nS[i][k] = T(0);
                }
    };

    // ---- entering boundary plane: I prescribed (bottom: Planck at the local
    // temperature, top: zero), w0 = 0
    prefetch(0);
    {
        const long k0 = (long)(up ? 0 : nz - 1) * nplane;
#pragma unroll
        for (int i = 0; i < MAXP; ++i) {
            if (!valid[i]) continue;
            T ch[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) ch[c] = T(0);
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                if (k >= nfl) continue;
                const T Ib = up ? a.ib[(long)(f0 + k) * nplane + nodeq[i]] : T(0);
                ch[3 * k] = Ib;
                ch[3 * k + 1] = nchi[i][k];
                ch[3 * k + 2] = nS[i][k];
                const long o = ((long)slot * a.nfreq + f0 + k) * nvox + k0 + nodeq[i];
                a.jx[o] = T(rpb) * wray * Ib;
                a.ux[o] = T(rpb) * wray;
                if (a.jm) a.jm[o] = T(rpb) * wray * Ib;
            }
            if (nz > 1)
                for (int j = 0; j < rpb; ++j)
                    store_node(ch, xq[i], yq[i], sstep[0][j].sx, sstep[0][j].sy, 0, j);
        }
    }
    if (nz > 1) prefetch(1);
    if (cl) cluster_barrier();
    else __syncthreads();

    for (int t = 1; t < nz; ++t) {
        const long kp = (long)(up ? t : nz - 1 - t) * nplane;
        const T *prev = buf + ((t - 1) & 1) * plane_el;
        const bool write = t + 1 < nz;
        // the next step's constants go to the other half of sstep, which the
        // previous step read; the barrier at the end of this step orders them
        if (write && threadIdx.x < rpb)
            sstep[(t + 1) & 1][threadIdx.x] = a.steps[(long)(r0 + threadIdx.x) * nz + t + 1];
        T cchi[MAXP][NF], cS[MAXP][NF];
#pragma unroll
        for (int i = 0; i < MAXP; ++i)
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                cchi[i][k] = nchi[i][k];
                cS[i][k] = nS[i][k];
            }
        if (write) prefetch(t + 1);
#pragma unroll
        for (int i = 0; i < MAXP; ++i) {
            if (!valid[i]) continue;
            T sp[NF], su[NF], sw[NF], si[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) sp[k] = su[k] = sw[k] = si[k] = T(0);
            for (int j = 0; j < rpb; ++j) {
                const PlaneStep<T> st = sstep[t & 1][j];
                const T *c00 = prev + j * ray_el + corq[i];
                const T *c10 = c00 + CS, *c01 = c00 + pitch, *c11 = c01 + CS;
                T ch[NCH];
#pragma unroll
                for (int vv = 0; vv < NV; ++vv) {
                    T A[VW], B[VW], C[VW], D[VW];
                    ld16(c00 + vv * VW, A);
                    ld16(c10 + vv * VW, B);
                    ld16(c01 + vv * VW, C);
                    ld16(c11 + vv * VW, D);
#pragma unroll
                    for (int e = 0; e < VW; ++e)
                        ch[vv * VW + e] = vv * VW + e < 3 * NF
                                              ? st.w00 * A[e] + st.w10 * B[e] + st.w01 * C[e] +
                                                    st.w11 * D[e]
                                              : T(0);
                }
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    if (k >= nfl) continue;
                    const T I_up = ch[3 * k], chi_up = ch[3 * k + 1], S_up = ch[3 * k + 2];
                    const T x = (chi_up + cchi[i][k]) * st.half_s;
                    T ex, w0, wup, u;
                    ScWeights<T>::eval(x, sc_rcp(x), et, ex, w0, wup, u);
                    const T part = I_up * ex + wup * S_up;   // I - w0 S
                    const T I = part + w0 * cS[i][k];
                    sp[k] += part;
                    su[k] += u;
                    sw[k] += w0;
                    si[k] += I;
                    ch[3 * k] = I;
                    ch[3 * k + 1] = cchi[i][k];
                    ch[3 * k + 2] = cS[i][k];
                }
                if (write) store_node(ch, xq[i], yq[i], st.sx, st.sy, t & 1, j);
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                if (k >= nfl) continue;
                const long v = (long)(f0 + k) * nvox + kp + nodeq[i];
                const long o = (long)slot * a.nfreq * nvox + v;
                a.jx[o] = wray * (sp[k] + a.sc[v] * sw[k]);
                a.ux[o] = wray * (su[k] + a.oc[v] * sw[k]);
                if (a.jm) a.jm[o] = wray * si[k];
            }
        }
        if (write) {
            if (cl) cluster_barrier();
            else __syncthreads();
        }
    }
}

// MAXT threads at most, 128 registers (65536 / (MAXT x MINB)): two blocks of
// 256 or four of 128 can share an SM where shared memory allows
template <typename T, int NF, int MAXT>
__global__ void __launch_bounds__(MAXT, 512 / MAXT) ml_plane_kernel(const MlPlaneArgs<T> a) {
    ml_plane_body<T, NF>(a);
}

template <typename T, int NF>
inline size_t ml_plane_smem_t(int rows, int nx, int rpb) {
    return 2ull * rpb * (rows + 1) * (nx + 1) * mlplane::node_stride<T>(NF) * sizeof(T);
}

// launch (a non-null) or occupancy query (a null: *n = clusters, or blocks
// per SM for one band, the GPU holds at once)
template <typename T, int NF, int MAXT>
static cudaError_t ml_plane_go(const MlPlaneArgs<T> *a, int bands, int rows, int nx, int rpb,
                               int nfreq, int threads, cudaStream_t st, int *n) {
    cudaError_t e = cudaFuncSetAttribute(ml_plane_kernel<T, NF, MAXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMlPlaneMaxSmem);
    if (e == cudaSuccess && bands > kPortableBands)
        e = cudaFuncSetAttribute(ml_plane_kernel<T, NF, MAXT>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(bands, (nfreq + NF - 1) / NF, 2 * (12 / rpb));
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = ml_plane_smem_t<T, NF>(rows, nx, rpb);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = bands;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = bands > 1 ? 1 : 0;
    if (a) return cudaLaunchKernelEx(&cfg, ml_plane_kernel<T, NF, MAXT>, *a);
    if (bands == 1)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            n, ml_plane_kernel<T, NF, MAXT>, threads, cfg.dynamicSmemBytes);
    return cudaOccupancyMaxActiveClusters(n, ml_plane_kernel<T, NF, MAXT>, &cfg);
}

template <typename T>
static cudaError_t ml_plane_dispatch(const MlPlaneArgs<T> *a, int nf_block, int bands, int rows,
                                     int nx, int rpb, int nfreq, int threads, cudaStream_t st,
                                     int *n) {
    if (threads < 32 || threads > 512 || threads % 32 || rpb < 1 || 12 % rpb)
        return cudaErrorInvalidValue;
    auto go = [&](auto nf_tag) -> cudaError_t {
        constexpr int NF = decltype(nf_tag)::value;
        if constexpr (sizeof(T) == 8 && NF > 1) {
            // FP64 with more than one frequency per block spills at 128 registers
            return cudaErrorInvalidValue;
        } else {
            if (threads <= 128)
                return ml_plane_go<T, NF, 128>(a, bands, rows, nx, rpb, nfreq, threads, st, n);
            if (threads <= 256)
                return ml_plane_go<T, NF, 256>(a, bands, rows, nx, rpb, nfreq, threads, st, n);
            return ml_plane_go<T, NF, 512>(a, bands, rows, nx, rpb, nfreq, threads, st, n);
        }
    };
    switch (nf_block) {
        case 1: return go(std::integral_constant<int, 1>{});
        case 2: return go(std::integral_constant<int, 2>{});
        case 4: return go(std::integral_constant<int, 4>{});
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mg3d
