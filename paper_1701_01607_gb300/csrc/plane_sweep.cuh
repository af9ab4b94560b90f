// Formal solution with shifted plane storage: the linear short-characteristics
// sweep of a static atmosphere in complete redistribution (Sec. 3), laid out
// so that every node finds its upwind corners at fixed offsets from itself.
//
// The upwind crossing of a (ray, step) lies at the same horizontal offset
// (ix0 + tx, iy0 + ty) cells from every node of the plane (periodic in x and
// y, Sec. 4.2).  So when plane k is finished, each node's values are stored
// already shifted by the offset of the step that will read them: node (x, y)
// goes to position ((x - ix0') mod nx, (y - iy0') mod ny) of the stored frame,
// where (ix0', iy0') belongs to the next step.  The next step then reads the
// four corners of node (x, y) at positions (x, y), (x + 1, y), (x, y + 1) and
// (x + 1, y + 1) of that frame: the same four offsets for every node, with no
// wrap, band or peer arithmetic on the reading side.
//
// One thread-block cluster per (ray, group of frequencies): the cluster's
// blocks split the stored frame in bands of rows.  A block owns rows
// [rank*rows, rank*rows + myrows) of the frame, plus one halo row (the first
// row of the next band, or row 0 after the last band) and one pad column
// (a copy of column 0), so all four corners of its nodes are in its own
// shared memory.  Writes carry the shift instead: a node's values go to the
// block that owns its stored row (distributed shared memory, st.shared::cluster)
// and, for the first row of a band or column 0, also to the halo row or pad
// column that duplicates it.  Two planes are kept (read k-1, write k); one
// cluster barrier per plane orders the writes of a step before the reads of
// the next and the reads of a step before the overwrite two steps later.
//
// A second completion scheme (stage 3) replaces the barrier's release fence
// with transaction-counted stores: values bound for another block go by
// st.async, which counts its bytes on an mbarrier in the receiving block, and
// each block waits on its own mbarrier for the bytes its plane receives from
// other blocks (stores within a block are ordered by __syncthreads).  The
// reads of a step must still end, cluster-wide, before the plane they came
// from is overwritten two steps later; a relaxed cluster barrier (no fence)
// arrives at the end of a step and waits just before the first store of the
// next.  Every wait on an mbarrier is bounded in time: past the bound the
// kernel records MG3D_STATUS_WAIT in the status word, stops waiting and runs
// to the end, so the host reports an error instead of a hung launch.
//
// Channels: per stored node the intensities of the group's frequencies in
// slot order, then chi0 and S of the node's plane (so the upwind chi0 and S
// are interpolated with the intensities, from the same corners), padded to
// whole 16-byte vectors; the node stride is an odd number of vectors, so the
// 16-byte loads of a warp's consecutive nodes do not conflict in banks.
//
// Slots: frequencies are taken in pairs.  For the two-level atom phi(x) =
// phi(-x), so a pair of mirror frequencies shares the optical depth of every
// short characteristic and hence the weights e^-x, w0, w_up, u (evaluated once
// per slot); a slot whose two frequencies differ in phi evaluates them twice,
// a slot of one frequency leaves its second channel unused.
//
// Per node the block accumulates, over its frequencies,
//   Jeff = sum w phi (I - w0 S)   and   U = sum w phi (1 - w0)
// (Sec. 2.1, the diagonal operator of MALI) into the partial slot of its
// (ray, group); the rate kernel adds the slots in a fixed order.
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "mg3d_internal.h"
#include "sc_step.cuh"

namespace mg3d {

namespace plane {

template <typename T>
__host__ __device__ constexpr int vec_width() { return 16 / (int)sizeof(T); }
// channels per node: 2 NP intensities, chi0, S, padded to whole vectors
template <typename T, int NP>
__host__ __device__ constexpr int channels() {
    return (2 * NP + 2 + vec_width<T>() - 1) / vec_width<T>() * vec_width<T>();
}
// node stride in elements: an odd number of 16-byte vectors
template <typename T, int NP>
__host__ __device__ constexpr int node_stride() {
    return ((channels<T, NP>() / vec_width<T>()) | 1) * vec_width<T>();
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned cluster_addr(unsigned a, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// 16-byte store of (v[0..VW-1]) at a shared::cluster address (this block's
// or another block's shared memory; a launch without clusters is a cluster of
// one block), unconditional or under a predicate.  No memory clobber: the
// stores go to the plane being written, which no thread reads before the
// barrier (whose asm carries the clobber) that ends the step.
__device__ __forceinline__ void st16(unsigned a, const float *v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]));
}
__device__ __forceinline__ void st16(unsigned a, const double *v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v[0]), "d"(v[1]));
}
__device__ __forceinline__ void st16_if(bool c, unsigned a, const float *v) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
        "@p st.shared::cluster.v4.f32 [%1], {%2, %3, %4, %5};\n\t}" ::"r"((int)c),
        "r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]));
}
__device__ __forceinline__ void st16_if(bool c, unsigned a, const double *v) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
        "@p st.shared::cluster.v2.f64 [%1], {%2, %3};\n\t}" ::"r"((int)c),
        "r"(a), "d"(v[0]), "d"(v[1]));
}
// one 16-byte vector of shared memory into registers
__device__ __forceinline__ void ld16(const float *p, float *o) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void ld16(const double *p, double *o) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    o[0] = v.x;
    o[1] = v.y;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}

// Split phases of a cluster barrier without memory ordering (the async
// scheme orders its data through mbarriers and __syncthreads)
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}
// 16-byte store into another block's shared memory that completes 16 bytes of
// the transaction count of the mbarrier at `bar` (a shared::cluster address
// in the same block), under a predicate
__device__ __forceinline__ void st16_async_if(bool c, unsigned a, const float *v, unsigned bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
        "@p st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%1], "
        "{%2, %3, %4, %5}, [%6];\n\t}" ::"r"((int)c),
        "r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void st16_async_if(bool c, unsigned a, const double *v,
                                              unsigned bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
        "@p st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%1], "
        "{%2, %3}, [%4];\n\t}" ::"r"((int)c),
        "r"(a), "d"(v[0]), "d"(v[1]), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the one arrival of a phase, with the bytes the phase is to receive
__device__ __forceinline__ void mbar_arrive_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits until the phase of parity `parity` of the mbarrier completes, at most
// kWaitLimitNs; false when the bound ran out.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
static __device__ __noinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Short-characteristics weights of optical path x (>= 0) for the linear
// step I = I_up e^-x + w_up S_up + w0 S0:  u = (1 - e^-x)/x, w0 = 1 - u,
// w_up = u - e^-x.  Below a threshold the closed form cancels, and the
// Taylor series of w0 and w_up (e^-x = 1 - w0 - w_up) replace it.
//   FP32: e^-x = 2^(-x log2 e) and 1/x by the hardware approximations (within
//   2 ulp, ample for the FP32 formal solution); series below x = 0.1.
//   FP64: Tang's table-driven e^-x (exp_neg) and 1/x from the caller
//   (1/dtau0 times 1/phi); series below x ~ 1e-3, tested on the high word of x
//   (a positive double orders like its bit pattern), which keeps the test off
//   the FP64 pipe.
struct Weights32 {
    static __device__ __forceinline__ void series(float x, float &ex, float &w0, float &wup,
                                                  float &u) {
        w0 = x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f -
                                                 x * (1.0f / 120.0f - x * (1.0f / 720.0f)))));
        wup = x * (0.5f - x * (1.0f / 3.0f - x * (1.0f / 8.0f -
                                                  x * (1.0f / 30.0f - x * (1.0f / 144.0f)))));
        u = 1.0f - w0;
        ex = u - wup;
    }
    static __device__ __forceinline__ void closed(float x, float, const ExpNegTable &, float &ex,
                                                  float &w0, float &wup, float &u) {
        ex = ex2_approx(x * -1.44269504088896341f);
        const float ix = rcp_approx(x);
        u = fmaf(-ex, ix, ix);
        w0 = 1.0f - u;
        wup = u - ex;
    }
    static __device__ __forceinline__ void eval(float x, float ix, const ExpNegTable &et,
                                                float &ex, float &w0, float &wup, float &u) {
        if (x < 0.1f) series(x, ex, w0, wup, u);
        else closed(x, ix, et, ex, w0, wup, u);
    }
};

struct Weights64 {
    static __device__ __forceinline__ void series(double x, double &ex, double &w0, double &wup,
                                                  double &u) {
        // the coefficients as products with the rounded reciprocals: a division
        // would cost an FP64 reciprocal iteration each
        w0 = x * (0.5 - x * (1.0 / 6.0 - x * (1.0 / 24.0 - x * (1.0 / 120.0 - x * (1.0 / 720.0)))));
        wup = x * (0.5 - x * (1.0 / 3.0 - x * (1.0 / 8.0 - x * (1.0 / 30.0 - x * (1.0 / 144.0)))));
        u = 1.0 - w0;
        ex = u - wup;
    }
    static __device__ __forceinline__ void closed(double x, double inv_x, const ExpNegTable &et,
                                                  double &ex, double &w0, double &wup,
                                                  double &u) {
        ex = exp_neg_hi(x, et);
        u = fma(-ex, inv_x, inv_x);
        w0 = 1.0 - u;
        wup = u - ex;
    }
    static __device__ __forceinline__ void eval(double x, double inv_x, const ExpNegTable &et,
                                                double &ex, double &w0, double &wup, double &u) {
        // 0x3F50624D is the high word of 1e-3: x below 1e-3 (up to the low word)
        if (__double2hiint(x) < 0x3F50624D) series(x, ex, w0, wup, u);
        else closed(x, inv_x, et, ex, w0, wup, u);
    }
};

template <typename T>
struct WeightsOf;
template <>
struct WeightsOf<float> {
    using W = Weights32;
};
template <>
struct WeightsOf<double> {
    using W = Weights64;
};

// 1/dtau0 for the FP64 weights (FP32 takes 1/x per slot instead): the
// hardware approximation of the reciprocal (about 23 correct bits) refined by
// two Newton-Raphson steps r <- r + r (1 - d r), each of which doubles the
// correct bits, so the result is within about an ulp (the closed-form weights
// only use it where x >= 1e-3, where dtau0 is far from 0 and from overflow).
__device__ __forceinline__ double node_rcp(double d) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ float node_rcp(float) { return 0.0f; }

}  // namespace plane

// The body of the kernel for ray blockIdx.z and frequency group blockIdx.y.
template <typename T, int NP, bool AS>
__device__ __forceinline__ void plane_sweep_body(const PlaneArgs<T> &a) {
    using namespace plane;
    constexpr int VW = vec_width<T>();
    constexpr int NCH = channels<T, NP>();
    constexpr int NV = NCH / VW;
    constexpr int CS = node_stride<T, NP>();
    constexpr int CHI = 2 * NP, SRC = 2 * NP + 1;
    using W = typename WeightsOf<T>::W;

    const int r = blockIdx.z, g = blockIdx.y;
    const int nb = a.bands;
    const bool cl = nb > 1;
    const bool as = AS && cl;               // the async completion scheme
    const int rank = (int)cluster_rank();   // 0 in a launch without clusters
    const int nx = a.nx, ny = a.ny, nz = a.nz, rows = a.rows;
    const int y0 = rank * rows;
    const int myrows = min(rows, ny - y0);
    const int lastrows = ny - (nb - 1) * rows;   // rows of the last band
    const int pitch = (nx + 1) * CS;             // one stored row, elements
    const int plane_el = (rows + 1) * pitch;     // one stored plane, elements
    const int nplane = nx * ny;                  // the host keeps nvox below 2^31
    const bool up = (a.up_mask >> r) & 1u;
    const long slot = (long)r * a.ngroups + g;
    T *__restrict__ pj = a.pj + slot * (long)nplane * nz;
    T *__restrict__ pu = a.pu + slot * (long)nplane * nz;
    const PlaneSlot<T> *__restrict__ gs = a.slots + (long)g * NP;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const unsigned buf_addr = smem_addr(buf);
    __shared__ double exp_tab[kExpTab];
    __shared__ PlaneSlot<T> stab[NP];
    // async scheme: one mbarrier per plane buffer, one phase per filling
    __shared__ __align__(8) unsigned long long full_bar[2];
    const unsigned bar_addr = smem_addr(full_bar);
    if (as && threadIdx.x == 0) {
        mbar_init(bar_addr, 1);
        mbar_init(bar_addr + 8, 1);
        mbar_init_fence();
    }
    if (sizeof(T) == 8)
        for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) exp_tab[i] = a.exp_tab[i];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) stab[i] = gs[i];
    __syncthreads();
    const ExpNegTable et{exp_tab, a.exp_l1, a.exp_l2};
    const int nslot = a.nslot_last > 0 && g == a.ngroups - 1 ? a.nslot_last : NP;

    // Block-uniform slot facts.  The fast path covers groups whose NP slots
    // are all active and mirror pairs (equal phi and w phi), except that the
    // last slot may hold one frequency (the line centre); other groups take
    // the general path with per-slot tests.
    T wsum = 0, phimin = 0, phimax = 0;
    bool fast = nslot == NP;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int fl = stab[p].flags;
        wsum += stab[p].wphi_a + stab[p].wphi_b;
        if (p < nslot) {
            const T ph = stab[p].phi_a;
            phimin = p == 0 ? ph : min(phimin, ph);
            phimax = p == 0 ? ph : max(phimax, ph);
            if (fl & kHasB) {
                phimin = min(phimin, stab[p].phi_b);
                phimax = max(phimax, stab[p].phi_b);
            }
        }
        if (p < NP - 1 && fl != (kHasB | kShared)) fast = false;
        if ((fl & kHasB) && (!(fl & kShared) || stab[p].wphi_a != stab[p].wphi_b)) fast = false;
    }
    const bool lastb = (stab[NP - 1].flags & kHasB) != 0;

    // FP32 keeps the slot tables in registers for the whole sweep; FP64 (bound
    // by its FP64 pipe, not by issue) reads them from shared memory where used
    constexpr bool kRegTabs = sizeof(T) == 4;
    T r_phi[NP], r_wa[NP], r_wu[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (kRegTabs) {
            r_phi[p] = stab[p].phi_a;
            r_wa[p] = stab[p].wphi_a;
            r_wu[p] = stab[p].wu_a;
        }
    }
    auto phi_a = [&](int p) { return kRegTabs ? r_phi[p] : stab[p].phi_a; };
    auto wphi_a = [&](int p) { return kRegTabs ? r_wa[p] : stab[p].wphi_a; };
    auto wu_a = [&](int p) { return kRegTabs ? r_wu[p] : stab[p].wu_a; };

    // The nodes of this thread, the same at every step: q = tid + i*nth for
    // i < MAXP (the host keeps the band within that many passes).
    constexpr int MAXP = plane_max_pass(NP, sizeof(T) == 8);
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

    // Stores the channels of node (x, y) into the frame of the next step,
    // shifted by (sx, sy), in buffer `par`, with its pad and halo copies
    // (predicated stores: a node of column 0 also fills the pad column, a
    // node of a band's first row also the halo row of the band before it).
    auto store_node = [&](const T *ch, int x, int y, int sx, int sy, int par) {
        int xs = x - sx;
        xs += xs < 0 ? nx : 0;
        int ys = y - sy;
        ys += ys < 0 ? ny : 0;
        const int ob = band_of(ys, a.rmagic);
        const int lr = ys - ob * rows;
        const int hb = ob == 0 ? nb - 1 : ob - 1;   // the band whose halo row is ys
        const int hr = hb == nb - 1 ? lastrows : rows;
        const unsigned col = (unsigned)((par * plane_el + xs * CS) * (int)sizeof(T));
        const unsigned base = cluster_addr(buf_addr, (unsigned)ob) +
                              col + (unsigned)(lr * pitch * (int)sizeof(T));
        const unsigned hbase = cluster_addr(buf_addr, (unsigned)hb) +
                               col + (unsigned)(hr * pitch * (int)sizeof(T));
        const unsigned padoff = (unsigned)(nx * CS * (int)sizeof(T));
        const bool pad = xs == 0, halo = lr == 0;
        if constexpr (AS) {
            if (as) {
                // to another block: st.async counted on that block's mbarrier
                // of buffer `par`; within the block: plain stores
                const unsigned bar = cluster_addr(bar_addr + 8u * par, (unsigned)ob);
                const unsigned hbar = cluster_addr(bar_addr + 8u * par, (unsigned)hb);
                const bool rem = ob != rank, hrem = hb != rank;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const T *cv = ch + v * VW;
                    if (rem) {
                        st16_async_if(true, base + v * 16, cv, bar);
                        st16_async_if(pad, base + padoff + v * 16, cv, bar);
                    } else {
                        st16(base + v * 16, cv);
                        st16_if(pad, base + padoff + v * 16, cv);
                    }
                    if (hrem) {
                        st16_async_if(halo, hbase + v * 16, cv, hbar);
                        st16_async_if(halo && pad, hbase + padoff + v * 16, cv, hbar);
                    } else {
                        st16_if(halo, hbase + v * 16, cv);
                        st16_if(halo && pad, hbase + padoff + v * 16, cv);
                    }
                }
                return;
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            st16(base + v * 16, ch + v * VW);
            st16_if(pad, base + padoff + v * 16, ch + v * VW);
            st16_if(halo, hbase + v * 16, ch + v * VW);
            st16_if(halo && pad, hbase + padoff + v * 16, ch + v * VW);
        }
    };

    // chi0 and S of the thread's nodes on the next plane are loaded one step
    // ahead into registers, so that the global-memory latency overlaps the
    // current step and the barrier instead of opening each step.
    T nchi[MAXP], nS[MAXP];
    auto prefetch = [&](int t) {
        const int kp = (up ? t : nz - 1 - t) * nplane;
#pragma unroll
        for (int i = 0; i < MAXP; ++i)
            if (valid[i]) {
                nchi[i] = a.chi0[kp + nodeq[i]];
                nS[i] = a.S[kp + nodeq[i]];
            }
    };

    // Async scheme: the bytes buffer `par` of this block receives from other
    // blocks when the plane is stored with row shift sy.  Stored row ys (a
    // row of the band, or the halo row: the next band's first row, row 0
    // after the last band) holds source row (ys + sy) mod ny, all of its nx
    // nodes and the pad copy, written by the block that owns that row.  Warp
    // 0 counts the rows with another owner; its lane 0 posts the phase's one
    // arrival with the byte count.
    auto expect_fill = [&](int sy, int par) {
        if (threadIdx.x >= 32) return;
        int cnt = 0;
        for (int j = threadIdx.x; j <= myrows; j += 32) {
            const int ys = j < myrows ? y0 + j : (rank == nb - 1 ? 0 : y0 + rows);
            int ysrc = ys + sy;
            ysrc -= ysrc >= ny ? ny : 0;
            cnt += band_of(ysrc, a.rmagic) != rank ? 1 : 0;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (threadIdx.x == 0)
            mbar_arrive_expect(bar_addr + 8u * par, (unsigned)(cnt * (nx + 1) * NV * 16));
    };
    bool waits_ok = true;   // false once a bounded wait ran out
    auto wait_fill = [&](int s) {   // buffer s & 1 holds the plane stored at step s
        if (waits_ok && !mbar_wait_bounded(bar_addr + 8u * (s & 1), (unsigned)((s >> 1) & 1))) {
            waits_ok = false;
            if (a.status) atomicOr(a.status, kPlaneStatusWait);
        }
    };
    if (as && nz > 1) {
        // every block's mbarriers are initialised before any store reaches them
        cluster_barrier();
        expect_fill(a.steps[(long)r * nz].sy, 0);
    }

    // ---- entering boundary plane: I prescribed (bottom: Planck at the local
    // temperature, top: zero), so w0 = 0 and 1 - w0 = 1
    prefetch(0);
    {
        const int k0 = (up ? 0 : nz - 1) * nplane;
        const PlaneStep<T> sp = a.steps[(long)r * nz];
#pragma unroll
        for (int i = 0; i < MAXP; ++i) {
            if (!valid[i]) continue;
            const T Ib = up ? a.bbot[nodeq[i]] : T(0);
            T ch[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) ch[c] = c < 2 * NP ? Ib : T(0);
            ch[CHI] = nchi[i];
            ch[SRC] = nS[i];
            pj[k0 + nodeq[i]] = Ib * wsum;
            pu[k0 + nodeq[i]] = wsum;
            if (nz > 1) store_node(ch, xq[i], yq[i], sp.sx, sp.sy, 0);
        }
    }
    if (nz > 1) prefetch(1);
    if (cl && !as) cluster_barrier();
    else __syncthreads();

    // Regime of a node's weights: every slot in closed form, every slot by
    // series, or a per-slot choice.  FP32 compares dtau0 with the thresholds
    // 0.1/phi_min and 0.1/phi_max; FP64 compares the high words of dtau0 and
    // of 1e-3/phi (integer compares, off the FP64 pipe), a conservative test
    // whose border cases take the per-slot choice.
    const T thr = sizeof(T) == 8 ? T(1e-3) : T(0.1);
    const T d_all_closed = thr / phimin, d_all_series = thr / phimax;
    const int hi_closed = sizeof(T) == 8 ? __double2hiint((double)d_all_closed) : 0;
    const int hi_series = sizeof(T) == 8 ? __double2hiint((double)d_all_series) : 0;
    auto regime = [&](T dtau0) {   // 0 closed, 1 series, 2 mixed
        if constexpr (sizeof(T) == 8) {
            const int hd = __double2hiint((double)dtau0);
            return hd > hi_closed ? 0 : (hd < hi_series ? 1 : 2);
        } else {
            return dtau0 >= d_all_closed ? 0 : (dtau0 < d_all_series ? 1 : 2);
        }
    };

    auto run = [&](auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
        // channel c is interpolated when it carries a frequency of an active
        // slot, or chi0 or S; the others (the second channel of a
        // one-frequency slot, slots past the last group's end, padding) hold 0
        auto live = [&](int c) {
            if (c == CHI || c == SRC) return true;
            if (c >= 2 * NP) return false;
            if (FAST) return c != 2 * NP - 1 || lastb;
            const int p = c >> 1;
            return p < nslot && ((c & 1) == 0 || (stab[p].flags & kHasB));
        };
        // the step constants are loaded one step ahead as well
        PlaneStep<T> sp_next = a.steps[(long)r * nz + (nz > 1 ? 1 : 0)];
        for (int t = 1; t < nz; ++t) {
            const int kp = (up ? t : nz - 1 - t) * nplane;
            const T *prev = buf + ((t - 1) & 1) * plane_el;
            const PlaneStep<T> sp = sp_next;
            const bool write = t + 1 < nz;
            if (write) sp_next = a.steps[(long)r * nz + t + 1];
            T cchi[MAXP], cS[MAXP];
#pragma unroll
            for (int i = 0; i < MAXP; ++i) {
                cchi[i] = nchi[i];
                cS[i] = nS[i];
            }
            if (write) prefetch(t + 1);
            if (as) {
                // the other blocks' part of the plane stored at step t - 1
                wait_fill(t - 1);
                if (write) {
                    expect_fill(sp.sy, t & 1);
                    // every block's reads of this buffer (step t - 1) are over
                    if (t >= 2) cluster_wait();
                }
            }
#pragma unroll
            for (int i = 0; i < MAXP; ++i) {
                // FP64 takes its nodes one after the other (its pipe, not
                // latency, bounds it, and overlapping two nodes would spill)
                if (sizeof(T) == 8 && i > 0) asm volatile("" ::: "memory");
                if (!valid[i]) continue;
                const int v = kp + nodeq[i];
                const T chi_loc = cchi[i];
                const T S_loc = cS[i];
                // the four upwind corners, interpolated channel by channel
                const T *c00 = prev + corq[i];
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
                        ch[vv * VW + e] = live(vv * VW + e) ? sp.w00 * A[e] + sp.w10 * B[e] +
                                                                  sp.w01 * C[e] + sp.w11 * D[e]
                                                            : T(0);
                }
                const T chi_up = ch[CHI], S_up = ch[SRC];
                const T dtau0 = (chi_up + chi_loc) * sp.half_s;
                const T inv_dtau0 = node_rcp(dtau0);
                T cj = 0, cu = 0;
                // new intensities of slot p's frequencies from its weights
                auto apply = [&](int p, bool two, T ex, T w0, T wup, T u) {
                    cu = fma(wu_a(p), u, cu);
                    const T wupS = wup * S_up;
                    const T pa = fma(ch[2 * p], ex, wupS);
                    if (two) {
                        const T pb = fma(ch[2 * p + 1], ex, wupS);
                        cj = fma(wphi_a(p), pa + pb, cj);
                        ch[2 * p + 1] = fma(w0, S_loc, pb);
                    } else {
                        cj = fma(wphi_a(p), pa, cj);
                    }
                    ch[2 * p] = fma(w0, S_loc, pa);
                };
                if constexpr (FAST) {
                    // every slot a mirror pair except possibly the last
                    auto slots = [&](auto mode_tag) {
                        constexpr int MODE = decltype(mode_tag)::value;
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const T x = dtau0 * phi_a(p);
                            const T ix = sizeof(T) == 8 ? inv_dtau0 * stab[p].iphi_a : T(0);
                            T ex, w0, wup, u;
                            if (MODE == 0) W::closed(x, ix, et, ex, w0, wup, u);
                            else if (MODE == 1) W::series(x, ex, w0, wup, u);
                            else W::eval(x, ix, et, ex, w0, wup, u);
                            apply(p, p < NP - 1 || lastb, ex, w0, wup, u);
                        }
                    };
                    const int rg = regime(dtau0);
                    if (rg == 0) slots(std::integral_constant<int, 0>{});
                    else if (rg == 1) slots(std::integral_constant<int, 1>{});
                    else slots(std::integral_constant<int, 2>{});
                } else {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (p >= nslot) continue;
                        const int fl = stab[p].flags;
                        T ex, w0, wup, u;
                        W::eval(dtau0 * phi_a(p), sizeof(T) == 8 ? inv_dtau0 * stab[p].iphi_a : T(0),
                                et, ex, w0, wup, u);
                        cu = fma(wu_a(p), u, cu);
                        T wupS = wup * S_up;
                        T part = fma(ch[2 * p], ex, wupS);
                        cj = fma(wphi_a(p), part, cj);
                        ch[2 * p] = fma(w0, S_loc, part);
                        if (fl & kHasB) {
                            if (!(fl & kShared)) {
                                W::eval(dtau0 * stab[p].phi_b,
                                        sizeof(T) == 8 ? inv_dtau0 * stab[p].iphi_b : T(0), et,
                                        ex, w0, wup, u);
                                cu = fma(stab[p].wu_b, u, cu);
                                wupS = wup * S_up;
                            }
                            part = fma(ch[2 * p + 1], ex, wupS);
                            cj = fma(stab[p].wphi_b, part, cj);
                            ch[2 * p + 1] = fma(w0, S_loc, part);
                        }
                    }
                }
                pj[v] = cj;
                pu[v] = cu;
                if (write) {
                    ch[CHI] = chi_loc;
                    ch[SRC] = S_loc;
                    store_node(ch, xq[i], yq[i], sp.sx, sp.sy, t & 1);
                }
            }
            if (write) {
                if (as) {
                    __syncthreads();
                    if (t + 2 < nz) cluster_arrive_relaxed();
                } else if (cl) {
                    cluster_barrier();
                } else {
                    __syncthreads();
                }
            }
        }
    };
    if (fast) run(std::true_type{});
    else run(std::false_type{});
    // no block leaves while another may still address its shared memory
    if (as && nz > 1) cluster_barrier();
}

// MAXT: block-size bound the kernel is compiled for; MINB: resident blocks
// per SM it must fit (the register budget).
template <typename T, int NP, int MAXT, int MINB, bool AS>
__global__ void __launch_bounds__(MAXT, MINB) plane_sweep_kernel(const PlaneArgs<T> a) {
    plane_sweep_body<T, NP, AS>(a);
}

// ------------------------------------------------------------- launching

template <typename T, int NP>
inline size_t plane_smem_t(int rows, int nx) {
    return 2ull * (rows + 1) * (nx + 1) * plane::node_stride<T, NP>() * sizeof(T);
}

// Kernel attributes and the launch configuration of shape s (dynamic shared
// memory, clusters of `bands` blocks); a is used by the launch only.
template <typename T, int NP, int MAXT, int MINB, bool AS>
static cudaError_t plane_config(const SweepShape &s, int nx, cudaStream_t st,
                                cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr) {
    // the limit is the same for every launch, so a CUDA graph that captured a
    // launch needing more shared memory than a later one still replays
    cudaError_t e = cudaFuncSetAttribute(plane_sweep_kernel<T, NP, MAXT, MINB, AS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxPlaneSmem);
    if (e == cudaSuccess && s.bands > kPortableBands)
        e = cudaFuncSetAttribute(plane_sweep_kernel<T, NP, MAXT, MINB, AS>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(s.bands, s.ngroups, kRays);
    cfg->blockDim = dim3(s.threads, 1, 1);
    cfg->dynamicSmemBytes = plane_smem_t<T, NP>(s.rows, nx);
    cfg->stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s.bands;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = s.bands > 1 ? 1 : 0;   // one band: a plain launch
    return cudaSuccess;
}

// launch (a non-null) or occupancy query (a null: *n = clusters, or blocks
// per SM for one band, the GPU holds at once)
template <typename T, int NP, int MAXT, int MINB, bool AS>
static cudaError_t plane_go(const PlaneArgs<T> *a, const SweepShape &s, int nx, cudaStream_t st,
                            int *n) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = plane_config<T, NP, MAXT, MINB, AS>(s, nx, st, &cfg, attr);
    if (e != cudaSuccess) return e;
    if (a) return cudaLaunchKernelEx(&cfg, plane_sweep_kernel<T, NP, MAXT, MINB, AS>, *a);
    if (s.bands == 1)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            n, plane_sweep_kernel<T, NP, MAXT, MINB, AS>, s.threads, cfg.dynamicSmemBytes);
    return cudaOccupancyMaxActiveClusters(n, plane_sweep_kernel<T, NP, MAXT, MINB, AS>, &cfg);
}

// register budget: lean 0 the full budget of MAXT threads (one block per SM),
// lean 1 (FP32 only) two blocks of 512 or four of 256 per SM (64 registers);
// FP32 blocks of up to 1024 threads for one or two slots
template <typename T, int NP, bool AS>
static cudaError_t plane_go_np(const PlaneArgs<T> *a, const SweepShape &s, int nx,
                               cudaStream_t st, int *n) {
    if constexpr (sizeof(T) == 4) {
        if (s.threads > 512) {
            // 1024 threads (64 registers): small slot counts only
            if constexpr (NP <= 2) {
                if (s.lean == 0) return plane_go<T, NP, 1024, 1, AS>(a, s, nx, st, n);
            }
            return cudaErrorInvalidValue;
        }
        if (s.lean == 1)
            return s.threads <= 256 ? plane_go<T, NP, 256, 4, AS>(a, s, nx, st, n)
                                    : plane_go<T, NP, 512, 2, AS>(a, s, nx, st, n);
        return s.threads <= 256 ? plane_go<T, NP, 256, 1, AS>(a, s, nx, st, n)
                                : plane_go<T, NP, 512, 1, AS>(a, s, nx, st, n);
    } else {
        // the FP64 body does not fit 64 registers without spilling: no lean
        // variant; 448 threads leave it up to 146 registers
        if (s.lean != 0 || s.threads > 512) return cudaErrorInvalidValue;
        if (s.threads <= 256) return plane_go<T, NP, 256, 1, AS>(a, s, nx, st, n);
        if (s.threads <= 448) return plane_go<T, NP, 448, 1, AS>(a, s, nx, st, n);
        return plane_go<T, NP, 512, 1, AS>(a, s, nx, st, n);
    }
}

template <typename T, bool AS>
static cudaError_t plane_dispatch(const PlaneArgs<T> *a, const SweepShape &s, int nx,
                                  cudaStream_t st, int *n) {
    if (s.threads < 32 || s.threads > kPlaneMaxThreads || s.threads % 32 || s.lean < 0 ||
        s.lean > 1)
        return cudaErrorInvalidValue;
    switch (s.np) {
        case 1: return plane_go_np<T, 1, AS>(a, s, nx, st, n);
        case 2: return plane_go_np<T, 2, AS>(a, s, nx, st, n);
        case 3: return plane_go_np<T, 3, AS>(a, s, nx, st, n);
        case 5: return plane_go_np<T, 5, AS>(a, s, nx, st, n);
        case 8: return plane_go_np<T, 8, AS>(a, s, nx, st, n);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mg3d
