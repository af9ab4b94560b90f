// Allocation-free formal solution.
//
// Some callers cannot allocate device memory at the time they need a formal
// solution: code running inside another framework's memory pool that forbids
// foreign cudaMalloc calls, allocation-free sections of a real-time or
// embedded pipeline, or a process that has already handed all device memory
// to a caching allocator.  mg3d_formal_solve_noalloc serves them: the caller
// passes device inputs and outputs, and the scratch the sweep needs (partial
// sums per ray, the per-plane upwind geometry and the frequency tables) lives
// in one fixed-size array in the library's device image, which every GPU that
// loads the library holds until the process exits.
//
// The array's name is only a host-side stand-in in host code; its device
// address is obtained once per device with cudaGetSymbolAddress (on the first
// call made while that device is current) and passed to the kernels.  With
// lazy module loading (the CUDA default) that first lookup is also when the
// device reserves the array, so it can fail for lack of memory (MG3D_E_OOM)
// if the caller's allocator already holds the device's memory; the same
// one-time set-up fills the exponential table from the host.  All calls share
// the array, so calls whose work overlaps on the GPU race; each call rewrites
// every other scratch entry it reads, so nothing carries over from one call to
// the next.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "mg3d.h"
#include "mg3d_internal.h"

namespace mg3d {

void record_error(const std::string &msg);

namespace {

constexpr long kMaxNodes = MG3D_NOALLOC_MAX_NODES;
constexpr int kMaxNz = MG3D_NOALLOC_MAX_NZ;
constexpr int kMaxFreq = MG3D_NOALLOC_MAX_FREQ;

// Layout of the scratch array, in doubles.
constexpr long kOffPj = 0;
constexpr long kOffPu = kOffPj + (long)kRays * kMaxNodes;
constexpr long kOffGeom = kOffPu + (long)kRays * kMaxNodes;
constexpr long kGeomDoubles = (long)kRays * kMaxNz * (sizeof(StepGeom) / sizeof(double));
constexpr long kOffPhi = kOffGeom + kGeomDoubles;
constexpr long kOffInvPhi = kOffPhi + kMaxFreq;
constexpr long kOffWphi = kOffInvPhi + kMaxFreq;
constexpr long kOffExpTab = kOffWphi + kMaxFreq;
constexpr long kScratchDoubles = kOffExpTab + kExpTab;
static_assert(sizeof(StepGeom) % sizeof(double) == 0, "geometry entries pack into doubles");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        record_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return MG3D_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        record_error("device index beyond the allocation-free path's table");
        return MG3D_E_ARG;
    }
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess) {
            // the table of 2^(j/256) the sweep's FP64 exp uses, correctly
            // rounded on the host: written once, read by every call
            double tab[kExpTab], l1 = 0.0, l2 = 0.0;
            exp_neg_constants(tab, &l1, &l2);
            e = cudaMemcpyToSymbol(g_noalloc_scratch, tab, sizeof(tab),
                                   kOffExpTab * sizeof(double), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            const bool oom = e == cudaErrorMemoryAllocation;
            cudaGetLastError();
            record_error(std::string(oom ? "allocation-free scratch could not be reserved on "
                                           "this device (first call, device memory full): "
                                         : "allocation-free scratch set-up: ") +
                         cudaGetErrorString(e));
            return oom ? MG3D_E_OOM : MG3D_E_CUDA;
        }
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return MG3D_OK;
}

// A4 directions (per octant the permutations of (a, a, b)), upwind geometry
// of every (ray, step) and the frequency tables, written into the scratch.
__global__ void noalloc_tables_kernel(int nx, int ny, int nz, double dx, double dy,
                                      const double *__restrict__ z, double a, int nfreq,
                                      double x_max, double *scratch) {
    if (!(a > 0.0)) a = sqrt((4.0 - sqrt(6.4)) / 12.0);
    const double b = sqrt(1.0 - 2.0 * a * a);
    StepGeom *geom = reinterpret_cast<StepGeom *>(scratch + kOffGeom);
    const int total = kRays * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int r = i / nz, t = i - r * nz;
        const int oct = r / 3, p = r % 3;
        const double ax = p == 0 ? b : a, ay = p == 1 ? b : a, az = p == 2 ? b : a;
        const double mx = (oct & 1) ? -ax : ax;
        const double my = (oct & 2) ? -ay : ay;
        const double mz = (oct & 4) ? -az : az;
        StepGeom g{0, 0, 0.0, 0.0, 0.0};
        if (t > 0) {
            const bool up = mz > 0;
            const int k = up ? t : nz - 1 - t;
            const int kp = up ? k - 1 : k + 1;
            const double s = fabs(z[k] - z[kp]) / fabs(mz);
            const double sx = -s * mx / dx, sy = -s * my / dy;
            const double fx = floor(sx), fy = floor(sy);
            long ix = (long)fx % nx, iy = (long)fy % ny;
            if (ix < 0) ix += nx;
            if (iy < 0) iy += ny;
            g.ix0 = (int)ix;
            g.iy0 = (int)iy;
            g.tx = sx - fx;
            g.ty = sy - fy;
            g.s = s;
        }
        geom[i] = g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double *phi = scratch + kOffPhi, *inv_phi = scratch + kOffInvPhi;
        double *wphi = scratch + kOffWphi;
        double sum = 0.0;
        for (int f = 0; f < nfreq; ++f) {
            const double x = nfreq == 1 ? 0.0 : x_max * (2 * f - (nfreq - 1)) / (nfreq - 1);
            double w = nfreq == 1 ? 1.0 : 2.0 * x_max / (nfreq - 1);
            if (nfreq > 1 && (f == 0 || f == nfreq - 1)) w *= 0.5;
            phi[f] = exp(-x * x) / sqrt(M_PI);
            inv_phi[f] = 1.0 / phi[f];
            wphi[f] = w * phi[f];
            sum += wphi[f];
        }
        for (int f = 0; f < nfreq; ++f) wphi[f] /= sum * kRays;
    }
}

// Jeff and U: the 24 ray partials of every node added in ray order.
__global__ void noalloc_reduce_kernel(long nvox, const double *__restrict__ pj,
                                      const double *__restrict__ pu, double *__restrict__ jeff,
                                      double *__restrict__ u) {
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox;
         v += (long)gridDim.x * blockDim.x) {
        double J = 0.0, U = 0.0;
        for (int s = 0; s < kRays; ++s) {
            J += pj[(long)s * nvox + v];
            U += pu[(long)s * nvox + v];
        }
        jeff[v] = J;
        u[v] = U;
    }
}

}  // namespace
}  // namespace mg3d

using namespace mg3d;

extern "C" int mg3d_formal_solve_noalloc(int nx, int ny, int nz, double dx, double dy,
                                         const double *z_dev, const mg3d_atom *atom,
                                         double quad_a, const double *chi0_dev,
                                         const double *S_dev, const double *bbot_dev,
                                         double *jeff_dev, double *u_dev, void *cuda_stream) {
    if (!atom || !z_dev || !chi0_dev || !S_dev || !bbot_dev || !jeff_dev || !u_dev) {
        record_error("null argument");
        return MG3D_E_ARG;
    }
    if (!std::isfinite(quad_a) || (quad_a > 0.0 && 2.0 * quad_a * quad_a >= 1.0)) {
        record_error("quadrature parameter a must be finite and below 1/sqrt(2) "
                     "(a <= 0 selects the default A4 set)");
        return MG3D_E_ARG;
    }
    if (nx < 1 || ny < 1 || nz < 2 || !(dx > 0.0) || !(dy > 0.0)) {
        record_error("grid needs nx, ny >= 1, nz >= 2 and dx, dy > 0");
        return MG3D_E_ARG;
    }
    const long nvox = (long)nx * ny * nz;
    if (nvox > kMaxNodes || nz > kMaxNz) {
        record_error("grid of " + std::to_string(nx) + "x" + std::to_string(ny) + "x" +
                     std::to_string(nz) + " nodes exceeds the allocation-free limit of " +
                     std::to_string(kMaxNodes) + " nodes and " + std::to_string(kMaxNz) +
                     " planes");
        return MG3D_E_ARG;
    }
    if (atom->gamma_prd != 0.0 || atom->a_damp != 0.0) {
        record_error("the allocation-free call takes Doppler profiles and complete "
                     "redistribution (gamma_prd and a_damp 0)");
        return MG3D_E_ARG;
    }
    const int nf = atom->n_freq;
    if (nf < 1 || nf > kMaxFreq || !(atom->x_max >= 0.0)) {
        record_error("n_freq must be 1.." + std::to_string(kMaxFreq) + " on the allocation-free path");
        return MG3D_E_ARG;
    }
    // one frequency group (24 partial slots); the fewest bands that fit
    SweepShape shape{nf, 1, 0, 0, 0};
    for (int bands = 1; bands <= kPortableBands && bands <= ny; ++bands) {
        const int rows = (ny + bands - 1) / bands;
        if ((long)(bands - 1) * rows >= ny) continue;
        SweepShape s{nf, 1, bands, rows, 0};
        if (sweep_smem_bytes(MG3D_PREC_F64, s, nx) <= kMaxSweepSmem) {
            shape = s;
            break;
        }
    }
    if (shape.bands == 0) {
        record_error("plane too large for the sweep's shared memory on the allocation-free path "
                     "(all n_freq intensity planes of a row band, at most 8 bands of 200 KB)");
        return MG3D_E_ARG;
    }
    const int band = shape.rows * nx;
    const int passes = (band + kMaxSweepThreads - 1) / kMaxSweepThreads;
    int th = ((band + passes - 1) / passes + 31) / 32 * 32;
    shape.threads = th < 32 ? 32 : th;

    double *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != MG3D_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    noalloc_tables_kernel<<<(kRays * nz + 255) / 256, 256, 0, st>>>(
        nx, ny, nz, dx, dy, z_dev, quad_a, nf, atom->x_max, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        double tab_unused[kExpTab], l1 = 0.0, l2 = 0.0;
        exp_neg_constants(tab_unused, &l1, &l2);
        unsigned up_mask = 0;
        for (int r = 0; r < kRays; ++r)
            if (!((r / 3) & 4)) up_mask |= 1u << r;
        SweepArgs<double> a{nx, ny, nz, nf, shape.ng, shape.ngroups, shape.rows, up_mask,
                            chi0_dev, S_dev, bbot_dev,
                            reinterpret_cast<const StepGeom *>(scratch + kOffGeom),
                            scratch + kOffPhi, scratch + kOffInvPhi, scratch + kOffWphi,
                            scratch + kOffPj, scratch + kOffPu, scratch + kOffExpTab, l1, l2};
        e = launch_sweep_f64(a, shape, st);
    }
    if (e == cudaSuccess) {
        long blocks = (nvox + 255) / 256;
        noalloc_reduce_kernel<<<(int)(blocks < 4864 ? blocks : 4864), 256, 0, st>>>(
            nvox, scratch + kOffPj, scratch + kOffPu, jeff_dev, u_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        record_error(std::string("allocation-free formal solution: ") + cudaGetErrorString(e));
        return MG3D_E_CUDA;
    }
    return MG3D_OK;
}
