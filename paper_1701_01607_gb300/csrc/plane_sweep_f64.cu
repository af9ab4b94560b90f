// Shifted-plane sweep (plane_sweep.cuh), FP64 instances, and the host-side
// helpers shared by both precisions.
#include "plane_sweep.cuh"

namespace mg3d {

bool plane_np_supported(int np) {
    for (int i = 0; i < kPlaneNpCount; ++i)
        if (kPlaneNp[i] == np) return true;
    return false;
}

size_t plane_smem_bytes(int prec, int np, int rows, int nx) {
    const int vw = prec == 0 ? 2 : 4;                   // elements per 16-byte vector
    const int nch = (2 * np + 2 + vw - 1) / vw * vw;    // channels, whole vectors
    const int stride = ((nch / vw) | 1) * vw;           // odd number of vectors
    return 2ull * (rows + 1) * (nx + 1) * stride * (prec == 0 ? 8 : 4);
}

cudaError_t launch_plane_sweep_f64(const PlaneArgs<double> &a, const SweepShape &s,
                                   cudaStream_t st) {
    if (s.plane == 2) return launch_plane_async_f64(a, s, st);
    return plane_dispatch<double, false>(&a, s, a.nx, st, nullptr);
}

cudaError_t plane_active_clusters_f32(const SweepShape &s, int nx, int *n);

cudaError_t plane_active_clusters(int prec, const SweepShape &s, int nx, int *n) {
    *n = 0;
    if (prec != 0) return plane_active_clusters_f32(s, nx, n);
    if (s.plane == 2) return plane_async_clusters_f64(s, nx, n);
    return plane_dispatch<double, false>(nullptr, s, nx, 0, n);
}

}  // namespace mg3d
