// Shifted-plane sweep (plane_sweep.cuh) with transaction-counted stores
// between blocks, FP64 instances.
#include "plane_sweep.cuh"

namespace mg3d {

cudaError_t launch_plane_async_f64(const PlaneArgs<double> &a, const SweepShape &s,
                                   cudaStream_t st) {
    return plane_dispatch<double, true>(&a, s, a.nx, st, nullptr);
}

cudaError_t plane_async_clusters_f64(const SweepShape &s, int nx, int *n) {
    return plane_dispatch<double, true>(nullptr, s, nx, 0, n);
}

}  // namespace mg3d
