// Shifted-plane sweep (plane_sweep.cuh), FP32 instances.
#include "plane_sweep.cuh"

namespace mg3d {

cudaError_t launch_plane_sweep_f32(const PlaneArgs<float> &a, const SweepShape &s,
                                   cudaStream_t st) {
    if (s.plane == 2) return launch_plane_async_f32(a, s, st);
    return plane_dispatch<float, false>(&a, s, a.nx, st, nullptr);
}

cudaError_t plane_active_clusters_f32(const SweepShape &s, int nx, int *n) {
    if (s.plane == 2) return plane_async_clusters_f32(s, nx, n);
    return plane_dispatch<float, false>(nullptr, s, nx, 0, n);
}

}  // namespace mg3d
