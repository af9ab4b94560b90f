// Multi-level shifted-plane sweep (ml_plane.cuh): instances and host helpers.
#include "mg3d.h"
#include "ml_plane.cuh"

namespace mg3d {

size_t ml_plane_smem_bytes(int prec, int nf, int rows, int nx, int rpb) {
    return prec == MG3D_PREC_F64 ? 2ull * rpb * (rows + 1) * (nx + 1) *
                                       mlplane::node_stride<double>(nf) * sizeof(double)
                                 : 2ull * rpb * (rows + 1) * (nx + 1) *
                                       mlplane::node_stride<float>(nf) * sizeof(float);
}

cudaError_t launch_ml_plane_f64(const MlPlaneArgs<double> &a, int nf_block, int threads,
                                cudaStream_t st) {
    return ml_plane_dispatch<double>(&a, nf_block, a.bands, a.rows, a.nx, a.rpb, a.nfreq,
                                     threads, st, nullptr);
}

cudaError_t launch_ml_plane_f32(const MlPlaneArgs<float> &a, int nf_block, int threads,
                                cudaStream_t st) {
    return ml_plane_dispatch<float>(&a, nf_block, a.bands, a.rows, a.nx, a.rpb, a.nfreq,
                                    threads, st, nullptr);
}

cudaError_t ml_plane_active_clusters(int prec, int nf_block, int bands, int rows, int nx,
                                     int rpb, int nfreq, int threads, int *n) {
    *n = 0;
    if (prec == MG3D_PREC_F64)
        return ml_plane_dispatch<double>(nullptr, nf_block, bands, rows, nx, rpb, nfreq,
                                         threads, 0, n);
    return ml_plane_dispatch<float>(nullptr, nf_block, bands, rows, nx, rpb, nfreq, threads, 0,
                                    n);
}

}  // namespace mg3d
