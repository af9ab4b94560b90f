// Throughput probe of the arithmetic pipes the formal solution runs on.
//
// The sweep kernels are bound by arithmetic, not by memory, so their roofline
// needs the peak rates of the instructions they execute: FP32 fused
// multiply-add (the FMA pipes, 128 lanes per SM per clock nominally), the
// multi-function unit's ex2 and rcp approximations (the FP32 e^-x and 1/x),
// and FP64 fused multiply-add (the FP64 pipe).  Each probe kernel runs eight
// independent dependency chains per thread on enough blocks to fill every SM,
// so the rate it reaches is the pipe's throughput, not its latency.  The
// chains are contractions (or reciprocal pairs) that stay finite for any
// number of iterations, and their sum is written out so nothing is removed.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "mg3d.h"

namespace mg3d {

void record_error(const std::string &msg);

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float ex2_neg(float x) {
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x));
    return r;
}
__device__ __forceinline__ float rcp_f(float x) {
    float r;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// OP 0: FP32 FMA, 1: ex2, 2: rcp (each followed by one FMA, which runs on
// another pipe), 3: FP64 FMA; iters x kChains operations per thread
template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(int iters, double *out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (OP == 3) {
        double d[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) d[c] = 0.25 + 1e-3 * c + 1e-9 * tid;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) d[c] = fma(d[c], -0.999, 1.0);
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += d[c];
        out[tid] = s;
    } else {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 0.5f + 1e-3f * c + 1e-9f * tid;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (OP == 0) a[c] = fmaf(a[c], -0.999f, 1.0f);
                if (OP == 1) a[c] = ex2_neg(a[c]);     // a <- 2^-a, stays in (0, 1]
                if (OP == 2) a[c] = fmaf(rcp_f(a[c]), 0.5f, 0.5f);  // a <- 1/(2a) + 1/2, to 1
            }
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += a[c];
        out[tid] = s;
    }
}

template <int OP>
cudaError_t probe_one(int iters, int blocks, double *out, int reps, double *rate) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // launch 0 warms up
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) {
            probe_kernel<OP><<<blocks, 256>>>(iters, out);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) *rate = (double)blocks * 256 * iters * kChains / (best * 1e-3);
    return e;
}

}  // namespace
}  // namespace mg3d

using namespace mg3d;

extern "C" int mg3d_probe_alu_peaks(int reps, double *out_host) {
    if (reps < 1 || reps > 100 || !out_host) {
        record_error("mg3d_probe_alu_peaks: reps must be 1..100 and out_host non-null");
        return MG3D_E_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 8 * (sms > 0 ? sms : 1);
    double *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(double));
    // iterations sized for launches of a few to a few tens of milliseconds
    if (e == cudaSuccess) e = probe_one<0>(20000, blocks, out, reps, &out_host[0]);
    if (e == cudaSuccess) e = probe_one<1>(4000, blocks, out, reps, &out_host[1]);
    if (e == cudaSuccess) e = probe_one<2>(4000, blocks, out, reps, &out_host[2]);
    if (e == cudaSuccess) e = probe_one<3>(400, blocks, out, reps, &out_host[3]);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        record_error(std::string("mg3d_probe_alu_peaks: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return MG3D_E_CUDA;
    }
    return MG3D_OK;
}
