// cn_probe.cu -- cn_measure_fp64_rate: the throughput of the device's FP64 pipe,
// the denominator of the binary64 path's ALU roofline.
//
// Every thread of a grid of 4 CTAs per multiprocessor runs kChains independent
// chains of binary64 operations (FMA v = v a + b, or addition v = v + b) for a
// fixed number of iterations; the rate is the operations of the grid over the
// best of five CUDA-event timings.  The operands are passed at run time
// (a = 0.999999, b = 1e-9: generic values, the chains stay normal numbers), so
// the compiler cannot fold them.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cn.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kProbeThreads = 256;

// iters arrives at run time and the outer loop stays rolled, so every iteration
// issues the kChains independent operations back to back (a trip count known to
// the compiler let it regroup the chains and measured latency, not throughput)
template <bool kFma>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_rate(double* out, int iters, double a, double b) {
    double v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = 1e-3 * threadIdx.x + k;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) v[k] = kFma ? fma(v[k], a, b) : v[k] + b;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += v[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <bool kFma>
cudaError_t time_rate(double* out, unsigned grid, double* rate) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int r = 0; r < 6 && e == cudaSuccess; ++r) {  // the first run warms up
        e = cudaEventRecord(e0, nullptr);
        if (e == cudaSuccess) k_fp64_rate<kFma><<<grid, kProbeThreads>>>(out, kIters, 0.999999, 1e-9);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) *rate = (double)grid * kProbeThreads * (double)kIters * kChains / (best * 1e-3);
    return e;
}

}  // namespace

extern "C" cn_status cn_measure_fp64_rate(double* fma_per_s, double* add_per_s) {
    if (!fma_per_s || !add_per_s) return CN_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CN_ERR_CUDA;
    const unsigned grid = 4u * (unsigned)sms;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return CN_ERR_OOM;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = time_rate<true>(out, grid, fma_per_s);
    if (e == cudaSuccess) e = time_rate<false>(out, grid, add_per_s);
    cudaFree(out);
    return e == cudaSuccess ? CN_OK : CN_ERR_CUDA;
}
