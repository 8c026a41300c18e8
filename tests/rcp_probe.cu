// Device build of the binary64 reciprocal of the FP64 kernels (d_rcp in
// cn_arith.cuh) next to CUDA's own division 1.0 / q, for test_gpu_rcp.py.
// Every thread handles at most one element i < n.
#include <cuda_runtime.h>

#include "../paper_2205_00856_b300/csrc/cn_arith.cuh"

__global__ void k_rcp_probe(const double* q, double* y, double* ref, int* ok, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool k = true;
    y[i] = cnb::d_rcp(q[i], k);
    ok[i] = k;
    ref[i] = 1.0 / q[i];
}

// Host arrays in and out; returns a cudaError_t code (0 on success).
extern "C" int rcp_probe(const double* q, double* y, double* ref, int* ok, long n) {
    double *dq = nullptr, *dy = nullptr, *dr = nullptr;
    int* dk = nullptr;
    const size_t b = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMalloc(&dq, b);
    if (e == cudaSuccess) e = cudaMalloc(&dy, b);
    if (e == cudaSuccess) e = cudaMalloc(&dr, b);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(dq, q, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_rcp_probe<<<(unsigned)((n + 255) / 256), 256>>>(dq, dy, dr, dk, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, b, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ref, dr, b, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ok, dk, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(dq);
    cudaFree(dy);
    cudaFree(dr);
    cudaFree(dk);
    return (int)e;
}
