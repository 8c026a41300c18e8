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

// The FMA forms of binary64 addition, subtraction and multiplication (d_add,
// d_sub, d_mul: fma with 1 or -0 from constant memory) next to the plain
// operations, element i of out holding (d_add, a + b, d_sub, a - b, d_mul, a b,
// d_add_int: the addition on the integer pipe).
__global__ void k_fma_form_probe(const double* a, const double* b, double* out, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = a[i], y = b[i];
    double* o = out + 7 * i;
    o[0] = cnb::d_add(x, y);
    o[1] = __dadd_rn(x, y);
    o[2] = cnb::d_sub(x, y);
    o[3] = __dsub_rn(x, y);
    o[4] = cnb::d_mul(x, y);
    o[5] = __dmul_rn(x, y);
    o[6] = cnb::d_add_int(x, y);
}

extern "C" int fma_form_probe(const double* a, const double* b, double* out, long n) {
    double *da = nullptr, *db = nullptr, *dout = nullptr;
    const size_t bytes = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMalloc(&da, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&db, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 7 * bytes);
    if (e == cudaSuccess) e = cudaMemcpy(da, a, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, b, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_fma_form_probe<<<(unsigned)((n + 255) / 256), 256>>>(da, db, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 7 * bytes, cudaMemcpyDeviceToHost);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dout);
    return (int)e;
}

// The complex reciprocal crcp<double> (integer arithmetic) on the device: z and w
// interleaved (re, im), ok per element.
__global__ void k_crcp_probe(const double* z, double* w, int* ok, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool k = true;
    const cnb::cx<double> r = cnb::crcp(cnb::mk(z[2 * i], z[2 * i + 1]), k);
    w[2 * i] = r.re;
    w[2 * i + 1] = r.im;
    ok[i] = k;
}

extern "C" int crcp_probe(const double* z, double* w, int* ok, long n) {
    double *dz = nullptr, *dw = nullptr;
    int* dk = nullptr;
    const size_t b = 2 * sizeof(double) * (size_t)n;
    cudaError_t e = cudaMalloc(&dz, b);
    if (e == cudaSuccess) e = cudaMalloc(&dw, b);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(dz, z, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_crcp_probe<<<(unsigned)((n + 255) / 256), 256>>>(dz, dw, dk, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(w, dw, b, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ok, dk, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(dz);
    cudaFree(dw);
    cudaFree(dk);
    return (int)e;
}

// The FMA on the integer pipe (d_fma_int) next to the device's fma, element i of out
// holding (d_fma_int(x, y, z), fma(x, y, z)).
__global__ void k_fma_int_probe(const double* x, const double* y, const double* z, double* out, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[2 * i] = cnb::d_fma_int(x[i], y[i], z[i]);
    out[2 * i + 1] = __fma_rn(x[i], y[i], z[i]);
}

extern "C" int fma_int_probe(const double* x, const double* y, const double* z, double* out, long n) {
    double *dx = nullptr, *dy = nullptr, *dz = nullptr, *dout = nullptr;
    const size_t bytes = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMalloc(&dx, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dy, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dz, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 2 * bytes);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dy, y, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dz, z, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_fma_int_probe<<<(unsigned)((n + 255) / 256), 256>>>(dx, dy, dz, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 2 * bytes, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dy);
    cudaFree(dz);
    cudaFree(dout);
    return (int)e;
}
