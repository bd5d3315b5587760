// Test helper (not part of the library): evaluates the FP64 division that
// the per-node arithmetic uses on the device (lbm::fdiv: hardware
// approximate reciprocal refined by two Newton-Raphson steps) next to
// CUDA's correctly rounded a / b, for tests/test_gpu_fdiv.py.
#include <cuda_runtime.h>

#include "../paper_1809_08683_gb300/csrc/lbm_node.cuh"

__global__ void k_fdiv(const double* a, const double* b, double* q_lbm, double* q_ieee, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    q_lbm[i] = lbm::fdiv(a[i], b[i]);
    q_ieee[i] = __ddiv_rn(a[i], b[i]);
}

// Host arrays of n doubles; returns 0 on success, else the CUDA error code.
extern "C" int fdiv_check(const double* a, const double* b, double* q_lbm, double* q_ieee, int n) {
    double* d = nullptr;
    const size_t bytes = (size_t)n * sizeof(double);
    cudaError_t e = cudaMalloc(&d, 4 * bytes);
    if (e != cudaSuccess) return (int)e;
    cudaMemcpy(d, a, bytes, cudaMemcpyHostToDevice);
    cudaMemcpy(d + n, b, bytes, cudaMemcpyHostToDevice);
    k_fdiv<<<(n + 255) / 256, 256>>>(d, d + n, d + 2 * n, d + 3 * n, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        cudaMemcpy(q_lbm, d + 2 * n, bytes, cudaMemcpyDeviceToHost);
        cudaMemcpy(q_ieee, d + 3 * n, bytes, cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    return (int)e;
}
