// FP64 fused-multiply-add throughput of the current device: the roofline denominator of the
// sweep kernels (which are bound by the FP64 pipe).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>

#include "../../include/msqoc.h"

namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

// 8 independent FMA chains per thread; the result is stored so the work cannot be removed
__global__ void __launch_bounds__(PEAK_THREADS) k_dfma_peak(double* out, int iters, double a, double b) {
    double x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = threadIdx.x * 1e-9 + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" msqoc_status msqoc_measure_fp64_peak(double* tflops) {
    if (!tflops) return MSQOC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MSQOC_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8;
    double* out = nullptr;
    if (cudaMalloc(&out, size_t(grid) * PEAK_THREADS * sizeof(double)) != cudaSuccess) return MSQOC_ERR_OUT_OF_MEMORY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 4000;
    k_dfma_peak<<<grid, PEAK_THREADS>>>(out, 100, 1.0000001, 1e-7);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        k_dfma_peak<<<grid, PEAK_THREADS>>>(out, iters, 1.0000001, 1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return MSQOC_ERR_CUDA;
    const double flops = 2.0 * PEAK_CHAINS * double(iters) * grid * PEAK_THREADS;
    *tflops = flops / (double(best) * 1e-3) / 1e12;
    return MSQOC_OK;
}
