// wb_peak.cu -- FMA throughput micro-benchmark (measurement helper for the
// ALU roofline of the sweep kernels; not part of the paper's method).
//
// Each thread runs 8 independent FMA chains for a fixed number of
// iterations; the grid is a multiple of the SM count so every SM is busy.
// The result is stored so the chains cannot be removed.
#include "../../include/wombat_gb300.h"

#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = x[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == T(-1.2345)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int run(double* tflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WB_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WB_ECUDA;
    const int blocks = nsm * 8, threads = 256;
    const int iters = sizeof(T) == 4 ? 1 << 14 : 1 << 9;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return WB_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-7);
    fma_chains<T><<<blocks, threads>>>(out, iters, a, b);   // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; r++) fma_chains<T><<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return WB_ECUDA;
    const double flops = 5.0 * 2.0 * 8.0 * double(iters) * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return WB_OK;
}

}  // namespace

extern "C" int wb_alu_peak(int precision, double* tflops) {
    if (!tflops) return WB_EINVAL;
    if (precision == WB_FP32) return run<float>(tflops);
    if (precision == WB_FP64) return run<double>(tflops);
    return WB_EINVAL;
}
