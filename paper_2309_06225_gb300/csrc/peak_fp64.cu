// FP64 FMA throughput microbenchmark (measurement tool; see include/grf_peak.h).
#include <cuda_runtime.h>

#include "grf_peak.h"

namespace {
__global__ void dfma_chains(int iters, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a0 = 1.0 + 1e-9 * t, a1 = a0 + 0.1, a2 = a0 + 0.2, a3 = a0 + 0.3;
    double a4 = a0 + 0.4, a5 = a0 + 0.5, a6 = a0 + 0.6, a7 = a0 + 0.7;
    const double b = 0.99999999, c = 1e-8;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}
}  // namespace

extern "C" int grf_peak_fp64(int blocks, int threads, int iters, double* out_dev, float* ms_out, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -3;
    dfma_chains<<<blocks, threads, 0, st>>>(iters, out_dev);
    cudaEventRecord(e0, st);
    dfma_chains<<<blocks, threads, 0, st>>>(iters, out_dev);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e == cudaSuccess ? 0 : -3;
}
