// FP64 throughput microbenchmark (measurement tool; see include/grf_peak.h): independent chains
// of FP64 instructions per thread, the instruction kind selectable, so that the pipe's issue
// rate can be measured with a mix of kinds like the stage kernel's as well as with FMAs alone.
#include <cuda_runtime.h>

#include "grf_peak.h"

namespace {
// CH independent chains per thread, each advanced `iters` times by an instruction of the kind:
// 0 DFMA, 1 DADD, 2 DMUL, 3 the mix DADD : DMUL : DFMA = 1 : 1 : 2 (per group of 4 chains),
// 4 DFMA with each chain's own multiplier and addend registers, 5 DFMA with one integer
// multiply-add beside each (other pipes busy as in a real kernel). The operands keep every chain
// bounded and non-constant.
template <int CH, int KIND>
__global__ void fp64_chains(int iters, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a[CH], bm[CH], ca[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        a[c] = 1.0 + 1e-9 * t + 0.01 * c;
        bm[c] = 0.99999999 - 1e-10 * c - 1e-15 * t;
        ca[c] = 1e-8 * (1.0 + 0.1 * c);
    }
    const double b = 0.99999999, cc = 1e-8, m = 1.0000000001;
    unsigned h = 2654435761u * (unsigned)t;
#pragma unroll 2
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int kind = KIND == 3 ? ((c & 3) == 0 ? 1 : ((c & 3) == 1 ? 2 : 0)) : KIND;
            if (kind == 0) a[c] = fma(a[c], b, cc);
            else if (kind == 1) a[c] = a[c] + (i & 1 ? -cc : cc);
            else if (kind == 2) a[c] = a[c] * (i & 1 ? b : m);
            else if (kind == 4) a[c] = fma(a[c], bm[c], ca[c]);
            else {
                a[c] = fma(a[c], b, cc);
                h = h * 1664525u + (unsigned)c;
            }
        }
    }
    double s = (double)(h & 1u) * 1e-300;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += a[c];
    out[t] = s;
}

template <int CH>
void launch(int kind, int blocks, int threads, int iters, double* out, cudaStream_t st) {
    switch (kind) {
        case 1: fp64_chains<CH, 1><<<blocks, threads, 0, st>>>(iters, out); break;
        case 2: fp64_chains<CH, 2><<<blocks, threads, 0, st>>>(iters, out); break;
        case 3: fp64_chains<CH, 3><<<blocks, threads, 0, st>>>(iters, out); break;
        case 4: fp64_chains<CH, 4><<<blocks, threads, 0, st>>>(iters, out); break;
        case 5: fp64_chains<CH, 5><<<blocks, threads, 0, st>>>(iters, out); break;
        default: fp64_chains<CH, 0><<<blocks, threads, 0, st>>>(iters, out); break;
    }
}
}  // namespace

extern "C" int grf_peak_fp64(int kind, int chains, int blocks, int threads, int iters, int launches, double* out_dev,
                             float* ms_out, void* stream) {
    if (kind < 0 || kind > 5 || (chains != 4 && chains != 8 && chains != 16) || blocks < 1 || threads < 32 ||
        threads > 1024 || iters < 1 || launches < 1 || !out_dev || !ms_out)
        return -1;
    cudaStream_t st = (cudaStream_t)stream;
    auto one = [&]() {
        if (chains == 4) launch<4>(kind, blocks, threads, iters, out_dev, st);
        else if (chains == 8) launch<8>(kind, blocks, threads, iters, out_dev, st);
        else launch<16>(kind, blocks, threads, iters, out_dev, st);
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -3;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -3; }
    one();  // warm-up
    cudaEventRecord(e0, st);
    for (int l = 0; l < launches; ++l) one();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e == cudaSuccess ? 0 : -3;
}
