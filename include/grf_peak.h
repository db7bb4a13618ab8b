/*
 * grf_peak.h -- FP64 throughput microbenchmark (libgrf_peak.so), the measured denominator of
 * the FP64 roofline of the evolution kernels. Not part of the method: a measurement tool.
 */
#ifndef GRF_PEAK_H
#define GRF_PEAK_H
#ifdef __cplusplus
extern "C" {
#endif
/* Runs `blocks` x `threads` threads, each advancing 8 independent FP64 FMA chains for
 * `iters` iterations (16 * iters flops per thread), once untimed and once timed with CUDA
 * events on `stream`. out_dev: device buffer of blocks*threads doubles (keeps the chains
 * live). *ms_out (host): timed duration in milliseconds. Returns 0, or -3 on a CUDA error.
 * Synchronises `stream`. */
int grf_peak_fp64(int blocks, int threads, int iters, double* out_dev, float* ms_out, void* stream);
#ifdef __cplusplus
}
#endif
#endif
