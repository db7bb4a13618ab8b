/*
 * grf_peak.h -- FP64 throughput microbenchmark (libgrf_peak.so), the measured denominator of
 * the FP64 roofline of the evolution kernels. Not part of the method: a measurement tool.
 */
#ifndef GRF_PEAK_H
#define GRF_PEAK_H
#ifdef __cplusplus
extern "C" {
#endif
/* Runs `blocks` x `threads` threads, each advancing `chains` (4, 8 or 16) independent chains of
 * FP64 instructions for `iters` iterations; kind 0: DFMA, 1: DADD, 2: DMUL, 3: the mix
 * DADD : DMUL : DFMA = 1 : 1 : 2, 4: DFMA with per-chain operand registers, 5: DFMA with an
 * integer multiply-add beside each. One untimed launch, then `launches` back-to-back launches timed
 * together with CUDA events on `stream`. FP64 instructions executed in the timed region:
 * launches * blocks * threads * chains * iters. out_dev: device buffer of blocks * threads
 * doubles (keeps the chains live). *ms_out (host): the timed duration in milliseconds.
 * Returns 0, -1 on a bad argument, or -3 on a CUDA error. Synchronises `stream`. */
int grf_peak_fp64(int kind, int chains, int blocks, int threads, int iters, int launches, double* out_dev,
                  float* ms_out, void* stream);
#ifdef __cplusplus
}
#endif
#endif
