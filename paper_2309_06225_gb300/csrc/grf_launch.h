// Host-side launchers of the heavy kernels (each lives in its own translation unit so the
// library builds in parallel).
#pragma once

#include <cuda_runtime.h>

#include "grf.h"
#include "grf_point.cuh"

namespace grf {
struct Geom;
struct StageArgs;

// The per-launch coefficients of a parameter set (every entry point builds them this way).
inline Coeffs make_coeffs(const grf_params* p) {
    Coeffs c;
    c.kappa1 = p->kappa1; c.kappa2 = p->kappa2; c.kappa3 = p->kappa3;
    c.shift_F = p->shift_F; c.eta = p->eta; c.lam = p->lambda; c.g2 = p->g2; c.g3 = p->g3;
    c.inv_1pa = 1.0 / (1.0 + p->a0);
    c.a_1pa = p->a0 / (1.0 + p->a0);
    c.bK = 3.0 * p->b0 / (4.0 * (1.0 + p->b0));
    c.bTh = 1.0 / (2.0 * (1.0 + p->b0));
    c.beta_kind = p->beta_kind;
    c.beta_kappa = p->beta_kappa;
    c.decoupled = p->decoupled;
    c.advection = p->advection;
    return c;
}

void launch_stage(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const StageArgs& a);
void launch_stage_decoupled(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                            const StageArgs& a);
void launch_stage_folded(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                         const StageArgs& a);
// 4th-order scheme with lopsided advection; 6th-order scheme (centred / lopsided advection)
void launch_stage_lopsided(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                           const StageArgs& a);
// 4th-order scheme, centred advection, every coupling (both decoupled modes compiled in)
void launch_stage_general(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                          const StageArgs& a);
void launch_stage6(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                   const StageArgs& a);
void launch_stage6_lopsided(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                            const StageArgs& a);
void launch_rhs6(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s, double* rhs,
                 double ko, int* status);
void launch_constraints6(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s,
                         double* out4, double* part, double* dens, double* psi4, double3 origin,
                         double* hyp = nullptr);
void launch_rhs(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s, double* rhs,
                double ko, int* status);
void launch_constraints(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s,
                        double* out4, double* part, double* dens, double* psi4, double3 origin,
                         double* hyp = nullptr);
// Outer boundaries (grf_boundary.cu): the extrapolation fill of all ghosts of s, and the
// Sommerfeld ghost update of one RK4 stage (stage 0..3) or, with stage -1, the ghosts' right-hand
// side written to out (a.src the state).
void launch_extrapolate(const Geom& g, double* s, cudaStream_t st);
void launch_sommerfeld(int stage, const Geom& g, const StageArgs& a, double* out, double x0, double y0, double z0,
                       cudaStream_t st);
// Waveform modes of a field on a sphere (grf_extract.cu; grf_extract_modes validates the box).
int extract_modes(const grf_box* box, const Geom& g, const double* f_re, const double* f_im, int spin,
                  const grf_sphere* sphere, int ntheta, int nphi, int lmax, double* modes_host, void* ws,
                  size_t ws_bytes, cudaStream_t st);
// Records a CUDA error for grf_last_cuda_error() and returns GRF_ECUDA.
int record_cuda_error(cudaError_t e);
}  // namespace grf
