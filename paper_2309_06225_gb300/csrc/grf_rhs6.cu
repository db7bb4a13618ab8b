// Single-state RHS and constraint kernels of the 6th-order scheme (4 ghost layers).
#include "grf_diag.cuh"
#include "grf_launch.h"

namespace grf {

// Blocks of (32, 4, 1) threads (block gather, as rk4_stage6_kernel). LOP: lopsided advection.
template <int LOP>
__global__ void __launch_bounds__(128) rhs6_kernel(Geom g, Coeffs c, const double* __restrict__ s,
                                                   double* __restrict__ rhs, double ko, int* status) {
    __shared__ YzRows6 sh;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z;
    yz_rows_fill6(g, s, i, blockIdx.y * 4, threadIdx.y, k, lane, sh);
    __syncthreads();
    const int jc = min(j, g.ny + 2);
    const long long p = gidx(g, min(i, g.nx + 2) + NG6, jc + NG6, k + NG6);
    PointIn in;
    double kos[NFIELDS], adv[LOP ? NFIELDS : 1];
    WarpRow6 wr;
    warp_row_halo6(g, s, i - lane, jc, k, lane, wr);
    gather6_block<LOP>(g, s, p, in, kos, adv, wr, sh, threadIdx.y);
    if (i >= g.nx || j >= g.ny) return;
    double r[NFIELDS];
    bool ok = true;
    point_rhs<double, double, -1, LOP>(c, in, r, nullptr, ok, adv);
    if (!ok) atomicOr(status, 1);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) rhs[f * g.fstride + p] = r[f] + ko * kos[f];
}

void launch_rhs6(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s, double* rhs,
                 double ko, int* status) {
    if (c.advection) rhs6_kernel<kLopsided><<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
    else rhs6_kernel<0><<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
}

void launch_constraints6(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s,
                         double* out4, double* part, double* dens, double* psi4, double3 origin, double* hyp) {
    if (psi4 || hyp) constraints_kernel<6, 1><<<grid, block, 0, st>>>(g, c, s, out4, part, dens, psi4, origin, hyp);
    else constraints_kernel<6, 0><<<grid, block, 0, st>>>(g, c, s, out4, part, dens, psi4, origin, hyp);
}

}  // namespace grf
