// RK4 stage kernels of the 4th-order scheme with centred advection for every coupling function
// and the cubic Horndeski term (the default instantiations compile only the linear and quadratic
// couplings, without the cubic term). The decoupled mode is
// a compile-time instantiation here too, so the bits equal those of the batched kernels.
#include "grf_kernels.cuh"
#include "grf_launch.h"

namespace grf {
void launch_stage_general(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                          const StageArgs& a) {
    if (c.decoupled) {
        switch (stage) {
            case 0: rk4_stage_kernel<0, 1, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
            case 1: rk4_stage_kernel<1, 1, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
            case 2: rk4_stage_kernel<2, 1, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
            default: rk4_stage_kernel<3, 1, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
        }
        return;
    }
    switch (stage) {
        case 0: rk4_stage_kernel<0, 0, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
        case 1: rk4_stage_kernel<1, 0, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
        case 2: rk4_stage_kernel<2, 0, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
        default: rk4_stage_kernel<3, 0, 0, 1><<<grid, block, 0, st>>>(g, c, a); break;
    }
}
}  // namespace grf
