// RK4 stage kernels of the decoupled mode (4dST without backreaction), one instantiation per
// stage, in their own translation unit so the library builds in parallel.
#include "grf_kernels.cuh"
#include "grf_launch.h"

namespace grf {
void launch_stage_decoupled(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                            const StageArgs& a) {
    switch (stage) {
        case 0: rk4_stage_kernel<0, 1, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 1: rk4_stage_kernel<1, 1, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 2: rk4_stage_kernel<2, 1, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        default: rk4_stage_kernel<3, 1, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
    }
}
}  // namespace grf
