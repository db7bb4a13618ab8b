// Folded RK4 stage kernels (boxes whose x-extent is not a multiple of 32), one instantiation
// per stage, in their own translation unit so the library builds in parallel.
#include "grf_kernels.cuh"
#include "grf_launch.h"

namespace grf {
void launch_stage_folded(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                         const StageArgs& a) {
    if (c.decoupled) {
        switch (stage) {
            case 0: rk4_stage_fold_kernel<0, 1><<<grid, block, 0, st>>>(g, c, a); break;
            case 1: rk4_stage_fold_kernel<1, 1><<<grid, block, 0, st>>>(g, c, a); break;
            case 2: rk4_stage_fold_kernel<2, 1><<<grid, block, 0, st>>>(g, c, a); break;
            default: rk4_stage_fold_kernel<3, 1><<<grid, block, 0, st>>>(g, c, a); break;
        }
        return;
    }
    switch (stage) {
        case 0: rk4_stage_fold_kernel<0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 1: rk4_stage_fold_kernel<1, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 2: rk4_stage_fold_kernel<2, 0><<<grid, block, 0, st>>>(g, c, a); break;
        default: rk4_stage_fold_kernel<3, 0><<<grid, block, 0, st>>>(g, c, a); break;
    }
}
}  // namespace grf
