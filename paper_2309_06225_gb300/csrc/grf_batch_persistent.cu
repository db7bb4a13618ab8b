// The persistent variant of the batched RK4 (GRF_BATCH_PERSISTENT): one cooperative launch of
// co-resident blocks that loop over the work list for every stage and step, separated by grid
// barriers whose spin is bounded.
// The stages of one launch read states that other blocks wrote before the previous grid barrier,
// so the stencil loads must be coherent (L2), not the read-only path.
#define GRF_COHERENT_LOADS 1
#include "grf_batch.cuh"

namespace grf {

// Grid-wide barrier for a cooperative launch. Thread 0 of each block arrives on a counter;
// the last arrival resets it and bumps the generation. Waiting is bounded by `timeout`
// clock cycles: on expiry the status word gets bit 2 and false is returned (the caller
// returns from the kernel), so a barrier can never hang the device.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long timeout, int* status) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > timeout) {
                    atomicOr(status, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(128, 3) batch_persistent_kernel(const BoxDesc* __restrict__ boxes,
                                                               const TileDesc* __restrict__ tiles, int ntiles,
                                                               int nsteps, unsigned* bar, int* status,
                                                               long long timeout) {
    __shared__ YzRows sh;
    for (int n = 0; n < nsteps; ++n) {
#pragma unroll 1
        for (int s = 0; s < 4; ++s) {
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const TileDesc td = tiles[t];
                const bool dec = boxes[td.box].c.decoupled != 0;
                const bool lop = boxes[td.box].c.advection != 0;
                switch (s) {
                    case 0: lop ? batch_tile_call<0, -1, 1>(boxes, td, status, sh)
                                : (dec ? batch_tile_call<0, 1, 0>(boxes, td, status, sh) : batch_tile_call<0, 0, 0>(boxes, td, status, sh)); break;
                    case 1: lop ? batch_tile_call<1, -1, 1>(boxes, td, status, sh)
                                : (dec ? batch_tile_call<1, 1, 0>(boxes, td, status, sh) : batch_tile_call<1, 0, 0>(boxes, td, status, sh)); break;
                    case 2: lop ? batch_tile_call<2, -1, 1>(boxes, td, status, sh)
                                : (dec ? batch_tile_call<2, 1, 0>(boxes, td, status, sh) : batch_tile_call<2, 0, 0>(boxes, td, status, sh)); break;
                    default: lop ? batch_tile_call<3, -1, 1>(boxes, td, status, sh)
                                 : (dec ? batch_tile_call<3, 1, 0>(boxes, td, status, sh) : batch_tile_call<3, 0, 0>(boxes, td, status, sh)); break;
                }
            }
            if (!grid_barrier(bar, gridDim.x, timeout, status)) return;
        }
    }
}

cudaError_t batch_persistent_attributes() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, (const void*)batch_persistent_kernel);
}

cudaError_t batch_persistent_occupancy(int nthreads, int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persistent_kernel, nthreads, 0);
}

cudaError_t launch_batch_persistent(dim3 grid, dim3 block, const BoxDesc* boxes, const TileDesc* tiles, int ntiles,
                                    int nsteps, unsigned* bar, int* status, long long timeout, cudaStream_t st) {
    void* args[] = {(void*)&boxes, (void*)&tiles, (void*)&ntiles, (void*)&nsteps, (void*)&bar, (void*)&status,
                    (void*)&timeout};
    return cudaLaunchCooperativeKernel((const void*)batch_persistent_kernel, grid, block, args, 0, st);
}

}  // namespace grf
