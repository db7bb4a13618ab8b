// grf_rk4_step_noalloc: the RK4 step for callers that cannot allocate device memory.
//
// Its three stage buffers live in one file-scope __device__ array of fixed size instead of a
// caller-provided workspace. Every GPU that loads the library holds this array until the
// process exits. No cudaMalloc/cudaFree or allocating library routine is called.
#include <cstdint>
#include <mutex>

#include "grf.h"

namespace {

// The fixed scratch: two stage states and the RK4 accumulator of one box.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GRF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device. In host code the array's name
// is only a host-side stand-in, so the address is looked up (once per device, with that device
// current) and cached.
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return GRF_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GRF_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return GRF_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GRF_OK;
}

}  // namespace

extern "C" {

int grf_rk4_step_noalloc(const grf_box* box, const grf_params* params, double* state, double dt, int nsteps,
                         grf_stream_t stream) {
    const size_t need = grf_workspace_bytes(box, GRF_OP_RK4);
    if (need == 0) return GRF_EINVAL;
    if (need > (size_t)GRF_NOALLOC_SCRATCH_BYTES) return GRF_ETOOLARGE;
    void* ws = nullptr;
    const int r = scratch_address(&ws);
    if (r != GRF_OK) return r;
    return grf_rk4_step(box, params, state, dt, nsteps, ws, (size_t)GRF_NOALLOC_SCRATCH_BYTES, stream);
}

}  // extern "C"
