// C-ABI entry points of libgrf.so (declared in include/grf.h).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <mutex>

#include "grf.h"
#include "grf_kernels6.cuh"
#include "grf_launch.h"

namespace grf {

char g_cuda_msg[256] = "";

__global__ void ko_kernel(Geom g, const double* __restrict__ s, double* __restrict__ rhs, double ko) {
    int i, j, k;
    if (!interior_thread(g, i, j, k)) return;
    const long long p = gidx(g, i + NG, j + NG, k + NG);
    for (int f = 0; f < NFIELDS; ++f) rhs[f * g.fstride + p] += ko * ko6(s + f * g.fstride, p, g.pitch, g.plane);
}

// The 6th-order scheme's dissipation: rhs += ko sum_d Delta^8_d u (ko = -sigma / (256 dx)).
__global__ void ko8_kernel(Geom g, const double* __restrict__ s, double* __restrict__ rhs, double ko) {
    int i, j, k;
    if (!interior_thread(g, i, j, k)) return;
    const long long p = gidx(g, i + NG6, j + NG6, k + NG6);
    for (int f = 0; f < NFIELDS; ++f) rhs[f * g.fstride + p] += ko * ko8(s + f * g.fstride, p, g.pitch, g.plane);
}

// Periodic ghost fill: one thread per ghosted (i, j) column and field; walks k.
__global__ void ghost_fill_kernel(Geom g, double* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    if (i >= g.NX || j >= g.NY) return;
    const int ng = g.ng;
    auto wrap = [ng](int a, int n) { int x = (a - ng) % n; if (x < 0) x += n; return x + ng; };
    const int wi = wrap(i, g.nx), wj = wrap(j, g.ny);
    const bool ghost_ij = (wi != i) || (wj != j);
    double* u = s + f * g.fstride;
    for (int k = 0; k < g.NZ; ++k) {
        const int wk = wrap(k, g.nz);
        if (!ghost_ij && wk == k) continue;
        u[gidx(g, i, j, k)] = u[gidx(g, wi, wj, wk)];
    }
}

// Mirror-plane ghost fill: every ghost point with a coordinate below the box takes its mirror
// image times the component's parity. GRF_BC_REFLECT_LOW (all = 0): only ghosts whose other
// coordinates are interior or low (the high faces are left as given); GRF_BC_REFLECT_LOW_SOMMERFELD
// (all = 1): also those beyond a high face in another axis, images of evolved high-face ghosts.
// One thread per (i, j) column and field; walks k.
__global__ void reflect_fill_kernel(Geom g, double* __restrict__ s, int all) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    const int ng = g.ng;
    const int ex = all ? g.NX : g.nx + ng, ey = all ? g.NY : g.ny + ng, ez = all ? g.NZ : g.nz + ng;
    if (i >= ex || j >= ey) return;
    double* u = s + (long long)f * g.fstride;
    const int a = i < ng ? 2 * ng - 1 - i : i, b = j < ng ? 2 * ng - 1 - j : j;
    const int mij = (i < ng ? 1 : 0) | (j < ng ? 2 : 0);
    for (int k = 0; k < ez; ++k) {
        const int m = mij | (k < ng ? 4 : 0);
        if (m == 0) continue;
        u[gidx(g, i, j, k)] = mirror_sign(f, m) * u[gidx(g, a, b, k < ng ? 2 * ng - 1 - k : k)];
    }
}

// Ghost preparation for one slab of z-planes [K0, K1) of the host-to-device pipeline of
// grf_rk4_step_host. Periodic: in-plane (x, y) wrap of the ghost columns of `s`; the z-ghost
// planes themselves were copied from the interior planes they are images of, so after this the
// planes hold what a full periodic refill gives. Frozen: the ghost points of `s` are copied into
// the stage buffers A and B, which carry the caller's ghosts through the stages.
__global__ void slab_ghost_kernel(Geom g, double* __restrict__ s, double* __restrict__ A, double* __restrict__ B,
                                  int K0, int K1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const long long fo = (long long)blockIdx.z * g.fstride;
    if (i >= g.NX || j >= g.NY) return;
    if (g.periodic) {
        auto wrap = [](int a, int n) { int x = (a - NG) % n; if (x < 0) x += n; return x + NG; };
        const int wi = wrap(i, g.nx), wj = wrap(j, g.ny);
        if (wi == i && wj == j) return;
        for (int k = K0; k < K1; ++k) s[fo + gidx(g, i, j, k)] = s[fo + gidx(g, wi, wj, k)];
    } else {  // frozen and mirror boxes: the ghosts go to A and B; mirror boxes rebuild their low ones
        const bool ghost_ij = i < NG || i >= g.nx + NG || j < NG || j >= g.ny + NG;
        const int mij = (i < NG ? 1 : 0) | (j < NG ? 2 : 0);
        const bool low_ij = i < g.nx + NG && j < g.ny + NG;
        for (int k = K0; k < K1; ++k) {
            if (!ghost_ij && k >= NG && k < g.nz + NG) continue;
            const long long q = fo + gidx(g, i, j, k);
            double v = s[q];
            if (g.reflect && low_ij && k < g.nz + NG) {  // a mirrored ghost: its source is interior
                const int m = mij | (k < NG ? 4 : 0);
                v = mirror_sign((int)blockIdx.z, m) *
                    s[fo + gidx(g, i < NG ? 2 * NG - 1 - i : i, j < NG ? 2 * NG - 1 - j : j, k < NG ? 2 * NG - 1 - k : k)];
                s[q] = v;
            }
            A[q] = v;
            B[q] = v;
        }
    }
}

// Copy of up to 81 contiguous runs (offsets and lengths in doubles) between page-locked host
// memory and device memory by the SMs (grf_rk4_step_host). On GB300 the copy engines lose most of
// their host-link bandwidth after, and while, the FP64 kernels run; loads and stores issued by a
// few dozen blocks keep the full link rate and take few block slots from the concurrent stages.
constexpr int kMaxRuns = 81;
struct CopyRuns {
    int n;
    long long dst[kMaxRuns], src[kMaxRuns], len[kMaxRuns];
};

template <bool V2>
__global__ void __launch_bounds__(256) run_copy_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                       CopyRuns r) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int q = 0; q < r.n; ++q) {
        if (V2) {  // 16-byte units, 4 in flight per thread
            const double2* s = reinterpret_cast<const double2*>(src + r.src[q]);
            double2* d = reinterpret_cast<double2*>(dst + r.dst[q]);
            const long long n = r.len[q] / 2;
            long long i = t0;
            for (; i + 3 * stride < n; i += 4 * stride) {
                const double2 a = s[i], b = s[i + stride], c = s[i + 2 * stride], e = s[i + 3 * stride];
                d[i] = a;
                d[i + stride] = b;
                d[i + 2 * stride] = c;
                d[i + 3 * stride] = e;
            }
            for (; i < n; i += stride) d[i] = s[i];
        } else {
            const double* s = src + r.src[q];
            double* d = dst + r.dst[q];
            const long long n = r.len[q];
            for (long long i = t0; i < n; i += stride) d[i] = s[i];
        }
    }
}

// Deterministic final reduction of the per-block partials (single block, fixed order).
__global__ void norms_final_kernel(const double* __restrict__ part, long long nblocks, double npts, double* __restrict__ out8) {
    __shared__ double red[8][256];
    const int t = threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long b = t; b < nblocks; b += 256)
        for (int m = 0; m < 8; ++m) acc[m] = (m & 1) ? fmax(acc[m], part[b * 8 + m]) : acc[m] + part[b * 8 + m];
    for (int m = 0; m < 8; ++m) red[m][t] = acc[m];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int m = 0; m < 8; ++m)
                red[m][t] = (m & 1) ? fmax(red[m][t], red[m][t + w]) : red[m][t] + red[m][t + w];
        __syncthreads();
    }
    if (t == 0)
        for (int m = 0; m < 8; ++m) out8[m] = (m & 1) ? red[m][0] : sqrt(red[m][0] / npts);
}

__global__ void finite_kernel(Geom g, const double* __restrict__ s, int* flag) {
    int i, j, k;
    if (!interior_thread(g, i, j, k)) return;
    const long long p = gidx(g, i + g.ng, j + g.ng, k + g.ng);
    for (int f = 0; f < NFIELDS; ++f)
        if (!isfinite(s[f * g.fstride + p])) { atomicOr(flag, 1); return; }
}


int record_cuda_error(cudaError_t e) {
    std::snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return GRF_ECUDA;
}
}  // namespace grf

using namespace grf;

namespace {

__device__ int g_status;

int cuda_fail(cudaError_t e) { return grf::record_cuda_error(e); }

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRF_OK : cuda_fail(e);
}

bool box_ok(const grf_box* b) {
    if (!b) return false;
    if ((b->ng != NG && b->ng != NG6) || b->nx < 1 || b->ny < 1 || b->nz < 1 || !(b->dx > 0.0)) return false;
    if (b->pitch < (long long)b->nx + 2 * b->ng) return false;
    if (b->bc != GRF_BC_PERIODIC && b->bc != GRF_BC_FROZEN && b->bc != GRF_BC_REFLECT_LOW && b->bc != GRF_BC_EXTRAPOLATE &&
        b->bc != GRF_BC_SOMMERFELD && b->bc != GRF_BC_REFLECT_LOW_SOMMERFELD)
        return false;
    if (b->bc != GRF_BC_FROZEN && (b->nx < b->ng || b->ny < b->ng || b->nz < b->ng)) return false;
    return true;
}

Geom make_geom(const grf_box* b) {
    Geom g;
    g.nx = b->nx; g.ny = b->ny; g.nz = b->nz;
    g.NX = b->nx + 2 * b->ng; g.NY = b->ny + 2 * b->ng; g.NZ = b->nz + 2 * b->ng;
    g.ng = b->ng;
    g.pitch = b->pitch;
    g.plane = b->pitch * g.NY;
    g.fstride = g.plane * g.NZ;
    g.dx = b->dx;
    g.periodic = (b->bc == GRF_BC_PERIODIC);
    g.reflect = (b->bc == GRF_BC_REFLECT_LOW || b->bc == GRF_BC_REFLECT_LOW_SOMMERFELD);
    return g;
}

bool params_ok(const grf_params* p) {
    if (!p) return false;
    if (p->beta_kind != GRF_BETA_LINEAR && p->beta_kind != GRF_BETA_QUADRATIC && p->beta_kind != GRF_BETA_EXPONENTIAL)
        return false;
    if (p->beta_kind == GRF_BETA_EXPONENTIAL && !(p->beta_kappa >= 0.0 && p->beta_kappa < 1e300)) return false;
    if (!(1.0 + p->a0 > 0.0) || !(1.0 + p->b0 > 0.0)) return false;
    if (p->advection != 0 && p->advection != 1) return false;
    return true;
}

// sigma times the dissipation factor of the box's scheme: sigma / (64 dx) with the 6th difference
// (4th order), -sigma / (256 dx) with the 8th difference (6th order); both damp the grid's
// Nyquist mode at sigma / dx per direction.
double ko_factor(const Geom& g, double sigma) {
    return g.ng == NG6 ? -sigma / (256.0 * g.dx) : sigma / (64.0 * g.dx);
}

const dim3 kBlock(32, 4, 1);

dim3 interior_grid(const Geom& g) {
    return dim3((g.nx + kBlock.x - 1) / kBlock.x, (g.ny + kBlock.y - 1) / kBlock.y, (g.nz + kBlock.z - 1) / kBlock.z);
}

// x-points per warp row of the stage launch: 32 (one row per warp, the block gather), or a
// folded 16 / 8 when that fills enough more lanes of a box whose x-extent is not a multiple of 32
// to pay for the per-thread gather, whose extra FP64 work and less coalesced loads cost about
// 15% with rows of 16 and 35% with rows of 8 (measured: 48^3 folded to rows of 16 runs 17%
// faster; 100^3 folded to rows of 4 ran 3% slower than unfolded).
// Folding also cuts the number of blocks, so it is used only when the folded grid still fills
// at least one wave of resident blocks (3 per SM); a smaller box ran 10% slower folded (13^3).
int fold_width(const Geom& g, const grf_params* p) {
    const int nx = g.nx;
    // the folded kernel: 4th order, centred advection, linear or quadratic coupling
    if (nx % 32 == 0 || g.ng != NG || p->advection || p->beta_kind == GRF_BETA_EXPONENTIAL) return 32;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 32;
    }
    int best = 32;
    double best_eff = (double)nx / (32.0 * ((nx + 31) / 32));
    for (int w : {16, 8}) {
        const double cost = (w == 16) ? 1.15 : 1.35;
        const double eff = (double)nx / ((double)w * ((nx + w - 1) / w)) / cost;
        const int rows = 4 * (32 / w);
        const long long blocks = (long long)((nx + w - 1) / w) * ((g.ny + rows - 1) / rows) * g.nz;
        if (eff > best_eff + 1e-12 && blocks >= 3LL * sms) { best = w; best_eff = eff; }
    }
    return best;
}

// Stage launch grid for `planes` z-planes with row width w (blocks of 32 x 4 x 1 threads).
dim3 stage_grid(const Geom& g, int planes, int w) {
    const int rows = 4 * (32 / w);
    return dim3((unsigned)((g.nx + w - 1) / w), (unsigned)((g.ny + rows - 1) / rows), (unsigned)planes);
}

size_t state_bytes(const Geom& g) { return sizeof(double) * (size_t)NFIELDS * (size_t)g.fstride; }

int* status_ptr() {
    int* p = nullptr;
    cudaGetSymbolAddress((void**)&p, g_status);
    return p;
}

// Ghosts read by the next right-hand side: periodic wrap, mirror images, or extrapolation;
// frozen and Sommerfeld ghosts are state as given.
int fill_ghosts(const Geom& g, int bc, double* s, cudaStream_t st) {
    if (bc == GRF_BC_EXTRAPOLATE) {
        launch_extrapolate(g, s, st);
        return check_launch();
    }
    if (g.reflect) {
        const int all = bc == GRF_BC_REFLECT_LOW_SOMMERFELD;
        dim3 blk(32, 8, 1), grd(((all ? g.NX : g.nx + g.ng) + 31) / 32, ((all ? g.NY : g.ny + g.ng) + 7) / 8, NFIELDS);
        reflect_fill_kernel<<<grd, blk, 0, st>>>(g, s, all);
        return check_launch();
    }
    if (!g.periodic) return GRF_OK;
    dim3 blk(32, 8, 1), grd((g.NX + 31) / 32, (g.NY + 7) / 8, NFIELDS);
    ghost_fill_kernel<<<grd, blk, 0, st>>>(g, s);
    return check_launch();
}

size_t constraint_partials(const Geom& g) {
    dim3 grd = interior_grid(g);
    return (size_t)grd.x * grd.y * grd.z;
}

// ---- host-to-host stepping (grf_rk4_step_host): per-device copy stream and events
constexpr int kMaxSlabs = 16;
constexpr int kMaxDevices = 64;

struct CopyPipe {
    bool ready = false;
    cudaStream_t copy = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t h2d[kMaxSlabs] = {}, s4[kMaxSlabs] = {};
};

std::mutex g_pipe_mu;
CopyPipe g_pipe[kMaxDevices];

void destroy_pipe(CopyPipe& p) {
    if (p.copy) cudaStreamDestroy(p.copy);
    for (cudaEvent_t* e : {&p.start, &p.done})
        if (*e) cudaEventDestroy(*e);
    for (int s = 0; s < kMaxSlabs; ++s) {
        if (p.h2d[s]) cudaEventDestroy(p.h2d[s]);
        if (p.s4[s]) cudaEventDestroy(p.s4[s]);
    }
    p = CopyPipe();
}

// The current device's copy stream and events, created on first use (caller holds g_pipe_mu).
int pipe_for_current_device(CopyPipe*& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return GRF_EINVAL;
    CopyPipe& p = g_pipe[dev];
    if (!p.ready) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p.copy, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
        for (int s = 0; s < kMaxSlabs && e == cudaSuccess; ++s) {
            e = cudaEventCreateWithFlags(&p.h2d[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.s4[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            destroy_pipe(p);
            return cuda_fail(e);
        }
        p.ready = true;
    }
    out = &p;
    return GRF_OK;
}

// Ghosted z-planes [K0, K1) of all fields as contiguous runs (offsets and lengths in doubles).
// The source of a run is the same planes, except for host -> device copies of periodic boxes,
// where the source of a z-ghost plane is the interior plane it is an image of (the host's ghosts
// are not read).
void plane_runs(const Geom& g, int K0, int K1, bool image_source, CopyRuns& r) {
    r.n = 0;
    int K = K0;
    while (K < K1) {
        int end, shift = 0;
        if (K < NG) {
            end = std::min(K1, NG);
            shift = (image_source && g.periodic) ? g.nz : 0;
        } else if (K < g.nz + NG) {
            end = std::min(K1, g.nz + NG);
        } else {
            end = K1;
            shift = (image_source && g.periodic) ? -g.nz : 0;
        }
        for (int f = 0; f < NFIELDS; ++f) {
            const long long off = (long long)f * g.fstride;
            r.dst[r.n] = off + (long long)K * g.plane;
            r.src[r.n] = off + (long long)(K + shift) * g.plane;
            r.len[r.n] = (long long)(end - K) * g.plane;
            ++r.n;
        }
        K = end;
    }
}

// The device address of a page-locked (cudaHostAlloc'ed or registered) host buffer, nullptr for
// pageable memory, whose copies then go through cudaMemcpyAsync.
const double* device_view(const double* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? (const double*)a.devicePointer : nullptr;
}

constexpr int kCopyBlocks = 48;  // enough blocks to reach the host-link rate, few enough to share the SMs

// Copies the runs from src to dst on `st`: by the SMs when both sides are device-addressable
// (dev_src / dev_dst non-null), else one cudaMemcpyAsync per run.
cudaError_t copy_runs(const CopyRuns& r, const double* src, const double* dev_src, double* dst, double* dev_dst,
                      cudaMemcpyKind kind, cudaStream_t st) {
    if (r.n == 0) return cudaSuccess;
    if (dev_src && dev_dst) {
        bool v2 = (((uintptr_t)dev_src | (uintptr_t)dev_dst) & 15) == 0;
        for (int q = 0; q < r.n; ++q) v2 = v2 && ((r.src[q] | r.dst[q] | r.len[q]) & 1) == 0;
        if (v2) run_copy_kernel<true><<<kCopyBlocks, 256, 0, st>>>(dev_src, dev_dst, r);
        else run_copy_kernel<false><<<kCopyBlocks, 256, 0, st>>>(dev_src, dev_dst, r);
        return cudaGetLastError();
    }
    for (int q = 0; q < r.n; ++q) {
        cudaError_t e = cudaMemcpyAsync(dst + r.dst[q], src + r.src[q], (size_t)r.len[q] * sizeof(double), kind, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char* grf_error_string(int code) {
    switch (code) {
        case GRF_OK: return "ok";
        case GRF_EINVAL: return "invalid argument (sizes, pointers, ng != 3, pitch, bc or parameters)";
        case GRF_EWORKSPACE: return "workspace too small or not 256-byte aligned";
        case GRF_ECUDA: return "CUDA error (see grf_last_cuda_error)";
        case GRF_ENONFINITE: return "non-finite value in the state";
        case GRF_ESINGULAR: return "singular coupled 7x7 system at some grid point";
        case GRF_ETIMEOUT: return "bounded device wait timed out";
        case GRF_ETOOLARGE: return "box too large for the fixed scratch of grf_rk4_step_noalloc (3 states > GRF_NOALLOC_SCRATCH_BYTES)";
        default: return "unknown error code";
    }
}

const char* grf_last_cuda_error(void) { return g_cuda_msg; }

size_t grf_workspace_bytes(const grf_box* box, int op) {
    if (!box_ok(box)) return 0;
    Geom g = make_geom(box);
    switch (op) {
        case GRF_OP_RHS: return 0;
        case GRF_OP_RK4: return 3 * state_bytes(g);
        case GRF_OP_CONSTRAINTS: return (constraint_partials(g) * 8 + 8) * sizeof(double) + 256;
        default: return 0;
    }
}

int grf_fill_ghosts(const grf_box* box, double* state, grf_stream_t stream) {
    if (!box_ok(box) || !state) return GRF_EINVAL;
    return fill_ghosts(make_geom(box), box->bc, state, (cudaStream_t)stream);
}

int grf_rhs(const grf_box* box, const grf_params* params, double* state, double* rhs, void* ws, size_t ws_bytes,
            grf_stream_t stream) {
    (void)ws; (void)ws_bytes;
    if (!box_ok(box) || !params_ok(params) || !state || !rhs) return GRF_EINVAL;
    Geom g = make_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    int r = fill_ghosts(g, box->bc, state, st);
    if (r) return r;
    launch_rhs(interior_grid(g), kBlock, st, g, make_coeffs(params), state, rhs, ko_factor(g, params->sigma_ko),
               status_ptr());
    if (box->bc == GRF_BC_SOMMERFELD || box->bc == GRF_BC_REFLECT_LOW_SOMMERFELD) {  // evolved ghosts' RHS
        StageArgs a{};
        a.src = state;
        launch_sommerfeld(-1, g, a, rhs, box->x0, box->y0, box->z0, st);
    }
    return check_launch();
}

int grf_ko_dissipation(const grf_box* box, double sigma, const double* state, double* rhs_accum, grf_stream_t stream) {
    if (!box_ok(box) || !state || !rhs_accum) return GRF_EINVAL;
    Geom g = make_geom(box);
    if (g.ng == NG6)
        ko8_kernel<<<interior_grid(g), kBlock, 0, (cudaStream_t)stream>>>(g, state, rhs_accum, ko_factor(g, sigma));
    else
        ko_kernel<<<interior_grid(g), kBlock, 0, (cudaStream_t)stream>>>(g, state, rhs_accum, ko_factor(g, sigma));
    return check_launch();
}

int grf_rk4_step(const grf_box* box, const grf_params* params, double* state, double dt, int nsteps, void* ws,
                 size_t ws_bytes, grf_stream_t stream) {
    if (!box_ok(box) || !params_ok(params) || !state || nsteps < 0) return GRF_EINVAL;
    Geom g = make_geom(box);
    const size_t sb = state_bytes(g);
    if (!ws || ws_bytes < 3 * sb || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    if (nsteps == 0) return GRF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    double* A = (double*)ws;
    double* B = (double*)((char*)ws + sb);
    double* acc = (double*)((char*)ws + 2 * sb);
    int r = fill_ghosts(g, box->bc, state, st);
    if (r) return r;
    if (box->bc == GRF_BC_FROZEN || box->bc == GRF_BC_REFLECT_LOW) {  // the stage buffers carry the caller's ghosts
        cudaError_t e = cudaMemcpyAsync(A, state, sb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B, state, sb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const Coeffs c = make_coeffs(params);
    StageArgs a;
    a.dt = dt;
    a.ko = ko_factor(g, params->sigma_ko);
    a.min_chi = params->min_chi;
    a.min_lapse = params->min_lapse;
    a.enforce = params->enforce_algebraic;
    a.status = status_ptr();
    a.k0 = 0;
    a.fold = fold_width(g, params);
    a.un = state;
    a.acc = acc;
    const dim3 grd = stage_grid(g, g.nz, a.fold);
    // outer boundaries after each stage: Sommerfeld ghosts take the same stage update, extrapolated
    // ghosts are refilled from the stage's new interior; behind mirror planes the images of the
    // evolved high-face ghosts follow their update
    auto boundary = [&](int stage) {
        if (box->bc == GRF_BC_SOMMERFELD) launch_sommerfeld(stage, g, a, nullptr, box->x0, box->y0, box->z0, st);
        else if (box->bc == GRF_BC_EXTRAPOLATE) launch_extrapolate(g, a.dst, st);
        else if (box->bc == GRF_BC_REFLECT_LOW_SOMMERFELD) {
            launch_sommerfeld(stage, g, a, nullptr, box->x0, box->y0, box->z0, st);
            fill_ghosts(g, box->bc, a.dst, st);
        }
    };
    for (int n = 0; n < nsteps; ++n) {
        a.src = state; a.dst = A;
        launch_stage(0, grd, kBlock, st, g, c, a);
        boundary(0);
        a.src = A; a.dst = B;
        launch_stage(1, grd, kBlock, st, g, c, a);
        boundary(1);
        a.src = B; a.dst = A;
        launch_stage(2, grd, kBlock, st, g, c, a);
        boundary(2);
        a.src = A; a.dst = state;
        launch_stage(3, grd, kBlock, st, g, c, a);
        boundary(3);
        r = check_launch();
        if (r) return r;
    }
    return GRF_OK;
}

int grf_rk4_step_host(const grf_box* box, const grf_params* params, const double* host_in, double* host_out,
                      double* state, double dt, int nsteps, void* ws, size_t ws_bytes, grf_stream_t stream) {
    if (!box_ok(box) || !params_ok(params) || !host_in || !host_out || !state || nsteps < 0) return GRF_EINVAL;
    Geom g = make_geom(box);
    const size_t sb = state_bytes(g);
    if (!ws || ws_bytes < 3 * sb || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_pipe_mu);
    CopyPipe* pp = nullptr;
    int r = pipe_for_current_device(pp);
    if (r) return r;
    const CopyPipe& P = *pp;
    cudaError_t e = cudaEventRecord(P.start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.copy, P.start, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    const double* dev_in = device_view(host_in);
    double* dev_out = const_cast<double*>(device_view(host_out));
    CopyRuns runs;
    if (nsteps == 0) {  // the state makes the round trip unchanged
        runs.n = 1;
        runs.dst[0] = runs.src[0] = 0;
        runs.len[0] = (long long)(sb / sizeof(double));
        e = copy_runs(runs, host_in, dev_in, state, state, cudaMemcpyHostToDevice, P.copy);
        if (e == cudaSuccess) e = copy_runs(runs, state, state, host_out, dev_out, cudaMemcpyDeviceToHost, P.copy);
        if (e == cudaSuccess) e = cudaEventRecord(P.done, P.copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P.done, 0);
        return e == cudaSuccess ? GRF_OK : cuda_fail(e);
    }
    // The slab pipeline below is laid out for 3 ghost layers whose ghosts are images or frozen state.
    // Other boxes (4 ghost layers; extrapolated or Sommerfeld ghosts) copy the whole state in, run
    // the device step, and copy it out, with the same stream ordering.
    if (box->ng != NG || box->bc == GRF_BC_EXTRAPOLATE || box->bc == GRF_BC_SOMMERFELD ||
        box->bc == GRF_BC_REFLECT_LOW_SOMMERFELD) {
        runs.n = 1;
        runs.dst[0] = runs.src[0] = 0;
        runs.len[0] = (long long)(sb / sizeof(double));
        e = copy_runs(runs, host_in, dev_in, state, state, cudaMemcpyHostToDevice, P.copy);
        if (e == cudaSuccess) e = cudaEventRecord(P.h2d[0], P.copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P.h2d[0], 0);
        if (e != cudaSuccess) return cuda_fail(e);
        const int r = grf_rk4_step(box, params, state, dt, nsteps, ws, ws_bytes, stream);
        if (r) return r;
        e = cudaEventRecord(P.s4[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P.copy, P.s4[0], 0);
        if (e == cudaSuccess) e = copy_runs(runs, state, state, host_out, dev_out, cudaMemcpyDeviceToHost, P.copy);
        if (e == cudaSuccess) e = cudaEventRecord(P.done, P.copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P.done, 0);
        return e == cudaSuccess ? GRF_OK : cuda_fail(e);
    }
    double* A = (double*)ws;
    double* B = (double*)((char*)ws + sb);
    double* acc = (double*)((char*)ws + 2 * sb);
    // Slab s = interior planes [lo(s), hi(s)); its copy chunk = ghosted planes [clo(s), chi(s)), the
    // first and last chunks also holding the z-ghost planes. Q >= 4 planes, so the planes a slab's
    // stencils read (up to interior plane hi + 2) lie in chunks s-1, s and s+1.
    const int Q = std::max(4, (g.nz + kMaxSlabs - 1) / kMaxSlabs);
    const int S = (g.nz + Q - 1) / Q;
    auto lo = [&](int s) { return s * Q; };
    auto hi = [&](int s) { return std::min(g.nz, (s + 1) * Q); };
    auto clo = [&](int s) { return s == 0 ? 0 : lo(s) + NG; };
    auto chi = [&](int s) { return s == S - 1 ? g.NZ : hi(s) + NG; };
    const Coeffs c = make_coeffs(params);
    StageArgs a;
    a.dt = dt;
    a.ko = ko_factor(g, params->sigma_ko);
    a.min_chi = params->min_chi;
    a.min_lapse = params->min_lapse;
    a.enforce = params->enforce_algebraic;
    a.status = status_ptr();
    a.un = state;
    a.acc = acc;
    a.fold = fold_width(g, params);
    const dim3 full = stage_grid(g, g.nz, a.fold);
    auto slab_grid = [&](int s) { return stage_grid(g, hi(s) - lo(s), a.fold); };
    const dim3 gblk(32, 8, 1), ggrd((g.NX + 31) / 32, (g.NY + 7) / 8, NFIELDS);

    for (int s = 0; s < S && e == cudaSuccess; ++s) {
        plane_runs(g, clo(s), chi(s), true, runs);
        e = copy_runs(runs, host_in, dev_in, state, state, cudaMemcpyHostToDevice, P.copy);
        if (e == cudaSuccess) e = cudaEventRecord(P.h2d[s], P.copy);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    for (int n = 0; n < nsteps; ++n) {
        a.src = state;
        a.dst = A;
        if (n == 0) {  // first stage, slab by slab as the planes arrive
            for (int s = 0; s <= S; ++s) {
                if (s < S) {
                    e = cudaStreamWaitEvent(st, P.h2d[s], 0);
                    if (e != cudaSuccess) return cuda_fail(e);
                    slab_ghost_kernel<<<ggrd, gblk, 0, st>>>(g, state, A, B, clo(s), chi(s));
                }
                if (s >= 1) {
                    a.k0 = lo(s - 1);
                    launch_stage(0, slab_grid(s - 1), kBlock, st, g, c, a);
                }
            }
        } else {
            a.k0 = 0;
            launch_stage(0, full, kBlock, st, g, c, a);
        }
        a.k0 = 0;
        a.src = A; a.dst = B;
        launch_stage(1, full, kBlock, st, g, c, a);
        a.src = B; a.dst = A;
        launch_stage(2, full, kBlock, st, g, c, a);
        a.src = A; a.dst = state;
        if (n < nsteps - 1) {
            launch_stage(3, full, kBlock, st, g, c, a);
        } else {  // last stage, slab by slab, each finished slab copied out behind the next
            for (int s = 0; s < S; ++s) {
                a.k0 = lo(s);
                launch_stage(3, slab_grid(s), kBlock, st, g, c, a);
                e = cudaEventRecord(P.s4[s], st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(P.copy, P.s4[s], 0);
                plane_runs(g, lo(s) + NG, hi(s) + NG, false, runs);
                if (e == cudaSuccess) e = copy_runs(runs, state, state, host_out, dev_out, cudaMemcpyDeviceToHost, P.copy);
                if (e != cudaSuccess) return cuda_fail(e);
            }
        }
        r = check_launch();
        if (r) return r;
    }
    // z-ghost planes (periodic images written by the first and last slabs; frozen: as given)
    plane_runs(g, 0, NG, false, runs);
    e = copy_runs(runs, state, state, host_out, dev_out, cudaMemcpyDeviceToHost, P.copy);
    plane_runs(g, g.nz + NG, g.NZ, false, runs);
    if (e == cudaSuccess) e = copy_runs(runs, state, state, host_out, dev_out, cudaMemcpyDeviceToHost, P.copy);
    if (e == cudaSuccess) e = cudaEventRecord(P.done, P.copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P.done, 0);
    return e == cudaSuccess ? GRF_OK : cuda_fail(e);
}

int grf_constraints(const grf_box* box, const grf_params* params, double* state, double* out4, double* norms_host,
                    void* ws, size_t ws_bytes, grf_stream_t stream) {
    if (!box_ok(box) || !params_ok(params) || !state || !out4) return GRF_EINVAL;
    Geom g = make_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = constraint_partials(g);
    if (norms_host) {
        if (!ws || ws_bytes < (nb * 8 + 8) * sizeof(double) || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    }
    int r = fill_ghosts(g, box->bc, state, st);
    if (r) return r;
    double* part = norms_host ? (double*)ws : nullptr;
    launch_constraints(interior_grid(g), kBlock, st, g, make_coeffs(params), state, out4, part, nullptr, nullptr,
                       make_double3(0.0, 0.0, 0.0));
    r = check_launch();
    if (r || !norms_host) return r;
    double* out8 = part + nb * 8;
    norms_final_kernel<<<1, 256, 0, st>>>(part, (long long)nb, (double)g.nx * g.ny * g.nz, out8);
    r = check_launch();
    if (r) return r;
    cudaError_t e = cudaMemcpyAsync(norms_host, out8, 8 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? GRF_OK : cuda_fail(e);
}

int grf_energy_densities(const grf_box* box, const grf_params* params, double* state, double* out3,
                         grf_stream_t stream) {
    if (!box_ok(box) || !params_ok(params) || !state || !out3) return GRF_EINVAL;
    Geom g = make_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    int r = fill_ghosts(g, box->bc, state, st);
    if (r) return r;
    launch_constraints(interior_grid(g), kBlock, st, g, make_coeffs(params), state, nullptr, nullptr, out3, nullptr,
                       make_double3(0.0, 0.0, 0.0));
    return check_launch();
}

int grf_weyl_psi4(const grf_box* box, const grf_params* params, double* state, double* out2, grf_stream_t stream) {
    if (!box_ok(box) || !params_ok(params) || !state || !out2) return GRF_EINVAL;
    Geom g = make_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    int r = fill_ghosts(g, box->bc, state, st);
    if (r) return r;
    launch_constraints(interior_grid(g), kBlock, st, g, make_coeffs(params), state, nullptr, nullptr, nullptr, out2,
                       make_double3(box->x0, box->y0, box->z0));
    return check_launch();
}

int grf_hyperbolicity(const grf_box* box, const grf_params* params, double* state, double* out4, grf_stream_t stream) {
    if (!box_ok(box) || !params_ok(params) || !state || !out4) return GRF_EINVAL;
    Geom g = make_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    int r = fill_ghosts(g, box->bc, state, st);
    if (r) return r;
    launch_constraints(interior_grid(g), kBlock, st, g, make_coeffs(params), state, nullptr, nullptr, nullptr, nullptr,
                       make_double3(0.0, 0.0, 0.0), out4);
    return check_launch();
}

int grf_extract_modes(const grf_box* box, const double* f_re, const double* f_im, int spin, const grf_sphere* sphere,
                      int ntheta, int nphi, int lmax, double* modes_host, void* ws, size_t ws_bytes,
                      grf_stream_t stream) {
    if (!box_ok(box)) return GRF_EINVAL;
    return extract_modes(box, make_geom(box), f_re, f_im, spin, sphere, ntheta, nphi, lmax, modes_host, ws, ws_bytes,
                         (cudaStream_t)stream);
}

int grf_check_status(grf_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    int h = 0, z = 0;
    e = cudaMemcpyFromSymbol(&h, g_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_status, &z, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
    return h ? GRF_ESINGULAR : GRF_OK;
}

int grf_check_finite(const grf_box* box, const double* state, void* ws, size_t ws_bytes, grf_stream_t stream) {
    if (!box_ok(box) || !state) return GRF_EINVAL;
    if (!ws || ws_bytes < 256 || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    Geom g = make_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    int* flag = (int*)ws;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e);
    finite_kernel<<<interior_grid(g), kBlock, 0, st>>>(g, state, flag);
    int r = check_launch();
    if (r) return r;
    int h = 0;
    e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    return h ? GRF_ENONFINITE : GRF_OK;
}

}  // extern "C"
