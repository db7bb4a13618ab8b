// One box (periodic or with frozen ghosts) evolved as px x py x pz patches with a halo exchange
// after every RK4 stage (domain decomposition on one device; the calls are declared in grf.h).
//
// The stage work of all patches is one launch of the batched stage kernel over the patches' tiles
// (each patch a frozen-ghost box: the stage reads its ghosts and writes its interior only). After
// the stage, the exchange writes every ghost point of every patch from the interior of the patch
// that owns the point in the box (periodic: every ghost point; frozen: the ghost points inside the
// box, the others keep the caller's values). The stage arithmetic per point is that of grf_rk4_step
// and its inputs are the same values, so the results are the same bits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "grf.h"
#include "grf_batch.cuh"
#include "grf_launch.h"
#include "grf_shell.cuh"

namespace grf {

// The level's patch layout, passed by value to the exchange and copy kernels.
struct PatchTable {
    int p[3];                                      // patches per axis
    int n[3];                                      // the box's interior points per axis
    int periodic;                                  // 1: periodic box, 0: frozen ghosts
    int off[3][GRF_MAX_PATCHES_PER_AXIS + 1];      // first interior point of each patch, per axis
    double* ptr[GRF_MAX_PATCHES];                  // the patch states (device)
};

__host__ __device__ __forceinline__ long long patch_pitch(int nx) { return ((long long)nx + 2 * NG + 3) / 4 * 4; }

__host__ __device__ __forceinline__ Geom patch_geom(const PatchTable& t, int a, int b, int c) {
    Geom g;
    g.nx = t.off[0][a + 1] - t.off[0][a];
    g.ny = t.off[1][b + 1] - t.off[1][b];
    g.nz = t.off[2][c + 1] - t.off[2][c];
    g.NX = g.nx + 2 * NG; g.NY = g.ny + 2 * NG; g.NZ = g.nz + 2 * NG;
    g.ng = NG;
    g.pitch = patch_pitch(g.nx);
    g.plane = g.pitch * g.NY;
    g.fstride = g.plane * g.NZ;
    g.dx = 0.0;  // not used by the copies
    g.periodic = 0;
    g.reflect = 0;
    return g;
}

// The patch along one axis that owns interior point x of the box (the last with off <= x).
__device__ __forceinline__ int owner(const int* off, int p, int x) {
    int a = 0;
    while (a + 1 < p && off[a + 1] <= x) ++a;
    return a;
}

// One thread per ghost point of patch blockIdx.y; 27 fields each. In a frozen box the ghost points
// outside the box are skipped.
__global__ void __launch_bounds__(256) halo_exchange_kernel(PatchTable t) {
    const int q = blockIdx.y;
    const int a = q % t.p[0], b = (q / t.p[0]) % t.p[1], c = q / (t.p[0] * t.p[1]);
    const Geom g = patch_geom(t, a, b, c);
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= shell_count(g, 0)) return;
    int i, j, k;
    shell_point(g, 0, s, i, j, k);
    // the point in the box's interior indices (ghost layers reach at most 3 beyond it)
    int x = t.off[0][a] + i - NG, y = t.off[1][b] + j - NG, z = t.off[2][c] + k - NG;
    if (!t.periodic && (x < 0 || x >= t.n[0] || y < 0 || y >= t.n[1] || z < 0 || z >= t.n[2])) return;
    x += x < 0 ? t.n[0] : (x >= t.n[0] ? -t.n[0] : 0);
    y += y < 0 ? t.n[1] : (y >= t.n[1] ? -t.n[1] : 0);
    z += z < 0 ? t.n[2] : (z >= t.n[2] ? -t.n[2] : 0);
    const int oa = owner(t.off[0], t.p[0], x), ob = owner(t.off[1], t.p[1], y), oc = owner(t.off[2], t.p[2], z);
    const Geom h = patch_geom(t, oa, ob, oc);
    const double* __restrict__ src =
        t.ptr[oa + t.p[0] * (ob + t.p[1] * oc)] +
        gidx(h, x - t.off[0][oa] + NG, y - t.off[1][ob] + NG, z - t.off[2][oc] + NG);
    double* __restrict__ dst = t.ptr[q] + gidx(g, i, j, k);
#pragma unroll 9
    for (int f = 0; f < NFIELDS; ++f) dst[(long long)f * g.fstride] = src[(long long)f * h.fstride];
}

// One thread per point of patch blockIdx.y: to_patch, every point of the patch, ghosts included,
// from the same point of the box (the patch's ghosted block lies inside the box's); otherwise the
// box's interior from the patch's.
__global__ void __launch_bounds__(256) patch_copy_kernel(PatchTable t, Geom box, double* __restrict__ s, int to_patch) {
    const int q = blockIdx.y;
    const int a = q % t.p[0], b = (q / t.p[0]) % t.p[1], c = q / (t.p[0] * t.p[1]);
    const Geom g = patch_geom(t, a, b, c);
    const int h = to_patch ? NG : 0;  // extent beyond the interior
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = g.nx + 2 * h, plane = row * (g.ny + 2 * h);
    if (r >= plane * (g.nz + 2 * h)) return;
    const int k = (int)(r / plane) - h, j = (int)((r % plane) / row) - h, i = (int)(r % row) - h;
    double* p = t.ptr[q] + gidx(g, i + NG, j + NG, k + NG);
    double* w = s + gidx(box, t.off[0][a] + i + NG, t.off[1][b] + j + NG, t.off[2][c] + k + NG);
#pragma unroll 9
    for (int f = 0; f < NFIELDS; ++f) {
        if (to_patch) p[(long long)f * g.fstride] = w[(long long)f * box.fstride];
        else w[(long long)f * box.fstride] = p[(long long)f * g.fstride];
    }
}

}  // namespace grf

using namespace grf;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool level_ok(const grf_patch_level* L) {
    if (!L) return false;
    const grf_box& b = L->box;
    if (b.ng != NG || (b.bc != GRF_BC_PERIODIC && b.bc != GRF_BC_FROZEN) || !(b.dx > 0.0)) return false;
    if (b.nx < 1 || b.ny < 1 || b.nz < 1 || b.pitch < (long long)b.nx + 2 * NG) return false;
    if (b.bc == GRF_BC_PERIODIC && (b.nx < NG || b.ny < NG || b.nz < NG)) return false;
    const int p[3] = {L->px, L->py, L->pz}, n[3] = {b.nx, b.ny, b.nz};
    for (int d = 0; d < 3; ++d)
        if (p[d] < 1 || p[d] > GRF_MAX_PATCHES_PER_AXIS || p[d] > n[d]) return false;
    return (long long)p[0] * p[1] * p[2] <= GRF_MAX_PATCHES;
}

int npatches(const grf_patch_level* L) { return L->px * L->py * L->pz; }

// The layout table (level_ok holds); ptrs may be null (geometry only).
PatchTable table_of(const grf_patch_level* L, double* const* ptrs) {
    PatchTable t;
    std::memset(&t, 0, sizeof(t));
    t.p[0] = L->px; t.p[1] = L->py; t.p[2] = L->pz;
    t.n[0] = L->box.nx; t.n[1] = L->box.ny; t.n[2] = L->box.nz;
    t.periodic = L->box.bc == GRF_BC_PERIODIC;
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a <= t.p[d]; ++a) t.off[d][a] = (int)((long long)a * t.n[d] / t.p[d]);
    if (ptrs)
        for (int q = 0; q < npatches(L); ++q) t.ptr[q] = ptrs[q];
    return t;
}

Geom geom_at(const PatchTable& t, int q) {
    return patch_geom(t, q % t.p[0], (q / t.p[0]) % t.p[1], q / (t.p[0] * t.p[1]));
}

size_t patch_state_bytes(const Geom& g) { return sizeof(double) * (size_t)NFIELDS * (size_t)g.fstride; }

bool ptrs_ok(const grf_patch_level* L, double* const* ptrs) {
    if (!ptrs) return false;
    for (int q = 0; q < npatches(L); ++q)
        if (!ptrs[q]) return false;
    return true;
}

int launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRF_OK : record_cuda_error(e);
}

struct PatchLayout {
    size_t boxes, tiles, bufs, total;
    long long ntiles;
};

PatchLayout patch_layout(const PatchTable& t, int np) {
    PatchLayout L;
    L.ntiles = 0;
    size_t bufs = 0;
    for (int q = 0; q < np; ++q) {
        const Geom g = geom_at(t, q);
        const int w = batch_row_width(g.nx);
        const int rows = 4 * (32 / w);
        L.ntiles += (long long)((g.nx + w - 1) / w) * ((g.ny + rows - 1) / rows) * g.nz;
        bufs += 3 * align_up(patch_state_bytes(g));
    }
    L.boxes = kAlign;  // the status word lives at the start
    L.tiles = L.boxes + align_up(sizeof(BoxDesc) * (size_t)np);
    L.bufs = L.tiles + align_up(sizeof(TileDesc) * (size_t)L.ntiles);
    L.total = L.bufs + bufs;
    return L;
}

}  // namespace

extern "C" {

int grf_patch_box(const grf_patch_level* level, int index, grf_box* out) {
    if (!level_ok(level) || !out || index < 0 || index >= npatches(level)) return GRF_EINVAL;
    const PatchTable t = table_of(level, nullptr);
    const int a = index % t.p[0], b = (index / t.p[0]) % t.p[1], c = index / (t.p[0] * t.p[1]);
    const Geom g = patch_geom(t, a, b, c);
    const grf_box& B = level->box;
    grf_box r;
    std::memset(&r, 0, sizeof(r));
    r.nx = g.nx; r.ny = g.ny; r.nz = g.nz;
    r.ng = NG;
    r.dx = B.dx;
    r.x0 = B.x0 + t.off[0][a] * B.dx;
    r.y0 = B.y0 + t.off[1][b] * B.dx;
    r.z0 = B.z0 + t.off[2][c] * B.dx;
    r.bc = GRF_BC_FROZEN;
    r.pitch = g.pitch;
    *out = r;
    return GRF_OK;
}

int grf_patch_copy(const grf_patch_level* level, double* box_state, double* const* patches, int direction,
                   grf_stream_t stream) {
    if (!level_ok(level) || !box_state || !ptrs_ok(level, patches) || (direction != 0 && direction != 1))
        return GRF_EINVAL;
    const PatchTable t = table_of(level, patches);
    const grf_box& B = level->box;
    Geom box;
    box.nx = B.nx; box.ny = B.ny; box.nz = B.nz;
    box.NX = B.nx + 2 * NG; box.NY = B.ny + 2 * NG; box.NZ = B.nz + 2 * NG;
    box.ng = NG;
    box.pitch = B.pitch;
    box.plane = B.pitch * box.NY;
    box.fstride = box.plane * box.NZ;
    box.dx = B.dx;
    box.periodic = 1;
    box.reflect = 0;
    const int h = direction == 0 ? 2 * NG : 0;
    long long most = 0;
    for (int q = 0; q < npatches(level); ++q) {
        const Geom g = geom_at(t, q);
        const long long n = (long long)(g.nx + h) * (g.ny + h) * (g.nz + h);
        if (n > most) most = n;
    }
    const dim3 grd((unsigned)((most + 255) / 256), (unsigned)npatches(level), 1);
    patch_copy_kernel<<<grd, 256, 0, (cudaStream_t)stream>>>(t, box, box_state, direction == 0);
    return launch_status();
}

// The halo exchange as data. Along one axis, the ghosted index range [0, n_a + 6) of patch a maps
// to the box's interior point x = off[a] + g - 3 (wrapped in a periodic box; outside a frozen box
// there is nothing to copy), owned by patch o with index x - off[o] + 3. Runs of consecutive g
// with the same owner and consecutive source indices are the axis's segments; a block of the
// plan is one segment per axis, except the patch's own interior (the identity on all three).
namespace {
struct AxisRun { int g0, len, owner, s0; bool self; };

std::vector<AxisRun> axis_runs(const PatchTable& t, int d, int a) {
    std::vector<AxisRun> runs;
    const int n = t.off[d][a + 1] - t.off[d][a], N = t.n[d];
    for (int g = 0; g < n + 2 * NG; ++g) {
        int x = t.off[d][a] + g - NG;
        if (x < 0 || x >= N) {
            if (!t.periodic) continue;
            x = (x % N + N) % N;
        }
        int o = 0;
        while (o + 1 < t.p[d] && t.off[d][o + 1] <= x) ++o;
        const int sg = x - t.off[d][o] + NG;
        const bool self = (o == a && sg == g);
        if (!runs.empty()) {
            AxisRun& r = runs.back();
            if (r.owner == o && r.self == self && r.g0 + r.len == g && r.s0 + r.len == sg) {
                ++r.len;
                continue;
            }
        }
        runs.push_back({g, 1, o, sg, self});
    }
    return runs;
}
}  // namespace

int grf_halo_plan(const grf_patch_level* level, grf_halo_block* blocks, int max_blocks) {
    if (!level_ok(level) || max_blocks < 0 || (max_blocks > 0 && !blocks)) return GRF_EINVAL;
    const PatchTable t = table_of(level, nullptr);
    int count = 0;
    for (int q = 0; q < npatches(level); ++q) {
        const int a = q % t.p[0], b = (q / t.p[0]) % t.p[1], c = q / (t.p[0] * t.p[1]);
        const std::vector<AxisRun> rx = axis_runs(t, 0, a), ry = axis_runs(t, 1, b), rz = axis_runs(t, 2, c);
        for (const AxisRun& z : rz)
            for (const AxisRun& y : ry)
                for (const AxisRun& x : rx) {
                    if (x.self && y.self && z.self) continue;
                    if (count < max_blocks) {
                        grf_halo_block& k = blocks[count];
                        k.dst = q;
                        k.src = x.owner + t.p[0] * (y.owner + t.p[1] * z.owner);
                        k.dst_i = x.g0; k.dst_j = y.g0; k.dst_k = z.g0;
                        k.src_i = x.s0; k.src_j = y.s0; k.src_k = z.s0;
                        k.ni = x.len; k.nj = y.len; k.nk = z.len;
                    }
                    ++count;
                }
    }
    return count;
}

int grf_halo_exchange(const grf_patch_level* level, double* const* patches, grf_stream_t stream) {
    if (!level_ok(level) || !ptrs_ok(level, patches)) return GRF_EINVAL;
    const PatchTable t = table_of(level, patches);
    long long most = 0;
    for (int q = 0; q < npatches(level); ++q) {
        const long long n = shell_count(geom_at(t, q), 0);
        if (n > most) most = n;
    }
    const dim3 grd((unsigned)((most + 255) / 256), (unsigned)npatches(level), 1);
    halo_exchange_kernel<<<grd, 256, 0, (cudaStream_t)stream>>>(t);
    return launch_status();
}

size_t grf_patches_workspace_bytes(const grf_patch_level* level) {
    if (!level_ok(level)) return 0;
    return patch_layout(table_of(level, nullptr), npatches(level)).total;
}

int grf_patches_rk4(const grf_patch_level* level, const grf_params* params, double* const* patches, double dt,
                    int nsteps, grf_halo_fn exchange, void* exchange_ctx, void* ws, size_t ws_bytes, int* status_host,
                    grf_stream_t stream) {
    if (!level_ok(level) || !params || !batch_params_ok(params) || !ptrs_ok(level, patches) || nsteps < 0)
        return GRF_EINVAL;
    const int np = npatches(level);
    const PatchTable t = table_of(level, nullptr);
    const PatchLayout L = patch_layout(t, np);
    if (L.ntiles > 0x7fffffffLL) return GRF_EINVAL;
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & (kAlign - 1))) return GRF_EWORKSPACE;
    if (nsteps == 0) return GRF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    int* status = (int*)base;
    BoxDesc* dboxes = (BoxDesc*)(base + L.boxes);
    TileDesc* dtiles = (TileDesc*)(base + L.tiles);

    // descriptors: every patch a frozen-ghost box with the level's couplings and time step
    std::vector<BoxDesc> hb(np);
    std::vector<TileDesc> ht;
    ht.reserve((size_t)L.ntiles);
    std::vector<double*> bufA(np), bufB(np), un(patches, patches + np);
    size_t off = L.bufs;
    for (int q = 0; q < np; ++q) {
        grf_box pb;
        grf_patch_box(level, q, &pb);
        BoxDesc& d = hb[q];
        batch_box_desc(d, &pb, params, dt);
        const size_t sb = align_up(patch_state_bytes(d.g));
        d.un = patches[q];
        d.A = bufA[q] = (double*)(base + off);
        d.B = bufB[q] = (double*)(base + off + sb);
        d.acc = (double*)(base + off + 2 * sb);
        off += 3 * sb;
        const int w = batch_row_width(pb.nx);
        const int rows = 4 * (32 / w);
        for (int k = 0; k < pb.nz; ++k)
            for (int j = 0; j < pb.ny; j += rows)
                for (int i = 0; i < pb.nx; i += w) ht.push_back(TileDesc{q, i, j, k, w});
    }
    cudaError_t e = cudaMemcpyAsync(dboxes, hb.data(), sizeof(BoxDesc) * np, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtiles, ht.data(), sizeof(TileDesc) * ht.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, kAlign, st);
    if (e != cudaSuccess) return record_cuda_error(e);  // (pageable sources: staged before the calls return)
    if (level->box.bc == GRF_BC_FROZEN)  // the stage buffers carry the ghosts outside the box
        for (int q = 0; q < np && e == cudaSuccess; ++q) {
            const size_t sb = patch_state_bytes(hb[q].g);
            e = cudaMemcpyAsync(bufA[q], patches[q], sb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(bufB[q], patches[q], sb, cudaMemcpyDeviceToDevice, st);
        }
    if (e != cudaSuccess) return record_cuda_error(e);

    auto halo = [&](std::vector<double*>& bufs) -> int {
        return exchange ? exchange(exchange_ctx, level, bufs.data(), stream)
                        : grf_halo_exchange(level, bufs.data(), stream);
    };
    const dim3 block(32, 4, 1);
    int r = halo(un);
    if (r) return r;
    for (int n = 0; n < nsteps; ++n) {
        // stage outputs: A, B, A, then the patch states (batch_tile's buffer order)
        launch_batch_stage(0, L.ntiles, block, st, dboxes, dtiles, status);
        if ((r = launch_status()) || (r = halo(bufA))) return r;
        launch_batch_stage(1, L.ntiles, block, st, dboxes, dtiles, status);
        if ((r = launch_status()) || (r = halo(bufB))) return r;
        launch_batch_stage(2, L.ntiles, block, st, dboxes, dtiles, status);
        if ((r = launch_status()) || (r = halo(bufA))) return r;
        launch_batch_stage(3, L.ntiles, block, st, dboxes, dtiles, status);
        if ((r = launch_status()) || (r = halo(un))) return r;
    }
    if (status_host) {
        e = cudaMemcpyAsync(status_host, status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return record_cuda_error(e);
        if (*status_host & 1) return GRF_ESINGULAR;
    }
    return GRF_OK;
}

size_t grf_patches_constraints_workspace_bytes(const grf_patch_level* level) {
    if (!level_ok(level)) return 0;
    size_t most = 0;
    for (int q = 0; q < npatches(level); ++q) {
        grf_box pb;
        grf_patch_box(level, q, &pb);
        const size_t n = grf_workspace_bytes(&pb, GRF_OP_CONSTRAINTS);
        if (n > most) most = n;
    }
    return most;
}

int grf_patches_constraints(const grf_patch_level* level, const grf_params* params, double* const* patches,
                            double* const* out4, double* norms_host, void* ws, size_t ws_bytes, grf_stream_t stream) {
    if (!level_ok(level) || !params || !ptrs_ok(level, patches) || !ptrs_ok(level, out4)) return GRF_EINVAL;
    double sq[4] = {0, 0, 0, 0}, mx[4] = {0, 0, 0, 0};
    long long total = 0;
    for (int q = 0; q < npatches(level); ++q) {
        grf_box pb;
        grf_patch_box(level, q, &pb);
        double n8[8];
        const int r = grf_constraints(&pb, params, patches[q], out4[q], norms_host ? n8 : nullptr, ws, ws_bytes,
                                      stream);
        if (r) return r;
        if (!norms_host) continue;
        const long long n = (long long)pb.nx * pb.ny * pb.nz;
        for (int m = 0; m < 4; ++m) {
            sq[m] += n8[2 * m] * n8[2 * m] * (double)n;  // the patch's sum of squares
            mx[m] = n8[2 * m + 1] > mx[m] ? n8[2 * m + 1] : mx[m];
        }
        total += n;
    }
    if (norms_host)
        for (int m = 0; m < 4; ++m) {
            norms_host[2 * m] = std::sqrt(sq[m] / (double)total);
            norms_host[2 * m + 1] = mx[m];
        }
    return GRF_OK;
}

}  // extern "C"
