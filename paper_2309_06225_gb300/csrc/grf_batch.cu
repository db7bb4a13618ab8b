// Batched RK4 over many boxes (uneven AMR-like boxes, coupling sweeps): a flattened work list
// of (box, tile) items, each box with its own geometry, couplings and time step.
//
// Variants (grf_batch_config.variant):
//   GRF_BATCH_GRAPH       the per-stage launches over the whole work list as one CUDA graph
//                         (a chain of kernel nodes built with the graph API, cached and replayed);
//   GRF_BATCH_PERSISTENT  one cooperative launch of co-resident blocks that loop over the work
//                         list for every stage and step, separated by grid barriers whose spin
//                         is bounded (a barrier that times out latches GRF_ETIMEOUT and every
//                         block returns);
//   GRF_BATCH_STREAM      the per-stage launches without a graph.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "grf.h"
#include "grf_batch.cuh"
#include "grf_launch.h"

namespace grf {

template <int STAGE>
__global__ void __launch_bounds__(128, 3) batch_stage_kernel(const BoxDesc* __restrict__ boxes,
                                                          const TileDesc* __restrict__ tiles, int ntiles, int* status) {
    __shared__ YzRows sh;
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const TileDesc td = tiles[t];
    // the decoupled mode and lopsided advection are compile-time instantiations (as in the single-box
    // kernels, whose bits these must match); the full theory with centred advection stays inlined
    const Coeffs& c = boxes[td.box].c;
    if (c.advection) batch_tile_call<STAGE, -1, 1>(boxes, td, status, sh);
    else if (c.decoupled) batch_tile_call<STAGE, 1, 0>(boxes, td, status, sh);
    else batch_tile<STAGE, 0, 0>(boxes, td, status, sh);
}

__global__ void batch_ghost_fill_kernel(const BoxDesc* __restrict__ boxes, int box) {
    const BoxDesc& d = boxes[box];
    const Geom& g = d.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    if (i >= g.NX || j >= g.NY) return;
    auto wrap = [](int a, int n) { int x = (a - NG) % n; if (x < 0) x += n; return x + NG; };
    const int wi = wrap(i, g.nx), wj = wrap(j, g.ny);
    const bool ghost_ij = (wi != i) || (wj != j);
    double* u = d.un + f * g.fstride;
    for (int k = 0; k < g.NZ; ++k) {
        const int wk = wrap(k, g.nz);
        if (!ghost_ij && wk == k) continue;
        u[gidx(g, i, j, k)] = u[gidx(g, wi, wj, wk)];
    }
}

bool batch_params_ok(const grf_params* p) {
    if (p->beta_kind != GRF_BETA_LINEAR && p->beta_kind != GRF_BETA_QUADRATIC && p->beta_kind != GRF_BETA_EXPONENTIAL)
        return false;
    if (p->beta_kind == GRF_BETA_EXPONENTIAL && !(p->beta_kappa >= 0.0 && p->beta_kappa < 1e300)) return false;
    if (!(1.0 + p->a0 > 0.0) || !(1.0 + p->b0 > 0.0)) return false;
    return p->advection == 0 || p->advection == 1;
}

void batch_box_desc(BoxDesc& d, const grf_box* b, const grf_params* p, double dt) {
    std::memset(&d, 0, sizeof(d));
    Geom& g = d.g;
    g.nx = b->nx; g.ny = b->ny; g.nz = b->nz;
    g.NX = b->nx + 6; g.NY = b->ny + 6; g.NZ = b->nz + 6;
    g.ng = NG;
    g.pitch = b->pitch;
    g.plane = b->pitch * g.NY;
    g.fstride = g.plane * g.NZ;
    g.dx = b->dx;
    g.periodic = (b->bc == GRF_BC_PERIODIC);
    g.reflect = 0;  // mirror boxes are not accepted here
    d.c = make_coeffs(p);
    d.dt = dt;
    d.ko = p->sigma_ko / (64.0 * b->dx);
    d.min_chi = p->min_chi;
    d.min_lapse = p->min_lapse;
    d.enforce = p->enforce_algebraic;
}

// A box whose x-extent is not a multiple of 32 would leave lanes idle through the whole stage;
// its tiles are folded instead, each warp covering 32 / w rows of w = 8 or 16 points, whichever
// fills the most lanes (the folded tiles take the per-thread gather).
int batch_row_width(int nx) {
    if (nx % 32 == 0) return 32;
    int best = 32;
    double best_eff = (double)nx / (32.0 * ((nx + 31) / 32));
    for (int w : {16, 8}) {
        const double eff = (double)nx / ((double)w * ((nx + w - 1) / w));
        if (eff > best_eff + 1e-12) { best = w; best_eff = eff; }
    }
    return best;
}

void launch_batch_stage(int stage, long long ntiles, dim3 block, cudaStream_t st, const BoxDesc* boxes,
                        const TileDesc* tiles, int* status) {
    const dim3 grid((unsigned)ntiles);
    switch (stage) {
        case 0: batch_stage_kernel<0><<<grid, block, 0, st>>>(boxes, tiles, (int)ntiles, status); break;
        case 1: batch_stage_kernel<1><<<grid, block, 0, st>>>(boxes, tiles, (int)ntiles, status); break;
        case 2: batch_stage_kernel<2><<<grid, block, 0, st>>>(boxes, tiles, (int)ntiles, status); break;
        default: batch_stage_kernel<3><<<grid, block, 0, st>>>(boxes, tiles, (int)ntiles, status); break;
    }
}

}  // namespace grf

using namespace grf;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool item_ok(const grf_batch_item& it) {
    const grf_box* b = &it.box;
    if (b->ng != 3 || b->nx < 1 || b->ny < 1 || b->nz < 1 || !(b->dx > 0.0)) return false;
    if (b->pitch < (long long)b->nx + 6) return false;
    if (b->bc != GRF_BC_PERIODIC && b->bc != GRF_BC_FROZEN) return false;
    if (b->bc == GRF_BC_PERIODIC && (b->nx < 3 || b->ny < 3 || b->nz < 3)) return false;
    return it.state != nullptr;
}

bool cfg_ok(const grf_batch_config* c) {
    if (!c) return false;
    if (c->tile_x < 1 || c->tile_y < 1 || c->tile_z < 1) return false;
    const long long n = (long long)c->tile_x * c->tile_y * c->tile_z;
    if (n > 128 || n < 32) return false;
    return c->variant >= GRF_BATCH_GRAPH && c->variant <= GRF_BATCH_STREAM;
}

Geom geom_of(const grf_box* b) {
    static const grf_params kAny{};  // only the geometry is used
    BoxDesc d;
    batch_box_desc(d, b, &kAny, 0.0);
    return d.g;
}

size_t state_bytes_of(const Geom& g) { return sizeof(double) * (size_t)NFIELDS * (size_t)g.fstride; }

// x-points per tile row for a box: folded rows (batch_row_width) with 32 x 4 x 1 tiles, else the
// tile's width.
int row_width(const grf_box* b, const grf_batch_config* c) {
    if (!(c->tile_x == 32 && c->tile_y == 4 && c->tile_z == 1)) return c->tile_x;
    return batch_row_width(b->nx);
}

long long tiles_of(const grf_box* b, const grf_batch_config* c) {
    const int w = row_width(b, c);
    const int rows = c->tile_y * (c->tile_x / w);
    return (long long)((b->nx + w - 1) / w) * ((b->ny + rows - 1) / rows) * ((b->nz + c->tile_z - 1) / c->tile_z);
}

struct Layout {
    size_t ctrl, boxes, tiles, bufs, total;
    long long ntiles;
};

Layout layout(const grf_batch_item* items, int n, const grf_batch_config* c) {
    Layout L;
    L.ntiles = 0;
    size_t bufs = 0;
    for (int i = 0; i < n; ++i) {
        L.ntiles += tiles_of(&items[i].box, c);
        bufs += 3 * align_up(state_bytes_of(geom_of(&items[i].box)));
    }
    L.ctrl = 0;
    L.boxes = kAlign;
    L.tiles = L.boxes + align_up(sizeof(BoxDesc) * (size_t)n);
    L.bufs = L.tiles + align_up(sizeof(TileDesc) * (size_t)L.ntiles);
    L.total = L.bufs + bufs;
    return L;
}

// one cached executable graph (re-used when the same batch is stepped again); the lookup, rebuild
// and launch hold g_graph_mutex, and the key includes the device, so host threads calling
// grf_batched_rk4 concurrently (on any devices) never launch or destroy each other's graph
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int device = -1;
    cudaStream_t stream = nullptr;
    const void* ws = nullptr;
    int nsteps = -1;
    long long ntiles = -1;
    int tx = 0, ty = 0, tz = 0;
    std::vector<char> key;
};
GraphCache g_graph;
std::mutex g_graph_mutex;

int cuda_err(cudaError_t e) { return grf::record_cuda_error(e); }

bool debug_on() {
    static const bool on = std::getenv("GRF_DEBUG_BATCH") != nullptr;
    return on;
}
#define DBG(...)                                              \
    do {                                                      \
        if (debug_on()) {                                     \
            std::fprintf(stderr, "[grf_batched_rk4] " __VA_ARGS__); \
            std::fprintf(stderr, "\n");                       \
            std::fflush(stderr);                              \
        }                                                     \
    } while (0)

// The 4 x nsteps stage launches as an explicitly built graph: a chain of kernel nodes.
cudaError_t build_stage_graph(int nsteps, long long ntiles, dim3 block, const BoxDesc* boxes, const TileDesc* tiles,
                              int* status, cudaGraphExec_t* exec) {
    const void* funcs[4] = {(const void*)batch_stage_kernel<0>, (const void*)batch_stage_kernel<1>,
                            (const void*)batch_stage_kernel<2>, (const void*)batch_stage_kernel<3>};
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    int nt = (int)ntiles;
    void* args[4] = {(void*)&boxes, (void*)&tiles, (void*)&nt, (void*)&status};
    cudaGraphNode_t prev = nullptr;
    for (int n = 0; n < nsteps && e == cudaSuccess; ++n)
        for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
            cudaKernelNodeParams kp;
            std::memset(&kp, 0, sizeof(kp));
            kp.func = (void*)funcs[s];
            kp.gridDim = dim3((unsigned)ntiles);
            kp.blockDim = block;
            kp.sharedMemBytes = 0;
            kp.kernelParams = args;
            kp.extra = nullptr;
            cudaGraphNode_t node = nullptr;
            e = cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
            prev = node;
        }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

void launch_stages(int nsteps, long long ntiles, dim3 block, cudaStream_t st, const BoxDesc* boxes,
                   const TileDesc* tiles, int* status) {
    for (int n = 0; n < nsteps; ++n)
        for (int s = 0; s < 4; ++s) launch_batch_stage(s, ntiles, block, st, boxes, tiles, status);
}

}  // namespace

extern "C" {

size_t grf_batched_workspace_bytes(const grf_batch_item* items, int nitems, const grf_batch_config* cfg) {
    if (!items || nitems < 1 || !cfg_ok(cfg)) return 0;
    for (int i = 0; i < nitems; ++i)
        if (!item_ok(items[i])) return 0;
    return layout(items, nitems, cfg).total;
}

int grf_batched_rk4(const grf_batch_item* items, int nitems, const grf_params* params, int nparams, int nsteps,
                    const grf_batch_config* cfg, void* ws, size_t ws_bytes, int* status_host, grf_stream_t stream) {
    if (!items || nitems < 1 || !params || nparams < 1 || nsteps < 0 || !cfg_ok(cfg)) return GRF_EINVAL;
    for (int i = 0; i < nitems; ++i) {
        if (!item_ok(items[i])) return GRF_EINVAL;
        const int pi = items[i].params_index;
        if (pi < 0 || pi >= nparams) return GRF_EINVAL;
        if (!batch_params_ok(&params[pi])) return GRF_EINVAL;
    }
    const Layout L = layout(items, nitems, cfg);
    DBG("entry: %d boxes, %lld tiles, ws %zu of %zu bytes, variant %d, tile %dx%dx%d", nitems, L.ntiles, ws_bytes,
        L.total, cfg->variant, cfg->tile_x, cfg->tile_y, cfg->tile_z);
    if (L.ntiles > 0x7fffffffLL) return GRF_EINVAL;
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & (kAlign - 1))) return GRF_EWORKSPACE;
    if (nsteps == 0) return GRF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    unsigned* bar = (unsigned*)(base + L.ctrl);
    int* status = (int*)(base + L.ctrl + 64);
    BoxDesc* dboxes = (BoxDesc*)(base + L.boxes);
    TileDesc* dtiles = (TileDesc*)(base + L.tiles);

    // descriptors (host side), then one upload
    std::vector<BoxDesc> hb(nitems);
    std::vector<TileDesc> ht;
    ht.reserve((size_t)L.ntiles);
    size_t off = L.bufs;
    for (int b = 0; b < nitems; ++b) {
        const grf_batch_item& it = items[b];
        const grf_params* p = &params[it.params_index];
        BoxDesc& d = hb[b];
        batch_box_desc(d, &it.box, p, it.dt);
        const size_t sb = align_up(state_bytes_of(d.g));
        d.un = it.state;
        d.A = (double*)(base + off);
        d.B = (double*)(base + off + sb);
        d.acc = (double*)(base + off + 2 * sb);
        off += 3 * sb;
        const int w = row_width(&it.box, cfg);
        const int rows = cfg->tile_y * (cfg->tile_x / w);
        for (int k = 0; k < it.box.nz; k += cfg->tile_z)
            for (int j = 0; j < it.box.ny; j += rows)
                for (int i = 0; i < it.box.nx; i += w) ht.push_back(TileDesc{b, i, j, k, w});
    }
    cudaError_t e = cudaMemcpyAsync(dboxes, hb.data(), sizeof(BoxDesc) * nitems, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtiles, ht.data(), sizeof(TileDesc) * ht.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, kAlign, st);
    if (e != cudaSuccess) return cuda_err(e);
    // ghosts: periodic boxes refill theirs; frozen boxes hand theirs to the stage buffers
    for (int b = 0; b < nitems; ++b) {
        const Geom& g = hb[b].g;
        if (g.periodic) {
            dim3 blk(32, 8, 1), grd((g.NX + 31) / 32, (g.NY + 7) / 8, NFIELDS);
            batch_ghost_fill_kernel<<<grd, blk, 0, st>>>(dboxes, b);
        } else {
            const size_t sb = state_bytes_of(g);
            e = cudaMemcpyAsync(hb[b].A, hb[b].un, sb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hb[b].B, hb[b].un, sb, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_err(e);
        }
    }
    e = cudaGetLastError();
    DBG("descriptors uploaded, ghosts prepared (%s)", cudaGetErrorName(e));
    if (e != cudaSuccess) return cuda_err(e);
    // load the stage kernels before any graph work
    for (const void* f : {(const void*)batch_stage_kernel<0>, (const void*)batch_stage_kernel<1>,
                          (const void*)batch_stage_kernel<2>, (const void*)batch_stage_kernel<3>}) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return cuda_err(e);
    }
    e = batch_persistent_attributes();
    if (e != cudaSuccess) return cuda_err(e);
    DBG("kernels loaded");

    const dim3 block(cfg->tile_x, cfg->tile_y, cfg->tile_z);
    int variant = cfg->variant;

    if (variant == GRF_BATCH_STREAM) {
        launch_stages(nsteps, L.ntiles, block, st, dboxes, dtiles, status);
        e = cudaGetLastError();
        DBG("stream: launched (%s)", cudaGetErrorName(e));
    } else if (variant == GRF_BATCH_GRAPH) {
        // key: everything the graph's launches depend on
        std::vector<char> key(sizeof(BoxDesc) * nitems);
        std::memcpy(key.data(), hb.data(), key.size());
        int device = -1;
        e = cudaGetDevice(&device);
        if (e != cudaSuccess) return cuda_err(e);
        std::lock_guard<std::mutex> lock(g_graph_mutex);
        const bool hit = g_graph.exec && g_graph.device == device && g_graph.stream == st && g_graph.ws == ws &&
                         g_graph.nsteps == nsteps &&
                         g_graph.ntiles == L.ntiles && g_graph.tx == cfg->tile_x && g_graph.ty == cfg->tile_y &&
                         g_graph.tz == cfg->tile_z && g_graph.key == key;
        DBG("graph: cache %s", hit ? "hit" : "miss");
        if (!hit) {
            if (g_graph.exec) {  // an executable graph still in flight is freed when it completes
                cudaGraphExecDestroy(g_graph.exec);
                g_graph.exec = nullptr;
            }
            e = build_stage_graph(nsteps, L.ntiles, block, dboxes, dtiles, status, &g_graph.exec);
            DBG("graph: built (%s)", cudaGetErrorName(e));
            if (e != cudaSuccess) { g_graph.exec = nullptr; return cuda_err(e); }
            g_graph.device = device; g_graph.stream = st; g_graph.ws = ws; g_graph.nsteps = nsteps; g_graph.ntiles = L.ntiles;
            g_graph.tx = cfg->tile_x; g_graph.ty = cfg->tile_y; g_graph.tz = cfg->tile_z; g_graph.key = key;
        }
        e = cudaGraphLaunch(g_graph.exec, st);
        DBG("graph: launched (%s)", cudaGetErrorName(e));
    } else {  // persistent cooperative launch
        int dev = 0, nsm = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int nthreads = cfg->tile_x * cfg->tile_y * cfg->tile_z;
        if (e == cudaSuccess) e = batch_persistent_occupancy(nthreads, &per_sm);
        if (e != cudaSuccess) return cuda_err(e);
        if (per_sm < 1) return GRF_EINVAL;
        if (cfg->blocks_per_sm > 0 && cfg->blocks_per_sm < per_sm) per_sm = cfg->blocks_per_sm;
        long long nb = (long long)per_sm * nsm;
        if (nb > L.ntiles) nb = L.ntiles;
        const long long timeout = cfg->barrier_timeout_cycles > 0 ? cfg->barrier_timeout_cycles : 20000000000LL;
        DBG("persistent: %lld blocks (%d per SM x %d SMs)", nb, per_sm, nsm);
        e = launch_batch_persistent(dim3((unsigned)nb), block, dboxes, dtiles, (int)L.ntiles, nsteps, bar, status,
                                    timeout, st);
        DBG("persistent: launched (%s)", cudaGetErrorName(e));
    }
    if (e != cudaSuccess) return cuda_err(e);
    if (status_host) {
        DBG("waiting for status");
        e = cudaMemcpyAsync(status_host, status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_err(e);
        if (*status_host & 2) return GRF_ETIMEOUT;
        if (*status_host & 1) return GRF_ESINGULAR;
    }
    return GRF_OK;
}

}  // extern "C"
