/*
 * grf.h -- C ABI of the GB300 library (libgrf.so) for the modified-CCZ4 + 4-derivative
 * scalar-tensor (4dST) evolution hot path of GRFolres (arXiv:2309.06225).
 *
 * What is computed (paper, section "Key features"): the fields of the 4dST theory
 * (R + X + g2 X^2 + beta(phi) L_GB, X = -1/2 (d phi)^2) evolved in the modified moving
 * puncture gauge with the CCZ4 formulation, 4th-order centred finite differences and
 * 4th-order Runge-Kutta time integration, on a ghosted 3D box with periodic (or frozen)
 * ghosts, plus Kreiss-Oliger dissipation and constraint monitoring ("Diagnostics").
 * The Gauss-Bonnet and X^2 couplings make d_t K_ij and d_t Pi appear on both sides of
 * the equations ("still second order equations of motion", section "Summary"): they are
 * found by a 7x7 linear solve at every grid point.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * State layout: 27 FP64 fields, structure of arrays, field-major:
 *     state[f * fstride + (k * (ny + 2 ng) + j) * pitch + i]
 * with ghosted indices 0 <= i < nx + 2 ng (x fastest), fstride = (nz + 2 ng) * (ny + 2 ng) * pitch.
 * Field order: 0 chi | 1-6 h11 h12 h13 h22 h23 h33 | 7 K | 8-13 A11..A33 | 14 Theta |
 *              15-17 Gamma^i | 18 lapse | 19-21 shift^i | 22-24 B^i | 25 phi | 26 Pi.
 * Ownership: every double* argument is a DEVICE pointer owned by the caller, except where
 * marked "host". The library never allocates or frees memory; scratch space is passed in
 * as `ws` (device, 256-byte aligned, at least grf_workspace_bytes(box, op) bytes).
 * Streams: every call is asynchronous on `stream` (0 = legacy default stream) unless it
 * says it synchronises.
 * Errors: 0 on success, a negative GRF_E* code otherwise; grf_error_string() describes it.
 * A launch failure is returned as GRF_ECUDA and its CUDA message is kept for
 * grf_last_cuda_error(). Per-point failures detected inside kernels (a singular coupled
 * system) are latched in a device flag and reported by grf_check_status().
 */
#ifndef GRF_H
#define GRF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* grf_stream_t; /* same type as cudaStream_t */

enum {
    GRF_OK = 0,
    GRF_EINVAL = -1,       /* bad sizes, null pointers, ng not 3 or 4, pitch too small */
    GRF_EWORKSPACE = -2,   /* ws too small or misaligned */
    GRF_ECUDA = -3,        /* a CUDA call failed; see grf_last_cuda_error() */
    GRF_ENONFINITE = -4,   /* non-finite value found by grf_check_finite() */
    GRF_ESINGULAR = -5,    /* some point's coupled 7x7 system had a vanishing pivot */
    GRF_ETIMEOUT = -6,     /* a bounded device-side wait gave up */
    GRF_ETOOLARGE = -7     /* box too large for the fixed scratch of grf_rk4_step_noalloc */
};

enum {
    GRF_BC_PERIODIC = 0,
    GRF_BC_FROZEN = 1,
    GRF_BC_REFLECT_LOW = 2,
    GRF_BC_EXTRAPOLATE = 3,
    GRF_BC_SOMMERFELD = 4,
    GRF_BC_REFLECT_LOW_SOMMERFELD = 5
};
enum { GRF_BETA_LINEAR = 0, GRF_BETA_QUADRATIC = 1, GRF_BETA_EXPONENTIAL = 2 };
enum { GRF_OP_RHS = 0, GRF_OP_RK4 = 1, GRF_OP_CONSTRAINTS = 2 };

/* Grid box. Points sit at x = x0 + (i - ng) dx (ghosted index i). The ghost width chooses the
 * finite-difference scheme ("Accuracy": 4th- and 6th-order stencils):
 *   ng = 3: centred 4th-order first / second / mixed differences, Kreiss-Oliger dissipation
 *           sigma/(64 dx) sum_d Delta^6_d, lopsided advection on offsets -1..3;
 *   ng = 4: centred 6th-order differences, dissipation -sigma/(256 dx) sum_d Delta^8_d,
 *           lopsided advection on offsets -2..4.
 * 4-ghost boxes are accepted by every call but grf_batched_rk4, grf_tlm_rk4 and the split-box
 * calls (grf_patch_level). */
typedef struct {
    int nx, ny, nz;       /* interior points per axis, each >= 1 (periodic, mirror: >= ng) */
    int ng;               /* ghost layers: 3 or 4 (above) */
    double dx;            /* grid spacing, > 0 */
    double x0, y0, z0;    /* coordinates of interior point (0,0,0) */
    int bc;               /* GRF_BC_PERIODIC: ghosts refilled by periodic wrap;
                             GRF_BC_FROZEN: ghosts are read as given and never written;
                             GRF_BC_REFLECT_LOW: the three low faces are mirror planes (half a
                             cell below the first point; "Boundary Conditions", reflective),
                             their ghosts rebuilt from the interior with each component's
                             parity; ghosts on the high faces are read as given. Needs n >= ng.
                             Not accepted by grf_batched_rk4, grf_tlm_rk4 and the split-box calls.
                           GRF_BC_EXTRAPOLATE ("Boundary Conditions", extrapolating): every ghost
                             is refilled before each right-hand side by linear extrapolation along
                             one axis, u(last + m) = u(last) + m (u(last) - u(last - 1)), axis by
                             axis (x-ghosts on rows of interior y, z; then y-ghosts on rows of any x
                             and interior z; then z-ghosts on rows of any x, y).
                           GRF_BC_SOMMERFELD ("Boundary Conditions", Sommerfeld / radiative): the
                             ghosts are evolved state. Each ghost point takes the RK4 stages of
                             d_t u = -(u - u_inf)/r - (x^i/r) d_i u, r = |x| (radiation centre at
                             the coordinate origin, speed 1), u_inf = 1 for chi, h_11, h_22, h_33
                             and the lapse and 0 for the rest; d_i is the 2nd-order one-sided
                             difference into the box along axes on which the point lies beyond
                             the interior, centred 2nd-order along the others. Meant for boxes
                             that contain the origin (outer faces, where the one-sided differences
                             are upwind). Needs n >= ng.
                           GRF_BC_REFLECT_LOW_SOMMERFELD: mirror planes at the three low faces and
                             Sommerfeld at the high faces, for the octant of a problem with the
                             three reflection symmetries about the origin. Every ghost beyond a
                             high face with no coordinate below the box is evolved by the radiative
                             condition (centred differences along the axes where it is inside, the
                             mirror images supplying the points below the box); every ghost with
                             a coordinate below the box is a mirror image, refilled after each
                             stage. Needs n >= ng.
                           Extrapolating and Sommerfeld boxes (also behind mirror planes) are not
                             accepted by grf_batched_rk4, grf_tlm_rk4 and the split-box calls. */
    long long pitch;      /* doubles per x row, >= nx + 2 ng */
} grf_box;

/* Theory, gauge and numerical parameters (modified puncture gauge with constant a, b;
 * beta(phi) = lambda phi, lambda phi^2 / 2, or lambda / (2 kappa) (1 - exp(-kappa phi^2)), the
 * exponential coupling of spin-induced scalarisation ("Statement of Need"); the X^2 coupling is
 * the constant g2; the cubic Horndeski coupling g3). The action is
 *   (1/16 pi) int sqrt(-g) [R + X + g2 X^2 + g3 X box(phi) + beta(phi) L_GB],  X = -1/2 (d phi)^2. */
typedef struct {
    double kappa1, kappa2, kappa3;   /* CCZ4 constraint damping */
    double shift_F, eta;             /* Gamma-driver: d_t shift = F B / (1 + a) - ..., d_t B = d_t Gamma - eta B */
    double a0, b0;                   /* modified-gauge functions a(x) = a0, b(x) = b0 (0, 0: standard gauge) */
    double lambda, g2;               /* Gauss-Bonnet coupling constant, X^2 coupling */
    double sigma_ko;                 /* Kreiss-Oliger strength sigma */
    double min_chi, min_lapse;       /* floors applied after every RK stage */
    int beta_kind;                   /* GRF_BETA_LINEAR, GRF_BETA_QUADRATIC or GRF_BETA_EXPONENTIAL */
    int enforce_algebraic;           /* 1: trace-free A_ij and the floors after every stage */
    int decoupled;                   /* 0: full 4dST; 1: without backreaction onto the metric
                                        ("Key features"): the metric evolves by vacuum CCZ4 in the
                                        same gauge, the scalar by its full equation on that metric */
    int advection;                   /* 0: centred differences in the advection terms beta^k d_k u;
                                        1: lopsided differences, one point further towards the side
                                        beta^k points to (every beta^k d_k of an evolved field, those
                                        inside the coupled 4dST system included). 1 is not accepted by
                                        grf_tlm_rk4 */
    double beta_kappa;               /* kappa >= 0 of GRF_BETA_EXPONENTIAL (ignored by the other kinds) */
    double g3;                       /* cubic Horndeski coupling ("Key features": the cubic Horndeski
                                        theory): the action gains g3 X box(phi), G3(phi, X) = g3 X;
                                        0 gives 4dST alone */
} grf_params;

/* d_t of all 27 fields at the interior points of `state` (modified CCZ4 + 4dST, section
 * "Key features"), including Kreiss-Oliger dissipation (the box's scheme, see grf_box).
 * The ghost layers of `state` are first refilled as the box's boundary type says (periodic
 * wrap, mirror images, extrapolation; the interior is not modified); frozen and Sommerfeld
 * ghosts are read as given. rhs: same layout as state; interior entries are written, and for
 * GRF_BC_SOMMERFELD also every ghost entry (the radiative right-hand side). ws may be NULL. */
int grf_rhs(const grf_box* box, const grf_params* params, double* state, double* rhs,
            void* ws, size_t ws_bytes, grf_stream_t stream);

/* Advance `state` in place by nsteps classical RK4 steps of size dt (section "Key
 * features": 4th-order Runge-Kutta). k_s = RHS(u_{s-1}) with dissipation; u_1 = u_n +
 * dt/2 k_1, u_2 = u_n + dt/2 k_2, u_3 = u_n + dt k_3, u_{n+1} = u_n + dt/6 (k_1 + 2k_2 +
 * 2k_3 + k_4); every written state gets the algebraic enforcement when enabled.
 * ws: >= grf_workspace_bytes(box, GRF_OP_RK4) bytes (two stage states + an accumulator). */
int grf_rk4_step(const grf_box* box, const grf_params* params, double* state, double dt,
                 int nsteps, void* ws, size_t ws_bytes, grf_stream_t stream);

/* grf_rk4_step from host memory to host memory, with the host<->device copies overlapped with
 * the first and the last RK stage (the time stepping of section "Key features"; the overlap
 * has no counterpart in the paper, whose states never leave the node's memory).
 *   host_in:  host, the state in the layout above (27 * pitch * (ny+6) * (nz+6) doubles).
 *             GRF_BC_PERIODIC: only interior values are read (ghosts are rebuilt by periodic
 *             wrap, as grf_rk4_step does); GRF_BC_FROZEN: ghosts are read as given.
 *   host_out: host, same size; receives the state after nsteps steps, ghosts included.
 *             May equal host_in.
 *   state:    device buffer of the same size; overwritten, and on completion it holds the
 *             same result as host_out.
 *   ws:       as for grf_rk4_step.
 * The state is copied in slabs of z-planes (at most 16) on a high-priority copy stream owned by
 * the library; each slab's first-stage launch waits only for the planes its stencils read. The
 * last stage runs slab by slab and each finished slab is copied to host_out while the next is
 * computed. Page-locked buffers are copied by a small kernel (48 blocks) that reads or writes
 * host memory directly, which keeps the full host-link rate while the stages run; pageable
 * buffers are copied with cudaMemcpyAsync. Results are bit-identical to: copy host_in to state,
 * grf_rk4_step, copy state to host_out. The stage kernels run on `stream`; the copies are
 * ordered after the work already queued on `stream`, and later work on `stream` is ordered
 * after the last copy, so host_out is
 * complete once `stream` is synchronised. Host buffers should be page-locked (cudaHostAlloc,
 * cudaHostRegister, pinned torch tensors); pageable buffers give the same results, but their
 * copies are staged by the driver and overlap the kernels poorly.
 * The first call on a device creates that device's copy stream and events (no memory is
 * allocated); make it before any stream capture. Calls from several host threads are
 * serialised while they queue work. The slab pipeline serves boxes with 3 ghost layers whose
 * ghosts are periodic or mirror images or frozen; other boxes (4 ghost layers, extrapolated or
 * Sommerfeld ghosts) copy the whole state in by the same copy path, run grf_rk4_step and copy it
 * out, without the overlap. Errors: GRF_EINVAL (box, params, null pointers, nsteps < 0),
 * GRF_EWORKSPACE, GRF_ECUDA. */
int grf_rk4_step_host(const grf_box* box, const grf_params* params, const double* host_in,
                      double* host_out, double* state, double dt, int nsteps, void* ws,
                      size_t ws_bytes, grf_stream_t stream);

/* Hamiltonian and momentum constraints (section "Key features", Diagnostics):
 *   H = R + K^2 - K_ij K^ij - 16 pi rho,  M_i = D_j K^j_i - D_i K - 8 pi S_i,
 * with the full 4dST rho and S_i. out4: device, 4 fields in the state layout (H, M1, M2,
 * M3; interior entries written). norms_host (host, may be NULL): 8 doubles
 * {L2(H), max|H|, L2(M1), max|M1|, L2(M2), max|M2|, L2(M3), max|M3|} over the interior,
 * L2 = sqrt(mean of squares). Synchronises `stream` when norms_host is given.
 * ws: >= grf_workspace_bytes(box, GRF_OP_CONSTRAINTS) bytes when norms_host is given. */
int grf_constraints(const grf_box* box, const grf_params* params, double* state, double* out4,
                    double* norms_host, void* ws, size_t ws_bytes, grf_stream_t stream);

/* Energy densities of the three scalar terms of the action ("Diagnostics": the energy densities
 * associated with the different scalar terms), in the 8 pi rho units of the equations:
 *   out3[0] = X term        = (Pi^2 + |D phi|^2) / 4
 *   out3[1] = g2 X^2 term   = g2 (X Pi^2 - X^2 / 2),  X = (Pi^2 - |D phi|^2) / 2
 *   out3[2] = beta(phi) L_GB term = -4 G_S^ij Phi_ij  (Phi = nabla nabla beta, G_S the Einstein
 *             tensor of the Gauss block)
 * Their sum is the 8 pi rho that enters the equations (with backreaction). out3: device, 3 fields
 * in the state layout, interior entries written. Ghosts of `state` are refilled as for grf_rhs. */
int grf_energy_densities(const grf_box* box, const grf_params* params, double* state, double* out3,
                         grf_stream_t stream);

/* rhs_accum += sigma/(64 dx) sum_{d=x,y,z} (u_-3 - 6u_-2 + 15u_-1 - 20u_0 + 15u_+1 - 6u_+2 + u_+3)
 * for all 27 fields at the interior points (Kreiss-Oliger dissipation). Ghosts of
 * `state` must be valid (call grf_fill_ghosts first for periodic boxes). */
int grf_ko_dissipation(const grf_box* box, double sigma, const double* state, double* rhs_accum,
                       grf_stream_t stream);

/* Periodic wrap of the 3 ghost layers of all 27 fields (no-op for GRF_BC_FROZEN). */
int grf_fill_ghosts(const grf_box* box, double* state, grf_stream_t stream);

/* Scratch bytes needed by an operation (GRF_OP_*) on this machine. */
size_t grf_workspace_bytes(const grf_box* box, int op);

/* Returns (and clears) the per-point status latched by kernels since the last call:
 * GRF_OK or GRF_ESINGULAR. Synchronises `stream`. */
int grf_check_status(grf_stream_t stream);

/* GRF_ENONFINITE if any interior value of the 27 fields is NaN/Inf, else GRF_OK.
 * ws: >= 256 bytes. Synchronises `stream`. */
int grf_check_finite(const grf_box* box, const double* state, void* ws, size_t ws_bytes,
                     grf_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Batched evolution of many independent boxes (uneven AMR-like box sets, coupling sweeps).
 * The paper evolves boxes of a block-structured AMR hierarchy ("Adaptive Mesh Refinement",
 * section "Key features"); this call advances a set of independent boxes, each with its own
 * geometry, boundary type, couplings and time step, by nsteps RK4 steps, with all boxes'
 * points in one flattened work list of (box, tile) items.
 * ------------------------------------------------------------------------------------- */
enum { GRF_BATCH_GRAPH = 1, GRF_BATCH_PERSISTENT = 2, GRF_BATCH_STREAM = 3 };

typedef struct {
    grf_box box;          /* this box's geometry and boundary type */
    double* state;        /* device: this box's state (layout above), advanced in place */
    int params_index;     /* index of this box's entry in the params array */
    double dt;            /* this box's time step */
} grf_batch_item;

typedef struct {
    int variant;          /* GRF_BATCH_GRAPH: the 4 x nsteps stage launches as one CUDA graph (kernel-node
                             chain, cached and replayed when the same batch is stepped again);
                             GRF_BATCH_PERSISTENT: one cooperative launch of co-resident blocks looping
                             over the work list, grid barriers between stages;
                             GRF_BATCH_STREAM: the stage launches issued directly */
    int tile_x, tile_y, tile_z;        /* threads per block / points per tile; product in [32, 128] */
    int blocks_per_sm;                 /* persistent: resident blocks per SM (0: as many as fit) */
    long long barrier_timeout_cycles;  /* persistent: spin limit of one grid barrier (0: 2e10 cycles);
                                          on expiry the call reports GRF_ETIMEOUT, no block hangs */
} grf_batch_config;

/* Scratch bytes for grf_batched_rk4: descriptors, tile list and three state-sized buffers per
 * box. 0 if an item or the configuration is invalid. */
size_t grf_batched_workspace_bytes(const grf_batch_item* items, int nitems, const grf_batch_config* cfg);

/* Advance every box by nsteps RK4 steps (same scheme as grf_rk4_step, per box). items, params
 * and cfg are host arrays read during the call. status_host (host, may be NULL): when given,
 * the call synchronises `stream` and returns GRF_ETIMEOUT / GRF_ESINGULAR if a barrier timed
 * out or a coupled system was singular. */
int grf_batched_rk4(const grf_batch_item* items, int nitems, const grf_params* params, int nparams, int nsteps,
                    const grf_batch_config* cfg, void* ws, size_t ws_bytes, int* status_host, grf_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * One box split into patches (domain decomposition). GRFolres distributes the boxes of
 * a level over processes and fills each box's ghost cells from its neighbours before every
 * right-hand side ("Key features": parallelism, AMR). Here the box's interior is
 * cut into px x py x pz patches, each a state of its own (frozen-ghost layout, below); every RK4
 * stage advances all patches' points in one launch, and a halo exchange then refills every
 * patch's ghosts from the interiors of the patches that own those points (in a box with frozen
 * ghosts, the patches' ghost points outside the box keep the values they were given). The exchange is a
 * separate step behind a function pointer, so a caller can put its own in its place (one that
 * moves halos between devices or processes, say); the built-in one is grf_halo_exchange.
 * With the built-in exchange the patches' interiors after grf_patches_rk4 equal, bit for bit,
 * those of grf_rk4_step on the whole box.
 *
 * Patch (a, b, c), index a + px (b + py c), covers the interior points
 * [floor(a nx / px), floor((a + 1) nx / px)) along x, and likewise along y and z.
 * ------------------------------------------------------------------------------------- */
#define GRF_MAX_PATCHES_PER_AXIS 16
#define GRF_MAX_PATCHES 256

typedef struct {
    grf_box box;          /* the whole box: ng = 3; GRF_BC_PERIODIC (nx, ny, nz >= 3) or GRF_BC_FROZEN */
    int px, py, pz;       /* patches per axis: 1 .. GRF_MAX_PATCHES_PER_AXIS and at most the axis'
                             points; px py pz <= GRF_MAX_PATCHES */
} grf_patch_level;

/* Host only. The geometry of patch `index`: its interior extent, ng = 3, dx of the box, the
 * centre of its first interior point (box origin + offset dx), bc GRF_BC_FROZEN (its ghosts are
 * written by the exchange) and pitch = interior x-extent + 6 rounded up to a multiple of 4.
 * Every patch state passed to the calls below has this layout. GRF_EINVAL on a bad level,
 * index or null pointer. */
int grf_patch_box(const grf_patch_level* level, int index, grf_box* out);

/* Copies between a whole-box state (the layout of level->box) and the patches. direction 0:
 * every point of every patch, ghosts included, from the same point of the box (an exchange then
 * rewrites the ghosts that lie inside the box, or all of them in a periodic box, so only a frozen
 * box's ghosts need be set); 1: the box's interior from the patches' interiors (its ghosts are
 * left unchanged). patches is a
 * host array of px py pz device pointers. Asynchronous on `stream`. */
int grf_patch_copy(const grf_patch_level* level, double* box_state, double* const* patches, int direction,
                   grf_stream_t stream);

/* The built-in halo exchange: every ghost point of every patch (all 27 fields) that lies in the
 * box (periodic: all of them, wrapped) takes the value of the same point of the box, read from
 * the interior of the patch that owns it; the others are left unchanged.
 * patches: host array of px py pz device pointers (read during the call). Asynchronous on
 * `stream`. */
int grf_halo_exchange(const grf_patch_level* level, double* const* patches, grf_stream_t stream);

/* The exchange as data, for exchanges between devices or processes: every ghost point that
 * grf_halo_exchange writes belongs to exactly one block of this plan, which copies it (all 27
 * fields) from the interior of the owning patch. A block is a rectangular range of ghosted
 * indices of patch `dst`, starting at (dst_i, dst_j, dst_k), that equals the range of patch `src`
 * starting at (src_i, src_j, src_k), both of extent (ni, nj, nk) (periodic boxes: the wrapped
 * points). The patch's own interior is not part of the plan. */
typedef struct {
    int dst, src;             /* patch indices a + px (b + py c) */
    int dst_i, dst_j, dst_k;  /* first point of the block in patch dst (ghosted indices) */
    int src_i, src_j, src_k;  /* first point in patch src (ghosted indices, inside its interior) */
    int ni, nj, nk;           /* extent */
} grf_halo_block;

/* Host only. Writes the first min(count, max_blocks) blocks of the level's plan to `blocks`
 * (NULL with max_blocks = 0 to query) and returns the plan's block count, or GRF_EINVAL for a bad
 * level or arguments. Blocks are ordered by destination patch. */
int grf_halo_plan(const grf_patch_level* level, grf_halo_block* blocks, int max_blocks);

/* A halo exchange that grf_patches_rk4 calls on the patches' current buffers (a host array of
 * px py pz device pointers in grf_patch_box layouts, valid for the call only): before the first
 * step on the patch states, then after every stage on the buffers that stage wrote. It must fill
 * every ghost point as grf_halo_exchange does, in order on `stream` (or synchronised with it), and
 * return GRF_OK; another return value ends grf_patches_rk4 with that value. */
typedef int (*grf_halo_fn)(void* ctx, const grf_patch_level* level, double* const* patches, grf_stream_t stream);

/* Scratch bytes for grf_patches_rk4: descriptors, tile list and three state-sized buffers per
 * patch. 0 for a bad level. */
size_t grf_patches_workspace_bytes(const grf_patch_level* level);

/* Advance the whole box, held as its patches (host array of px py pz device pointers, interiors
 * valid, and in a frozen box the ghosts outside it; advanced in place), by nsteps RK4 steps of size dt with the scheme of grf_rk4_step
 * (4th order, ng = 3; centred or lopsided advection, every coupling kind). exchange: NULL for
 * grf_halo_exchange, else the caller's, called with exchange_ctx. status_host (host, may be NULL):
 * when given, the call synchronises `stream` and returns GRF_ESINGULAR if a coupled system was
 * singular. Errors: GRF_EINVAL (bad level, params, pointers or nsteps < 0), GRF_EWORKSPACE
 * (ws null, smaller than grf_patches_workspace_bytes or not 256-byte aligned), GRF_ECUDA. */
int grf_patches_rk4(const grf_patch_level* level, const grf_params* params, double* const* patches, double dt,
                    int nsteps, grf_halo_fn exchange, void* exchange_ctx, void* ws, size_t ws_bytes, int* status_host,
                    grf_stream_t stream);

/* Scratch bytes for grf_patches_constraints (the largest patch's grf_constraints scratch); 0 for a
 * bad level. */
size_t grf_patches_constraints_workspace_bytes(const grf_patch_level* level);

/* The constraints of the whole box from its patches (the patches' ghosts as the last exchange left
 * them): grf_constraints on every patch, writing its H, M1, M2, M3 into out4[q] (host array of
 * px py pz device pointers, 4 fields each in the patch's layout), and, when norms_host is given,
 * the 8 norms of grf_constraints over the whole box's interior, combined on the host from the
 * patches' sums of squares and maxima (the one reduction of a few scalars that a run over several
 * devices would all-reduce). The per-point values equal grf_constraints on the whole box bit for
 * bit; the L2 norms differ from it by the order of summation only. Synchronises `stream` when
 * norms_host is given. Errors as grf_constraints, GRF_EINVAL for a bad level or pointer array. */
int grf_patches_constraints(const grf_patch_level* level, const grf_params* params, double* const* patches,
                            double* const* out4, double* norms_host, void* ws, size_t ws_bytes, grf_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Differentiation of an extracted scalar signal (the paper extracts scalar waveforms on
 * spheres, section "Key features": Diagnostics). The signal is
 *   L = sum_{n=1..nsteps} dt * sum_{q=1..26} w_q phi(c + R x_q, t_n)
 * (26-point degree-7 rule on the sphere of radius R about c, trilinear interpolation of phi on
 * the interior points, evaluated after every RK4 step). grf_tlm_rk4 advances the state exactly
 * like grf_rk4_step and, at the same time, three tangent states (forward-mode derivatives):
 * every operation of the step is differentiated, so after the call loss[1 + k] is the exact
 * derivative of loss[0] in direction k.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    double radius;        /* R > 0; the sphere must stay inside the interior points */
    double cx, cy, cz;    /* centre c */
} grf_sphere;

/* Scratch bytes for grf_tlm_rk4: 12 state-sized buffers (stage states and accumulators of the
 * value and the 3 tangents) plus 256 bytes. */
size_t grf_tlm_workspace_bytes(const grf_box* box);

/* state: device, advanced in place (as grf_rk4_step). tangents: device, 3 consecutive states in
 * the same layout holding d state / d theta_k (the caller seeds them, e.g. d(initial state)/d
 * amplitude), advanced in place. dparams: host, 6 doubles {d lambda/d theta_k, d g2/d theta_k}
 * for k = 0, 1, 2 (g3, when non-zero, is held fixed). loss: device, 4 doubles {L, dL/dtheta_0..2},
 * ACCUMULATED (zero it first).
 * Synchronises `stream`; GRF_EINVAL if the sphere leaves the interior, GRF_ESINGULAR if a
 * coupled system was singular. */
int grf_tlm_rk4(const grf_box* box, const grf_params* params, const double* dparams, double* state, double* tangents,
                double dt, int nsteps, const grf_sphere* sphere, double* loss, void* ws, size_t ws_bytes,
                grf_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Reverse mode (discrete adjoint) of the same evolution and signal, with RK4-step
 * checkpointing ("Key features": scalar waveform diagnostics -- the signal whose gradient is
 * taken). grf_signal_forward evolves the state and stores a checkpoint every
 * `checkpoint_every` steps; grf_adjoint_rk4 then runs backwards from them: each segment's step
 * states are recomputed from its checkpoint, each step's stage states from its step state,
 * and every stage is reversed by a reverse-mode re-evaluation of the pointwise map (right-hand
 * side, Kreiss-Oliger term, stage update and enforcement) followed by the transposed stencils.
 * The result is the exact gradient (to rounding) of
 *     J = loss_bar * L + <state_bar_in, state_N>   (interior points, all 27 fields)
 * with respect to the initial state's interior values and to (lambda, g2).
 * Accepted boxes: 3 ghost layers, periodic or frozen ghosts; params: centred advection, any
 * coupling kind, with or without backreaction, with or without the cubic term (g3 is held fixed:
 * no derivative is taken with respect to it). Calls on one device must not overlap in time:
 * the tape's device pointers are held in one constant of the library, set by each call.
 * ------------------------------------------------------------------------------------- */

/* Scratch bytes of grf_signal_forward and grf_adjoint_rk4 (0 for an unsupported box):
 * 9 + checkpoint_every state-sized buffers, 171 derivative-adjoint fields, and the reverse-mode
 * tapes of one wave of points: min(interior points, 155,648) tape columns of about 166 KB each
 * (25.8 GB at full width; 34.1 GB in all for the 96^3 box with a checkpoint every 20 steps). */
size_t grf_adjoint_workspace_bytes(const grf_box* box, int checkpoint_every);

/* Evolves `state` (device, in place, ghosts filled first) by nsteps RK4 steps exactly as
 * grf_rk4_step does, writes the state before steps 0, c, 2c, ... (c = checkpoint_every) to
 * `checkpoints` (device, ceil(nsteps / c) consecutive states of the box's layout) and sets
 * `loss` (device, 1 double) to L. Synchronises `stream`. Errors: GRF_EINVAL (box, params,
 * pointers, nsteps < 0, c < 1, or a sphere sample outside the interior), GRF_EWORKSPACE,
 * GRF_ESINGULAR, GRF_ECUDA. */
int grf_signal_forward(const grf_box* box, const grf_params* params, double* state, double dt, int nsteps,
                       const grf_sphere* sphere, int checkpoint_every, double* checkpoints, double* loss, void* ws,
                       size_t ws_bytes, grf_stream_t stream);

/* Reverse sweep over the checkpoints of grf_signal_forward (same box, params, dt, nsteps,
 * sphere and checkpoint_every). state_bar: device state, IN the cotangent of the final state's
 * interior (zeros for L alone), OUT the gradient of J with respect to the initial state's
 * interior values (ghost entries unused). param_bar: device, 2 doubles, OUT dJ/d lambda and
 * dJ/d g2. loss_bar: host scalar, the cotangent of L. Deterministic (fixed summation orders).
 * Synchronises `stream`. Errors as grf_signal_forward; GRF_EWORKSPACE also if a point's tape
 * overflowed. */
int grf_adjoint_rk4(const grf_box* box, const grf_params* params, const double* checkpoints, double dt, int nsteps,
                    const grf_sphere* sphere, int checkpoint_every, double loss_bar, double* state_bar,
                    double* param_bar, void* ws, size_t ws_bytes, grf_stream_t stream);

/* out (device, 1 double) = sum over interior points of x * y for field `field` (0..26), or over
 * all 27 fields (field = -1), in a fixed order (deterministic). ws: device, 256-byte aligned,
 * at least 304 doubles. Asynchronous. Used for gradients with respect to parameters of the
 * initial data (<state_bar, d state_0 / d theta>). */
int grf_state_dot(const grf_box* box, const double* x, const double* y, int field, double* out, void* ws,
                  size_t ws_bytes, grf_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Waveform extraction on spheres ("Diagnostics": tensor and scalar gravitational waveforms).
 * Modes of a field f = f_re + i f_im on the sphere of radius R about c,
 *   a_lm = integral over the sphere of f(c + R n) conj(sY_lm(theta, phi)) dOmega,
 * l = 0 .. lmax, m = -l .. l, theta from the z axis, phi from x towards y, spin weight s = 0
 * (scalar waveforms, e.g. the scalar field phi) or -2 (tensor waveforms, from Psi_4). sY_lm:
 * Goldberg et al.'s sum formula with the Condon-Shortley phase (s = 0: the usual Y_lm).
 * Quadrature: ntheta Gauss-Legendre nodes in cos(theta) times nphi equally spaced phi (exact for
 * band limits below 2 ntheta in theta and nphi in phi); f is interpolated at each sample with
 * the tensor product of 4-point Lagrange polynomials (4th order) on the points i0-1 .. i0+2.
 * ------------------------------------------------------------------------------------- */

/* Hyperbolicity diagnostics of the 4dST equations ("Research projects": the loss of
 * hyperbolicity of the theory; "Key features": diagnostics) at the interior points, 4 fields in the
 * state's layout (device, out4):
 *   0  det M, the determinant of the per-point linear system for (d_t K_ij, d_t Pi) with each
 *      unknown's own coefficient normalised to 1 (1 without coupling). Where it vanishes the
 *      equations do not determine the time derivatives (the solve reports GRF_ESINGULAR);
 *   1  det(g_eff^ab) / det(g^ab) for the principal symbol of the scalar equation,
 *      g_eff^ab = (1 + 2 g2 X) g^ab - 2 g2 nabla^a phi nabla^b phi + 2 g3 (box(phi) g^ab - nabla^a
 *      nabla^b phi); without the cubic term (1 + 2 g2 X)^3 (1 + 6 g2 X);
 *   2  -g_eff^nn = 1 + 2 g2 X + 2 g2 Pi^2 + 2 g3 tr(nabla_i nabla_j phi) (positive while the slice
 *      normal is timelike for the scalar's characteristic cone);
 *   3  the smallest pivot of Gaussian elimination with partial pivoting of that normalised system,
 *      over its largest entry (1 without coupling; small where the solve nears a lost pivot).
 * The state's ghosts are refilled as for grf_rhs. Asynchronous. GRF_EINVAL for a bad box, params or
 * pointer. */
int grf_hyperbolicity(const grf_box* box, const grf_params* params, double* state, double* out4, grf_stream_t stream);

/* Weyl scalar Psi_4, the source of the tensor waveforms: Psi_4 = C_abcd n^a mbar^b n^c mbar^d
 * with n = (u - e_r)/sqrt2, m = (e_theta + i e_phi)/sqrt2, u the slice normal and (e_r, e_theta,
 * e_phi) the triad orthonormalised (Gram-Schmidt with respect to gamma, in that order) from the
 * coordinate directions (x, y, z), (x z, y z, -(x^2 + y^2)), (-y, x, 0) about the coordinate
 * origin. On a null tetrad the Ricci terms of the Weyl tensor drop out, so Psi_4 is evaluated from
 * the Riemann blocks (Gauss, Codazzi, and the Ricci equation with d_t K_ij solved as for the
 * right-hand side). 0 on the polar axis x = y = 0. out2: device, 2 fields in the state layout
 * (re, im), interior entries written. Ghosts of `state` are refilled as for grf_rhs. */
int grf_weyl_psi4(const grf_box* box, const grf_params* params, double* state, double* out2, grf_stream_t stream);

/* Scratch bytes for grf_extract_modes (the rule, the ring sums, the modes); 0 if out of range. */
size_t grf_extract_workspace_bytes(int ntheta, int lmax);

/* f_re, f_im: device, single fields in the state layout of `box` (e.g. state + f * fstride;
 * f_im may be NULL for a real field), read as given, ghosts included where the stencils reach.
 * 1 <= ntheta <= 512, 1 <= nphi <= 2048, 0 <= lmax <= 12, spin 0 or -2. modes_host: host,
 * 2 (lmax + 1)^2 doubles, (re, im) of a_lm at index l^2 + l + m (0 for l < |spin|).
 * Synchronises `stream`. GRF_EINVAL if an argument is out of range or a sample's stencil would
 * leave the ghosted box; GRF_EWORKSPACE if ws is too small or not 256-byte aligned. */
int grf_extract_modes(const grf_box* box, const double* f_re, const double* f_im, int spin, const grf_sphere* sphere,
                      int ntheta, int nphi, int lmax, double* modes_host, void* ws, size_t ws_bytes,
                      grf_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * No-allocation variant (the paper has no counterpart: this is a library convenience).
 * Some callers cannot call cudaMalloc: code that runs inside an already-captured CUDA
 * graph region, host frameworks that hand out device pointers but own all allocation, or
 * embedded/real-time callers that forbid allocation after start-up. For them this entry point
 * runs the same RK4 step as grf_rk4_step with its scratch (two stage states and the RK4
 * accumulator) in a fixed file-scope device array of GRF_NOALLOC_SCRATCH_BYTES bytes that every
 * GPU loading the library holds until the process exits. It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   - Limit: 3 x state bytes <= GRF_NOALLOC_SCRATCH_BYTES (48 MiB: e.g. a 32^3 box, 12.5 MB per
 *     state); larger boxes are rejected with GRF_ETOOLARGE before any work.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current) and caches it; make that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents; nothing in it needs to
 *     start at zero (every value is written before it is read). Calls that overlap on the GPU
 *     (other streams, other host threads) race on the array: serialise them.
 * Arguments, layout and errors otherwise as grf_rk4_step. */
#define GRF_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
int grf_rk4_step_noalloc(const grf_box* box, const grf_params* params, double* state, double dt, int nsteps,
                         grf_stream_t stream);

const char* grf_error_string(int code);
const char* grf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GRF_H */
