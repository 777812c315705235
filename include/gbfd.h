/*
 * gbfd.h -- C ABI of libgbfd, a single-GPU (GB300, sm_103a) solver for the
 * isothermal compressible hydrodynamics of Pekkila et al. (2017), "Methods
 * for compressible fluid simulation on GPUs using high-order finite
 * differences": sixth-order central differences (Eqs. 6-9) for the
 * right-hand side of Eqs. 1-3, fused with the 2N-storage third-order
 * Runge-Kutta substep (Eq. 10, Algorithms 2 and 3) on a periodic 3D grid.
 *
 * Conventions shared by every entry point
 *  - Every call returns a gbfd_status and never aborts the process.  After a
 *    failure, gbfd_last_error(ctx) holds a one-line reason.
 *  - Device memory is owned by the caller: gbfd_init receives one
 *    workspace buffer (size from gbfd_workspace_bytes) and never allocates
 *    device memory itself.  The context object is host memory owned by the
 *    library and released by gbfd_destroy.
 *  - All device work is enqueued asynchronously on the CUDA stream given to
 *    gbfd_init; only gbfd_get_state to host memory, gbfd_diagnostics,
 *    gbfd_cfl_dt and gbfd_sync wait for that stream.
 *  - A state is nfields arrays [nz][ny][nx] (x fastest) of the fields
 *    (lnrho, u_x, u_y, u_z[, s]), laid out one after the other.  nfields is
 *    4 for entropy_mode 0 (the paper's isothermal model, no energy variable)
 *    and 5 for entropy_mode 1 (a passive entropy field, ds/dt = -u.grad s,
 *    with no feedback on the flow).
 *  - The grid is periodic in every axis (Sect. 4); point i of an axis sits
 *    at i L/N (Sect. 2.3).
 *  - Not thread-safe per context: calls on one context must not overlap.
 */
#ifndef GBFD_H
#define GBFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBFD_ABI_VERSION 2

typedef enum {
    GBFD_OK = 0,
    GBFD_ERR_INVALID_ARG = 1, /* a size, pointer or parameter was rejected  */
    GBFD_ERR_WORKSPACE = 2,   /* workspace too small or not 256-B aligned   */
    GBFD_ERR_CUDA = 3,        /* a CUDA runtime call failed (see last_error) */
    GBFD_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up          */
    GBFD_ERR_UNSUPPORTED = 5, /* valid request this build does not provide   */
    GBFD_ERR_STATE = 6        /* context unusable after an earlier error     */
} gbfd_status;

/* Arithmetic of the solver (spec precision forms).
 * FP64: FP64 storage and arithmetic.
 * FP32: FP32 storage, stencils and update.
 * FP32_ACC64: FP32 storage and stencils; the RK3 register update
 *   w <- alpha w + dt rhs and u <- u + beta w of Eq. 10 is done in FP64 in
 *   registers and rounded to FP32 storage.
 * FP32_ACC64_W64: as FP32_ACC64, but the 2N register w (u-tilde) is also
 *   stored in FP64.
 * FP32_ACCFF: as FP32_ACC64, with the update carried in float-float
 *   arithmetic (each value an unevaluated sum of two FP32 numbers, products
 *   and sums made error-free, Dekker 1971 / Knuth) on the FP32 units instead
 *   of the FP64 pipe; w stored in FP32.  55-point form only. */
enum {
    GBFD_FP64 = 0,
    GBFD_FP32 = 1,
    GBFD_FP32_ACC64 = 2,
    GBFD_FP32_ACC64_W64 = 3,
    GBFD_FP32_ACCFF = 4
};

/* Stencil form (Sect. 4.1 and 4.2).
 * 55P: single pass; grad(div u) from Eq. 7 and the bidiagonal Eq. 8.
 * 19P: two passes (Algorithm 3); pass 1 stores div u, pass 2 adds
 *      (nu/3) grad(div u) with Eq. 6 applied to the stored divergence. */
enum { GBFD_55P = 0, GBFD_19P = 1 };

typedef struct {
    int32_t nx, ny, nz;   /* points per axis; nx % 4 == 0, all >= 8           */
    int32_t precision;    /* GBFD_FP64 / GBFD_FP32 / GBFD_FP32_ACC64[_W64]     */
    int32_t form;         /* GBFD_55P / GBFD_19P                               */
    int32_t entropy_mode; /* 0: 4 fields (isothermal); 1: + passive entropy s */
    double lx, ly, lz;    /* box lengths L_i (> 0)                             */
    double cs;            /* isothermal sound speed c_s (>= 0), Eq. 2         */
    double nu;            /* kinematic viscosity nu (>= 0), Eq. 2             */
    int32_t bc_z;         /* GBFD_BC_PERIODIC (0) or GBFD_BC_WALL (1)          */
    int32_t reserved;     /* 0                                                */
} gbfd_params;

/* Boundary condition along z (Sect. 4: ghost zones carry the boundary
 * conditions; Algorithm 1's "compute boundary conditions" step).
 * PERIODIC: every axis periodic (the paper's runs); z spacing lz / nz.
 * WALL: x and y periodic; z bounded by two impermeable, free-slip walls
 * through the first and last grid planes, which sit at z = 0 and z = lz
 * (z spacing lz / (nz - 1)).  Three ghost planes below and above the
 * interior are filled after every substep (and between the two passes of
 * the 19-point form, for the stored divergence) with the mirror images of
 * the interior about the wall planes: even (f(-k) = f(k)) for lnrho, u_x,
 * u_y, s and the divergence, odd (f(-k) = -f(k)) for u_z.  The paper defines
 * no condition besides periodic; this one is the mirror reading of its
 * ghost zones, whose solution is the periodic one of the mirror-extended
 * state.  The initial state should have u_z = 0 on both wall planes.  Not
 * available with the forcing, the batch or the correction network
 * (UNSUPPORTED).
 * EXCHANGE: the box is one z-slab of a larger periodic domain split along z
 * (the domain decomposition the paper names as the route to several GPUs,
 * Sect. 7): x and y periodic, z spacing lz / nz, and the three ghost planes
 * below and above the slab are the neighbouring slabs' boundary planes,
 * which the caller moves between substeps with gbfd_halo_pack /
 * gbfd_halo_unpack (one exchange of the five fields per substep; the
 * 19-point form would need a second one for the divergence between its
 * passes and is not provided: INVALID_ARG).  55-point form only. */
enum { GBFD_BC_PERIODIC = 0, GBFD_BC_WALL = 1, GBFD_BC_EXCHANGE = 2 };

/* FP64 reductions over the current state (grid cell volume dV = prod L_i/N_i):
 * mass = dV sum exp(lnrho); ekin = dV sum exp(lnrho)|u|^2/2;
 * umax = max |u| (Euclidean); urms = sqrt(mean |u|^2);
 * rms[f] = sqrt(mean f^2), maxabs[f] = max |f| per field (0 for an absent
 * entropy field); nonfinite = 1 when any value of the state is NaN/Inf. */
typedef struct {
    double mass, ekin, umax, urms;
    double rms[5];
    double maxabs[5];
    int32_t nonfinite;
    int32_t nfields;
} gbfd_diag;

typedef struct gbfd_ctx gbfd_ctx;

/* Bytes of device workspace gbfd_init needs for these parameters (0 when the
 * parameters are invalid).  Holds two padded state buffers (ping-pong, the
 * separate in/out arrays of Sect. 4), the 2N register u-tilde, the
 * divergence field of the 19-point form, a staging area for state copies
 * and reduction scratch. */
size_t gbfd_workspace_bytes(const gbfd_params *p);

/* Create a context.  `workspace` is a device pointer (256-byte aligned) to
 * `workspace_bytes` >= gbfd_workspace_bytes(p) bytes that the caller keeps
 * alive until gbfd_destroy; `stream` is a cudaStream_t (NULL = legacy default
 * stream).  The state is zero after init.  Errors: INVALID_ARG (p or out
 * NULL, bad sizes), WORKSPACE, CUDA. */
gbfd_status gbfd_init(const gbfd_params *p, void *workspace, size_t workspace_bytes, void *stream,
                      gbfd_ctx **out);

/* Release the context (not the caller's workspace).  NULL is accepted. */
gbfd_status gbfd_destroy(gbfd_ctx *ctx);

/* Copy a full state into the solver.  `src` holds nfields*nz*ny*nx values,
 * FP64 if src_is_fp64 else FP32, in host memory (src_on_device = 0) or
 * device memory (src_on_device = 1).  Pinned host memory mapped into the
 * device address space is read in place by the copy kernel over the
 * CPU-GPU link (asynchronous, no staging copy); pageable host memory is
 * staged through the workspace.  Values are converted to the storage
 * precision.  The host buffer may be reused once the call's work on the
 * stream has completed. */
gbfd_status gbfd_set_state(gbfd_ctx *ctx, const void *src, int src_on_device, int src_is_fp64);

/* Copy the current state out, same layout as gbfd_set_state.  A host
 * destination is complete when the call returns (the stream is
 * synchronised; unless GBFD_OPT_HOST_ASYNC is set); pinned host memory is written in place by the copy kernel,
 * pageable memory through the workspace.  A device destination is written
 * asynchronously.  Errors: INVALID_ARG (dst NULL), CUDA; with a host
 * destination also TIMEOUT, as gbfd_sync reports it (the state copied out is
 * then not to be trusted). */
gbfd_status gbfd_get_state(gbfd_ctx *ctx, void *dst, int dst_on_device, int dst_is_fp64);

/* Advance `nsteps` >= 0 full RK3 steps of length dt (> 0, finite): three
 * substeps each of Eq. 10 with alpha = (0, -5/9, -153/128) and
 * beta = (1/3, 15/16, 8/15) (Williamson's 2N-storage RK3; the paper leaves
 * the coefficients to the chosen scheme and fixes alpha_1 = 0), the
 * right-hand side of Eqs. 1-3 with the body force f = 0, in the form chosen
 * at init.  Asynchronous. */
gbfd_status gbfd_rk3_step(gbfd_ctx *ctx, double dt, int nsteps);

/* One substep s in {0, 1, 2} of Eq. 10 (Algorithm 2 or 3), for tests that
 * compare single substeps; s = 0 ignores the old u-tilde (alpha_1 = 0).
 * Asynchronous. */
gbfd_status gbfd_substep(gbfd_ctx *ctx, int s, double dt);

/* FP64 reductions of the current state (struct above).  Synchronises. */
gbfd_status gbfd_diagnostics(gbfd_ctx *ctx, gbfd_diag *out);

/* Time step from the current state: dt = min(cfl dmin / (max|u| + c_s),
 * cnu dmin^2 / nu) with dmin the smallest grid spacing (the paper gives no
 * rule; this is the helper used by the benchmarks).  Synchronises. */
gbfd_status gbfd_cfl_dt(gbfd_ctx *ctx, double cfl, double cnu, double *dt_out);

/* nsteps RK3 steps with the non-helical random-k body force of Sect. 6
 * (Eqs. 20-21) in Eq. 2: step n adds f(x) = N f_k cos(k.x + phi) to the
 * momentum equation, with the integer wave vector k[3n..3n+2] (physical
 * k_i = 2 pi k_i / L_i), phase phi[n], unit vector e[3n..3n+2] (not parallel
 * to k), N = f0 c_s sqrt(|k| c_s / dt) and f_k = (k x e) / sqrt(|k|^2 -
 * (k.e)^2); k, phi and e stay fixed over the step's three substeps.  The
 * paper draws k from an isotropic set kmin <= |k| <= kmax and phi, e at
 * random every step; the caller supplies the draws.  k, phi, e are host
 * arrays of 3n, n and 3n values.  Each step first fills per-axis phase
 * tables in the workspace (one small launch).  Every precision and form is
 * supported; the FP32 tile table's entries all run the default kernel when
 * forced.  Errors: INVALID_ARG (dt <= 0 or not finite, nsteps < 0, NULL
 * arrays, k = 0, k parallel to e, phi not finite), CUDA. */
gbfd_status gbfd_rk3_step_forced(gbfd_ctx *ctx, double dt, int nsteps, double f0, const int *k,
                                 const double *phi, const double *e);

/* Halo exchange of a bc_z = GBFD_BC_EXCHANGE context (Sect. 7's domain
 * decomposition along z; no counterpart kernel in the paper).  A message is
 * the three interior planes next to one side, every field, whole padded
 * planes: gbfd_halo_bytes(ctx) bytes (0 for other contexts).  pack(side)
 * copies this slab's planes 0..2 (side 0) or nz-3..nz-1 (side 1) into the
 * device buffer dst; unpack(side) writes the device buffer src into the
 * ghost planes -3..-1 (side 0) or nz..nz+2 (side 1).  So the lower
 * neighbour's side-1 message is unpacked into side 0 and the upper
 * neighbour's side-0 message into side 1, before every substep (after
 * gbfd_set_state too).  Both are stream-ordered device copies on the
 * context's stream.  Errors: UNSUPPORTED (other contexts), INVALID_ARG. */
size_t gbfd_halo_bytes(const gbfd_ctx *ctx);
gbfd_status gbfd_halo_pack(gbfd_ctx *ctx, int side, void *dst);
gbfd_status gbfd_halo_unpack(gbfd_ctx *ctx, int side, const void *src);

/* Wait for the context's stream and report any device-side error
 * (bounded waits that gave up -> TIMEOUT; CUDA errors -> CUDA). */
gbfd_status gbfd_sync(gbfd_ctx *ctx);

/* Diagnostics for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is an interface convenience.  It computes the
 * same FP64 reductions as gbfd_diagnostics, but needs no context and no
 * workspace: the caller passes a device state array (nfields arrays
 * [nz][ny][nx], FP64 if state_is_fp64 else FP32, the gbfd_set_state layout)
 * and a device buffer `out` of 16 doubles, filled asynchronously on `stream`
 * with mass, ekin, umax, urms, rms[5], maxabs[5], nonfinite (as 0.0/1.0), 0.
 * It is meant for code that may not call cudaMalloc (for example inside a
 * host callback or a stream-ordered section, where the implicit device
 * synchronisation of cudaMalloc/cudaFree would stall or deadlock, or inside a
 * framework whose allocator does not allow it).  It calls no allocating
 * routine: its partial sums live in a fixed file-scope device array of 1216 x
 * 16 doubles (155,648 bytes) that every GPU loading the library holds until
 * the process exits.  Any grid size within the limits below fits in it (each
 * block walks the grid rows in a grid-stride loop).  The array's device
 * address is looked up on the first call on each device (with that device
 * current), and again after that device's context was replaced (e.g. by
 * cudaDeviceReset).  Make that first call before any stream capture, and
 * where allocation is still allowed: with lazy module loading it is also the
 * call that loads the library's device code, which may allocate device
 * memory for the module; later calls allocate nothing.  All calls share the
 * array: calls whose work overlaps on the GPU race and must be ordered (same
 * stream, or events).
 * Limits: nfields 4 or 5; extents >= 1, nx*ny*nz <= 2^33; box lengths > 0.
 * Errors: INVALID_ARG (with gbfd_last_error(NULL)), CUDA. */
gbfd_status gbfd_diagnostics_noalloc(const void *state, int state_is_fp64, int nx, int ny, int nz,
                                     int nfields, double lx, double ly, double lz, void *stream,
                                     double *out);

/* Measured FP64 fused multiply-add rate of the current device, in TFLOP/s
 * (an FMA counts 2): independent FMA chains on every SM, best of four timed
 * launches on `stream` after two warm-ups (about 0.1 s in all; synchronises
 * the stream).  It is the roofline denominator of the FP64 path, whose
 * kernels the FP64 pipe bounds; no counterpart in the paper.  Errors:
 * INVALID_ARG (NULL output), CUDA. */
gbfd_status gbfd_fp64_fma_rate(void *stream, double *tflops);

/* Measured cost of one tcgen05 MMA (M = 128, K = 16, BF16 operands from
 * shared memory, FP32 accumulation in TMEM) with n columns, n in {16, 32,
 * 48, 64, 96, 128, 256}: one thread per SM issues 1,024 MMAs back to back
 * with the convolutions' operand strides; *cycles = SM clock cycles per MMA,
 * averaged over the SMs (synchronises `stream`; results in fixed device
 * arrays, no allocation).  It is the measurement behind the network
 * convolutions' MMA shape (their z taps stacked along N); no counterpart in
 * the paper.  Errors: INVALID_ARG (NULL output, unsupported n), TIMEOUT (a
 * bounded completion wait gave up), CUDA. */
gbfd_status gbfd_tc_mma_cycles(int n, void *stream, double *cycles);

/* Tuning options (no counterpart in the paper; used by the tests and the
 * autotuner).  GBFD_OPT_KERNEL_PATH: 0 = tiled kernels (TMA-staged shared
 * memory, the default), 1 = simple one-thread-per-point kernels reading
 * global memory.  GBFD_OPT_TILE_CONFIG: index into the tiled kernels' tile
 * table, -1 = built-in default.  Out-of-range values -> INVALID_ARG. */
enum {
    GBFD_OPT_KERNEL_PATH = 1,
    GBFD_OPT_TILE_CONFIG = 2,
    GBFD_OPT_FAULT_SKIP_COPY = 3,
    GBFD_OPT_HOST_PATH = 4,
    GBFD_OPT_HOST_ASYNC = 5
};
/* GBFD_OPT_HOST_PATH: 0 (default) = gbfd_set_state / gbfd_get_state access
 * pinned host buffers in place from the copy kernels; 1 = always copy host
 * buffers through the workspace with cudaMemcpyAsync. */
/* GBFD_OPT_HOST_ASYNC: 0 (default) = gbfd_get_state to host memory returns
 * with the copy complete; 1 = it only enqueues the copy on the context's
 * stream (with pinned host memory it then overlaps other streams' work; with
 * pageable memory the CUDA runtime may still wait).  The buffer is complete
 * once the stream reaches that point (gbfd_sync, which also reports a device
 * TIMEOUT, or any wait on the stream). */
/* GBFD_OPT_FAULT_SKIP_COPY (tests only): value j >= 0 makes the first CTA of
 * the two-points-per-thread tiled kernels skip the TMA copy of local plane j
 * of its first column (a column has its output planes + 6 local planes), so
 * its bounded mbarrier wait gives up after about 2 s, the launch ends early
 * and gbfd_sync reports GBFD_ERR_TIMEOUT with the context still usable; -1
 * (the default) turns it off. */
gbfd_status gbfd_set_option(gbfd_ctx *ctx, int key, int64_t value);

/* Tile autotuner (no counterpart in the paper; the paper tuned block shapes
 * and points per thread by hand, Sect. 5).  Times every entry of the tiled
 * kernels' tile table on the context's current state for `reps` RK3 steps
 * each and selects the fastest; the state is not advanced (the timed
 * substeps write the spare buffer and u-tilde only).  With a non-NULL
 * `cache_path`, a JSON file keyed by GPU name, grid, precision, form and
 * field count is read first (a hit skips the timing) and updated after.
 * Outputs (may be NULL): the chosen table index and its ms per RK3 step
 * (0 on a cache hit).  Synchronises the stream. */
gbfd_status gbfd_autotune(gbfd_ctx *ctx, int reps, const char *cache_path, int *best_cfg,
                          double *best_ms);

/* Number of kernel launches the context has enqueued since init. */
int64_t gbfd_launch_count(const gbfd_ctx *ctx);

/* One-line description of the last failure on this context ("" if none);
 * valid until the next call on the context.  ctx may be NULL (reports
 * failures of gbfd_init). */
const char *gbfd_last_error(const gbfd_ctx *ctx);

/* Static name of a status code. */
const char *gbfd_status_string(gbfd_status s);

/* ------------------------------------------------------------------------
 * Batched form (no counterpart in the paper; the paper advances one grid).
 * nbox independent periodic cubic boxes, box b with n[b]^3 points (n[b] a
 * multiple of 4 in 8..1024), side lengths[b], viscosity nu[b], common c_s,
 * FP32 storage and arithmetic, the 55-point fused substep of Algorithm 2.
 * Each substep of all boxes is one persistent launch over a work list of
 * equal-cost columns (box, 32 x 8 tile, z-chunk); a run of nsteps RK3 steps
 * is captured once as a CUDA graph (per nsteps and buffer parity) and
 * replayed.  Per-box states use the gbfd_set_state layout.
 * ------------------------------------------------------------------------ */
typedef struct gbfd_batch gbfd_batch;

/* Workspace bytes for the batch (0 when the sizes are invalid). */
size_t gbfd_batch_workspace_bytes(int nbox, const int32_t *n, int entropy_mode);

/* Create a batch on the caller's 256-byte aligned device workspace; no
 * device allocation inside (one private non-blocking stream is created for
 * graph capture).  Errors: INVALID_ARG, WORKSPACE, CUDA. */
gbfd_status gbfd_batch_init(int nbox, const int32_t *n, const double *lengths, const double *nu,
                            double cs, int entropy_mode, void *workspace, size_t workspace_bytes,
                            void *stream, gbfd_batch **out);
gbfd_status gbfd_batch_destroy(gbfd_batch *b);

/* Copy one box's state in/out (host or device, FP32 or FP64).  Host copies
 * synchronise the stream (the staging area is shared by the boxes). */
gbfd_status gbfd_batch_set_state(gbfd_batch *b, int box, const void *src, int src_on_device,
                                 int src_is_fp64);
gbfd_status gbfd_batch_get_state(gbfd_batch *b, int box, void *dst, int dst_on_device,
                                 int dst_is_fp64);

/* Advance every box nsteps RK3 steps, box b with time step dt[b] (> 0,
 * finite; host array of nbox values, copied before the call returns). */
gbfd_status gbfd_batch_step(gbfd_batch *b, const double *dt, int nsteps);

/* FP64 diagnostics of one box (synchronises). */
gbfd_status gbfd_batch_diagnostics(gbfd_batch *b, int box, gbfd_diag *out);

/* Wait for the stream; TIMEOUT when a bounded device wait gave up (an
 * mbarrier wait in a column, or a dataflow item's wait for its box's
 * previous substep), after which the batch stays usable. */
gbfd_status gbfd_batch_sync(gbfd_batch *b);

/* Options (no counterpart in the paper):
 * GBFD_BATCH_OPT_GRAPH: 1 = replay CUDA graphs (default), 0 = direct launches;
 * GBFD_BATCH_OPT_ZCHUNK: planes per work item: 8, 16, 32 (default), 64;
 * GBFD_BATCH_OPT_GRID: persistent CTAs per launch (0 = SMs x resident CTAs);
 * GBFD_BATCH_OPT_KERNEL: column routine: 0 = two-plane packed on 32 x 8
 *   tiles (default), 1 = lagged output with TMEM on 32 x 8 (weights read from
 *   shared memory), 2 = two-plane packed on 64 x 8;
 * GBFD_BATCH_OPT_DATAFLOW: 1 = all substeps of a gbfd_batch_step in ONE
 *   persistent launch, work items ordered by substep and each waiting
 *   (bounded, about 2 s) for its box's previous substep through a per-box
 *   completion counter (default); 0 = one launch per substep;
 * GBFD_BATCH_OPT_FAULT_STALL (tests): the dataflow work item with this index
 *   is never counted as done, so its box's next substep runs into the
 *   bounded wait (TIMEOUT at gbfd_batch_sync); -1 = off (default).
 * Out-of-range values -> INVALID_ARG.  gbfd_batch_get_option reads them back
 * (GRID: the grid in use). */
enum {
    GBFD_BATCH_OPT_GRAPH = 1,
    GBFD_BATCH_OPT_ZCHUNK = 2,
    GBFD_BATCH_OPT_GRID = 3,
    GBFD_BATCH_OPT_KERNEL = 4,
    GBFD_BATCH_OPT_DATAFLOW = 5,
    GBFD_BATCH_OPT_FAULT_STALL = 6
};
gbfd_status gbfd_batch_set_option(gbfd_batch *b, int key, int64_t value);
gbfd_status gbfd_batch_get_option(const gbfd_batch *b, int key, int64_t *value);

/* Autotuner of the batch: times `steps` RK3 steps (dt = 0, which leaves the
 * state's values unchanged) for every column routine x z-chunk length x
 * launch mode (dataflow or per substep), keeps the fastest; its z-chunk and
 * time per step are returned (outputs may be NULL; the rest is readable with
 * gbfd_batch_get_option). */
gbfd_status gbfd_batch_autotune(gbfd_batch *b, int steps, int *best_zc, double *best_ms);

int64_t gbfd_batch_launch_count(const gbfd_batch *b);
const char *gbfd_batch_last_error(const gbfd_batch *b);

/* ------------------------------------------------------------------------
 * Learned coarse-grid correction (no counterpart in the paper).  A small
 * network corrects a coarse FP32 solver state after each RK3 step:
 *   state += std_out * net((state - mean_in) / std_in)   per channel,
 * net = conv3 . GELU . conv2 . GELU . conv1, each a periodic 3x3x3
 * cross-correlation y[o,p] = b[o] + sum_{c,t} W[o,c,t] x[c,p+t] (channels
 * 5 -> 32 -> 32 -> 5, exact GELU).  BF16 weights and activations, FP32
 * accumulation: the convolutions and their input gradients run as
 * implicit GEMMs on the tcgen05 tensor cores; weight gradients are FP32
 * sums over the grid; Adam keeps FP32 master weights.
 * Compact state arrays are [batch][5][n][n][n] FP32 on the device (the fifth
 * channel is ignored when nf = 4).  Parameters are exchanged in FP32, layer
 * by layer: W1 [32][5][3][3][3], b1 [32], W2 [32][32][3][3][3], b2 [32],
 * W3 [5][32][3][3][3], b3 [5] (gbfd_cnn_param_count() floats).
 * ------------------------------------------------------------------------ */
typedef struct gbfd_cnn gbfd_cnn;

/* Workspace for a network on an n^3 grid training on up to `batch` samples
 * at once (0 when invalid: n in 4..512, batch * n^3 <= 2^30). */
size_t gbfd_cnn_workspace_bytes(int n, int batch);
/* Create on a 1024-byte aligned device workspace (no device allocation). */
gbfd_status gbfd_cnn_init(int n, int batch, void *workspace, size_t workspace_bytes, void *stream,
                          gbfd_cnn **out);
gbfd_status gbfd_cnn_destroy(gbfd_cnn *c);
int gbfd_cnn_param_count(void);
/* Host FP32 parameters in / out (set resets the Adam moments). */
gbfd_status gbfd_cnn_set_params(gbfd_cnn *c, const float *params);
gbfd_status gbfd_cnn_get_params(gbfd_cnn *c, float *params);
/* Per-channel input mean/std and output std (5 values each, host). */
gbfd_status gbfd_cnn_set_norm(gbfd_cnn *c, const float *mean_in, const float *std_in,
                              const float *std_out);
/* Normalised network output ys [batch][5][n^3] of device states xs. */
gbfd_status gbfd_cnn_forward(gbfd_cnn *c, const float *xs, int nf, int batch, float *ys);
/* Loss (mean over batch, channel and point of (net(x) - (t - x)/std_out)^2)
 * and its gradient w.r.t. the parameters (host, param_count floats; NULL
 * skips the copy); xs are coarse-stepped states, ts the targets.
 * Synchronises. */
gbfd_status gbfd_cnn_gradients(gbfd_cnn *c, const float *xs, const float *ts, int nf, int batch,
                               float *grads, double *loss);
/* One Adam step (beta = 0.9, 0.999, eps 1e-8) on the same loss; the loss
 * before the step is returned when `loss` is non-NULL (synchronises then). */
gbfd_status gbfd_cnn_train_step(gbfd_cnn *c, const float *xs, const float *ts, int nf, int batch,
                                float lr, double *loss);
/* Apply the correction to the current state of an FP32 cubic context of the
 * network's grid (on the context's stream). */
gbfd_status gbfd_cnn_apply(gbfd_cnn *c, gbfd_ctx *ctx);
/* nsteps of: one RK3 step, then the correction. */
gbfd_status gbfd_step_corrected(gbfd_ctx *ctx, gbfd_cnn *c, double dt, int nsteps);
/* Centred box filter of an FP32 cubic context's state to an r times coarser
 * grid (r even): per axis weights (1/2, 1, ..., 1, 1/2) / r over fine offsets
 * -r/2..r/2 about fine vertex r I; out is [nf][nc^3] FP32 on the device. */
gbfd_status gbfd_box_filter(gbfd_ctx *fine, int r, float *out);
int64_t gbfd_cnn_launch_count(const gbfd_cnn *c);
const char *gbfd_cnn_last_error(const gbfd_cnn *c);
/* Launch-shape options (tests; no counterpart in the paper).
 * GBFD_CNN_OPT_CONV_GRID: CTAs per convolution launch, each walking an equal
 * share of the 256-point tiles (0 = default, one per SM); a small value
 * makes every CTA loop over many tiles.  GBFD_CNN_OPT_WGRAD_PARTS: CTAs of
 * the weight-gradient sums, 1..296 (0 = default 296).  Results agree to
 * rounding whatever the values; out-of-range values -> INVALID_ARG. */
enum { GBFD_CNN_OPT_CONV_GRID = 1, GBFD_CNN_OPT_WGRAD_PARTS = 2 };
gbfd_status gbfd_cnn_set_option(gbfd_cnn *c, int key, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* GBFD_H */
