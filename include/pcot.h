/*
 * pcot.h -- C ABI of the GB300 (sm_103a) engine for time-iterated affine star
 * stencils under the tile schedules studied in "PCOT: Cache Oblivious Tiling
 * of Polyhedral Programs" (Ranasinghe, Prajapati, Yuki, Rajopadhye;
 * arXiv 1802.00166).
 *
 * Problem statement (Sec. 3.1, Sec. 4.1, Sec. 4.2): a fully permutable affine
 * loop nest over a rectangular spatial domain repeated for T time steps.  The
 * loop body is the star-stencil point update
 *
 *     u^{t+1}[x] = c_0 u^t[x] + sum_{axis a} sum_{o in -r..-1, +1..+r} c_{a,o} u^t[x + o e_a]
 *
 * (the Jacobi-1D 3-point, Heat-2D 5-point and Jacobi-3D 7-point kernels of
 * Sec. 5.1.2 and Appendix A), with the two-buffer t%2 storage of the
 * Appendix A example.  Three schedules compute the identical result:
 *   PCOT_SWEEP  one pass over the grid per time step (the untiled loop nest);
 *   PCOT_SLT    single-level tiling: time blocks of depth k executed in
 *               lexicographic order, spatial tiles of a block concurrently
 *               (Sec. 3.3, "Single-Level Tiling");
 *   PCOT_COT    the recursive divide-and-conquer order of Sec. 4 applied to
 *               the lattice of (time block, spatial tile) leaves after time
 *               skewing, run by one persistent kernel with dependency counters
 *               in place of the OpenMP task waits of Sec. 4.2.
 *   PCOT_SKEW   (2-D Dirichlet grids) parallelogram tiles of the skewed space
 *               (t, t+i, t+j) -- the tiles of Sec. 3.1 after the skew of Sec.
 *               4.3.2, which recompute nothing -- run by the same persistent
 *               executor in wavefront order, or in the recursive order of Sec.
 *               4 when cot_threshold is set.  tile[0], tile[1] are the tile's
 *               skewed extents (default 32, 64), time_depth its steps
 *               (default 4), tile[2] the threads per CTA (32..512, a multiple
 *               of 32; default 256).  Every point is computed once, in the
 *               loop nest's rounding: FP64 exact mode is bitwise the sweep.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Coefficients: ncoeffs = 1 + 2*dims*radius doubles, ordered centre, then
 *    axis 0 (slowest) .. axis dims-1 (fastest); per axis offsets -r..-1 then
 *    +1..+r.  PCOT_F64_EXACT accumulates in exactly that order; the FMA
 *    modes (PCOT_F32, PCOT_F64) accumulate the same terms with the axis-0
 *    +1 neighbour moved last (see Precision).
 *  Grid layout: row-major, the last axis contiguous (stride 1).  `sizes` are
 *    the INTERIOR sizes n_a.  Dirichlet grids store n_a + 2r entries per axis;
 *    the outer ring of width r holds fixed boundary values that are never
 *    written.  Periodic grids store n_a entries per axis and wrap.
 *  Strides: `strides` (element strides per axis, last entry 1) may be NULL for
 *    the contiguous layout.  A padded pitch whose byte size is a multiple of
 *    16 (and a 16-byte-aligned base) lets the kernels use 16-byte vector
 *    accesses; other layouts are accepted and run with narrower accesses.
 *  Precision: PCOT_F32 grids hold float and use fused multiply-add;
 *    PCOT_F64 grids hold double and use fused multiply-add; in both, every
 *    schedule evaluates a point with the same operations in the same order
 *    (centre product first, the axis-0 +1 term last), so the schedules agree
 *    with each other bitwise and with the exact definition within rounding;
 *    PCOT_F64_EXACT grids hold double and use separately rounded multiply and
 *    add in the order above, so results are bitwise identical to a plain
 *    IEEE-754 binary64 evaluation of the definition.
 *  Memory: every `grid` / `workspace` pointer is DEVICE memory owned by the
 *    caller unless a parameter says "host".  The handle owns only host-side
 *    plan caches and a small device status block allocated by pcot_create.
 *  Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Compute entry points are asynchronous: argument and
 *    launch errors are returned immediately, device-side errors (a dependency
 *    wait that timed out, an index outside a buffer) are reported by
 *    pcot_check.
 *  Errors: every entry point returns a pcot_status; nothing throws or aborts
 *    across the ABI.  A handle must not be used from two host threads at once.
 */
#ifndef PCOT_H
#define PCOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PCOT_OK = 0,
    PCOT_ERR_INVALID_ARG = 1,  /* NULL pointer, size < 1, wrong coefficient count, T < 0 ... */
    PCOT_ERR_UNSUPPORTED = 2,  /* dims / radius / tile shape this build has no kernel for     */
    PCOT_ERR_ALIGNMENT = 3,    /* pointer or stride not aligned to the element size          */
    PCOT_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed                */
    PCOT_ERR_OOM = 5,          /* workspace too small, or a host allocation failed           */
    PCOT_ERR_TIMEOUT = 6,      /* a device-side dependency wait gave up (see pcot_check)     */
    PCOT_ERR_BOUNDS = 7        /* a device-side index check failed (see pcot_check)          */
} pcot_status;

typedef enum { PCOT_DIRICHLET = 0, PCOT_PERIODIC = 1 } pcot_boundary;
typedef enum { PCOT_F32 = 0, PCOT_F64 = 1, PCOT_F64_EXACT = 2 } pcot_dtype;
typedef enum { PCOT_SWEEP = 0, PCOT_SLT = 1, PCOT_COT = 2, PCOT_AUTO = 3, PCOT_SKEW = 4 } pcot_schedule;

/*
 * Tile parameters (Sec. 3.3 "Tile Size": the tile size doubles as the
 * recursion's leaf size; Sec. 4.5 padding).
 *  tile[a]          output extent of a spatial tile along axis a (axis 0
 *                   slowest).  0 picks the default.  The kernels may round an
 *                   extent (the fastest axis to whole warps); pcot_plan_query
 *                   reports the extents actually used.
 *  time_depth       k, the number of time steps a tile advances in one pass
 *                   (the height of the trapezoid); 0 picks the default.
 *  cot_threshold[0] leaf orthant extent of the tile lattice in time blocks,
 *  cot_threshold[1+a]  ... and in tiles along axis a (the recursion's base-case
 *                   threshold, Sec. 4.2).  0 means 1.
 */
typedef struct {
    int32_t tile[3];
    int32_t time_depth;
    int32_t cot_threshold[4];
} pcot_tile_params;

typedef struct pcot_plan *pcot_handle;

/* Human-readable name of a status code (static storage, never NULL). */
const char *pcot_status_string(pcot_status s);

/*
 * Create a stencil handle.
 *  dims in {1,2,3}; radius must be 1 (the star stencils of Sec. 5.1.2);
 *  coeffs: ncoeffs = 1 + 2*dims*radius doubles (copied); boundary: Dirichlet
 *  ring or periodic wrap.  On success *out must be released with
 *  pcot_destroy.  Device resources of the handle (a small status block and a
 *  grid-sum partial buffer) are allocated on the current device by the first
 *  call that launches work; planning calls (pcot_plan_query) need no GPU.
 */
pcot_status pcot_create(int dims, int radius, const double *coeffs, int ncoeffs,
                        pcot_boundary boundary, pcot_handle *out);

/* Release a handle (waits for nothing: call after the last run completed). */
pcot_status pcot_destroy(pcot_handle h);

/*
 * Device workspace needed by pcot_run for this problem, step count and
 * schedule, in bytes (a twin of the grid with the same strides, plus the
 * per-run dependency counters and tile queue of PCOT_COT, which grow with the
 * number of time blocks).  `params` may be NULL (defaults).  For PCOT_AUTO:
 * the largest need over the picker's candidates (no GPU needed).  For
 * PCOT_SKEW: the twin plus a bound on its tile queue and counters.  A
 * schedule value outside the enum gives PCOT_ERR_INVALID_ARG.
 */
pcot_status pcot_workspace_bytes(pcot_handle h, const int64_t *sizes, const int64_t *strides,
                                 int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                                 const pcot_tile_params *params, size_t *bytes);

/*
 * Advance `grid` by T time steps (Sec. 4.2: the result of the original loop
 * nest, whatever the schedule).
 *  grid       device, in/out, layout as above; the result is in `grid` for
 *             every T (the library arranges an even number of buffer swaps).
 *  workspace  device scratch of at least pcot_workspace_bytes bytes, 256-byte
 *             aligned; its contents on entry are ignored and on exit are
 *             undefined.  The Dirichlet ring is copied into it by the call.
 *  workspace_bytes  size of `workspace`; a smaller size than the schedule
 *             needs returns PCOT_ERR_OOM before anything is launched.
 *  T          number of time steps, T >= 0; T = 0 returns PCOT_OK at once.
 *  schedule   PCOT_AUTO runs the schedule and tile parameters pcot_pick
 *             chooses for this problem (the learned picker, or the
 *             autotuner when no model is loaded; the first call for a
 *             problem makes the pick and synchronises, later calls reuse
 *             it); `params` is then ignored.
 *  params     NULL = defaults.
 * Asynchronous on `stream`; call pcot_check to surface device errors.
 */
pcot_status pcot_run(pcot_handle h, void *grid, void *workspace, size_t workspace_bytes,
                     const int64_t *sizes, const int64_t *strides, int64_t T, pcot_dtype dtype,
                     pcot_schedule schedule, const pcot_tile_params *params, void *stream);

/*
 * End-to-end variant of pcot_run for host-resident data: copies `host_grid`
 * (host memory, pinned for best speed, same layout) to `dev_grid`, runs
 * pcot_run, copies the result back into `host_grid`, and synchronises the
 * stream before returning (so it also reports device errors like pcot_check).
 */
pcot_status pcot_run_host(pcot_handle h, void *host_grid, void *dev_grid, void *workspace,
                          size_t workspace_bytes, const int64_t *sizes, const int64_t *strides, int64_t T,
                          pcot_dtype dtype, pcot_schedule schedule,
                          const pcot_tile_params *params, void *stream);

/*
 * Synchronise `stream` and read the handle's device status block: returns
 * PCOT_OK, PCOT_ERR_TIMEOUT (a dependency wait of the persistent executor
 * exceeded its limit; the kernel returned without hanging) or PCOT_ERR_BOUNDS,
 * and clears the block.  CUDA errors of the stream map to PCOT_ERR_CUDA.
 */
pcot_status pcot_check(pcot_handle h, void *stream);

/*
 * Describe the PCOT_COT plan for a problem (for inspection and the legality
 * tests).  Writes lattice[0] = number of time blocks run by the persistent
 * kernel, lattice[1+a] = tiles along axis a; tile_ext[a] = tile output extent
 * used; *depth = time steps per block; *n_tiles = number of queue entries.
 * If `queue` is non-NULL it receives n_tiles entries (capacity `cap`) in
 * execution order, each the linear lattice index
 * ((b * L_0 + i_0) * L_1 + i_1) * L_2 + i_2; `deps` (may be NULL) receives the
 * initial dependency count of each entry of `queue`.  `tail_steps` receives
 * the steps run after the persistent kernel by single-level launches.
 */
pcot_status pcot_plan_query(pcot_handle h, const int64_t *sizes, int64_t T, pcot_dtype dtype,
                            const pcot_tile_params *params, int32_t *lattice, int32_t *tile_ext,
                            int32_t *depth, int64_t *n_tiles, int64_t *tail_steps,
                            int32_t *queue, int32_t *deps, int64_t cap);

/*
 * Describe the PCOT_SKEW plan of a 2-D problem (no GPU needed; for the
 * planner tests).  lattice[3] = tiles along t, a = t+i, c = t+j; tile[3] =
 * (time_depth, tile[0], tile[1]) used; *n_tiles = non-empty tiles.  If
 * `queue` is non-NULL it receives the n_tiles lattice ids (b0 * L1 + b1) * L2
 * + b2 in execution order and `deps` (may be NULL) each one's number of
 * non-empty predecessors among its seven lower neighbours (capacity `cap`).
 */
pcot_status pcot_skew_plan_query(const int64_t *sizes, int64_t T, const pcot_tile_params *params,
                                 int32_t *lattice, int32_t *tile, int64_t *n_tiles, int32_t *queue,
                                 int32_t *deps, int64_t cap);

/*
 * Test hook: the persistent executor's dependency wait with a counter that
 * nothing releases.  Launches one CTA that waits on a count of 1 with a limit
 * of `timeout_ms` milliseconds; the kernel records PCOT_ERR_TIMEOUT in the
 * status block and returns.  pcot_check then returns PCOT_ERR_TIMEOUT.
 */
pcot_status pcot_test_wait_timeout(pcot_handle h, void *workspace, int32_t timeout_ms, void *stream);

/*
 * Conservation check (sum of the interior): *out_device (device, one double)
 * receives the FP64 sum of all interior values of `grid` (float grids are
 * widened before adding).  The reduction order is fixed by the problem size,
 * so repeated calls give bitwise identical sums.  Uses a partial-sum buffer
 * owned by the handle (allocated by pcot_create).
 */
pcot_status pcot_grid_sum(pcot_handle h, const void *grid, const int64_t *sizes,
                          const int64_t *strides, pcot_dtype dtype, double *out_device,
                          void *stream);

/* ------------------------------------------------------------------------
 * Batched runs: many independent 2-D Dirichlet grids (same stencil, dtype,
 * time depth and tile width; their own sizes, step counts, tile heights and
 * recursion thresholds) advanced by ONE persistent kernel.  Each grid's tiles
 * are ordered by the recursive schedule (Sec. 4.2) of its own lattice; the
 * per-grid queues are merged so that every grid progresses at the same
 * relative rate (ties: the grid with more tiles first), which keeps many
 * independent tiles in flight on all SMs.  The kernel records per-grid
 * completion times.  The launch sequence (counter reset, ring copy,
 * persistent kernel) is captured in a CUDA graph by pcot_batch_create and
 * replayed by pcot_batch_launch.
 *
 *  nb        number of grids (1 .. 65535)
 *  grids     HOST array of nb DEVICE pointers (each grid in/out, layout as for
 *            pcot_run; the result lands in the caller's grid)
 *  sizes     nb*2 interior sizes (row-major per grid)
 *  strides   nb*2 element strides, or NULL for contiguous grids
 *  T         nb step counts (>= 0)
 *  params    nb tile parameter sets or NULL; time_depth (1, 2, 4, 6 or 8
 *            for PCOT_F32; 1, 2 or 4 otherwise) and tile[1] (warps per tile via
 *            the tile width) are taken from params[0] for all grids; tile[0]
 *            and cot_threshold per grid
 *  workspace device scratch of pcot_batch_workspace_bytes bytes (queue,
 *            counters, descriptors and one twin per grid), 256-byte aligned;
 *            it must stay allocated and untouched while the batch exists
 *  done_ns   DEVICE array of nb+1 uint64 or NULL: [0] receives the
 *            %globaltimer (ns) when the first tile starts, [1+g] when grid g's
 *            last tile finished (latency of grid g = done_ns[1+g]-done_ns[0])
 * ------------------------------------------------------------------------ */
typedef struct pcot_batch_s *pcot_batch;

pcot_status pcot_batch_workspace_bytes(pcot_handle h, int nb, const int64_t *sizes,
                                       const int64_t *strides, const int64_t *T, pcot_dtype dtype,
                                       const pcot_tile_params *params, size_t *bytes);

pcot_status pcot_batch_create(pcot_handle h, int nb, void *const *grids, const int64_t *sizes,
                              const int64_t *strides, const int64_t *T, pcot_dtype dtype,
                              const pcot_tile_params *params, void *workspace,
                              size_t workspace_bytes, uint64_t *done_ns, void *stream,
                              pcot_batch *out);

/* Replay the captured graph on `stream` (asynchronous; pcot_check reports
 * device-side errors). */
pcot_status pcot_batch_launch(pcot_batch b, void *stream);

/* Release the graph and host plan (call after the last launch completed). */
pcot_status pcot_batch_destroy(pcot_batch b);

/* create + launch + synchronise + destroy; returns the pcot_check status. */
pcot_status pcot_run_batched(pcot_handle h, int nb, void *const *grids, const int64_t *sizes,
                             const int64_t *strides, const int64_t *T, pcot_dtype dtype,
                             const pcot_tile_params *params, void *workspace,
                             size_t workspace_bytes, uint64_t *done_ns, void *stream);

/* ------------------------------------------------------------------------
 * Exhaustive autotuner (the GPU counterpart of the tile-size exploration of
 * Sec. 5.1.5: every candidate timed, mean over repetitions).
 *  grid, workspace  as for pcot_run; the workspace must be large enough for
 *             every candidate (pcot_workspace_bytes of the largest); the grid
 *             CONTENTS ARE ADVANCED by the timing runs (use a scratch copy)
 *  ncand      number of candidates; schedules[i] and params[i] describe one
 *  reps       timed repetitions per candidate (after one untimed warm-up)
 *  ms_out     HOST array of ncand floats: mean milliseconds of one pcot_run,
 *             or -1 for a candidate the library rejects (unsupported shape,
 *             workspace too small)
 * Synchronous: returns after the last timing.
 * ------------------------------------------------------------------------ */
pcot_status pcot_autotune(pcot_handle h, void *grid, void *workspace, size_t workspace_bytes,
                          const int64_t *sizes, const int64_t *strides, int64_t T, pcot_dtype dtype,
                          int ncand, const pcot_schedule *schedules, const pcot_tile_params *params,
                          int reps, float *ms_out, void *stream);

/* ------------------------------------------------------------------------
 * Learned tile picker.  A 12-64-64-64-2 ReLU MLP (FP32, 9282 parameters in
 * one flat array: W1 (64x12, row = output), b1, W2 (64x64), b2, W3, b3,
 * W4 (2x64), b4) maps a normalised feature vector of (problem, schedule,
 * tile parameters) to two measured quantities, normalised: the log
 * milliseconds of a run and the log slowdown against the fastest candidate
 * of the same problem (capped at log 3).  Picks minimise the second.  Training
 * and inference run in the library's kernels; all pointers are DEVICE
 * pointers unless stated.  x is batch x 12, y and targets batch x 2, all
 * row-major.
 * ------------------------------------------------------------------------ */
int pcot_mlp_param_count(void);

/* Device scratch needed by pcot_mlp_grad for a batch. */
pcot_status pcot_mlp_scratch_bytes(int batch, size_t *bytes);

pcot_status pcot_mlp_forward(const float *params, const float *x, int batch, float *y, void *stream);

/* Gradient of L = (1/batch) sum 0.5 (y - target)^2 into grad (9282 floats)
 * and L into *loss (device, may be NULL); deterministic reduction order. */
pcot_status pcot_mlp_grad(const float *params, const float *x, const float *target, int batch,
                          float *grad, float *loss, void *scratch, size_t scratch_bytes,
                          void *stream);

/* One Adam step (Kingma and Ba) with bias correction; step counts from 1. */
pcot_status pcot_mlp_adam(float *params, const float *grad, float *m, float *v, int n, int step,
                          float lr, float beta1, float beta2, float eps, void *stream);

/* *out_index (device int) = argmin over rows of y[row * stride + col]. */
pcot_status pcot_mlp_argmin(const float *y, int n, int stride, int col, int *out_index, void *stream);

/*
 * Feature vector (12 floats, HOST) of one candidate, before normalisation:
 * [dims, log2 of the tiles per time block (0 for the sweep), log2 n_0,
 *  log2 n_1, log2 n_2 (0 when absent), log2 T,
 *  log2 tile_0, log2 tile_1, log2 tile_2 (extents actually used; the grid
 *  extents for the sweep), log2 k (0 for the sweep), log2 of the leaf
 *  orthant volume in tiles (PCOT_COT) or -1 (sweep / single-level), dtype].
 * Defined for the picker's schedules (sweep, single-level, recursive):
 * PCOT_AUTO and PCOT_SKEW give PCOT_ERR_UNSUPPORTED, other values
 * PCOT_ERR_INVALID_ARG.
 */
pcot_status pcot_features(pcot_handle h, const int64_t *sizes, int64_t T, pcot_dtype dtype,
                          pcot_schedule schedule, const pcot_tile_params *params, float *out12);

/*
 * The candidates the picker chooses among for this handle's stencil and a
 * dtype (the GPU counterpart of the tile sizes explored in Sec. 5.1.5): the
 * plain sweep; the single-level schedule over time depths and tile heights;
 * for Dirichlet grids the recursive order over depths, tile heights and leaf
 * orthants.  *count receives their number; with cap >= *count the HOST
 * arrays `schedules` and `params` receive them (cap = 0 only counts;
 * a smaller nonzero cap returns PCOT_ERR_OOM).  Needs no GPU.
 */
pcot_status pcot_candidates(pcot_handle h, pcot_dtype dtype, int cap, pcot_schedule *schedules,
                            pcot_tile_params *params, int *count);

/*
 * Load the picker's model into the handle: mlp_params (9282 floats, layout
 * above), feat_mean and feat_std (12 floats each, the normalisation of the
 * pcot_features vector), all HOST memory, copied.  Passing three NULLs
 * unloads the model, after which pcot_pick falls back to the autotuner.  A
 * new handle starts with the model the library was built with (trained on
 * this library's own autotuner records), if any.  Clears the picks cached
 * by earlier pcot_pick / PCOT_AUTO calls.
 */
pcot_status pcot_picker_load(pcot_handle h, const float *mlp_params, const float *feat_mean,
                             const float *feat_std);

/*
 * Schedule and tile parameters for a problem (sizes, T, dtype).  With a
 * model loaded: the MLP predicts every candidate of pcot_candidates
 * (forward and argmin kernels on the legacy default stream) and the one with
 * the least predicted slowdown is returned.  Without a model: the
 * exhaustive autotuner (pcot_autotune, two timed runs per candidate) runs on
 * a scratch grid of the problem's size with rows padded to 128 bytes, which
 * the call allocates and frees; the fastest measured candidate is returned.
 * Picks are cached in the handle per problem, so later calls (and PCOT_AUTO
 * runs) for the same problem return at once.  Synchronous.
 */
pcot_status pcot_pick(pcot_handle h, const int64_t *sizes, int64_t T, pcot_dtype dtype,
                      pcot_schedule *schedule, pcot_tile_params *params);

/*
 * The picker's building block with an explicit model and candidate list:
 * builds the features of the ncand candidates, normalises them with
 * mean/std (HOST, 12 + 12 floats), runs the MLP forward and argmin (of the
 * predicted slowdown, output 1) kernels with the DEVICE parameters
 * `mlp_params`, returns the index in *best (HOST).  `scratch` is device memory of at least ncand * (12 + 2) * 4 + 256
 * bytes.  Synchronous.
 */
pcot_status pcot_pick_among(pcot_handle h, const int64_t *sizes, int64_t T, pcot_dtype dtype,
                            const float *mlp_params, const float *feat_mean, const float *feat_std,
                            int ncand, const pcot_schedule *schedules, const pcot_tile_params *params,
                            void *scratch, int *best, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free variant of pcot_run (the paper has no counterpart).  It
 * serves callers that may not allocate device memory at the moment they
 * advance a grid: hosts that reserve all device memory up front and forbid
 * allocation afterwards (real-time and embedded systems, services with a
 * fixed memory budget), and library layers that are handed only a grid and a
 * stream and may not touch the caller's allocator.
 *
 * Runs PCOT_SWEEP or PCOT_SLT with pcot_run's depth and tile rules, but the
 * grid's twin is a fixed array of PCOT_NOALLOC_MAX_BYTES bytes that the
 * library reserves on every GPU that loads it, for the life of the process;
 * the call allocates nothing (no cudaMalloc, no host heap).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture.  Grids whose storage span
 * exceeds PCOT_NOALLOC_MAX_BYTES return PCOT_ERR_OOM; PCOT_COT and PCOT_AUTO
 * return PCOT_ERR_UNSUPPORTED.  All calls on one device share the array:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * on it and must be serialised by the caller.  The array keeps the previous
 * call's contents; the call rewrites every cell it reads (the ring is copied
 * in first), and only the grid's stored cells are written back (the padding
 * between rows of a strided grid is left untouched).  Tiles use plain loads
 * (no TMA ring), so no device status block is needed; launch errors are
 * returned, pcot_check is not required.
 * ------------------------------------------------------------------------ */
#define PCOT_NOALLOC_MAX_BYTES (32u * 1024u * 1024u)

pcot_status pcot_run_noalloc(pcot_handle h, void *grid, const int64_t *sizes, const int64_t *strides,
                             int64_t T, pcot_dtype dtype, pcot_schedule schedule,
                             const pcot_tile_params *params, void *stream);

/* ------------------------------------------------------------------------
 * Gauss-Seidel 2-D (GS-2D, one of the stencils of the paper's benchmark
 * suite, Sec. 5.1.2): T in-place steps over an (n0 + 2) x (n1 + 2) grid
 * with a fixed ring; one step visits the interior rows i = 1..n0 and, within
 * a row, the columns j = 1..n1 in increasing order and sets
 *   u[i][j] = (u[i-1][j-1] + u[i-1][j] + u[i-1][j+1] + u[i][j-1] + u[i][j]
 *              + u[i][j+1] + u[i+1][j-1] + u[i+1][j] + u[i+1][j+1]) / 9
 * (adds left to right, each rounded; one rounded division), so the north row
 * and the west neighbour are already this step's values.  The GPU runs tiles
 * of the skewed space (t, t + i, 2t + i + j) (Sec. 4.1), in which every
 * dependence has non-negative components, with a persistent executor:
 *   PCOT_SWEEP  tiles one step deep (time_depth 1), wavefront order;
 *   PCOT_SLT    tiles time_depth steps deep, wavefront order (tiles with
 *               equal b0 + b1 + b2 are independent and run together);
 *   PCOT_COT    the recursive order of Sec. 4.2-4.3 over the tile lattice
 *               (orthants with equal numbers of upper halves side by side).
 * Every dtype evaluates the definition's operations in its order: PCOT_F64
 * and PCOT_F64_EXACT are bitwise equal to the plain loop nest in binary64;
 * PCOT_F32 rounds each operation to binary32.
 *
 * sizes: {n0, n1} interior rows and columns.  strides: {row stride, 1} or
 * NULL (row stride n1 + 2).  params: tile = {ha, wc} skewed rows and
 * columns per tile (default 32, 128; ha * time_depth <= 1024 threads, wc >= 2),
 * time_depth = kt (default 1 for PCOT_SWEEP, else 8), cot_threshold[0..2] =
 * recursion leaf in tiles along (t, a, c) (default 32, 32, 32).  The handle
 * supplies the device status block (its coefficients are not used).  The
 * workspace (device, 256-byte aligned, pcot_gs2d_workspace_bytes) holds the
 * tile queue and dependency counters.  Asynchronous on `stream`; a
 * dependency wait that times out is reported by pcot_check.
 * ------------------------------------------------------------------------ */
pcot_status pcot_gs2d_workspace_bytes(const int64_t *sizes, int64_t T, pcot_schedule schedule,
                                      const pcot_tile_params *params, size_t *bytes);
pcot_status pcot_gs2d_run(pcot_handle h, void *grid, void *workspace, size_t workspace_bytes,
                          const int64_t *sizes, const int64_t *strides, int64_t T, pcot_dtype dtype,
                          pcot_schedule schedule, const pcot_tile_params *params, void *stream);
/*
 * The GS-2D tile plan without running it (host only, no GPU needed):
 * lattice[3] tiles along (t, a, c), tile[3] = {kt, ha, wc}, *n_tiles the
 * number of non-empty tiles; queue (n_tiles entries, linear ids
 * (b0 * L1 + b1) * L2 + b2 in execution order) and deps (L0 * L1 * L2
 * entries: predecessors of each id among its seven lower neighbours that hold
 * points) are filled up to cap entries when not NULL.
 */
pcot_status pcot_gs2d_plan_query(const int64_t *sizes, int64_t T, pcot_schedule schedule,
                                 const pcot_tile_params *params, int32_t *lattice, int32_t *tile,
                                 int64_t *n_tiles, int32_t *queue, int32_t *deps, int64_t cap);

/* ------------------------------------------------------------------------
 * FDTD-2D (the two-dimensional FDTD kernel of the paper's benchmark suite,
 * Sec. 5.1.2): three fields ex, ey, hz of nx x ny values (row stride s, the
 * same for all three; strides {s, 1} or NULL for s = ny) advanced T steps.
 * Step t:
 *   ey[0][j] = fict[t];  ey[i][j] -= 0.5 * (hz[i][j] - hz[i-1][j])   (i >= 1)
 *   ex[i][j] -= 0.5 * (hz[i][j] - hz[i][j-1])                          (j >= 1)
 *   hz[i][j] -= 0.7 * (((ex[i][j+1] - ex[i][j]) + ey[i+1][j]) - ey[i][j])
 *                                  (i <= nx-2, j <= ny-2; ex, ey of step t)
 * each product and difference separately rounded in that order (no fused
 * multiply-add): PCOT_F64 and PCOT_F64_EXACT are bitwise the loop nest in
 * binary64, PCOT_F32 rounds the same operations to binary32.  fict: T values
 * of the field type (device).  Schedules: PCOT_SWEEP one launch per step;
 * PCOT_SLT tiles of tile[0] x tile[1] outputs advanced time_depth steps in
 * shared memory (overlapped tiles, halo = time_depth; tiles at least
 * time_depth wide; defaults 32 x 32 x 4 for FP64, 48 x 64 x 8 for FP32);
 * PCOT_COT the same tiles as leaves of the recursive order over the
 * (block, tile) lattice run by the persistent executor (cot_threshold =
 * leaf in blocks, y-tiles, x-tiles; default 2, 256, 256), the remaining
 * T mod time_depth steps as one single-level block.  The workspace (device,
 * 256-byte aligned, pcot_fdtd2d_workspace_bytes) holds a second copy of the
 * three fields and the recursive schedule's queue; the result is always in
 * ex, ey, hz.  Asynchronous on `stream`; pcot_check reports device errors.
 * ------------------------------------------------------------------------ */
pcot_status pcot_fdtd2d_workspace_bytes(const int64_t *sizes, const int64_t *strides, int64_t T,
                                        pcot_dtype dtype, pcot_schedule schedule,
                                        const pcot_tile_params *params, size_t *bytes);
pcot_status pcot_fdtd2d_run(pcot_handle h, void *ex, void *ey, void *hz, const void *fict, void *workspace,
                            size_t workspace_bytes, const int64_t *sizes, const int64_t *strides, int64_t T,
                            pcot_dtype dtype, pcot_schedule schedule, const pcot_tile_params *params,
                            void *stream);

/* ------------------------------------------------------------------------
 * LU and Cholesky factorizations (the linear-algebra kernels of the paper's
 * benchmark suite, Sec. 5.1.2), whose iteration spaces are triangular: the
 * recursion over their bounding box skips empty orthants (Sec. 4.3).
 *
 * A: n x n binary64 matrix (device, 8-byte aligned), row-major with row
 * stride lda >= n elements, factored in place.
 *   PCOT_LA_LU        Gaussian elimination without pivoting: for k = 0..n-1,
 *                     A[i][k] /= A[k][k] (i > k), then
 *                     A[i][j] -= A[i][k] * A[k][j] (i, j > k); the result
 *                     holds the unit lower factor below the diagonal and the
 *                     upper factor on and above it.  No pivoting: a zero or
 *                     tiny pivot gives infinities or NaNs, as in the loops.
 *   PCOT_LA_CHOLESKY  lower Cholesky factor: for k = 0..n-1,
 *                     A[k][k] = sqrt(A[k][k]), A[i][k] /= A[k][k] (i > k),
 *                     A[i][j] -= A[i][k] * A[j][k] (k < j <= i); only the
 *                     lower triangle is read or written.
 * Each element receives its updates for k ascending, then its division (or
 * square root), so every schedule is bitwise the loops above: PCOT_F64 with
 * each update one fused multiply-add, PCOT_F64_EXACT with a rounded product
 * and a rounded difference.  PCOT_F32 is not supported.
 * Schedules: PCOT_SWEEP the plain loop over k (two launches per k);
 * PCOT_SLT tiles of b x b x b points of the (k, i, j) space, block step by
 * block step: a launch for the panels and one for the updates (the next
 * step's diagonal tile is factored inside the update launch, by the CTA that
 * updates that block);
 * PCOT_COT the same tiles in the recursive order over the tile lattice
 * (orthants with equal numbers of upper halves side by side, leaves
 * lexicographic), run by a persistent kernel that waits (bounded) on
 * per-tile dependency counters.  params: tile[0] = b (32 or 64, default 32),
 * cot_threshold[0..2] = recursion leaf in tiles along (k, i, j) (default
 * 2, 32, 32); other fields are ignored.  The workspace (device, 256-byte
 * aligned, pcot_la_workspace_bytes; 0 bytes except for PCOT_COT) holds the
 * queue and the counters.  The handle supplies the device status block (its
 * coefficients are not used).  Asynchronous on `stream`; a dependency wait
 * that times out is reported by pcot_check.
 * ------------------------------------------------------------------------ */
typedef enum { PCOT_LA_LU = 0, PCOT_LA_CHOLESKY = 1 } pcot_la_kind;

pcot_status pcot_la_workspace_bytes(pcot_la_kind kind, int64_t n, pcot_schedule schedule,
                                    const pcot_tile_params *params, size_t *bytes);
pcot_status pcot_la_run(pcot_handle h, pcot_la_kind kind, void *A, void *workspace, size_t workspace_bytes,
                        int64_t n, int64_t lda, pcot_dtype dtype, pcot_schedule schedule,
                        const pcot_tile_params *params, void *stream);
/*
 * The tile plan without running it (host only, no GPU needed): *L tiles per
 * side, *b the tile side, *n_tiles the number of non-empty tiles; queue
 * (n_tiles ids (kb * L + ib) * L + jb in execution order: lexicographic for
 * PCOT_SLT, recursive for PCOT_COT) and deps (L^3 entries: predecessors of
 * each id in the tile graph) are filled up to cap entries when not NULL.
 */
pcot_status pcot_la_plan_query(pcot_la_kind kind, int64_t n, pcot_schedule schedule,
                               const pcot_tile_params *params, int32_t *L, int32_t *b, int64_t *n_tiles,
                               int32_t *queue, int32_t *deps, int64_t cap);

/*
 * Number of kernels this handle has launched since it was created (sweep
 * steps, single-level blocks, persistent executors, ring copies, sums).
 * Host-side counter; lets a caller state how many of its GPU launches were
 * the library's.
 */
pcot_status pcot_launch_count(pcot_handle h, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* PCOT_H */
