/*
 * ebisu.h -- C ABI of the GB300 temporally blocked stencil library.
 *
 * The library runs many Jacobi time steps of a fixed-coefficient star or box
 * stencil on one GPU.  The update it computes is the one of Section 2.1 of
 * "Revisiting Temporal Blocking Stencil Optimizations" (ICS '23; Listings 1-3,
 * benchmark shapes of Table 2):
 *
 *     u_s(x) = sum_k c_k * u_{s-1}(x + o_k),   s = 1 .. steps,
 *
 * over every interior cell x, with the offsets o_k taken in canonical order
 * (lexicographic in (dz, dy, dx)) and the sum taken as
 *     acc = c_0 * u(o_0);  acc = fma(c_k, u(o_k), acc) for k = 1 .. P-1.
 * Temporal blocking (Sections 3-4: tile-by-tile execution, circular
 * multi-queue, lazy streaming) reorders these updates without changing them,
 * so the blocked path returns bit-for-bit what the one-step-per-launch path
 * (ebisu_run_naive) returns.
 *
 * Conventions shared by every entry point
 *   - Layout: row-major, x fastest.  2D grids are (ny, nx), 3D grids
 *     (nz, ny, nx); `dims` always lists interior extents slowest first.
 *   - Dirichlet grids are stored padded by `radius` cells on every side,
 *     (n + 2r) per axis; the pad holds fixed values that are read and never
 *     changed.  Periodic grids are stored unpadded, n per axis; neighbours
 *     wrap modulo n.
 *   - Storage types: EBISU_F64 (double), EBISU_F32 (float), EBISU_BF16
 *     (bfloat16, 2 bytes).  F64 computes in double.  F32 and BF16 compute in
 *     float with the coefficients rounded to float, and round every step's
 *     result to the storage type (round to nearest even, or for BF16 on
 *     request stochastically: ebisu_plan_set_rounding), including the
 *     intermediate steps inside a temporal block.
 *   - Memory: every pointer to grid data or workspace is a device pointer
 *     owned by the caller (unless a function says host pointer).  Plans own
 *     host memory only.  `stream` is a cudaStream_t (NULL = legacy default
 *     stream); work is enqueued asynchronously on it.
 *   - Errors: argument errors are returned synchronously and nothing is
 *     enqueued.  Errors found by the kernels (a dependency wait that ran out
 *     of time, a failed launch) are reported by ebisu_sync(), which waits
 *     for the stream and reads the status word in the workspace.
 */
#ifndef EBISU_H
#define EBISU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ebisu_plan_s* ebisu_plan_t;
typedef struct ebisu_batch_s* ebisu_batch_t;
typedef struct ebisu_server_s* ebisu_server_t;

enum ebisu_status {
    EBISU_OK = 0,
    EBISU_ERR_INVALID_ARG = 1,  /* a null pointer, a bad enum or size        */
    EBISU_ERR_UNSUPPORTED = 2,  /* radius/shape/size outside what is built    */
    EBISU_ERR_CUDA = 3,         /* a CUDA runtime call failed                 */
    EBISU_ERR_OOM = 4,          /* a host allocation failed                   */
    EBISU_ERR_BUDGET = 5,       /* serving: request exceeds the HBM budget    */
    EBISU_ERR_TIMEOUT = 6,      /* a device-side wait gave up (bounded spin)  */
    EBISU_ERR_DEVICE_FAULT = 7, /* a kernel reported an inconsistent state    */
    EBISU_ERR_NOT_READY = 8,    /* serving: the request has not finished      */
    EBISU_ERR_BUSY = 9          /* serving: queue full, request rejected      */
};

/* Shapes (Table 2): star = centre + axis offsets |k| <= r; box = every
 * offset with max|k| <= r; and two 3D order-1 sets the paper gives only by
 * point count -- poisson (19 points: the 27-point box without its corners)
 * and j3d17pt (17 points; the library's reading: poisson without the two
 * z-axis neighbours, i.e. the z = 0 plane's 3x3 box plus the four in-plane
 * axis neighbours (dy,dx) = (+-1,0), (0,+-1) in each plane z = +-1). */
enum ebisu_shape { EBISU_STAR = 0, EBISU_BOX = 1, EBISU_POISSON = 2, EBISU_J3D17PT = 3 };
enum ebisu_dtype { EBISU_F64 = 0, EBISU_F32 = 1, EBISU_BF16 = 2 };
enum ebisu_boundary { EBISU_DIRICHLET = 0, EBISU_PERIODIC = 1 };
enum ebisu_rounding { EBISU_ROUND_NEAREST = 0, EBISU_ROUND_STOCHASTIC = 1 };

/* Execution parameters of a plan (the tuner's search space, Sections 5-6):
 *   tile_x, tile_y : output tile extents in x and (3D only) y; the tile is
 *                    streamed along the slowest axis (y in 2D, z in 3D),
 *                    Section 2.1.3 / 3.
 *   tile_s         : length of the streamed band along the slowest axis
 *                    (0 = the whole axis).
 *   depth          : temporal block depth t (steps fused per pass, >= 1).
 *   ctas_per_sm    : resident CTAs per SM (the paper's minimal parallelism,
 *                    Section 6.1, is one 256-thread CTA per SM).
 *   threads        : threads per CTA (multiple of 32, <= 1024).
 *   variant        : 0 = temporally blocked persistent kernel (shared-
 *                    memory queues), 1 = naive one-step-per-launch kernel
 *                    (ebisu_run then takes the naive path), 2 = register-
 *                    streaming temporally blocked kernel: in 2D one warp per
 *                    128-column strip, every time level in registers; in 3D
 *                    one warp per 64-column patch streamed along z (FP64,
 *                    radius 1 and the 13-point star: 2 rows, depth 1; FP32
 *                    and BF16 radius 1: 4 rows, depth 2 or 3 for the star,
 *                    2 for the box, poisson and j3d17pt).
 *                    depth
 *                    must be one of ebisu_plan_rs_depths(), tile_s is the
 *                    rows (2D) or planes (3D) per segment, ctas_per_sm caps
 *                    the resident 128-thread CTAs, and tile_x / tile_y are
 *                    set to the strip's output width (128 - 2*depth*radius;
 *                    3D: 64 - 2*depth*radius, 2 fewer for FP32/BF16 at even
 *                    depth) and the patch's rows.  Batches run
 *                    2D variant-2 plans with the register-streaming kernel
 *                    and every other plan with variant 0, using the last
 *                    variant-0 parameters the plan held. */
typedef struct ebisu_params {
    int32_t tile_x;
    int32_t tile_y;
    int32_t tile_s;
    int32_t depth;
    int32_t ctas_per_sm;
    int32_t threads;
    int32_t variant;
    int32_t fused_variant;  /* set by ebisu_plan_tune: the faster temporally
                             * blocked build (0 or 2).  When the tuner picks
                             * the naive kernel (variant 1), the tile and
                             * depth fields are that build's parameters, so
                             * setting variant = fused_variant runs it. */
} ebisu_params;

/* Human-readable name of a status code (static string, never NULL). */
const char* ebisu_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int ebisu_version(void);

/* Create a plan (host only; no device memory is touched).
 *   ndim      : 2 or 3.
 *   dims      : host array of ndim interior extents, slowest first, each >= 1
 *               (periodic: each >= 2*radius+1).
 *   shape     : enum ebisu_shape (Table 2 of the paper).
 *   radius    : 1..3 for star, 1..2 for box, 1 for poisson and j3d17pt
 *               (3D only).
 *   coeffs    : host array of P weights in canonical offset order
 *               (P = 2*ndim*r+1 for star, (2r+1)^ndim for box, 19 for
 *               poisson, 17 for j3d17pt); copied.
 *   dtype     : storage type (enum ebisu_dtype).
 *   boundary  : EBISU_DIRICHLET (padded, fixed pad) or EBISU_PERIODIC.
 *   out       : receives the plan.
 * The execution parameters start at the cost model's choice (Section 5-6);
 * ebisu_plan_set_params or ebisu_plan_tune may replace them. */
int ebisu_plan_create(int ndim, const int64_t* dims, int shape, int radius,
                      const double* coeffs, int dtype, int boundary,
                      ebisu_plan_t* out);

/* Create a plan from an explicit offset list (any support set; Section
 * 2.1's update with the given offsets).
 *   offsets : host array of npts (dz, dy, dx) triples (2D: dz = 0), no
 *             repeats; the radius is the largest |component| (1..3).
 *   coeffs  : npts weights, one per offset (any order: the sum is taken in
 *             canonical order, as for the named shapes).
 * A list whose set is exactly a named shape's gets that shape's kernels.
 * Any other list runs on the box of its radius (radius <= 2) with zero
 * weights on the offsets it lacks: for finite values the sum is the same,
 * at the box's arithmetic cost.  A non-star list of radius 3 returns
 * EBISU_ERR_UNSUPPORTED.  Otherwise as ebisu_plan_create. */
int ebisu_plan_create_offsets(int ndim, const int64_t* dims, int npts,
                              const int32_t* offsets, const double* coeffs,
                              int dtype, int boundary, ebisu_plan_t* out);

/* Destroy a plan.  Plans may be destroyed while work that used them is still
 * in flight: launches copy what they need. */
int ebisu_plan_destroy(ebisu_plan_t plan);

/* Number of support points P of the plan's stencil. */
int ebisu_plan_npoints(ebisu_plan_t plan, int* npts);

/* Stored element count of the plan's grid (padded extents multiplied). */
int ebisu_plan_grid_elems(ebisu_plan_t plan, int64_t* elems);

/* Read or replace the execution parameters.  set_params validates them
 * against the device (shared memory, co-residency) and returns
 * EBISU_ERR_UNSUPPORTED if they cannot run. */
int ebisu_plan_get_params(ebisu_plan_t plan, ebisu_params* p);
int ebisu_plan_set_params(ebisu_plan_t plan, const ebisu_params* p);

/* Storage rounding of a BF16 plan (the paper's kernels are FP64 only; this
 * serves the reduced-precision forms).
 *   rounding : EBISU_ROUND_NEAREST (the default: every step's FP32 result
 *              rounded to nearest even) or EBISU_ROUND_STOCHASTIC (BF16
 *              storage only, else EBISU_ERR_UNSUPPORTED).
 *   seed     : seeds the random bits of stochastic rounding.
 * Round-to-nearest BF16 storage stagnates on long runs: an update smaller
 * than half a BF16 ulp (2^-9 relative) is discarded at every step, so the
 * error against the exact solution grows with the step count.  Stochastic
 * rounding rounds x up to the next BF16 value with probability equal to the
 * discarded fraction of an ulp, which keeps the rounding unbiased.  The
 * random bits are a function of (seed, step, cell) only:
 *   pcg(v)   = PCG hash (Jarzynski and Olano, JCGT 9(3), 2020): s = v *
 *              747796405 + 2891336453; w = ((s >> ((s >> 28) + 4)) ^ s) *
 *              277803737; pcg = (w >> 22) ^ w   (32-bit arithmetic)
 *   K        = pcg(lo32(seed) ^ pcg(hi32(seed)))
 *   K_t      = pcg(K ^ t), t = 1 .. steps, the step whose result is rounded
 *   rnd      = pcg(i + K_t), i = the cell's index in the stored array mod 2^32
 *   result   = BF16 with the upper 16 bits of (bits(x) + (rnd >> 16))
 * so the blocked, naive and batched kernels round every cell of every step
 * alike and return identical results.  Stochastic rounding runs in the
 * register-streaming build (2D; 3D radius 1) and the one-step kernel; a plan
 * on the shared-memory build moves to the register-streaming one (or to the
 * one-step kernel where there is none), and ebisu_plan_set_params rejects
 * variant 0 while the rounding is stochastic.  Host only. */
int ebisu_plan_set_rounding(ebisu_plan_t plan, int rounding, uint64_t seed);
int ebisu_plan_get_rounding(ebisu_plan_t plan, int* rounding, uint64_t* seed);

/* Ablation of the shared-memory build (variant 0), to measure what each
 * element of the method contributes -- the cumulative steps of the paper's
 * performance breakdown (Section 7.4: BASE, +CMQ, +PRE, +LST, +RST):
 *   EBISU_ABLATE_REGISTER_REUSE : FP32 cells one per thread from shared
 *                                 memory (no four-cells-per-thread reuse in
 *                                 registers; FP64 already works this way);
 *   EBISU_ABLATE_LAZY           : a barrier after every level, level s
 *                                 lagging level s-1 by r planes (instead of
 *                                 lag r+1 and one barrier per plane);
 *   EBISU_ABLATE_PREFETCH       : each input plane loaded and waited for in
 *                                 the iteration that uses it;
 *   EBISU_ABLATE_CIRCULAR       : queues that shift down one slot per plane
 *                                 by copying, instead of circular indexing.
 * mask must be a cumulative step: 0 (everything on), REGISTER_REUSE,
 * REGISTER_REUSE|LAZY, REGISTER_REUSE|LAZY|PREFETCH, or all four
 * (EBISU_ERR_INVALID_ARG otherwise).  Built for the two case-study stencils
 * only: the 2D 5-point and 3D 7-point star (radius 1), FP32 and FP64
 * storage (EBISU_ERR_UNSUPPORTED otherwise).  Results are unchanged (the
 * same FMA chains); only the speed differs.  Host only. */
enum ebisu_ablate {
    EBISU_ABLATE_PREFETCH = 1,
    EBISU_ABLATE_LAZY = 2,
    EBISU_ABLATE_REGISTER_REUSE = 4,
    EBISU_ABLATE_CIRCULAR = 8
};
int ebisu_plan_set_ablation(ebisu_plan_t plan, int mask);

/* Variable coefficients (an extension; the paper's weights are fixed):
 * with a field set, every step computes
 *     u_s(x) = sum_k c_k(x) * u_{s-1}(x + o_k)
 * in canonical offset order (acc = c_0(x) u(o_0), then FMAs), the weights of
 * cell x read from `field`: a DEVICE array of P arrays laid out like the
 * stored grid (array k starts at field + k * ebisu_plan_grid_elems; the
 * entries of pad cells are unused), in the accumulation type (double for
 * EBISU_F64, float for EBISU_F32 and EBISU_BF16), owned by the caller and
 * read during every run.  Every step reads P weights per cell, which no
 * temporal blocking can spare, so such plans run the one-step kernel
 * whatever their parameters; tuning, batches and the server refuse them
 * (EBISU_ERR_UNSUPPORTED), as do stochastic rounding and ablation.
 * field = NULL restores the plan's fixed coefficients.  Host only. */
int ebisu_plan_set_coefficient_field(ebisu_plan_t plan, const void* field);

/* Temporal depths built for the register-streaming kernel (variant 2) of
 * this plan's stencil and storage type (Section 4's temporal blocking with
 * the per-level queues held in registers): *shallow <= *deep.  3D plans: 1
 * and 1 for the FP64 7- and 13-point stars and radius-1 boxes (27-point,
 * poisson, j3d17pt), 2 and 3 for the FP32 and BF16 7-point stars, 2 and 2
 * for the FP32 and BF16 radius-1 boxes, else 0 and 0 (no such kernel).  Host only; never
 * fails for a valid plan. */
int ebisu_plan_rs_depths(ebisu_plan_t plan, int* shallow, int* deep);

/* Bytes of device workspace a run of this plan needs: a control block plus
 * one grid-sized ping-pong buffer (the paper's two time levels, Listing 4). */
int ebisu_plan_workspace_bytes(ebisu_plan_t plan, size_t* bytes);

/* Run `steps` time steps: out = S^steps(in), temporally blocked.
 *   in        : device grid, read only (unless in == out).
 *   out       : device grid of the same stored shape; its Dirichlet pad is
 *               copied from `in`.  in == out is allowed.
 *   steps     : >= 0; 0 copies in to out.
 *   workspace : device memory of ebisu_plan_workspace_bytes bytes, 256-byte
 *               aligned; must not be used by another call that overlaps on
 *               the GPU.
 *   stream    : cudaStream_t.
 * Enqueues work and returns; call ebisu_sync for device-side errors. */
int ebisu_run(ebisu_plan_t plan, const void* in, void* out, int64_t steps,
              void* workspace, void* stream);

/* The same result through the naive path: one kernel launch per time step,
 * each thread reading its neighbours straight from global memory, with the
 * same per-cell summation order.  This is the reference GPU path that the
 * blocked kernel must equal bit for bit. */
int ebisu_run_naive(ebisu_plan_t plan, const void* in, void* out,
                    int64_t steps, void* workspace, void* stream);

/* ebisu_run without a caller workspace and without any allocation.  The
 * paper has no counterpart; this is a deployment convenience.
 *
 * For callers that cannot allocate device memory or hand the library a
 * workspace: hosts that own all device memory through their own pool and
 * forbid outside allocations, programs whose memory budget is fixed at
 * start-up, and latency-critical loops where an allocation, which may
 * synchronise the device, is not acceptable.
 *
 * The workspace is a fixed 64 MiB array inside the library (one per device,
 * reserved when this part of the library is first loaded on that device and
 * held until the process exits), so the plan's ebisu_plan_workspace_bytes
 * must not exceed 64 MiB: about 8.3 M FP64, 16.7 M FP32 or 33 M BF16 stored
 * cells (a 2048 x 2048 FP64 grid fits).  Larger plans return
 * EBISU_ERR_UNSUPPORTED and nothing is enqueued.
 *   plan, in, out, steps, stream : as for ebisu_run (in == out allowed).
 *   wait : 0 = enqueue and return (the kernels' status stays in the array
 *          until ebisu_sync_static reads it or the next call on the device
 *          resets it, so read it before the next call); nonzero = also
 *          wait for the stream and return the kernels' status (as ebisu_sync
 *          would).
 * Every call looks up the array's device address with the caller's device
 * current (a host-side query that allocates nothing).  The array is reserved
 * when this part of the library is loaded on a device: at the first call
 * there under lazy module loading (the default), or when the context is
 * created under CUDA_MODULE_LOADING=EAGER.  The first call on a device
 * should therefore come before any stream capture.  The serving loop's HBM
 * budget does not count the array.  Every call on a device uses the same
 * array, and the array keeps what the last call left in it; each call resets
 * the part that must start at zero (the control block) itself.  Calls whose
 * work overlaps on the GPU, on different streams or threads, race on the
 * array: serialise them. */
int ebisu_run_static(ebisu_plan_t plan, const void* in, void* out,
                     int64_t steps, void* stream, int wait);

/* Status read for ebisu_run_static with wait = 0 (no counterpart in the
 * paper): wait for `stream`, then read and clear the status word the last
 * static run on the current device left in the library's array.  Returns
 * what ebisu_sync returns.  Allocates nothing. */
int ebisu_sync_static(void* stream);

/* Wait for `stream`, then read and clear the status word that kernels of
 * the last run on `workspace` left there.  Returns EBISU_OK, EBISU_ERR_CUDA
 * (a CUDA error, whose text ebisu_last_cuda_error gives) or the kernel's
 * status (EBISU_ERR_TIMEOUT, EBISU_ERR_DEVICE_FAULT). */
int ebisu_sync(void* workspace, void* stream);

/* Text of the last CUDA error seen by this thread (static or thread-local
 * storage, never NULL). */
const char* ebisu_last_cuda_error(void);

/* Empirical autotuning (Sections 6.3-6.4: the cost model prunes, the
 * measurement decides).  Times up to `max_candidates` parameter sets from the
 * cost model's ranking, plus the naive one-step kernel, on the caller's
 * buffers (in is not modified; out and workspace are overwritten) for `steps`
 * steps each.  The plan keeps the fastest fused-kernel parameters, with
 * `variant` = 1 if the naive kernel was faster still; `best_ms` (optional)
 * receives the fastest time.  Synchronises the stream. */
int ebisu_plan_tune(ebisu_plan_t plan, const void* in, void* out,
                    int64_t steps, void* workspace, int max_candidates,
                    double* best_ms, void* stream);

/* ebisu_plan_tune for a plan that will share the GPU: `share` (0 < share
 * <= 1) is the fraction of the GPU's resident warps it can expect, e.g. its
 * cells over a batch's total cells.  The candidates' streamed bands (tile_s)
 * are sized to fill that share instead of the whole GPU, so a batch member
 * keeps tall bands and little overlap; the timing itself runs the plan
 * alone.  share = 1 is ebisu_plan_tune. */
int ebisu_plan_tune_share(ebisu_plan_t plan, const void* in, void* out,
                          int64_t steps, void* workspace, int max_candidates,
                          double share, double* best_ms, void* stream);

/* Cost model of Section 5 for the plan's current parameters on this
 * device.  All outputs are optional (NULL to skip):
 *   pred_cells_per_s : practical attainable performance PP = P x V.
 *   bound            : 0 = global memory, 1 = shared memory, 2 = FP pipe.
 *   valid_fraction   : V, the useful share of the computed cells. */
int ebisu_plan_model(ebisu_plan_t plan, double* pred_cells_per_s, int* bound,
                     double* valid_fraction);

/* The paper's practical-attainable-performance model (Section 5) evaluated on
 * caller-supplied machine and kernel figures (host only; the tuner uses the
 * same code with this device's measured figures).
 *   Eq. 2-5:  T_gm = a_gm D_gm S / B_gm,  T_sm = a_sm D_sm t S / B_sm,
 *             T_cmp = a_cmp D_cmp t / THR_cmp;  T_stencil = max of the three.
 *   Eq. 7:    P = D_all t / T_stencil  (D_all = d_cmp).
 *   Eq. 8-9:  V_SMtile = prod over the (ndim-1) tiled axes of
 *             (tile - 2 rad (t-1)) / tile  -- the tile is the region computed
 *             in the first fused step; each further step loses rad per side.
 *   Eq. 11:   V_Dtile = T_stencil / (T_stencil + T_Dsync n).
 *   Eq. 1:    PP = P V (V per `tiling`).
 *   Eq. 17:   desired depth, SM tiling: t >= a_gm D_gm B_sm / (a_sm D_sm B_gm).
 *   Eq. 18-19: desired depth, device tiling with
 *             D_gm = tx ty + (tx + ty) 2 t rad, D_sm = tx ty.
 *   Eq. 23:   smallest square device-tile side 4 a_gm B_sm rad / (a_sm B_gm).
 * Every input is a plain number (units: cells, bytes, bytes/s, flop/s, s). */
typedef struct ebisu_model_in {
    double a_gm, a_sm, a_cmp;    /* accesses (or flops) per cell             */
    double d_gm, d_sm, d_cmp;    /* cells moved / cached / computed          */
    double s_cell;               /* bytes per cell                           */
    double b_gm, b_sm, thr_cmp;  /* bandwidths (B/s), FP throughput (flop/s) */
    double t;                    /* temporal depth                           */
    double t_dsync, n_sync;      /* device-wide sync cost (s), syncs per tile */
    double tile_x, tile_y, rad;  /* SM tile (first-step region) and radius   */
    int32_t ndim;                /* 2 or 3                                   */
    int32_t tiling;              /* 0 = SM tiling, 1 = device tiling         */
} ebisu_model_in;

typedef struct ebisu_model_out {
    double t_gm, t_sm, t_cmp, t_stencil; /* seconds                          */
    double p;                            /* attainable cells/s (Eq. 7)       */
    double v_smtile, v_dtile;            /* valid proportions (Eq. 8-11)     */
    double pp;                           /* practical attainable (Eq. 1)     */
    double depth_sm, depth_device;       /* desired depth (Eq. 17, 18-19)    */
    double min_device_tile;              /* Eq. 23                           */
    int32_t bound;                       /* 0 gm, 1 sm, 2 compute            */
    int32_t reserved;
} ebisu_model_out;

int ebisu_cost_model(const ebisu_model_in* in, ebisu_model_out* out);

/* FP64 reductions over the interior of a device grid (plan's layout and
 * storage type; values are widened to double):
 *   result[0] = sum, result[1] = L2 norm, result[2] = max |value|,
 * of `a`, or of (a - b) when b is not NULL.  `result` is a HOST array of 3
 * doubles.  Uses a fixed-order tree, so the result does not depend on the
 * launch.  Synchronises the stream. */
int ebisu_reduce(ebisu_plan_t plan, const void* a, const void* b,
                 double* result, void* workspace, void* stream);

/* Batched runs: n independent problems in one persistent launch per group
 * of plans that share (ndim, shape, radius, dtype); the boundary, sizes,
 * coefficients and parameters may differ.  The work table interleaves the
 * problems' temporal blocks, so items of one problem fill the dependency
 * waits of another.  Each result equals ebisu_run of the same problem alone,
 * bit for bit.
 *   plans, in, out, steps : host arrays of n entries (in/out hold device
 *                           pointers; in[i] == out[i] is allowed).
 *   workspace             : device memory of ebisu_batch_workspace_bytes
 *                           bytes, 256-byte aligned.
 * Groups launch concurrently: each on a stream of the batch's own, forked
 * from `stream` and joined back into it by events (so the whole launch stays
 * one unit on `stream`, and stays capturable into a CUDA graph).
 * ebisu_batch_run = create + launch + destroy.  To replay a batch cheaply,
 * ebisu_batch_create uploads the work tables into the workspace once
 * (synchronising the stream); ebisu_batch_launch then enqueues only stream
 * operations (a memset, device copies, kernel launches) and may be captured
 * into a CUDA graph; ebisu_batch_sync waits and returns the first kernel
 * status; ebisu_batch_destroy frees the host handle (any time after create).
 * The plans are copied at create time. */
int ebisu_batch_workspace_bytes(int n, const ebisu_plan_t* plans,
                                const int64_t* steps, size_t* bytes);
int ebisu_batch_run(int n, const ebisu_plan_t* plans, const void* const* in,
                    void* const* out, const int64_t* steps, void* workspace,
                    void* stream);
int ebisu_batch_create(int n, const ebisu_plan_t* plans, const void* const* in,
                       void* const* out, const int64_t* steps, void* workspace,
                       void* stream, ebisu_batch_t* batch);
int ebisu_batch_launch(ebisu_batch_t batch, void* stream);
int ebisu_batch_sync(ebisu_batch_t batch, void* stream);
int ebisu_batch_destroy(ebisu_batch_t batch);

/* Serving loop (continuous batching, host thread + CUDA streams).
 *   hbm_budget : bytes of device memory the server may hold for grids and
 *                workspaces; requests are admitted while they fit.
 *   max_slots  : launches (lanes) that may run on the device at once, 1..64;
 *                0 = scale with the budget (one per 4 GiB, 4 to 32).  Each
 *                lane runs one batched launch of the requests admitted
 *                together.
 * The server allocates and frees its own device memory inside the budget. */
int ebisu_serve_create(size_t hbm_budget, int max_slots, ebisu_server_t* out);

/* Submit a request: copy `in_dev` (device grid laid out as the plan says)
 * into a resident buffer, run `steps` steps when admitted, and write the
 * result to `out_dev`.  `in_dev` may be reused once ebisu_serve_poll reports
 * the request done.  The plan is copied.  Returns EBISU_ERR_BUDGET if the
 * request alone exceeds the budget and EBISU_ERR_BUSY if the queue already
 * holds its limit of waiting requests (admission control: the request is
 * dropped; the limit is 1024 unless ebisu_serve_set_max_queue changed it).
 * *ticket receives the request id. */
int ebisu_serve_submit(ebisu_server_t s, ebisu_plan_t plan, const void* in_dev,
                       void* out_dev, int64_t steps, uint64_t* ticket);

/* Non-blocking status of a request: *done = 1 once out_dev holds the
 * result; *latency_s = seconds from submit to completion (or so far). */
int ebisu_serve_poll(ebisu_server_t s, uint64_t ticket, int* done,
                     double* latency_s);

/* Block until the request finishes (or timeout_s passes: EBISU_ERR_NOT_READY). */
int ebisu_serve_wait(ebisu_server_t s, uint64_t ticket, double timeout_s,
                     double* latency_s);

/* Counters: stats[0] submitted, [1] completed, [2] rejected, [3] queued now,
 * [4] running now, [5] peak bytes held, [6] bytes held now. */
int ebisu_serve_stats(ebisu_server_t s, int64_t* stats);

/* Admission control: most requests that may wait in the queue (>= 1). */
int ebisu_serve_set_max_queue(ebisu_server_t s, int max_queue);

/* Scheduling and admission policy (not in the paper; serving only).
 *   order      : EBISU_SERVE_FIFO (arrival order, the default) or
 *                EBISU_SERVE_SHORTEST: least estimated work first, the
 *                estimate being the request's cell updates over half its
 *                stencil's roofline (HBM over 2S/t bytes, FMA rate over 2P
 *                flops) for its storage type and depth; a request's priority
 *                is that estimate minus the time it has already waited, so
 *                large requests are delayed, never starved.
 *   max_wait_s : > 0 = admission control on predicted delay: a request is
 *                refused (EBISU_ERR_BUSY) when the work already queued,
 *                estimated as above and scaled by the running mean of
 *                measured over estimated time of finished launches, exceeds
 *                max_wait_s seconds; 0 = off (the default). */
enum ebisu_serve_order { EBISU_SERVE_FIFO = 0, EBISU_SERVE_SHORTEST = 1 };
int ebisu_serve_set_policy(ebisu_server_t s, int order, double max_wait_s);

/* Cancel a request that has not started (EBISU_ERR_NOT_READY if it has). */
int ebisu_serve_cancel(ebisu_server_t s, uint64_t ticket);

/* Drain all requests, stop the thread, free device memory. */
int ebisu_serve_destroy(ebisu_server_t s);

/* Device microbenchmarks that fill the roofline and the cost model
 * (Section 6.1: Little's law needs measured throughputs).  All outputs are
 * HOST pointers, each optional:
 *   out[0] FP64 FMA rate (flop/s, 2 per FMA), out[1] FP32 FMA rate,
 *   out[2] shared-memory load bandwidth (byte/s), out[3] device-wide
 *   barrier latency (seconds), out[4] SM count, out[5] SM clock seen (Hz).
 * The rates also replace the figures the cost model (ebisu_plan_model, the
 * tuner's ranking) uses on this device for the rest of the process, so that
 * a roofline computed from them and the model agree.
 * Synchronises the device. */
int ebisu_probe_device(double* out);

#ifdef __cplusplus
}
#endif
#endif /* EBISU_H */
