/*
 * shadowaccrual.h -- C ABI of the GB300 shadow-accumulation library (libshadowaccrual.so).
 *
 * Problem (Sec. 3.1, Sec. 7.1 of Miranda et al., "Shadow Accrual Maps", TVCG 2019):
 * given a mesh of building triangles, a set of receivers (ground raster cells or facade
 * points) and a time period sampled as a table of sun directions, count for every
 * receiver the steps it spends in building shadow ("gross shadow", also in minutes) and
 * the longest run of consecutive shadowed steps within a day, maximised over days
 * ("continuous shadow").  The sun is a directional light (Sec. 3.2); every direction in
 * the table points TOWARD the sun and must have d_z > 0.
 *
 * Frame: ENU metres, x = east, y = north, z = up, flat ground at z = 0.
 *
 * Exact target (what every exact method reproduces):
 *   shadow(r, j) = 1 iff the ray o_r + t d_j, t > t_min, meets any triangle (two-sided);
 *   ground receiver at p:                o = p,               t_min = 1e-3 m
 *   facade receiver at p, outward n:     o = p + 1e-2 m * n,  t_min = 0
 *
 * Conventions for every call:
 *   - Handles (sa_scene, sa_sun, sa_receivers) own only their internal device memory;
 *     the caller owns every buffer it passes and keeps it alive for the call.
 *   - "dev" buffers are device pointers of the current CUDA device; "host" buffers are
 *     host pointers.  Functions with a `device_ptrs` flag accept either.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and is
 *     asynchronous unless stated otherwise.  Creation calls synchronise `stream` before
 *     returning so the handle is ready for use on any stream.
 *   - Errors are returned as sa_status; no exception crosses the ABI.  sa_last_error()
 *     gives a message for the calling thread's last failure.
 *   - Integer outputs are deterministic from run to run.
 */
#ifndef SHADOWACCRUAL_H
#define SHADOWACCRUAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SA_OK = 0,
    SA_ERR_INVALID_ARG = -1,        /* bad pointer, size, flag or direction */
    SA_ERR_CUDA = -2,               /* a CUDA runtime call failed */
    SA_ERR_OOM = -3,                /* device allocation failed */
    SA_ERR_SUN_BELOW_HORIZON = -4,  /* a sun direction has d_z <= 0 */
    SA_ERR_DEGENERATE = -5,         /* non-finite vertex or receiver coordinate */
    SA_ERR_TIMEOUT = -6,            /* a bounded device-side wait gave up */
    SA_ERR_INTERNAL = -7,           /* a device-side consistency check failed */
    SA_ERR_UNSUPPORTED = -8         /* method not defined for these receivers */
} sa_status;

/* Accumulation methods.  All five count the same quantity; the first four are exact
 * (equal to the definition above away from shadow boundaries), SA_IAM is the paper's
 * approximate inverse accrual map.
 *   SA_SWEEP_TRACE    plain per-step sweep: one any-hit ray per receiver and step
 *                     through the BVH (the per-minute ray-tracing baseline, Sec. 8.1).
 *   SA_SWEEP_RASTER   per-step shadow raster of ground receivers: each step projects
 *                     the triangles onto the ground separately (the per-minute
 *                     shadow-map baseline, Sec. 8.1).  Ground grids only.
 *   SA_ACCRUAL_TRACE  ray-traced accrual: one BVH traversal per receiver and block of
 *                     <= 64 steps, whose query is the whole fan of the block's rays
 *                     (the moving-shadow observation of Sec. 3.2 applied to rays).
 *   SA_ACCRUAL_SAM    shadow accrual map (Sec. 4): one pass over the geometry serves all
 *                     the steps of a block (ground grids: the receiver-space accrual
 *                     raster) or of a run of <= 32 steps (points: a light-space map
 *                     orthogonal to the run's middle direction, tested exactly per step;
 *                     SA_OPT_POINT_RUN sets the bound).
 *   SA_IAM            inverse accrual map (Sec. 5): L source levels traced from both
 *                     ends of each block, shadow lines drawn into per-step bit vectors.
 *                     Ground grids only; approximate by design. */
typedef enum {
    SA_SWEEP_TRACE = 0,
    SA_SWEEP_RASTER = 1,
    SA_ACCRUAL_TRACE = 2,
    SA_ACCRUAL_SAM = 3,
    SA_IAM = 4
} sa_method;

typedef struct sa_scene sa_scene;
typedef struct sa_sun sa_sun;
typedef struct sa_receivers sa_receivers;

/* Message of the calling thread's most recent failed call ("" if none). */
const char* sa_last_error(void);

/* Library version, (major << 16) | minor. */
int32_t sa_version(void);

/* Process-wide tuning options (set between calls; not thread-safe against running calls).
 *   SA_OPT_SWEEP_TRAVERSAL, SA_OPT_ACCRUAL_TRAVERSAL: BVH traversal of the ray-traced
 *   methods -- 1 warp-coherent (the 32 lanes of a warp walk the node list together), 2 one
 *   traversal per lane, 0 the default (per lane for the sweep, warp-coherent for the
 *   accrual, the faster of the two on the district workload).  Results do not depend on
 *   the option.
 *   SA_OPT_RASTER_RUN: at most this many steps the ground accrual raster tests per cell
 *   set-up (1..32, default 24), and SA_OPT_POINT_RUN: at most this many steps per
 *   light-space map of point receivers (1..32, default 27); each block is split into
 *   runs of balanced lengths within the bound.  The defaults are the fastest on the
 *   district workload.  Longer runs amortise the set-up, shorter runs bound the swept
 *   region more tightly.  Results do not depend on either option.
 *   SA_OPT_KERNEL_TIMING: 1 records a CUDA event pair on the launching stream around every
 *   launch of the main kernels (below), 0 (default) records nothing.  Launches inside a
 *   stream capture, and those of sa_accumulate_grid_noalloc, are never timed.
 *   SA_OPT_BATCH_TILE_SKIP: read by sa_batch_create.  1 (default): a work item whose tile
 *   no removed building and no tower can shadow during the interval keeps the base counts
 *   without rastering; 0: every tile of every region is rastered.  Results do not depend
 *   on the option; 0 exists to measure what the skipping saves.
 * sa_get_option returns the current value, or -1 for an unknown key. */
#define SA_OPT_SWEEP_TRAVERSAL 1
#define SA_OPT_ACCRUAL_TRAVERSAL 2
#define SA_OPT_RASTER_RUN 3
#define SA_OPT_KERNEL_TIMING 4
#define SA_OPT_POINT_RUN 5
#define SA_OPT_BATCH_TILE_SKIP 6
sa_status sa_set_option(int32_t key, int32_t value);
int32_t sa_get_option(int32_t key);

/* Kernel classes timed under SA_OPT_KERNEL_TIMING. */
#define SA_KERNEL_RASTER 0       /* ground accrual raster (Sec. 4) and per-step raster */
#define SA_KERNEL_SAM_POINTS 1   /* light-space accrual map of point receivers (Sec. 4) */
#define SA_KERNEL_ACCRUAL 2      /* ray-traced accrual */
#define SA_KERNEL_SWEEP 3        /* per-step ray sweep (Sec. 8.1 baseline) */
#define SA_KERNEL_IAM 4          /* inverse accrual map line drawing (Sec. 5) */
#define SA_KERNEL_GRAPH 5        /* direction graph: edge run summaries and day-path reduce (Sec. 6) */
#define SA_KERNEL_RASTER_BIN 6   /* triangle binning of the ground raster (count and fill passes) */
#define SA_KERNEL_CONTRIB 7      /* building contribution: fan traversal of the shadowed steps (Sec. 7.2) */
#define SA_KERNEL_CLASSES 8

/* Collect the timed launches recorded since the last collection: waits for their events,
 * ADDS each launch's duration in milliseconds to ms[class] and 1 to launches[class]
 * (arrays of n entries, host memory, either may be NULL; classes >= n are dropped), and
 * empties the record.  Errors: SA_ERR_INVALID_ARG (n < 0), SA_ERR_CUDA (an event failed;
 * the others are still added). */
sa_status sa_kernel_times(double* ms, int64_t* launches, int32_t n);

/* ---------------------------------------------------------------------------- scene
 * Build a scene from an indexed triangle mesh (Sec. 8.2: the city mesh): vertices
 * float [nv][3] and triangles int32 [nt][3] (0-based vertex indices), optional int32
 * [nt] building id per triangle (NULL: all 0), n_buildings > every id.  Buffers are
 * host (device_ptrs = 0) or device (device_ptrs = 1) memory; they are copied.
 * On the device this builds a linear BVH: 30-bit Morton codes of the triangle
 * centroids, a least-significant-digit radix sort, Karras' (2012) radix-tree topology,
 * bottom-up box refit, and a depth-first node order whose escape links allow stackless
 * traversal.  Zero-area triangles are kept but never hit.  Sizes and pointers are
 * checked on the host; the contents on the device, while the BVH is built (an index out
 * of range reads no memory), and the message names the first offending vertex or
 * triangle.  The call synchronises the stream.
 * Errors: SA_ERR_INVALID_ARG (NULL pointers, nt or nv < 0, nt > 2^30, n_buildings < 0,
 * a vertex index outside [0, nv), a building id outside [0, max(n_buildings, 1))),
 * SA_ERR_DEGENERATE (a non-finite coordinate of any vertex, used or not), SA_ERR_OOM,
 * SA_ERR_CUDA.  nt = 0 is allowed. */
sa_status sa_scene_from_mesh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                             const int32_t* tri_building, int32_t n_buildings,
                             int32_t device_ptrs, void* stream, sa_scene** out);

/* Build a scene from extruded building footprints (Sec. 8.2: the city is a mesh of extruded
 * OpenStreetMap footprints).  xy float [nv][2]: vertices of every footprint, each a convex
 * counter-clockwise polygon of >= 3 vertices; poly_off int32 [n_buildings + 1]: footprint b
 * is xy[poly_off[b] .. poly_off[b+1]); heights float [n_buildings] (> 0 m).  Building b
 * becomes a closed prism: walls split into nb = max(1, ceil(h_b / band_height)) bands
 * (band_height 0: one band), two triangles per band and edge, a roof fan and a bottom fan
 * at z = 0; triangle building ids are b.  Extrusion and BVH build run on the device.  The
 * band counts are fixed here, so sa_scene_set_heights keeps the topology.
 * Errors: SA_ERR_INVALID_ARG (sizes, non-convex or clockwise footprints, heights <= 0),
 * SA_ERR_DEGENERATE, SA_ERR_OOM, SA_ERR_CUDA. */
sa_status sa_scene_from_footprints(const float* xy, const int32_t* poly_off, int32_t n_buildings,
                                   const float* heights, float band_height, int32_t device_ptrs,
                                   void* stream, sa_scene** out);

/* Replace the heights of a footprint scene (host or device float [n_buildings]) and
 * rebuild its mesh and BVH (synchronises `stream`).  SA_ERR_UNSUPPORTED for mesh scenes. */
sa_status sa_scene_set_heights(sa_scene* scene, const float* heights, int32_t device_ptrs,
                               void* stream);

/* Release a scene (NULL is ignored). Synchronises the device first. */
void sa_scene_destroy(sa_scene* scene);

/* Declare (closed = 1) that every building of the scene is a closed solid whose triangles
 * are wound counter-clockwise seen from outside.  The projection of a closed solid is
 * covered by its faces that face the sun, so the raster methods then skip the others
 * (about half the work) with the same result; the ray-traced methods are unaffected.
 * Scenes from sa_scene_from_footprints are closed from the start.  Declaring an open
 * or inward-wound mesh closed gives wrong raster results. */
sa_status sa_scene_declare_closed(sa_scene* scene, int32_t closed);

/* Triangle and BVH node counts, number of buildings, minimum vertex z. */
sa_status sa_scene_info(const sa_scene* scene, int64_t* n_tris, int64_t* n_nodes,
                        int32_t* n_buildings, float* min_z);

/* ------------------------------------------------------------------------- sun table
 * Validate and partition a per-step sun-direction table (host memory): dirs float
 * [S][3] toward the sun, |d| within 1e-5 of 1 and d_z > 0; day_start int32 [D+1] with
 * day_start[0] = 0, non-decreasing, day_start[D] = S.  Steps of a day are consecutive
 * and equally spaced in time.  Each day is cut into consecutive blocks of at most
 * block_len steps (1..64; 0 picks 60, the paper's hourly interval of one-minute steps,
 * Sec. 3.2), so every step lies in exactly one block and blocks never cross days.
 * Errors: SA_ERR_INVALID_ARG, SA_ERR_SUN_BELOW_HORIZON, SA_ERR_OOM, SA_ERR_CUDA. */
sa_status sa_sun_create(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                        int32_t block_len, void* stream, sa_sun** out);
void sa_sun_destroy(sa_sun* sun);
/* The paper's short-interval sun (Sec. 3.2, and Sec. 4, where the accrual map draws every
 * step from the first and last direction of its interval): writes a table in which every
 * block (as sa_sun_create cuts it with the same block_len) keeps its first and last
 * directions d_1, d_n and the steps between move at a constant angular rate along the
 * great circle through them: step i (i' = i - 1 = 0 .. n-1) is d_1 rotated toward d_n by
 * i' theta / (n - 1), theta = angle(d_1, d_n).  This is what the paper's tangent law
 * draws on a shadow plane orthogonal to d_1, read with n - 1 in the denominator so that
 * the last step lands on d_n.  Pass the result to sa_sun_create with the same block_len
 * to run any method in the paper's mode; comparing with the exact table measures the
 * error of the linear-motion assumption.
 *   dirs, day_start: as for sa_sun_create (host, validated the same way).
 *   dirs_out: float [S][3] host; may be dirs itself.  Blocks of 1 or 2 steps are copied.
 * FP64 arithmetic, rounded once to FP32.  Errors: as sa_sun_create's checks. */
sa_status sa_sun_interpolate(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                             int32_t block_len, float* dirs_out);

/* Number of steps, days and blocks. */
sa_status sa_sun_info(const sa_sun* sun, int32_t* S, int32_t* D, int32_t* n_blocks);

/* The block partition sa_sun_create uses (host only, Sec. 3.2's hourly intervals cut per
 * day): each day k of n = day_start[k+1] - day_start[k] steps becomes ceil(n / block_len)
 * consecutive blocks whose sizes differ by at most one, the longer ones first (481 steps,
 * block_len 60: four blocks of 54 and five of 53).  block_len 1..64, 0 for 60.
 *   day_start: int32 [D + 1] host, from 0, non-decreasing.  *n_blocks (required) receives
 *   the count; j0 and K (int32 [n_blocks] host, nullable: call once with NULLs to size
 *   them) receive each block's first step and length; mask block b of sa_shadow_masks is
 *   block b here.
 * Errors: SA_ERR_INVALID_ARG (NULL day_start or n_blocks, D < 0, day_start not from 0 or
 * decreasing, block_len outside 0..64). */
sa_status sa_block_partition(const int32_t* day_start, int32_t D, int32_t block_len,
                             int32_t* n_blocks, int32_t* j0, int32_t* K);

/* ------------------------------------------------------------------------- receivers
 * Ground raster: nx * ny cells of side dx (> 0) with lower-left corner (x0, y0); the
 * receiver of cell (ix, iy) is its centre (x0 + (ix + 0.5) dx, y0 + (iy + 0.5) dx, 0)
 * and its output index is iy * nx + ix.  Nothing is allocated per cell. */
sa_status sa_receivers_grid(float x0, float y0, float dx, int32_t nx, int32_t ny,
                            sa_receivers** out);

/* Point receivers: pos float [n][3]; normal float [n][3] outward unit normals (facade
 * receivers) or NULL (ground receivers at their own z, using the ground rule).  Host or
 * device memory per device_ptrs (host memory is copied with cudaMemcpyAsync, so pinned
 * buffers transfer fastest); sorted internally along a Morton curve so a warp holds
 * neighbouring points.  The values are checked on the device while they are sorted; the
 * call synchronises `stream` once.  Outputs always come back in input order.
 * Errors: SA_ERR_INVALID_ARG, SA_ERR_DEGENERATE (non-finite position or normal; the
 * message names the first such point), SA_ERR_OOM, SA_ERR_CUDA. */
sa_status sa_receivers_points(const float* pos, const float* normal, int64_t n,
                              int32_t device_ptrs, void* stream, sa_receivers** out);
void sa_receivers_destroy(sa_receivers* recv);
int64_t sa_receivers_count(const sa_receivers* recv);

/* ------------------------------------------------------------------------ accumulate
 * Accumulate shadow over every step of `sun` for every receiver (Sec. 3.1):
 *   gross_steps      int32 [R] dev: shadowed steps (required)
 *   gross_minutes    float [R] dev: gross_steps * step_minutes (nullable)
 *   continuous_steps int32 [R] dev: longest run of consecutive shadowed steps inside a
 *                    day, maximised over days (nullable)
 * flags: SA_ACCUMULATE_INTO adds to gross_steps and takes the max with
 *        continuous_steps already in the buffers (progressive accumulation over several
 *        calls that each cover whole days, Sec. 7.1); otherwise they are overwritten.
 * iam_levels: source levels L for SA_IAM (1..8; 0 picks 3, the paper's choice, Sec. 8.2).
 * Scratch memory is taken from the stream-ordered allocator on `stream`.
 * Errors: SA_ERR_INVALID_ARG, SA_ERR_UNSUPPORTED (raster / IAM methods on point
 * receivers, or raster methods on a scene with geometry below z = 0), SA_ERR_OOM,
 * SA_ERR_CUDA. */
#define SA_ACCUMULATE_INTO 1
sa_status sa_accumulate(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                        float step_minutes, sa_method method, int32_t iam_levels,
                        int32_t flags, int32_t* gross_steps, float* gross_minutes,
                        int32_t* continuous_steps, void* stream);

/* Per-step shadow masks: masks uint64 [n_blocks][R] dev; bit k of masks[b][r] is
 * shadow(r, first step of block b + k).  Same methods as sa_accumulate. */
sa_status sa_shadow_masks(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                          sa_method method, int32_t iam_levels, uint64_t* masks, void* stream);

/* Height gradient of the shadow-minutes of a ground grid (no counterpart in the paper, which
 * motivates height trade-offs in its case studies, Sec. 9).  Objective: between consecutive
 * steps of a day the sun moves on the great circle through their directions, at constant
 * rate over step_minutes; a receiver counts step_minutes * chi over an interval whose end
 * statuses agree, and the shadowed part of it where its status flips once.
 *   S = sum_r w_r * (those minutes),  w_r = weights[r] (dev float [R], NULL = 1).
 * Writes dS_dh (dev float [n_buildings]) and, if S_out is non-NULL, S (dev double [1]).
 * Flips come from the forward step masks (ground accrual raster); each flip time and its
 * derivative with respect to the height of the building whose roof edge casts it are
 * computed in FP64.  Needs a scene from sa_scene_from_footprints and a ground grid.
 * Errors: SA_ERR_INVALID_ARG, SA_ERR_UNSUPPORTED, SA_ERR_OOM, SA_ERR_CUDA. */
sa_status sa_height_grad(const sa_scene* scene, const sa_receivers* grid, const sa_sun* sun,
                         float step_minutes, const float* weights, float* dS_dh, double* S_out,
                         void* stream);

/* ---------------------------------------------------------------- batched scenarios
 * Impact of development variants (Sec. 7.1: the impact of a new or replaced building is
 * the difference of the two states' accumulations), many variants x sun intervals in one
 * persistent, CUDA-graph-captured launch over a ground grid.
 * A variant adds tower triangles and removes base buildings (by building id of the base
 * scene); its receivers are a rectangle of the base grid.  All arrays are host memory,
 * copied at creation:
 *   tower_tris  float [n_tower_tris][9], z >= 0      tower_off   int32 [V + 1]
 *   removed_ids int32 [n_removed]                    removed_off int32 [V + 1]
 *   regions     int32 [V][4]: first cell ix0, iy0 and size nx, ny of the region */
typedef struct {
    int32_t n_variants;
    const float* tower_tris;
    const int32_t* tower_off;
    const int32_t* removed_ids;
    const int32_t* removed_off;
    const int32_t* regions;
} sa_variants;
typedef struct sa_batch sa_batch;

/* Create a batch: the base scene's triangles are binned once per block of every interval
 * and the base counts of the whole grid are computed per interval.  A work item (interval,
 * variant, tile) is rastered only if the shadow of a removed building or of a tower, swept
 * over the interval's sun directions, can reach the tile; the others take the base counts
 * (their impact is zero).  with_impact is kept for compatibility and may be 0 or 1.
 * The scene, grid and suns must outlive the batch.  Synchronises `stream`.
 * Errors: SA_ERR_INVALID_ARG (offsets, regions outside the grid, bad towers),
 * SA_ERR_UNSUPPORTED (point receivers, geometry below z = 0), SA_ERR_OOM, SA_ERR_CUDA. */
sa_status sa_batch_create(const sa_scene* base, const sa_receivers* grid, const sa_variants* v,
                          const sa_sun* const* intervals, int32_t n_intervals,
                          int32_t with_impact, void* stream, sa_batch** out);
void sa_batch_destroy(sa_batch* b);
/* Outputs hold n_intervals x (sum of region cells); interval-major, then variant, then the
 * region's cells row by row.  sa_batch_output_offset gives the first index of (interval,
 * variant), or -1.  sa_batch_work_items is the number of (interval, variant, tile) items. */
int64_t sa_batch_output_count(const sa_batch* b);
int64_t sa_batch_output_offset(const sa_batch* b, int32_t interval, int32_t variant);
int32_t sa_batch_work_items(const sa_batch* b);
int32_t sa_batch_affected_items(const sa_batch* b);
/* Run every item: counts int32 (gross shadowed steps per receiver, dev) and, if the batch
 * has base counts and impact is non-NULL, impact int32 = variant minus base (dev).  The
 * work runs as a CUDA graph (instantiated on the first call with these output pointers)
 * holding one persistent launch that drains a work queue. */
sa_status sa_batch_run(sa_batch* b, int32_t* counts, int32_t* impact, void* stream);
/* Autotuner: times 2 to 6 persistent CTAs per SM (as many as the raster kernels are built
 * to hold) x raster runs of 8, 16 or 24 steps on an eighth of the work items and keeps the
 * fastest; reports the choice. */
sa_status sa_batch_tune(sa_batch* b, int32_t* best_ctas, int32_t* best_run, void* stream);
/* Work counters of one batch run (counters [2] cell set-ups, [3] cell-step tests). */
sa_status sa_batch_work_counters(sa_batch* b, uint64_t* counters, void* stream);

/* Work counters of one accumulation (diagnostics for roofline accounting): runs `method`
 * with counting enabled and writes counters uint64 [4] dev.
 *   trace methods: [0] ray/fan-versus-box tests, [1] ray-versus-triangle tests per
 *   receiver lane.
 *   raster methods (ground grids): [0] work units (triangle, run of steps) that reached
 *   the tile's cells, [1] cells their row spans enumerated, [2] cell set-ups (cells not
 *   already shadowed at every step of the unit), [3] cell-step coverage tests.
 *   light-space map of point receivers: [0] receiver-triangle set-ups, [1] step tests.
 * The outputs of the accumulation itself are discarded. */
sa_status sa_work_counters(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                           sa_method method, uint64_t* counters, void* stream);

/* Bounds-checked build (diagnostics, for where no memory sanitiser can run).  The library built with -DSA_CHECKED (libshadowaccrual_checked.so) range-checks
 * every index its kernels take from data -- a BVH leaf's triangle, an escape link, a
 * binned triangle or receiver, a permutation entry, a tile cell, a building id -- before
 * using it.  The first index out of range is recorded (site, index, bound) and replaced by
 * one in range (an escape link by the end of the node list), so that no access leaves its
 * buffer and no loop runs on; the computing calls (sa_accumulate, sa_shadow_masks,
 * sa_accumulate_graph, sa_height_grad, sa_building_contribution, sa_batch_run,
 * sa_accumulate_grid_noalloc) then synchronise their stream and return SA_ERR_INTERNAL
 * naming the site.  In the plain build the checks compile to nothing.
 *   sa_checked_build: 1 for the checked build, 0 for the plain one.
 *   sa_check_status: synchronises the device and returns SA_ERR_INTERNAL if a violation
 *   was recorded since the last report (writing site, index and bound, each nullable, and
 *   clearing the record), SA_OK otherwise (always SA_OK in the plain build); SA_ERR_CUDA
 *   if the device reports an error. */
int32_t sa_checked_build(void);
sa_status sa_check_status(int32_t* site, int64_t* index, int64_t* bound);

/* Statistics of the library's device memory pool (diagnostics): stats uint64 [4] host gets
 *   [0] allocations the library has made from its pool since it was loaded (all devices),
 *   [1] their bytes, summed,
 *   [2] bytes the current device's pool holds reserved (0 before its first use),
 *   [3] the pool's high-water mark of bytes in use.
 * The pool is stream-ordered, one per device.  Calls take their scratch from it and return
 * it before they end; scenes, sun tables and point receivers keep their arrays from it
 * until they are destroyed (a batch uses cudaMalloc).  The pool keeps up to 4 GiB
 * reserved between calls.  Errors: SA_ERR_INVALID_ARG (NULL). */
sa_status sa_scratch_stats(uint64_t* stats);

/* --------------------------------------------------- long periods: the direction graph
 * Sec. 6: over many days the sun retraces nearly the same arcs.  Directions fall into bins,
 * quads of the hemisphere bounded by bin_deg in elevation (bands [k b, (k+1) b) above the
 * horizon) and in azimuth (sectors [m b, (m+1) b), azimuth from +y toward +x).  A block of
 * the sun table (as sa_sun_create cuts it) becomes the pair (bin of its first direction,
 * bin of its last direction); blocks with the same pair and the same number of steps are
 * one edge of the direction graph, numbered in order of first appearance, and its weight
 * is the number of blocks it stands for.  The paper uses 5 degree bins.  An edge's map is
 * computed from one of its blocks, which the paper leaves open: here the middle one in
 * time order (member (m - 1) / 2 of its m blocks), so that the map's sun lies inside the
 * spread of the suns it stands for.
 *
 * sa_direction_graph (host only): the graph of a sun table.  *n_blocks and *n_edges
 * (required) receive the counts; edge_of_block int32 [n_blocks], map_block int32
 * [n_edges] and weight int32 [n_edges] (host, each nullable: call once with NULLs to size
 * them) receive each block's edge, the block each edge's map is computed from, and each
 * edge's weight.
 * Errors: as sa_sun_create's checks, SA_ERR_INVALID_ARG (bin_deg outside (0, 90]). */
sa_status sa_direction_graph(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                             int32_t block_len, float bin_deg, int32_t* n_blocks, int32_t* n_edges,
                             int32_t* edge_of_block, int32_t* map_block, int32_t* weight);

/* Accumulation through the direction graph (Sec. 6, approximate): one shadow map per edge,
 * computed by `method` over the edge's map block, stands for every block of the edge.
 * gross = sum over edges of the edge's count times its weight (Eq. 1); the continuous
 * count stitches each day's path of edges in time order from each edge's leading,
 * longest and trailing runs, and takes the longest over the days.  Outputs and methods as
 * sa_accumulate (SA_ACCUMULATE_INTO is not offered); *n_edges (host, nullable) receives
 * the number of maps computed, against sa_sun_info's n_blocks for the exact result.  With
 * a bin_deg small enough that no two blocks share an edge the result is sa_accumulate's.
 * Scratch: 4 bytes per receiver and edge, plus the step masks of at most 4 GiB of edges
 * at a time.  Synchronises `stream` once per chunk of edges.  Errors: as sa_accumulate,
 * SA_ERR_INVALID_ARG (bin_deg outside (0, 90]). */
sa_status sa_accumulate_graph(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                              sa_method method, int32_t iam_levels, float bin_deg, float step_minutes,
                              int32_t* gross_steps, float* gross_minutes, int32_t* continuous_steps,
                              int32_t* n_edges, void* stream);

/* ---------------------------------------------------------------- analysis measures
 * Shadow area over a polygonal region (Sec. 7.2, "Analysis measures"): the sum, over the
 * cells of a ground grid whose centre lies inside the polygon (even-odd rule), of
 * shadow(p) x area(p), with shadow(p) = steps[p] / total_steps the fraction of the
 * interval's steps the cell is in shadow, and area(p) = dx^2.  Gross counts give the gross
 * area, continuous counts the continuous one.  The paper's shadow score over intervals is
 * sa_shadow_score.
 *   grid: from sa_receivers_grid.  steps: int32 [nx * ny] device, in output order (as
 *   sa_accumulate writes it).  poly_xy: float [n][2] host, n >= 3, a simple polygon of
 *   either orientation.  total_steps > 0 (the interval's steps, e.g. S of its sun table).
 *   *area (host) receives the area in square metres, summed in FP64.
 * Cell centres are rounded as the receivers' (FP32) and tested in FP64.  Synchronises
 * `stream`.  Errors: SA_ERR_INVALID_ARG (NULL, not a grid, n < 3, total_steps <= 0),
 * SA_ERR_DEGENERATE (non-finite vertex), SA_ERR_CUDA. */
sa_status sa_shadow_area(const sa_receivers* grid, const int32_t* steps, int32_t total_steps,
                         const float* poly_xy, int32_t n, void* stream, double* area);

/* Shadow score over several intervals (Sec. 7.2, "Analysis measures"; Table 3 gives one
 * weighting, by month): the sum over intervals t of w_t x (the shadow area of interval t
 * over the polygon), i.e. the sum over the region's cells of
 * sum_t w_t x steps_t[p] / total_steps_t x dx^2, computed in one pass over the cells.
 * Positive weights count shadow as a cost (summer), negative ones as a benefit (winter).
 *   grid: from sa_receivers_grid.  steps: int32 [n_intervals][nx * ny] device, interval t's
 *   per-cell counts (gross or continuous, as sa_accumulate writes them) at
 *   steps + t * nx * ny.  total_steps: int32 [n_intervals] host, each > 0 (the interval's
 *   steps).  weights: float [n_intervals] host, each in [-1, 1].  poly_xy, n: as
 *   sa_shadow_area.  *score (host) receives the score in square metres, summed in FP64.
 * With one interval and weight 1 this is sa_shadow_area.  Synchronises `stream`.  Errors:
 * SA_ERR_INVALID_ARG (NULL, not a grid, n < 3, n_intervals < 1, total_steps <= 0, a weight
 * outside [-1, 1]), SA_ERR_DEGENERATE (non-finite vertex), SA_ERR_CUDA. */
sa_status sa_shadow_score(const sa_receivers* grid, const int32_t* steps, int32_t n_intervals,
                          const int32_t* total_steps, const float* weights, const float* poly_xy,
                          int32_t n, void* stream, double* score);

/* Building contribution to the shadow of a region (Sec. 7.2, the contribution of each
 * building to the analysis measures): for every cell of a ground grid whose centre lies
 * inside the polygon (as in sa_shadow_area) and every step of `sun` at which the cell is in
 * shadow, the ray from the cell centre toward the sun is followed through the whole scene
 * and each building it meets beyond t_min = 1e-3 is credited dx^2 / S (S = the sun table's
 * steps).
 *   casting[b]: the area building b shadows on its own, over the interval (a cell-step
 *     shadowed by several buildings is credited to each of them, so the sum over buildings
 *     is at least the region's gross shadow area).
 *   nearest[b]: the area for which b holds the nearest hit along the ray; these partition
 *     the region's shadow: their sum plus stats[1] x dx^2 / S is its gross shadow area
 *     (sa_shadow_area of the gross counts with total_steps = S).
 *   scene: any (mesh or footprints); building ids are the ones the scene was built with.
 *   grid: from sa_receivers_grid.  poly_xy: float [n][2] host, n >= 3.
 *   casting, nearest: double [n_buildings] host.  stats: int64 [2] host, nullable:
 *     [0] cell-steps whose ray met more than 64 distinct buildings (those past the 64th
 *         are not credited in casting; nearest is exact); the call then returns
 *         SA_ERR_UNSUPPORTED, with every output written;
 *     [1] cell-steps the raster marks shadowed whose ray met no triangle beyond t_min in
 *         FP32 (rays that graze a shadow edge), credited to no building.
 * The shadowed steps come from the ground accrual raster (as SA_ACCRUAL_SAM computes
 * them); the call keeps its per-step masks, 8 bytes per cell and block of steps, and
 * rejects with SA_ERR_INVALID_ARG a grid and sun table whose masks exceed 4 GiB (split the
 * interval).  The buildings are found by one traversal per cell and run of <= 32 steps,
 * whose query is the fan of the run's rays (as SA_ACCRUAL_TRACE), testing every triangle
 * in the fan against the cell's shadowed steps with the exact ray test.  Synchronises
 * `stream`.  Errors: SA_ERR_INVALID_ARG (NULL, not a grid, n < 3), SA_ERR_DEGENERATE
 * (non-finite vertex), SA_ERR_UNSUPPORTED (geometry below z = 0, as for the raster
 * methods; a ray meeting more than 64 buildings, above), SA_ERR_OOM, SA_ERR_CUDA. */
sa_status sa_building_contribution(const sa_scene* scene, const sa_receivers* grid,
                                   const sa_sun* sun, const float* poly_xy, int32_t n,
                                   void* stream, double* casting, double* nearest,
                                   int64_t* stats);

/* ------------------------------------------------------------ allocation-free variant
 * The paper has no counterpart to this call; it exists for callers that cannot allocate
 * device memory while they run -- for example a host application that reserved the
 * device's memory for itself before loading this library, or a loop that must not pay
 * the allocator's synchronisation and latency.
 *
 * Same result as sa_accumulate(..., SA_ACCRUAL_SAM, ...) on a ground grid (the ground
 * accrual raster), but it calls no cudaMalloc, cudaMallocAsync, cudaFree or other
 * allocating routine: every scratch buffer (run state, tile bins, scan partials) comes
 * from one fixed device array of SA_NOALLOC_SCRATCH_BYTES (64 MiB) compiled into the
 * library, which every GPU that loads the library keeps until the process exits.  The
 * caller still passes the outputs (as for sa_accumulate; gross_minutes and
 * continuous_steps may be NULL).
 *   - grid must come from sa_receivers_grid with at most SA_NOALLOC_MAX_CELLS cells
 *     (2048 x 2048); larger grids are rejected with SA_ERR_INVALID_ARG.  Before writing
 *     any output the call sizes the triangle-tile bins of every block and cuts the blocks
 *     into chunks that fit the scratch; if a single block's bins do not fit, it returns
 *     SA_ERR_INVALID_ARG with every output untouched (use a shorter block_len, a smaller
 *     grid or sa_accumulate).
 *   - Every call looks up the array's device address in the current device's context
 *     (cudaGetSymbolAddress); the call runs on the current device.
 *   - A sun table with no steps gives zero counts (unchanged ones with
 *     SA_ACCUMULATE_INTO), as sa_accumulate does.
 *   - All calls in the process share the one array per device and it keeps the previous
 *     call's contents (each call clears what it needs).  Calls that can overlap on the GPU
 *     -- on different streams or threads of the same device -- race on it: serialise them.
 *   - Like the other raster methods it needs scene geometry at z >= 0
 *     (SA_ERR_UNSUPPORTED otherwise) and synchronises `stream` twice per chunk of blocks
 *     to size the bins (once in the sizing pass, once before rastering the chunk). */
#define SA_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
#define SA_NOALLOC_MAX_CELLS 4194304
sa_status sa_accumulate_grid_noalloc(const sa_scene* scene, const sa_receivers* grid,
                                     const sa_sun* sun, float step_minutes, int32_t flags,
                                     int32_t* gross_steps, float* gross_minutes,
                                     int32_t* continuous_steps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SHADOWACCRUAL_H */
