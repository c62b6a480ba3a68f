/*
 * cddt.h -- C ABI of the GB300 CDDT library (libcddt.so).
 *
 * Compressed Directional Distance Transform ray casting fused with the beam
 * sensor model of Monte Carlo localization (Walsh & Karaman, arXiv
 * 1705.01167).  Section citations below refer to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers whose name ends in _dev are device memory owned by the caller
 *    (for example torch tensors); the library never frees them.  Pointers
 *    ending in _host are host memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Calls that launch work are stream-ordered and return
 *    before it finishes unless stated otherwise.
 *  - A handle (cddt_t) owns all device memory of one CDDT: the zero-point
 *    store, the slice tables and a private copy of the occupancy grid (the
 *    update writes it).  A handle is bound to the device that was current
 *    when it was built; every call on it must run with that device current.
 *    A handle is not thread-safe: serialise calls on one handle.
 *  - Every call returns a cddt_status and never aborts the process.
 *    Argument errors are detected on the host before any launch.  A kernel
 *    that detects bad input (for example an out-of-map cell in an update)
 *    records CDDT_ERR_DEVICE in the handle's device status word and skips
 *    that item; cddt_get_status() reports and clears it.
 *  - Coordinates are in cells.  Cell (i, j) is grid[j*W + i], centred on
 *    the integer point (i, j); theta is in radians from +x toward +y.
 *  - The CUDA extension does no work on the CPU: without a CUDA device
 *    every call returns CDDT_ERR_CUDA.
 */
#ifndef CDDT_H
#define CDDT_H

#include <stdint.h>

#if defined(__GNUC__)
#define CDDT_API __attribute__((visibility("default")))
#else
#define CDDT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cddt_s *cddt_t;

typedef enum {
    CDDT_OK = 0,
    CDDT_ERR_ARG = 1,     /* invalid argument (detected on the host)               */
    CDDT_ERR_CUDA = 2,    /* a CUDA runtime call failed, or no CUDA device          */
    CDDT_ERR_OOM = 3,     /* device allocation failed                               */
    CDDT_ERR_PRUNED = 4,  /* incremental update of a pruned CDDT (Section IV-D)     */
    CDDT_ERR_TIMEOUT = 5, /* a bounded device-side wait gave up                     */
    CDDT_ERR_DEVICE = 6,  /* a kernel flagged bad input; see cddt_get_status        */
    CDDT_ERR_BOUNDS = 7   /* (CDDT_CHECKED builds) a gather failed its bounds check  */
} cddt_status;

/* Build flags. */
#define CDDT_ZP_U16 1u /* 16-bit zero points (Section IV-C, "16 bit integers")     */

/* Search layouts for queries (cddt_set_search).  Both give identical answers. */
#define CDDT_SEARCH_TREE 0   /* implicit 8-ary max-separator tree over each bin     */
#define CDDT_SEARCH_BINARY 1 /* branch-free binary search of the sorted bin          */

/* Beam sensor model (Section VI, "beam mode sensor model"; the mixture of the
 * textbook beam model).  p(z | z*) = z_hit p_hit + z_short p_short + z_max
 * p_max + z_rand p_rand with
 *   p_hit   = N(z; z*, sigma_hit^2), optionally divided by its mass on
 *             [0, max_range] when hit_truncnorm != 0
 *   p_short = lambda e^{-lambda z} / (1 - e^{-lambda z*}) for 0 <= z <= z*,
 *             z* > 0; else 0
 *   p_max   = 1 if z >= max_range else 0
 *   p_rand  = 1/max_range if z < max_range else 0
 * where z is the measured range clamped to [0, max_range] and z* the CDDT
 * range.  The weights are used as given (not renormalised). */
typedef struct {
    float z_hit, z_short, z_max, z_rand;
    float sigma_hit;
    float lambda_short;
    float max_range;
    int32_t hit_truncnorm;
} cddt_beam_model;

typedef struct {
    int32_t W, H, theta_disc, n_slices; /* n_slices = theta_disc / 2 stored slices   */
    float max_range;
    uint32_t flags;
    int32_t pruned;
    int64_t total_bins;
    int64_t n_zero_points;   /* zero points stored (after pruning / updates)      */
    int64_t n_edge_cells;    /* edge cells at build time                          */
    int64_t store_bytes;     /* bytes of the zero-point store incl. tree nodes    */
    int64_t max_bin;         /* largest bin                                       */
    float build_ms, prune_ms, update_ms; /* device time of the last such call     */
} cddt_stats;

/* Build a CDDT from an occupancy grid (Section IV-A, direct construction).
 *   grid_dev    uint8 [H][W], nonzero = occupied; read during the call only.
 *   W, H        1 .. 32767.
 *   theta_disc  N >= 2, even: directions 2 pi k / N over the full circle;
 *               N/2 slices are stored (Section IV-C symmetry).
 *   max_range   > 0, in cells; ranges are clamped to it.
 *   flags       0 or CDDT_ZP_U16.
 *   out         receives the handle.
 * Synchronises `stream` (allocation sizes depend on the zero-point count).
 * Errors: ARG, CUDA, OOM. */
CDDT_API cddt_status cddt_build(const uint8_t *grid_dev, int32_t W, int32_t H, int32_t theta_disc,
                       float max_range, uint32_t flags, void *stream, cddt_t *out);

/* Free every device buffer of the handle (synchronises the device first).
 * NULL is accepted. */
CDDT_API cddt_status cddt_destroy(cddt_t h);

/* Prune (Section IV-C, PCDDT): remove every zero point that no query from a
 * free cell can return; answers of such queries do not change.  A pruned
 * handle rejects cddt_update_cells (Section IV-D).  Synchronises `stream`.
 * Errors: ARG, CUDA, OOM, PRUNED (already pruned). */
CDDT_API cddt_status cddt_prune(cddt_t h, void *stream);

/* Incremental update (Section IV-D): apply n cell writes in order, later
 * writes to the same cell winning.  xy_dev int32 [n][2] = (x, y) cells,
 * occ_dev uint8 [n] (nonzero = occupied).  Afterwards the zero points equal
 * those of cddt_build on the updated grid, including obstacles revealed or
 * hidden by the edge-map erosion.  Writes outside the map are skipped and
 * flag CDDT_ERR_DEVICE.  May synchronise `stream` when the store must grow.
 * Errors: ARG, CUDA, OOM, PRUNED. */
CDDT_API cddt_status cddt_update_cells(cddt_t h, const int32_t *xy_dev, const uint8_t *occ_dev, int32_t n,
                              void *stream);

/* Ray casting (Section IV-B query, Section IV-C reverse search): n queries
 * pose_dev float [n][3] = (x, y, theta) -> range_dev float [n].  A query whose
 * nearest cell is occupied or off the map returns 0; a ray that meets no
 * zero point returns max_range.  sort_by_slice != 0 first orders the queries
 * by slice and direction (a counting sort on the device) so that the gathers
 * of one slice run together and reach DRAM about once per slice; the answers
 * are the same.  scratch: with sort_by_slice the handle keeps an internal
 * scratch of 16 bytes per query plus 4 bytes per (bucket, sort block) --
 * at most 1024 buckets, two per stored slice, and a few hundred blocks --
 * grown on demand (growing synchronises `stream`).  Errors: ARG, CUDA, OOM. */
CDDT_API cddt_status cddt_calc_range_many(cddt_t h, const float *pose_dev, float *range_dev, int64_t n,
                                 int32_t sort_by_slice, void *stream);

/* Ray casting as cddt_calc_range_many (unsorted), one query per thread,
 * with the latency of every warp of 32 consecutive queries: warp_cycles_dev
 * int64 [ceil(n / 32)] receives the SM clock cycles between the warp reading
 * its poses and its last range being written.  The GPU counterpart of the
 * paper's per-query completion times (its latency violins, Section V):
 * cycles per warp of queries, not per query.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_calc_range_timed(cddt_t h, const float *pose_dev, float *range_dev, int64_t n,
                                           int64_t *warp_cycles_dev, void *stream);

/* Slice-sorted ray casting that allocates no device memory.  The paper has
 * no counterpart: this entry point serves callers that cannot call
 * cudaMalloc while they run -- an application that reserves all device
 * memory up front and gives libraries fixed budgets, or a real-time loop that
 * forbids allocation after start-up.  It returns the same ranges as
 * cddt_calc_range_many(h, pose_dev, range_dev, n, 1, stream), but keeps its
 * scratch in one fixed buffer of about 4.7 MB that is part of the library's
 * device image (held on every device that loads the library until the
 * process exits) instead of memory the handle allocates.
 *   n            0 .. CDDT_NOALLOC_MAX_QUERIES queries (float [n][3] poses,
 *                float [n] ranges, device memory owned by the caller).
 *   theta_disc   of the handle at most CDDT_NOALLOC_MAX_THETA_DISC.
 * Larger inputs return CDDT_ERR_ARG without launching anything.
 * The first call on a device looks up the buffer's device address (a
 * one-time set-up per device, under a lock); make that first call before any
 * stream capture.  The address is kept for the life of the process, so the
 * entry point is not valid on a device after cudaDeviceReset of that device
 * (the reset discards the buffer the address points to).  Every call shares the one buffer, which keeps the last
 * call's contents (nothing in it needs to start at zero): calls whose GPU
 * work overlaps -- on different streams, or from different threads -- race
 * on it, so the caller must order them.  The call calls no cudaMalloc,
 * cudaFree or allocating library routine.  Errors: ARG, CUDA. */
#define CDDT_NOALLOC_MAX_QUERIES 262144
#define CDDT_NOALLOC_MAX_THETA_DISC 2048
CDDT_API cddt_status cddt_calc_range_many_noalloc(cddt_t h, const float *pose_dev, float *range_dev,
                                                  int64_t n, void *stream);

/* Fused sensor model (Section VI): for every particle p, log w_p =
 * sum_i log p(obs_i | z*_i), z*_i the CDDT range from (x_p, y_p) at theta_p +
 * beam_off_i (one float32 add).
 *   particles_dev float [P][3]; beam_off_dev, obs_dev float [B] (shared by all
 *   particles); logw_dev float [P]; ranges_dev float [P][B] or NULL.
 *   pair_offset D: 0, or the index distance between opposite beams
 *   (beam_off[i + D] - beam_off[i] = pi, B/2 <= D < B).  Paired beams whose
 *   directions fall on the same stored slice share one search (Section IV-C);
 *   D only affects speed, never the result.
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_sensor_weights(cddt_t h, const float *particles_dev, int64_t P,
                                const float *beam_off_dev, const float *obs_dev, int32_t B,
                                int32_t pair_offset, const cddt_beam_model *m, float *logw_dev,
                                float *ranges_dev, void *stream);

/* Adjoint of cddt_sensor_weights: grad_xy_dev float [P][2] = grad_logw_p *
 * d log w_p / d(x_p, y_p).  The range is linear in the rotated abscissa
 * x' = x cos(theta_k) + y sin(theta_k) (Section IV-B), so the derivative of
 * z* by (x, y) is -(cos, sin) of the discrete direction (+ for the reverse
 * search); it is 0
 * for a clamped range, a miss, and a particle in an occupied or off-map
 * cell.  The derivative in theta is 0 almost everywhere (theta is rounded to
 * a slice) and is not returned.  Recomputes the searches.
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_sensor_weights_backward(cddt_t h, const float *particles_dev, int64_t P,
                                         const float *beam_off_dev, const float *obs_dev,
                                         int32_t B, int32_t pair_offset, const cddt_beam_model *m,
                                         const float *grad_logw_dev, float *grad_xy_dev,
                                         void *stream);

/* Forward and adjoint in one pass: logw_dev [P] and grad_xy_dev [P][2] with
 * grad_logw = 1.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_sensor_weights_fwd_bwd(cddt_t h, const float *particles_dev, int64_t P,
                                        const float *beam_off_dev, const float *obs_dev,
                                        int32_t B, int32_t pair_offset, const cddt_beam_model *m,
                                        float *logw_dev, float *grad_xy_dev, void *stream);

/* ---------------------------------------------------------------- batched */

/* One filter of a batch: its CDDT, particles, scan and model.  Several
 * filters may share a handle (for example successive filter steps on one
 * map).  All pointers are owned by the caller and must stay valid while the
 * plan is used.  They are device memory, or page-locked host memory
 * (cudaHostAlloc / cudaMallocHost, which kernels address directly under
 * unified addressing): the plan's kernel then reads the particles and writes
 * the log-weights across the host link itself, with no separate copy; the
 * host may read logw once `stream` has passed the run. */
typedef struct {
    cddt_t map;
    const float *particles_dev; /* [P][3] */
    int64_t P;
    const float *beam_off_dev; /* [B] */
    const float *obs_dev;      /* [B] */
    int32_t B;
    int32_t pair_offset;
    cddt_beam_model model;
    float *logw_dev; /* [P] */
    /* outputs of cddt_plan_refine only (may be NULL otherwise): */
    float *grad_xy_dev;       /* [P][2] d log w / d(x, y) at the refined pose */
    float *particles_out_dev; /* [P][3] refined poses (may equal particles_dev) */
} cddt_filter;

typedef struct cddt_plan_s *cddt_plan;

/* Make a plan that weights many filters (maps of any size, any theta_disc,
 * any particle count) in one persistent launch.  Blocks take work items
 * (filter, particle range) from a device work queue.  The work table is
 * uploaded here; the plan keeps its own copy of the filter descriptors.
 * Synchronises `stream`.  Errors: ARG, CUDA, OOM. */
CDDT_API cddt_status cddt_plan_create(const cddt_filter *filters_host, int32_t n_filters, void *stream,
                             cddt_plan *out);

/* Pick block size, threads per particle and particles per work item by
 * timing candidate launches on `stream` (the plan's filters are evaluated
 * several times; outputs are overwritten).  Synchronises `stream`.
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_plan_autotune(cddt_plan p, void *stream);

/* Set the launch shape by hand: tpp in {1,2,4,8,16,32} threads per particle, ppi
 * particles per work item (multiple of 32 / tpp), block threads in {256,
 * 512}, regcap 0 (registers as the compiler needs) or 1 (capped so that 48
 * warps stay resident per SM).  A new shape discards a graph that
 * cddt_plan_launch_graph captured with the old one (its next call captures
 * again).  Errors: ARG. */
CDDT_API cddt_status cddt_plan_set_shape(cddt_plan p, int32_t tpp, int32_t ppi, int32_t block,
                                         int32_t regcap);
CDDT_API cddt_status cddt_plan_get_shape(cddt_plan p, int32_t *tpp, int32_t *ppi, int32_t *block,
                                         int32_t *regcap);

/* Run the plan on `stream`: reset the queue and launch once.  Safe to
 * capture in a CUDA graph.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_plan_run(cddt_plan p, void *stream);

/* Gradient pose refinement of every filter of the plan in one persistent
 * launch per key type (the differentiation extension; the range is linear
 * in the rotated abscissa, Section IV-B, so d log w / d(x, y) is the
 * adjoint of cddt_sensor_weights_backward).  Each particle, with its pose
 * held on chip, `steps` times evaluates log w and g = d log w / d(x, y) at
 * its pose and moves (x, y) += eta g / max(|g|, 1e-12), each operation a
 * correctly rounded float32 step in that order (theta is not changed); it
 * then evaluates once more.  Written per filter: logw_dev (the final log w),
 * grad_xy_dev (the final g) and particles_out_dev (the refined pose), which
 * must be set for every filter with P > 0; particles_out_dev may equal
 * particles_dev.  steps >= 0 (0: one forward + adjoint evaluation), eta >= 0,
 * tpp: lanes per particle, 0 to choose from the plan's size, else 1, 2, 4,
 * 8, 16, 32, 64, 128 or 256 (above 32 a particle spans several warps of a
 * block; results agree to float32 rounding of the per-particle sums across
 * tpp).  Safe to capture in a CUDA graph once it has run outside one
 * with the same tpp (its work table is uploaded on first use).
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_plan_refine(cddt_plan p, int32_t steps, float eta, int32_t tpp, void *stream);

/* Capture cddt_plan_run into a CUDA graph owned by the plan and launch that
 * graph on later calls of cddt_plan_launch_graph.  The capture happens on
 * the first call.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_plan_launch_graph(cddt_plan p, void *stream);

/* Number of work items of the plan. */
CDDT_API int64_t cddt_plan_items(cddt_plan p);

/* Work items per kernel launch of the next run: items_per_group int64 [4] for
 * (float32 keys, tree), (float32, binary search), (16-bit, tree), (16-bit,
 * binary search), after regrouping for any handle change.  Errors: ARG. */
CDDT_API cddt_status cddt_plan_groups(cddt_plan p, int64_t *items_per_group);

CDDT_API cddt_status cddt_plan_destroy(cddt_plan p);

/* ---------------------------------------------------------------- support */

/* Choose the search layout used by later queries (CDDT_SEARCH_*). */
CDDT_API cddt_status cddt_set_search(cddt_t h, int32_t search);

/* Size and timing figures of a handle.  Synchronises the device. */
CDDT_API cddt_status cddt_get_stats(cddt_t h, cddt_stats *out);

/* Synchronise the device and return the handle's device status word
 * (CDDT_OK, CDDT_ERR_DEVICE or CDDT_ERR_TIMEOUT), clearing it. */
CDDT_API cddt_status cddt_get_status(cddt_t h);

/* Copy the CDDT to host memory in plain CSR form, for checks and
 * checkpointing: slice_base_host int64 [n_slices + 1] (first global bin of
 * each slice), bin_start_host int64 [total_bins + 1], zp_host float
 * [n_zero_points] (for CDDT_ZP_U16 the dequantised values), each bin sorted
 * ascending.  Any pointer may be NULL to skip it.  Synchronises the device.
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_export(cddt_t h, int64_t *slice_base_host, int64_t *bin_start_host,
                        float *zp_host);

/* Checkpoint restore (no counterpart in the paper, which rebuilds a CDDT
 * instead): a new handle for the grid and parameters given, its store taken
 * from a CSR that cddt_export wrote for a handle with the same grid,
 * theta_disc, max_range and flags, instead of being constructed.  total_bins
 * is that handle's bin count (cddt_stats.total_bins; it must match the
 * parameters), bin_start_host int64 [total_bins + 1] and zp_host float
 * [bin_start_host[total_bins]] as cddt_export wrote them (each bin sorted
 * ascending; for CDDT_ZP_U16 the dequantised values, which re-quantise
 * exactly).  pruned != 0 marks a store exported from a pruned handle (updates
 * are then rejected, as on the original).  The host arrays are copied before
 * the call returns (it synchronises `stream`).  A CSR from another grid gives
 * a handle whose answers are not those of a build (no memory is accessed out
 * of bounds).  Errors: ARG (bad arguments, a bin count that does not match
 * the parameters, an unsorted bin), OOM, CUDA. */
CDDT_API cddt_status cddt_import(const uint8_t *grid_dev, int32_t W, int32_t H, int32_t theta_disc,
                                 float max_range, uint32_t flags, int32_t pruned, int64_t total_bins,
                                 const int64_t *bin_start_host, const float *zp_host, void *stream,
                                 cddt_t *out);

/* Copy the handle's occupancy grid and edge map (uint8 [H][W]) to the host.
 * Either pointer may be NULL.  Synchronises the device.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_export_grid(cddt_t h, uint8_t *grid_host, uint8_t *edge_host);

/* Per-launch work figures of a cddt_sensor_weights call with the same
 * arguments, for roofline accounting (no ranges or weights are produced):
 *   out_host int64 [7] = { traversals, beams cast, searches with a
 *   non-empty bin, sum over searches of ceil(log2(k_b + 1)) for bin size
 *   k_b, paired reverse beams, particles passing the occupancy check, sum
 *   over searches of the 32-byte sectors a binary search of the bin as a
 *   sorted CSR touches: 1 for its two offsets, plus (k_b > 0) 1 per probe
 *   while the remaining range spans more than one sector (8 float32 or 16
 *   16-bit keys) and 1 for the last sector }.
 * Synchronises `stream`.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_sensor_work(cddt_t h, const float *particles_dev, int64_t P,
                             const float *beam_off_dev, int32_t B, int32_t pair_offset,
                             int64_t *out_host, void *stream);

/* ---------------------------------------------------------------- filter steps */

/* The particle filter around the sensor model (Section I: a movement model
 * from odometry before the sensor model, resampling by belief after it).
 * The paper gives neither in equations; these are the standard forms (see
 * each).  Both work on F filters whose particles are consecutive segments of
 * one array: seg_start_dev int64 [F + 1] (device), non-decreasing, with
 * segment f = particles [seg_start[f], seg_start[f + 1]) and seg_start[F] =
 * P.  Random numbers are inputs, so a step is reproducible. */

/* Odometry motion model, in place: particles_dev float [P][3] (x, y, theta);
 * odom_dev float [F][3] the robot's motion since the last step, (dx, dy) in
 * its own frame and dtheta; noise_dev float [P][3] a noise sample per
 * particle (nx, ny, ntheta).  Each pose becomes x + a cos(theta) - b sin(theta),
 * y + a sin(theta) + b cos(theta), theta + dtheta + ntheta (wrapped into
 * [0, 2 pi) by one turn), a = dx + nx, b = dy + ny, in float32.
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_motion(float *particles_dev, int64_t P, const int64_t *seg_start_dev, int32_t F,
                                 const float *odom_dev, const float *noise_dev, void *stream);

/* Low-variance (systematic) resampling of each filter: weights
 * w_i = exp(logw_i - max logw) and running sums C_i in double; output
 * particle m of a filter of n particles is input particle
 * i = min{ i : C_i > (u0 + m) / n * C_{n-1} } (the last one if none).
 * Where exp(logw - max) is undefined: a filter with no log-weight above
 * -inf (all -inf or NaN) weighs every particle 1 (each is kept once, in
 * order); otherwise a NaN log-weight weighs 0, and when the largest is +inf
 * exactly the +inf particles weigh 1.
 * particles_dev float [P][3] and logw_dev float [P] in, out_dev float
 * [P][3] (not particles_dev) out,
 * index_dev int32 [P] (optional, NULL to skip) the chosen input index
 * within the filter, u0_dev float [F] one uniform offset in [0, 1) per
 * filter, scratch_dev double [P] the running sums.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_resample(const float *particles_dev, const float *logw_dev, const int64_t *seg_start_dev,
                                   int32_t F, const float *u0_dev, float *out_dev, int32_t *index_dev,
                                   double *scratch_dev, void *stream);

/* ---------------------------------------------------------------- baselines */

/* The Bresenham line caster of Section II (the paper's BL baseline) over the
 * handle's grid and max_range: pose_dev float [n][3] -> range_dev float [n].
 * The walk runs over the digital line from the query's cell floor(p + 1/2)
 * to floor(p + max_range (c, s) + 1/2) and stops at the first occupied cell;
 * (c, s) is the heading's direction by the baseline rule (float32: the
 * remainder modulo pi/2 in three fused parts, Taylor polynomials to degree
 * 9 and 10, within 2 ulp), the end point one fused multiply-add per
 * coordinate.  The range is the float32 distance from the query point to
 * the hit cell's centre, clamped to max_range; 0 from an occupied or
 * off-map cell or a non-finite coordinate; max_range when the walk leaves
 * the map or reaches its end without a hit.  Its cost grows with the free
 * distance along the ray (the long tail the paper measures).
 * Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_cast_bresenham(cddt_t h, const float *pose_dev, float *range_dev, int64_t n,
                                         void *stream);

/* The ray marching caster of Section II (the paper's RM baseline): a
 * Euclidean distance transform of the handle's grid, precomputed once, and a
 * march that advances each ray by the transform's value at the cell it
 * stands on.  The transform is a snapshot: after cddt_update the caller
 * builds a new one (the precomputation the paper names as ray marching's
 * cost on a changing map). */
typedef struct cddt_rm_s *cddt_rm;

/* Build the transform of handle h's current grid: float [H][W], cell (i, j)
 * at j * W + i holds the distance between its centre and the nearest
 * occupied cell's centre, the square root (double, rounded to float) of an
 * exact integer squared distance; W + H everywhere on a map without an
 * occupied cell.  4 * W * H bytes of device memory owned by the object, plus
 * 2 * W * H bytes of scratch during the build (stream-ordered).  Keeps h's
 * max_range.  The transform is written on `stream`: a caller that uses it on
 * another stream synchronises first.  Errors: ARG (NULL, or h not on the
 * current device), OOM, CUDA. */
CDDT_API cddt_status cddt_rm_build(cddt_t h, void *stream, cddt_rm *out);
CDDT_API cddt_status cddt_rm_destroy(cddt_rm r);
/* The transform's device pointer (owned by r, valid until destroy) and its
 * size in bytes; either out-pointer may be NULL.  Errors: ARG. */
CDDT_API cddt_status cddt_rm_distances(cddt_rm r, const float **dist_dev, int64_t *bytes);

/* Ray casts by marching: pose_dev float [n][3] -> range_dev float [n];
 * steps_dev int32 [n] (optional, NULL to skip) the transform reads of each
 * ray.  With (c, s) the heading's direction by the baseline rule (as
 * cddt_cast_bresenham) and t = 0, each sample reads the cell floor(fma(t, (c, s), (x, y)) + 1/2): off the
 * map ends the ray at max_range, a zero distance (an occupied cell) returns
 * t, otherwise t += distance, and t >= max_range returns max_range.  0 from
 * an occupied or off-map cell or a non-finite coordinate.  The returned
 * sample lies in an occupied cell, at or beyond the ray's true first
 * contact; a ray that grazes a corner can step past it.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_rm_calc_range_many(cddt_rm r, const float *pose_dev, float *range_dev,
                                             int32_t *steps_dev, int64_t n, void *stream);

/* ---------------------------------------------------------------- lookup table */

/* The paper's main comparison (Section II, Table I): a three-dimensional
 * lookup table of the range of every discrete state (cell centre (i, j),
 * direction theta_k = 2 pi k / N), 16-bit entries, built on the GPU by casting
 * every state through a CDDT; queries snap to their state. */
typedef struct cddt_lut_s *cddt_lut;

/* Build the table of handle h's map, theta_disc N and max_range (its
 * current store): uint16 [N][H][W], entry = round-half-up(range * scale),
 * scale = the largest power of two with max_range * scale <= 65535, so the
 * range read back is code / scale.  2 * W * H * N bytes of device memory,
 * owned by the table.  The table is written on `stream`: a caller that reads
 * it on another stream synchronises first.  Errors: ARG, OOM, CUDA. */
CDDT_API cddt_status cddt_lut_build(cddt_t h, void *stream, cddt_lut *out);
CDDT_API cddt_status cddt_lut_destroy(cddt_lut l);
/* Table bytes and scale; either pointer may be NULL.  Errors: ARG. */
CDDT_API cddt_status cddt_lut_info(cddt_lut l, int64_t *bytes, float *scale);

/* Ray casts by lookup: pose_dev float [n][3] -> range_dev float [n], the
 * entry of the query's nearest cell centre and direction index (as
 * cddt_calc_range_many discretises theta); 0 off the map or for a
 * non-finite theta.  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_lut_calc_range_many(cddt_lut l, const float *pose_dev, float *range_dev, int64_t n,
                                              void *stream);

/* The fused beam sensor model (as cddt_sensor_weights) over table reads:
 * F filters as segments of particles_dev float [P][3] (seg_start_dev int64
 * [F + 1], as cddt_motion), one scan per filter obs_dev float [F][B], shared
 * beam offsets beam_off_dev float [B]; logw_dev float [P].  Every beam is a
 * table read (no pairing).  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_lut_sensor_weights(cddt_lut l, const float *particles_dev, int64_t P,
                                             const int64_t *seg_start_dev, int32_t F, const float *beam_off_dev,
                                             const float *obs_dev, int32_t B, const cddt_beam_model *m,
                                             float *logw_dev, void *stream);

/* Measurement helper, no counterpart in the paper: read `sectors` 32-byte
 * sectors of the device buffer buf_dev (32-byte aligned; bytes >= 32, a
 * multiple of 32) at
 * pseudo-random sector indices (a hash of seed and the read's index), one
 * 256-bit load each, and XOR them into *sink_dev (device, one uint64) so
 * that the loads are not dead.  Timed by the caller, it gives the random
 * sector gather bandwidth of HBM (a buffer larger than L2) or of L2 (a
 * smaller one).  Errors: ARG, CUDA. */
CDDT_API cddt_status cddt_gather_probe(const void *buf_dev, int64_t bytes, int64_t sectors, uint64_t seed,
                                       uint64_t *sink_dev, void *stream);

/* A short message for a status code (static storage). */
CDDT_API const char *cddt_status_string(cddt_status s);

/* Library version, for checks that the right build is loaded. */
CDDT_API int32_t cddt_version(void);
/* 1 in a bounds-checked build (compiled with -DCDDT_CHECKED=1), else 0.  In
 * such a build every gather of the query, sensor-model, lookup-table build
 * and prune kernels from the slice table, the bin headers and the store is
 * checked against its buffer; one outside records CDDT_ERR_BOUNDS in the
 * handle's device status word (read and cleared by cddt_get_status) and
 * reads a zeroed dummy instead, so no kernel touches memory it does not own.
 * Results of a call that tripped a check are not valid.  Slower; for
 * testing. */
CDDT_API int32_t cddt_checked_build(void);

/* ---------------------------------------------------------------- tracing */

/* Per-call device timing without a profiler: while on (cddt_trace_enable(1),
 * or CDDT_TRACE=1 in the environment when the library first checks), every
 * C-ABI call that takes a stream records a CUDA event on it at entry and at
 * exit (none while the stream is being captured into a graph), which times
 * the device work the call enqueued plus any idle gap it left.  Off by
 * default; a call then pays one atomic load.  Errors: ARG (on not 0 or 1). */
CDDT_API cddt_status cddt_trace_enable(int32_t on);
/* Waits for the recorded events, then writes the summary since the last
 * report as CSV text into buf (cap bytes, NUL-terminated, truncated when
 * short; cap may be 0 with buf NULL) and clears it: a header line
 * "entry,calls,total_ms,mean_ms,min_ms,max_ms" and one line per traced
 * entry point.  *len (optional) receives the bytes the full text needs,
 * NUL included.  Errors: ARG. */
CDDT_API cddt_status cddt_trace_report(char *buf, int64_t cap, int64_t *len);

#ifdef __cplusplus
}
#endif

#endif /* CDDT_H */
