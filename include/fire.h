/*
 * fire.h -- C ABI of libfire: many independent stochastic cellular-automaton
 * fire-spread simulations on one GPU, each scored against a target burnt map.
 *
 * The method is that of Denham & Laneri, "Using efficient parallelization in
 * Graphic Processing Units to parameterize stochastic fire propagation
 * models" (arXiv:1701.03549):
 *   - Eq. 1 (Sec. 2.1): a burning cell ignites a neighbouring target cell
 *     with probability p = 1 / (1 + exp(-(b0 + b1 I_f + b2 psi + b3 omega +
 *     b4 sigma))), where I_f is the forest indicator, psi = cos(aspect - 315
 *     deg) for slopes above 5 degrees, omega = cos(wind bearing - bearing from
 *     the burning cell to the target) and sigma = slope / 100 when the target
 *     lies above the burning cell;
 *   - Sec. 2.1 rules: cells are burnable, burning, burnt or non-burnable; all
 *     cells update synchronously; a burning cell burns out after one step; a
 *     fire runs until no cell burns;
 *   - Sec. 2.3: random numbers come from the counter-based Philox generator;
 *   - Eq. 2 (Sec. 2.2): a simulation is scored against the reference burnt
 *     map by delta = (|A u A*| - |A n A*|) / |A|.
 *
 * Conventions used throughout this interface.
 *   Grid: row-major, row 0 is the northern edge and column 0 the western edge.
 *     The paper's ignition coordinates (x, y) are (col, row).
 *   Directions: d = 0..7 is the bearing 45*d degrees (N, NE, E, SE, S, SW, W,
 *     NW) of the step from a burning cell to a target cell.
 *   Angles: aspect is the bearing the slope faces (downslope), wind is the
 *     bearing the wind blows toward, both in degrees clockwise from north.
 *   Trials: a target cell with k burning neighbours runs k independent trials
 *     (so it ignites with probability 1 - prod(1 - p_i), Sec. 2.1); the trial
 *     of target cell c (= row * W + col) at step t from direction d succeeds
 *     iff u < T, where u is word d % 4 of Philox4x32-10 with counter
 *     (c, t, d / 4, 0) and key (seed & 0xffffffff, seed >> 32), and
 *     T = floor(p * 2^32) with p evaluated in double precision in the order
 *     of Eq. 1.  A simulation's result therefore depends only on its map,
 *     parameters, ignition and seed: not on its position in a batch, the batch
 *     size or the launch shape.
 *   Pointers: every pointer argument is a host pointer unless the call's
 *     flags contain FIRE_DEVICE_PTRS, in which case every array argument of
 *     that call (inputs and outputs) is a device pointer valid on the
 *     context's device.  The caller owns all argument buffers; the library
 *     copies inputs it keeps (maps, targets) and owns the device memory of
 *     contexts and maps until fire_destroy / fire_map_free.
 *   Streams: work is issued on the context's stream.  With host output
 *     pointers the call returns after the results have been copied back.
 *     With FIRE_DEVICE_PTRS the call is asynchronous unless FIRE_SYNC is set;
 *     argument errors that can only be seen on the device (an ignition
 *     outside the grid) are reported per simulation in fire_result.status.
 *   Errors: functions return FIRE_OK (0) or a negative FIRE_E* code;
 *     fire_last_error() describes the last failure on a context.  A context
 *     may be used by one host thread at a time.
 *   Limits: H, W >= 1; the grid is processed in 32 x 32 tiles and at most
 *     FIRE_MAX_TILES tiles are supported; n <= 2^31 - 1 simulations per call.
 *     A batch of n = 0 (simulations, results, groups) returns FIRE_OK at once
 *     and touches no buffer, so its pointers may be NULL.
 */
#ifndef FIRE_H
#define FIRE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of the ABI are exported with default visibility; everything else
 * in the library is hidden. */
#if defined(__GNUC__)
#define FIRE_API __attribute__((visibility("default")))
#else
#define FIRE_API
#endif

typedef struct fire_ctx fire_ctx;
typedef struct fire_map fire_map;

/* beta_0 .. beta_4 of Eq. 1 (baseline, forest, aspect, wind, slope). */
typedef struct { double b[5]; } fire_params;

/* Ignition cell (Sec. 2.1: "ignition point"); the paper's (x, y) = (col, row). */
typedef struct { int32_t row, col; } fire_cell;

/* Per-simulation result.
 *   burnt  |A*|: cells that burnt, ignition included;
 *   inter  |A n A*| against the map's target (0 without a target);
 *   target |A| of the map's target;
 *   steps  number of steps in which some cell was burning (1 when only the
 *          ignition burnt);
 *   status FIRE_STATUS_* bits;
 *   trials number of (target cell, burning neighbour) trials evaluated. */
typedef struct {
    uint32_t burnt, inter, target, steps, status, trials;
} fire_result;

enum {
    FIRE_OK = 0,
    FIRE_EINVAL = -1,     /* bad argument (sizes, NULL, non-finite params)   */
    FIRE_ENOMEM = -2,     /* device or host allocation failed                */
    FIRE_ECUDA = -3,      /* CUDA runtime error (launch, copy, sync)         */
    FIRE_EIGNITION = -4,  /* host ignition outside the grid / non-burnable   */
    FIRE_ETIMEOUT = -5,   /* a bounded device wait ran out                   */
    FIRE_ESTEPS = -6      /* a simulation reached the step cap               */
};

#define FIRE_MAX_TILES 16384

/* call flags */
#define FIRE_DEVICE_PTRS 1u  /* array arguments are device pointers          */
#define FIRE_WANT_STEPS 2u   /* fill burn_step (see fire_simulate_batch)     */
#define FIRE_SYNC 4u         /* block until the work has finished            */
#define FIRE_GRAPH 8u        /* capture the call's device work as a CUDA graph
                                once and replay it on later identical calls  */
#define FIRE_CELL_UNIFORM 16u /* the paper's own CUDA update (Sec. 2.3): one
                                uniform per target cell and step, word 0 of
                                Philox block (cell, step, 2, 0), succeeding iff
                                u < floor((1 - q) 2^32) with q the product of
                                (1 - p_d) over the burning neighbours in
                                increasing d, in double precision            */
#define FIRE_LONGEST_FIRST 128u /* fire_simulate_batch: hand the fires to the
                                GPU's blocks longest-first, by a key predicted
                                from each fire's parameters on the map (for
                                batches larger than the grid, up to 8192
                                fires); scheduling only, results unchanged   */
#define FIRE_TC_A_MN 32u      /* fire_tc_gemm: A stored MN-major (A[k][m])   */
#define FIRE_TC_B_MN 64u      /* fire_tc_gemm: B stored MN-major (B[k][n])   */

/* fire_result.status bits */
#define FIRE_STATUS_BORDER 1u        /* a burnt cell lies on the grid edge   */
#define FIRE_STATUS_STEP_CAP 2u      /* stopped at the step cap              */
#define FIRE_STATUS_BAD_IGNITION 4u  /* ignition outside grid/non-burnable   */
#define FIRE_STATUS_TIMEOUT 8u       /* a bounded device wait ran out        */
#define FIRE_STATUS_BAD_MAP 16u      /* map index outside the map table      */

/* fitness kinds */
#define FIRE_FITNESS_PAPER_DELTA 0  /* Eq. 2: (|AuA*| - |AnA*|) / |A|          */
#define FIRE_FITNESS_JACCARD 1      /* (|AuA*| - |AnA*|) / |AuA*|             */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to issue work on (NULL: the context creates and owns a stream; pass
 * cudaStreamLegacy, (void *)1, for the legacy default stream). */
FIRE_API int fire_create(fire_ctx **out, int device, void *cuda_stream);

/* Release a context and everything it owns (maps must be freed first). */
FIRE_API void fire_destroy(fire_ctx *ctx);

/* Text of the last error on this context ("" if none).  Owned by ctx. */
FIRE_API const char *fire_last_error(const fire_ctx *ctx);

/* Block until all work issued on the context's stream has finished.
 * Returns FIRE_ETIMEOUT (once) when a bounded device wait of earlier work ran
 * out: the context's error word, or the error word of the no-alloc scratch on
 * the context's device (fire_simulate_batch_noalloc). */
FIRE_API int fire_sync(fire_ctx *ctx);

/* Launch shape used by later simulation calls: warps per block (1..16),
 * blocks per SM (0: as many as fit), candidate-queue entries per block
 * (0: default; at least 64) and state placement (FIRE_STATE_AUTO: shared
 * memory when the grid's state fits, else a per-block global buffer;
 * FIRE_STATE_SHARED; FIRE_STATE_GLOBAL).  Results do not depend on any of
 * them (see Trials above); a shape that does not fit the device makes the
 * next simulation call fail with FIRE_EINVAL. */
#define FIRE_STATE_AUTO 0
#define FIRE_STATE_SHARED 1
#define FIRE_STATE_GLOBAL 2
FIRE_API int fire_set_launch(fire_ctx *ctx, int warps_per_block, int blocks_per_sm,
                             int queue_entries, int state_mode);

/* Test hook for the out-of-memory path: the growth of a context-owned
 * device buffer (argument staging, simulation state and frontier lists,
 * ordering scratch) that comes `after` growths from now fails as if
 * cudaMalloc had failed: the buffer is released, the call returns
 * FIRE_ENOMEM with a message naming the hook, and the context stays usable
 * (the next call grows the buffer again).  after = -1 turns the hook off;
 * it fires once.  Growths that find a large enough buffer do not count. */
FIRE_API int fire_debug_fail_alloc(fire_ctx *ctx, int after);


/* Upload the raster maps of one landscape (Sec. 2.1, Fig. 1) and precompute
 * the per-cell covariates of Eq. 1 on the device:
 *   veg[H*W]     uint8 vegetation code: 0 non-burnable, 1 forest, 2.. other
 *   elev[H*W]    elevation (any unit; only comparisons are used)
 *   slope[H*W]   slope in degrees
 *   aspect[H*W]  aspect in degrees (downslope bearing)
 *   wind[H*W]    wind direction in degrees (bearing blown toward)
 * cell_m is recorded for reference only.  The map starts without a target. */
FIRE_API int fire_maps_upload(fire_ctx *ctx, int H, int W, float cell_m,
                     const uint8_t *veg, const float *elev, const float *slope,
                     const float *aspect, const float *wind, uint32_t flags,
                     fire_map **out);

/* Free a map and its device memory. */
FIRE_API void fire_map_free(fire_map *map);

/* Grid shape of a map. */
FIRE_API int fire_map_shape(const fire_map *map, int *H, int *W);

/* Set the reference (target) burnt map A of Eq. 2: burnt[H*W] uint8, nonzero
 * means burnt.  |A| is counted on the device. */
FIRE_API int fire_target_upload(fire_ctx *ctx, fire_map *map, const uint8_t *burnt,
                       uint32_t flags);

/* Run n independent simulations on one map (Sec. 2.1 rules, Eq. 1, Sec. 2.3)
 * and score each against the map's target (Eq. 2 counts).
 *   params[n]     beta vectors (finite)
 *   ignitions[n]  ignition cells (must be burnable)
 *   seeds[n]      64-bit Philox keys, one per simulation
 *   out[n]        results
 *   burn_step     NULL, or n*H*W int32 written when FIRE_WANT_STEPS is set:
 *                 step at which each cell ignited (0 for the ignition cell),
 *                 -1 for burnable cells that did not burn, -2 for
 *                 non-burnable cells; simulation i occupies
 *                 burn_step[i*H*W .. (i+1)*H*W).
 *   max_steps     0 for no cap, else stop a fire after that many steps and
 *                 set FIRE_STATUS_STEP_CAP.
 * Host ignitions that are outside the grid or non-burnable make the call
 * return FIRE_EIGNITION before any work is issued; a map uploaded through a
 * context on another device is refused with FIRE_EINVAL. */
FIRE_API int fire_simulate_batch(fire_ctx *ctx, const fire_map *map, int n,
                        const fire_params *params, const fire_cell *ignitions,
                        const uint64_t *seeds, uint32_t max_steps,
                        uint32_t flags, fire_result *out, int32_t *burn_step);

/* The same simulations as fire_simulate_batch for callers that cannot let
 * the library allocate device memory: for example code running under a fixed
 * device-memory budget owned by another allocator, or a latency-bound loop
 * in which cudaMalloc's implicit device synchronisation is not acceptable.
 * (The paper has no counterpart; this is an integration convenience.)
 * Every array argument is a device pointer supplied by the caller
 * (FIRE_DEVICE_PTRS is implied); results are identical to
 * fire_simulate_batch's.  The call allocates nothing: its scratch (work
 * counter, error word, per-block state buffers) lives in one fixed device
 * array of 2 MiB that every GPU loading the library holds until the process
 * exits.  A map whose per-block state buffer does not fit in it (grids of
 * more than about 8191 tiles whose state also exceeds shared memory) is
 * rejected with FIRE_EINVAL before any work is issued.  The first call on a
 * device looks up the array's address once; make that first call before any
 * stream capture begins on the device.  All calls on a device share the
 * array and each clears its counter area before launching, so calls whose
 * work overlaps on the GPU race: serialise them.  Flags: FIRE_DEVICE_PTRS
 * (implied), FIRE_WANT_STEPS, FIRE_SYNC and FIRE_CELL_UNIFORM; any other flag
 * (FIRE_LONGEST_FIRST, FIRE_GRAPH: both need library-owned buffers) is
 * refused with FIRE_EINVAL, as is a map uploaded on another device than the
 * context's, before any work is issued.  Asynchronous unless FIRE_SYNC is
 * set (then a timed-out device wait returns FIRE_ETIMEOUT).  After an
 * asynchronous call, a timed-out wait shows as FIRE_STATUS_TIMEOUT in the
 * affected out[i].status and is returned as FIRE_ETIMEOUT by the next
 * fire_sync on the context (which reads and clears the array's error word),
 * provided no later no-alloc call on the device has cleared it first. */
FIRE_API int fire_simulate_batch_noalloc(fire_ctx *ctx, const fire_map *map,
                                         int n, const fire_params *params,
                                         const fire_cell *ignitions,
                                         const uint64_t *seeds,
                                         uint32_t max_steps, uint32_t flags,
                                         fire_result *out, int32_t *burn_step);

/* Uneven batch: n simulations over nmaps landscapes of different sizes in one
 * persistent launch.  maps[nmaps] is a host array of map handles (all on the
 * context's device); map_of_sim[n] gives each simulation's map index; the
 * other arguments are as in fire_simulate_batch (out[i] belongs to
 * simulation i; burn-step maps are not produced).  Simulations run largest
 * map first (a device-side counting sort), which shortens the tail of the
 * launch; results do not depend on the order.  With host pointers, map
 * indices, parameters and ignitions are checked before any work is issued
 * (FIRE_EINVAL / FIRE_EIGNITION); with FIRE_DEVICE_PTRS a bad map index or
 * ignition is reported per simulation (FIRE_STATUS_BAD_MAP /
 * FIRE_STATUS_BAD_IGNITION).
 * FIRE_GRAPH (with FIRE_DEVICE_PTRS, on a context created with a
 * non-default stream): the first call captures the ordering, counter reset
 * and simulation launch into a CUDA graph kept by the context; a later call
 * with the same maps, n, pointers, step cap and launch shape replays it, so
 * new inputs must be written into the same device buffers.  Graphs are
 * dropped when the context has to move one of its device buffers. */
FIRE_API int fire_simulate_multi(fire_ctx *ctx, int nmaps,
                                 const fire_map *const *maps,
                                 const int32_t *map_of_sim, int n,
                                 const fire_params *params,
                                 const fire_cell *ignitions,
                                 const uint64_t *seeds, uint32_t max_steps,
                                 uint32_t flags, fire_result *out);

/* Launch shape chosen by the autotuner. */
typedef struct {
    int32_t warps_per_block, blocks_per_sm, queue_entries, state_mode;
    float ms;   /* time of the best shape on the probe batch */
} fire_launch;

/* Time the simulation kernel on the given batch (as fire_simulate_multi;
 * map_of_sim may be NULL with host pointers, meaning map 0) with each of a
 * fixed list of launch shapes (warps per block, blocks per SM, queue
 * capacity, state placement), record the fastest for this largest-map tile
 * count in the context, and return it.  Later calls without an explicit
 * fire_set_launch override use it; results never depend on it.  flags:
 * FIRE_DEVICE_PTRS, and FIRE_LONGEST_FIRST (nmaps = 1 only, else FIRE_EINVAL;
 * map_of_sim is then ignored) to time the shapes as fire_simulate_batch runs
 * with that flag.  Each shape
 * runs once untimed and twice timed (the better time counts): the batch runs
 * three times per shape, twelve shapes (fewer when a shape does not fit). */
FIRE_API int fire_autotune(fire_ctx *ctx, int nmaps, const fire_map *const *maps,
                           const int32_t *map_of_sim, int n,
                           const fire_params *params, const fire_cell *ignitions,
                           const uint64_t *seeds, uint32_t flags,
                           fire_launch *best);

/* One generation of the genetic algorithm of the paper's Appendix B on the
 * device: elitism (the two best individuals carried over unchanged),
 * tournament selection between two individuals drawn at random (one draw per
 * new individual), one-point crossover of consecutive pairs, and per-gene
 * mutation whose probability decreases as the generations advance.
 *   genes_in[pop*genes], genes_out[pop*genes]  row-major individuals; the
 *                  two must not overlap (FIRE_EINVAL)
 *   fitness[pop]   lower is better; NaN ranks last; ties go to the lower index
 *   generation / total_gens   g and NG of the schedule below
 *   ga_seed        Philox key of this GA run
 *   lo[genes], hi[genes]      bounds of each gene
 * The paper leaves the constants open; this library uses: contestants
 * a = (w0 pop) >> 32 and b = (w1 pop) >> 32 from Philox block (j, g, 0, 0) for
 * new slot j; cut c = 1 + ((w0 (genes - 1)) >> 32) from block (j, g, 1, 0)
 * for the pair (j, j + 1); gene k of child j mutates when w0 < floor(pm 2^32)
 * of block (j, g, 2, k), pm = 0.2 (1 - g/NG) + 0.01, by
 * (2 w1 2^-32 - 1) 0.1 (hi_k - lo_k) (1 - g/NG), clamped to [lo_k, hi_k].
 * The result depends only on the arguments (bit-reproducible). */
FIRE_API int ga_step(fire_ctx *ctx, int pop, int genes, const double *genes_in,
                     const double *fitness, int generation, int total_gens,
                     uint64_t ga_seed, const double *lo, const double *hi,
                     uint32_t flags, double *genes_out);

/* Ignition cells of individuals that carry the ignition point as two genes
 * (Sec. 3, Table 3 and Appendix B: with the ignition unknown the genetic
 * algorithm searches seven parameters, the five of Eq. 1 plus x and y).  For
 * individual i of genes_in[n*genes] (row-major), gene gx is x (the column)
 * and gene gy is y (the row); each is clamped to the grid ([0, W - 1],
 * [0, H - 1]; a NaN counts as 0) and rounded half up, and the fire starts
 * from the burnable cell of the map's target burnt area nearest to that
 * point (squared distance, ties to the lower row-major index), so every
 * simulated fire starts inside the reference scar as the paper's do.  The
 * cell is written to ignitions[i*reps + r] for r < reps (the layout
 * fire_simulate_batch takes with each individual's reps replicates
 * consecutive).  Host or device pointers (FIRE_DEVICE_PTRS); FIRE_EINVAL
 * for bad sizes or indices, a map of another device, or a target without a
 * burnable cell.  Synchronous. */
FIRE_API int fire_snap_ignitions(fire_ctx *ctx, const fire_map *map, int n,
                                 int genes, int gx, int gy,
                                 const double *genes_in, int reps,
                                 uint32_t flags, fire_cell *ignitions);

/* Ignition-point search: the ignition treated as unknown and sought inside
 * the map's target scar (the paper's variable-ignition experiment).  A
 * lat_h x lat_w lattice of equal strips spans the scar's bounding box;
 * lattice point (a, b) sits at row r0 + floor((2a+1)(r1-r0+1) / (2 lat_h))
 * and column c0 + floor((2b+1)(c1-c0+1) / (2 lat_w)) and is moved to the
 * nearest burnable burnt cell (squared distance, ties to the lower row-major
 * index).  Each candidate c = a lat_w + b is simulated reps times with
 * `params` and seeds seed + c reps + r; fitness_map[c] is the replicate mean
 * of fitness `kind`.  The ensemble is the candidates with fitness <= cutoff
 * (or, if none, the best one); xy_mean_sd = {mean x, sd x, mean y, sd y} of
 * its ignitions with x = column, y = row (sample standard deviation, 0 for
 * a single candidate).  cells (nullable) receives the candidates as
 * (row, col) pairs.  FIRE_EINVAL when the target is empty or has no
 * burnable cell.  Synchronous. */
FIRE_API int ignition_search(fire_ctx *ctx, const fire_map *map,
                             const fire_params *params, int lat_h, int lat_w,
                             int reps, uint64_t seed, int kind, double cutoff,
                             uint32_t flags, double *fitness_map,
                             int32_t *cells, double xy_mean_sd[4]);

/* Mean of each of `groups` runs of per_group consecutive values (the fitness
 * of a GA individual over its replicate simulations), summed in index order
 * in double precision: out[groups].  With FIRE_DEVICE_PTRS, out must not
 * overlap values (FIRE_EINVAL); host buffers may, as they are staged. */
FIRE_API int fire_group_mean(fire_ctx *ctx, const double *values, int groups,
                             int per_group, uint32_t flags, double *out);

/* Fitness of n results (Eq. 2 or the Jaccard distance), double precision,
 * computed on the device.  A zero denominator gives NaN.  With
 * FIRE_DEVICE_PTRS, out must not overlap results (FIRE_EINVAL). */
FIRE_API int fire_fitness(fire_ctx *ctx, const fire_result *results, int n, int kind,
                 uint32_t flags, double *out);

/* Debug export of the ignition thresholds T = floor(p 2^32) of Eq. 1 for one
 * parameter vector: out[d*H*W + cell], int64 in [0, 2^32], every direction d
 * and cell (whether or not the source cell lies in the grid). */
FIRE_API int fire_thresholds(fire_ctx *ctx, const fire_map *map,
                    const fire_params *params, uint32_t flags, int64_t *out);

/* Debug export of the propagation probability p of Eq. 1 per direction and
 * cell: p32 as the simulation kernel's single-precision screen computes it,
 * p64 in double precision as the thresholds use it (either may be NULL). */
FIRE_API int fire_probabilities(fire_ctx *ctx, const fire_map *map,
                       const fire_params *params, uint32_t flags, float *p32,
                       double *p64);

/* Debug export of the precomputed covariates: psi, sig (= slope / 100), cos
 * and sin of the wind bearing (float[H*W] each) and cell flags (uint16[H*W]:
 * bit d < 8 target higher than the source of direction d, bit 8 forest, bit 9
 * burnable).  Any pointer may be NULL. */
FIRE_API int fire_map_features(fire_ctx *ctx, const fire_map *map, uint32_t flags,
                      float *psi, float *sig, float *cos_wind, float *sin_wind,
                      uint16_t *cell_flags);

/* Self-check of the single-precision screen that decides most trials: draws
 * n random (parameters, covariates, direction, u) cases from `seed`, decides
 * each through the screen and through the double-precision threshold, and
 * writes counts[0] = cases, counts[1] = cases sent to double precision,
 * counts[2] = cases where the two decisions differ (must be 0), and
 * max_err_ratio[0] = the largest |p32 - p64| seen, each divided by the
 * screen's error bound for its case (7.5e-9 |b3| + 5e-7, within 1e-6 for
 * |b3| <= 66; must stay below 1).  Host outputs. */
FIRE_API int fire_screen_selftest(fire_ctx *ctx, uint64_t n, uint64_t seed,
                         uint64_t counts[3], double max_err_ratio[1]);

/* Debug export of raw Philox4x32-10 blocks: out[4*i .. 4*i+3] is the block of
 * counter (c0 + i, c1, c2, c3) under key (k0, k1), for i < n. */
FIRE_API int fire_philox_blocks(fire_ctx *ctx, uint64_t n, const uint32_t ctr[4],
                       const uint32_t key[2], uint32_t flags, uint32_t *out);

/* Burn-out times (the paper burns every fuel out one step after ignition,
 * Sec. 2.1, and leaves fuel-consumption times to future work): as
 * fire_simulate_batch with the per-neighbour rule, except that a cell ignited
 * at step t stays burning for burn_time[cell] steps (t+1 .. t+burn_time) and
 * tries its unburnt neighbours at each of them with the same keyed draws
 * (counter (cell, step, d/4, 0)); burn_time = 1 everywhere gives exactly the
 * fires of fire_simulate_batch.  steps = the number of update steps run
 * while some cell was burning.
 *   burn_time  uint8[H*W] row-major, 1..250 on burnable cells (host values
 *              are checked; device values outside are clamped); per-fuel
 *              times are a table lookup by vegetation class on the caller's
 *              side.
 * Other arguments, layouts and errors as fire_simulate_batch;
 * FIRE_CELL_UNIFORM and FIRE_GRAPH are rejected (FIRE_EINVAL).  Runs the
 * bit-plane simulation kernel of fire_simulate_batch in its burn-time form
 * (state in global memory: the two state planes, two planes of the cells
 * still burning from earlier steps and one byte of fuel per cell per block),
 * at the launch shape set by fire_set_launch or the autotuner for the map's
 * tile count. */
FIRE_API int fire_simulate_burnout(fire_ctx *ctx, const fire_map *map, int n,
                                   const fire_params *params,
                                   const fire_cell *ignitions,
                                   const uint64_t *seeds, const uint8_t *burn_time,
                                   uint32_t max_steps, uint32_t flags,
                                   fire_result *out, int32_t *burn_step);

/* Tensor-core GEMM (tcgen05, BF16 operands, FP32 accumulation in tensor
 * memory): C[m][n] = sum_k A(m, k) B(n, k) for m < M, n < N, k < K.  The
 * paper has no counterpart: this is the tile the surrogate network's
 * convolutions run on, exported so that it can be checked on its own.
 *   A, B   device BF16 (uint16 bit patterns), 16-byte aligned; A is A[m][k]
 *          (K-major) or, with FIRE_TC_A_MN, A[k][m]; B is B[n][k] or, with
 *          FIRE_TC_B_MN, B[k][n].
 *   K      a multiple of 64; M a multiple of 8 with FIRE_TC_A_MN and N a
 *          multiple of 8 with FIRE_TC_B_MN.
 *   ksplit the K range is cut into ksplit parts run by separate CTAs and
 *          summed with FP32 atomics (C is cleared first); 1 = plain store.
 *   C      device FP32 [M][N], row-major, owned by the caller.
 * FIRE_DEVICE_PTRS is required.  Returns FIRE_EINVAL on a shape, alignment
 * or flag error; FIRE_ETIMEOUT (at the next fire_sync) if a bounded wait for
 * the tensor core ran out. */
FIRE_API int fire_tc_gemm(fire_ctx *ctx, int M, int N, int K, const uint16_t *A,
                          const uint16_t *B, int ksplit, uint32_t flags, float *C);

/* Self-check of the device-side timeout path (no counterpart in the paper).
 * One thread waits, with the bounded wait that every TMA and tensor-core
 * pipeline of the library uses, on an mbarrier phase that nothing completes.
 * The wait gives up after 2^31 SM clocks (about a second), sets the
 * context's error word, and the call returns FIRE_ETIMEOUT, as fire_sync
 * does after a real timeout, with the error word cleared and the context
 * usable.  Blocks.  Any other return value means the path is broken (an
 * error pending from earlier work is returned first, unchanged). */
FIRE_API int fire_wait_selftest(fire_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Learned surrogate (no counterpart in the paper).  A BF16 convolutional
 * network maps one parameter vector, the landscape and the ignition to a
 * per-cell burn probability on an S x S coarse grid (each coarse cell the
 * (H/S) x (W/S) block of fine cells); it is trained on burn fractions the
 * automaton produces and ranks GA offspring before they are simulated.
 *
 * Input x[n][S][S][16] BF16 (NHWC): channels 0..4 the fraction of fine cells
 * of vegetation class k (classes above 4 count as 4), 5 mean slope in
 * degrees / 45, 6/7 mean sin/cos of the aspect, 8/9 mean sin/cos of the wind
 * bearing, 10 one at the coarse cell of the ignition, 11..15 the parameters
 * / 10.  Network: 3x3 conv 16 -> 128, seven 3x3 convs 128 -> 128 with
 * dilations 1, 2, 4, ..., 64 (layer 1 has dilation 1), ReLU after each,
 * zero padding, a 1x1 head 128 -> 1 and a sigmoid; loss = mean binary
 * cross-entropy against the burn fraction.  Parameters are one FP32 vector
 * (fire_net_param_count() = 1,051,777 floats): per layer W[o][t][i]
 * (t = 3 t_y + t_x) then b[o], then the head's w[128] and b.  Convolutions
 * run on tcgen05 tensor cores with BF16 operands and FP32 accumulation;
 * activations and activation gradients are stored in BF16.
 *
 * Unless stated, array arguments are device pointers and FIRE_DEVICE_PTRS is
 * required; calls are asynchronous on the context's stream (FIRE_SYNC
 * blocks).  Errors: FIRE_EINVAL for shapes, NULLs, alignment or a missing
 * flag; FIRE_ENOMEM; FIRE_ECUDA; FIRE_ETIMEOUT (at the next fire_sync) when
 * a bounded tensor-core wait ran out.
 * ------------------------------------------------------------------------- */
#define FIRE_NET_CIN 16
#define FIRE_NET_C 128
#define FIRE_NET_LAYERS 8

typedef struct fire_net fire_net;

FIRE_API int64_t fire_net_param_count(void);

/* A network for S x S inputs (S a power of two in [8, 1024]) and batches of
 * up to max_batch samples (max_batch * S * S <= 2^24).  Allocates all
 * parameter, optimiser and activation buffers up front (about
 * 2 * 8 * max_batch * S * S * 256 bytes for activations and their
 * gradients); parameters start at zero: call fire_net_set_params. */
FIRE_API int fire_net_create(fire_ctx *ctx, int S, int max_batch, fire_net **out);
FIRE_API void fire_net_free(fire_net *net);

/* Load parameters (float[param_count], host, or device with
 * FIRE_DEVICE_PTRS), reset Adam's moments and step count, refresh the BF16
 * weight copies.  Blocks. */
FIRE_API int fire_net_set_params(fire_ctx *ctx, fire_net *net, const float *params,
                                 uint32_t flags);

/* Copy out float[param_count]: which = 0 parameters, 1 the gradient of the
 * last fire_net_backward, 2 / 3 Adam's first / second moments.  Host
 * destination, or device with FIRE_DEVICE_PTRS.  Blocks. */
FIRE_API int fire_net_get(fire_ctx *ctx, const fire_net *net, int which,
                          uint32_t flags, float *out);

/* Burn probabilities prob[n][S][S] (FP32) for inputs x[n][S][S][16] (BF16,
 * 16-byte aligned); n may exceed max_batch (run in chunks). */
FIRE_API int fire_net_forward(fire_ctx *ctx, fire_net *net, int n,
                              const uint16_t *x, uint32_t flags, float *prob);

/* Forward and backward over 1 <= n <= max_batch samples against labels
 * target[n][S][S] (FP32 in [0, 1]); leaves the gradient of the mean BCE in
 * the network (fire_net_get which = 1) and, when loss is not NULL, writes the
 * loss to the device double *loss. */
FIRE_API int fire_net_backward(fire_ctx *ctx, fire_net *net, int n,
                               const uint16_t *x, const float *target,
                               uint32_t flags, double *loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the
 * gradient of the last fire_net_backward and learning rate lr. */
FIRE_API int fire_net_adam(fire_ctx *ctx, fire_net *net, float lr, uint32_t flags);

/* Debug copy of a buffer of the last call for its first n samples: which =
 * 0 the BF16 activations of layer `layer` (0-based, [n][S][S][128]), 1 the
 * BF16 gradient of that layer's pre-activation times its ReLU mask (same
 * shape), 2 the FP32 probabilities [n][S][S] (layer ignored).  Blocks. */
FIRE_API int fire_net_buffer(fire_ctx *ctx, const fire_net *net, int which,
                             int layer, int n, uint32_t flags, void *out);

/* Coarse map planes[S][S][10] (FP32, channels 0..9 of the input) from the
 * fine rasters veg (uint8), slope, aspect, wind (FP32 degrees), each [H][W]
 * row-major; H and W multiples of S. */
FIRE_API int fire_net_planes(fire_ctx *ctx, int H, int W, int S, const uint8_t *veg,
                             const float *slope, const float *aspect,
                             const float *wind, uint32_t flags, float *planes);

/* Network inputs x[n][S][S][16] (BF16) from planes, params[n] and fine-grid
 * ignitions ign[n] of an H x W map. */
FIRE_API int fire_net_inputs(fire_ctx *ctx, int S, int H, int W, int n,
                             const float *planes, const fire_params *params,
                             const fire_cell *ign, uint32_t flags, uint16_t *x);

/* Training labels from the automaton: for each group g < groups, simulates
 * reps fires with params[g] and ign[g] (simulation i = g reps + r draws with
 * seed + i, exactly as fire_simulate_batch would), and writes
 * labels[g][S][S] = the fraction of the coarse cell's fine cells burnt,
 * averaged over the replicates.  results[groups * reps] (nullable) receives
 * the fire_result of each simulation.  FIRE_CELL_UNIFORM is honoured. */
FIRE_API int fire_net_labels(fire_ctx *ctx, const fire_map *map, int S, int groups,
                             int reps, const fire_params *params,
                             const fire_cell *ign, uint64_t seed,
                             uint32_t max_steps, uint32_t flags, float *labels,
                             fire_result *results);

/* The target's burnt fraction per coarse cell, frac[S][S] (FP32). */
FIRE_API int fire_net_target_frac(fire_ctx *ctx, const fire_map *map, int S,
                                  uint32_t flags, float *frac);

/* Screening: pred[s] = Eq. 2 (kind 0) or the Jaccard distance (kind 1)
 * computed with expected set sizes from prob[s] (E|A*| = c sum q, |A| =
 * c sum t, E|AnA*| = c sum q t, c = cells_per_coarse), and keep_idx[r] = the
 * candidate of rank r < keep by increasing pred (NaN last, ties to the lower
 * index). */
FIRE_API int fire_net_screen(fire_ctx *ctx, int S, int n, const float *prob,
                             const float *target_frac, double cells_per_coarse,
                             int kind, int keep, uint32_t flags, double *pred,
                             int32_t *keep_idx);

#ifdef __cplusplus
}
#endif

#endif /* FIRE_H */
