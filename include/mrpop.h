/*
 * mrpop.h -- C ABI of the GB300 motion-validation library for MR. POP
 * (multi-robot parallel optimizing planner, dRRT + AO-x).
 *
 * The library implements the data-parallel hot path of the planner:
 * interpolation of composite edges, forward kinematics of serial arms to
 * collision-sphere sets, sphere-vs-obstacle and robot-vs-robot sphere tests
 * with early exit, cost-filtered nearest-neighbour and radius queries over
 * state-cost trees, and path cost.
 *
 * Conventions for every call
 *   - Every call returns an mrpop_status and never aborts; on failure a
 *     message is available from mrpop_last_error() (thread-local).
 *   - "device" pointers are CUDA global-memory pointers on the current device
 *     (for example from torch tensors); "host" pointers are CPU memory.  The
 *     caller owns every buffer it passes and keeps it alive until the work on
 *     the given stream has completed.
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Kernels
 *     are enqueued asynchronously on it; outputs are valid once the stream
 *     reaches that point.
 *   - Composite configurations q = (q^1, ..., q^K) concatenate the robots'
 *     joint vectors in robot order (Sec. III-A); D = sum of the robots' dof.
 *     Batches are SoA float32 [D][n]: element (i, e) at ptr[i * n + e].
 *   - A problem handle owns device copies of its robots and obstacles; it may
 *     be used from one host thread at a time.  Its validation calls
 *     (mrpop_validate_edges[_ex], mrpop_edge_clearance, mrpop_validate_work,
 *     mrpop_autotune) hand out edges through one device work counter of the
 *     handle, which the last warp of each launch resets: launches on one
 *     handle must not overlap on the GPU.  Enqueue them on one stream, or
 *     order the streams (events); two handles never share a counter.
 */
#ifndef MRPOP_H
#define MRPOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MRPOP_OK = 0,
    MRPOP_EINVAL = 1,      /* an argument is out of range or inconsistent      */
    MRPOP_ENOMEM = 2,      /* a host or device allocation failed               */
    MRPOP_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed      */
    MRPOP_ECAPACITY = 4,   /* a tree, roadmap or path buffer is full           */
    MRPOP_ETIMEOUT = 5,    /* a bounded device wait gave up                    */
    MRPOP_ENOSOLUTION = 6, /* no path was found within the budget             */
    MRPOP_EBUSY = 7,       /* the object is in use by another request          */
    MRPOP_ECANCELLED = 8   /* a serving request was cancelled                  */
} mrpop_status;

/* Limits checked by mrpop_create_problem. */
#define MRPOP_MAX_ROBOTS 16
#define MRPOP_MAX_DOF 16             /* joints per robot                     */
#define MRPOP_MAX_LINKS 64           /* sum of dof over robots (= max D)     */
#define MRPOP_MAX_SPHERES_PER_LINK 16
#define MRPOP_MAX_OBSTACLES 1024     /* spheres + cuboids                    */
/* Edges needing more interpolation intervals than this (|qb - qa| >
 * MRPOP_MAX_EDGE_INTERVALS * resolution), or with non-finite coordinates, are
 * reported invalid without being checked. */
#define MRPOP_MAX_EDGE_INTERVALS (1 << 20)

typedef struct mrpop_problem mrpop_problem; /* opaque, library-owned */

/* A serial arm of revolute joints with standard DH rows (Sec. III-E: robots
 * are approximated by collision spheres attached to their links).
 *   dh          host [dof][4]  a, alpha, d, theta_offset of each joint
 *   q_lo, q_hi  host [dof]     joint limits (rad)
 *   sphere_link host [n_spheres] link (joint) index of each sphere,
 *               non-decreasing; at most MRPOP_MAX_SPHERES_PER_LINK per link
 *   sphere_xyzr host [n_spheres][4] centre in frame F_j' (joint j's frame
 *               after its rotation Rz(q_j + theta_offset_j)) and radius
 *   base        row-major 3x4 [R | t] pose of the first joint's frame; R a
 *               proper rotation (R^T R = I within 1e-3, det R > 0; EINVAL
 *               otherwise)
 *   self_mask   host [dof] or NULL: the adjacency mask used when the
 *               config's self_collision is 1.  Bit i of self_mask[j] (i < j)
 *               set means links i and j of this robot are tested against
 *               each other; bits i >= j must be zero (EINVAL otherwise).
 *               NULL selects every pair with j >= i + 2.  Ignored when
 *               self_collision is 0.
 * The frame after joint j is F_j' * Tz(d_j) * Tx(a_j) * Rx(alpha_j). */
typedef struct {
    int32_t dof;
    int32_t n_spheres;
    const float *dh;
    const float *q_lo;
    const float *q_hi;
    const int32_t *sphere_link;
    const float *sphere_xyzr;
    float base[12];
    const uint16_t *self_mask;
} mrpop_robot;

/* Obstacles (host arrays): spheres [n][4] = cx, cy, cz, r; cuboids [n][15] =
 * centre c[3], half extents h[3], R[9] row-major whose columns are the box
 * axes in the world frame. */
typedef struct {
    int32_t n_spheres;
    const float *spheres;
    int32_t n_cuboids;
    const float *cuboids;
} mrpop_obstacles;

/* Planner and checker parameters.
 *   resolution   edge discretisation step (rad); an edge qa->qb is checked at
 *                q_k = qa + (k/n)(qb - qa), k = 0..n, n = max(1, ceil(|qb-qa|_2
 *                / resolution)) computed in FP32 (Sec. III-E discretisation)
 *   margin       contact inflation (m): a pair is in contact when its centre
 *                distance is below r1 + r2 + margin
 *   delta        per-robot roadmap connection radius (rad) (Sec. III-A)
 *   n_per_round  roadmap samples per robot per ROADMAP call (Alg. 2)
 *   tree_cap, roadmap_cap   vertex capacities of planner trees / roadmaps
 *   max_iters    planner iteration cap per search call
 *   seed         planner random seed
 *   self_collision  0: a robot's spheres are never tested against its own
 *                (the default; free space per robot counts obstacles only);
 *                1: spheres of the link pairs that each robot's self_mask
 *                selects are tested too (by default links i and j >= i + 2;
 *                adjacent links may overlap at their joint) */
typedef struct {
    float resolution;
    float margin;
    float delta;
    int32_t n_per_round;
    int64_t tree_cap;
    int64_t roadmap_cap;
    int64_t max_iters;
    uint64_t seed;
    int32_t self_collision;
} mrpop_config;

/* Message of the last failed call on this thread ("" when none). */
const char *mrpop_last_error(void);

/* Creates a problem (Sec. III-A problem setup: K robots, obstacles, q_start,
 * q_goal).  robots: host [K]; obs: host; start, goal: host [D] (may be NULL
 * when only the primitives are used); cfg: host.  Copies every table to the
 * current CUDA device; the handle owns those copies.  Errors: EINVAL when a
 * limit above is exceeded or a table is malformed; ENOMEM / ECUDA from the
 * device copies. */
mrpop_status mrpop_create_problem(const mrpop_robot *robots, int32_t K,
                                  const mrpop_obstacles *obs, const float *start,
                                  const float *goal, const mrpop_config *cfg,
                                  mrpop_problem **out);

/* Releases the handle and its device memory after synchronising the device
 * work that may still use it.  NULL is accepted. */
mrpop_status mrpop_destroy_problem(mrpop_problem *p);

/* Composite dimension D, robot count K and total sphere count S. */
mrpop_status mrpop_problem_dims(const mrpop_problem *p, int32_t *D, int32_t *K,
                                int32_t *S);

/* Forward kinematics (Sec. III-E FK tracing) of n composite configurations
 * q (device SoA [D][n]) to world sphere centres out (device [3][S][n]:
 * coordinate c of sphere s of configuration i at out[(c * S + s) * n + i]).
 * Spheres are ordered by robot, then as given. */
mrpop_status mrpop_fk(mrpop_problem *p, const float *q, int64_t n, float *out,
                      void *cuda_stream);

/* Motion validation of n_edges composite edges (Alg. 2: (q_near, q_new) in
 * C^f; Sec. III-E two-stage check).  qa, qb: device SoA [D][n_edges].
 * valid: device uint8 [n_edges], 1 when every interpolated configuration is
 * free of robot-obstacle and robot-robot contact, else 0.  Work stops for an
 * edge at its first colliding checkpoint tile. */
mrpop_status mrpop_validate_edges(mrpop_problem *p, const float *qa, const float *qb,
                                  int64_t n_edges, uint8_t *valid, void *cuda_stream);

/* Same check with optional by-products (NULL to skip):
 *   length   device float [n_edges]  |qb - qa|_2 (FP32), the edge cost
 *   npoints  device int32 [n_edges]  interval count n of each edge */
mrpop_status mrpop_validate_edges_ex(mrpop_problem *p, const float *qa, const float *qb,
                                     int64_t n_edges, uint8_t *valid, float *length,
                                     int32_t *npoints, void *cuda_stream);

/* Minimum signed clearance (surface distance minus margin-free radii) over
 * every checkpoint and every tested pair of each edge, without culling or
 * early exit: device float [n_edges].  A diagnostic for distance parity; the
 * edge is valid exactly when this is >= margin. */
mrpop_status mrpop_edge_clearance(mrpop_problem *p, const float *qa, const float *qb,
                                  int64_t n_edges, float *min_clear, void *cuda_stream);

/* Work counters of mrpop_validate_edges on the same inputs, summed over the
 * batch, for roofline accounting (device int64 [MRPOP_WORK_COUNTERS],
 * overwritten):
 *   [0]  checkpoints evaluated             [1]  joint transforms
 *   [2]  checkpoint link-vs-obstacle-sphere bound tests (tile candidates only)
 *   [3]  checkpoint link-vs-link bound tests (tile candidates only)
 *   [4]  sphere-vs-sphere-obstacle tests   [5]  sphere-vs-cuboid tests
 *   [6]  robot-robot sphere-pair tests     [7]  point transforms (coarse
 *        centres and sphere centres)
 *   [8]  tile-level sphere tests (tile bound vs obstacle spheres, vs the
 *        bounding spheres of cuboids and vs the tile bounds of earlier
 *        robots' links)
 *   [9]  tile bounds built (one per tile and link: centroid and radius of the
 *        link's coarse spheres at the tile's 32 checkpoints)
 *   [10] checkpoint link-vs-cuboid box tests (tile candidates only)
 *   [11] tile-level box tests (tile bound vs cuboid, where the cuboid's
 *        bounding sphere is near the tile bound)
 * Per-checkpoint counts only include what that checkpoint decides: a
 * sphere-level test is counted only where the checkpoint's own link-level
 * test hit (the kernel may run more, warp-wide). */
#define MRPOP_WORK_COUNTERS 12
mrpop_status mrpop_validate_work(mrpop_problem *p, const float *qa, const float *qb,
                                 int64_t n_edges, int64_t *counters, void *cuda_stream);

/* Autotuner of the validation launch (the batching pattern's tuned launch
 * shape; the paper fixes its own launch for its GPU).  Times
 * mrpop_validate_edges on the caller's edges (device SoA [D][n_edges], n_edges
 * > 0; verdicts written to valid) for every candidate that fits: warps per
 * block 1, 2 or 4, checkpoints strided across the edge (order 0: every tile
 * samples the whole edge, so collisions end an edge early) or contiguous
 * (order 1: tighter tile bounds, better culling on free edges), and the fine
 * obstacle tests as one warp-wide pass over every obstacle any checkpoint's
 * coarse sphere hit (fine stage 0) or as work items dealt out to the lanes in
 * proportion to each checkpoint's coarse hits (fine stage 1, the paper's
 * load-proportional thread reassignment of Sec. III-E).  The fastest becomes
 * the problem's launch for later validation calls and planner steps.  config
 * (host int32 [3], may be NULL): warps, order, fine stage; ms_per_launch
 * (host, may be NULL): its mean time.  Synchronises the stream.  Verdicts do
 * not depend on the launch. */
mrpop_status mrpop_autotune(mrpop_problem *p, const float *qa, const float *qb, int64_t n_edges,
                            uint8_t *valid, int32_t *config, float *ms_per_launch,
                            void *cuda_stream);

/* Sets the validation launch directly: warps_per_block 0 (largest that fits),
 * 1, 2 or 4; order 0 (strided) or 1 (contiguous); fine_stage 0 (warp-wide
 * union) or 1 (reassigned work items), as described for mrpop_autotune.
 * Errors: EINVAL for any other value. */
mrpop_status mrpop_set_launch(mrpop_problem *p, int32_t warps_per_block, int32_t order,
                              int32_t fine_stage);

/* mrpop_set_launch plus the register budget of the kernel: registers 0
 * (compact: the compiler's choice, about 72 registers, the most warps per SM)
 * or 1 (wide: up to 128 registers, four blocks per SM, no spills where
 * many-arm scenes run their robot-robot fine tests).  mrpop_autotune times
 * both budgets too.  Errors: EINVAL for any other value. */
mrpop_status mrpop_set_launch_ex(mrpop_problem *p, int32_t warps_per_block, int32_t order,
                                 int32_t fine_stage, int32_t registers);

/* The problem's current validation launch (host int32 [4]): warps per
 * block, order, fine stage, register budget.  Errors: EINVAL for NULL. */
mrpop_status mrpop_get_launch(const mrpop_problem *p, int32_t *config);

/* ---------------------------------------------------------------------------
 * Tuned-launch cache.  mrpop_autotune, mrpop_nearest_autotune and
 * mrpop_neighbors_autotune keep their choice in a process-wide cache keyed by
 * (GPU architecture, shape of the work): for validation the problem's robot,
 * link, sphere and obstacle counts (mrpop_create_problem applies a cached
 * launch to a new problem of that shape); for NEAREST and NEIGHBORS the
 * dimension and the base-2 logarithms of the tree size and the batch size
 * (later calls of that shape use it).  The cache can be saved to and loaded
 * from a text file, one "<key> = <values>" line per entry.
 * ------------------------------------------------------------------------- */
mrpop_status mrpop_autotune_cache_save(const char *path);
/* Adds (or replaces) the file's entries; EINVAL on a malformed line. */
mrpop_status mrpop_autotune_cache_load(const char *path);
mrpop_status mrpop_autotune_cache_clear(void);

/* Counters of the library's stream-ordered scratch pool on the current
 * device (host int64 [3]): bytes in use, the high-water mark of bytes in use,
 * bytes reserved from the device.  The library takes every temporary device
 * buffer (split-tree NEAREST partials, the ordering arena of large NEAREST
 * batches, NEIGHBORS partials, path-cost partials, planner staging) from
 * this pool, which keeps up to 1 GiB of freed memory across
 * synchronisations.  reset_high 1 resets the high-water mark after reading
 * it.  A diagnostic with no paper counterpart.  Errors: EINVAL (NULL), ECUDA. */
mrpop_status mrpop_scratch_stats(int32_t reset_high, int64_t *stats);

/* Times mrpop_nearest_ex on the caller's inputs with the budget-ordered path
 * split into 2, 4 or 8 waves of (query block, tree slice) pieces per SM
 * capacity, keeps the fastest for calls of this shape and filter, and
 * reports it (*waves, host; *ms_per_call, host, may be NULL).  out_idx
 * receives the results.  Batches that take the small-batch path are timed
 * too, but the waves do not apply to them.  Synchronises the stream.
 * Errors: as mrpop_nearest_ex. */
mrpop_status mrpop_nearest_autotune(const float *tree, int64_t n_vertices, int64_t ld,
                                    int32_t dim, const float *queries, const float *budgets,
                                    int64_t n_queries, int32_t filter, int64_t *out_idx,
                                    int32_t *waves, float *ms_per_call, void *cuda_stream);

/* Times mrpop_neighbors on the caller's inputs with the vertex ranges sized
 * for 14, 54 or 216 warps per SM (few queries are split over vertex ranges
 * so that the GPU fills), keeps the fastest for calls of this shape and
 * reports it (*warps_per_sm, host).  Synchronises the stream.  Errors: as
 * mrpop_neighbors. */
mrpop_status mrpop_neighbors_autotune(const float *tree, int64_t n_vertices, int64_t ld,
                                      int32_t dim, const float *queries, int64_t n_queries,
                                      float delta, int64_t k_max, int64_t *out_idx,
                                      int64_t *out_cnt, int32_t *warps_per_sm,
                                      float *ms_per_call, void *cuda_stream);

/* NEAREST(V, q, c) of Alg. 2 for n_queries queries: among tree vertices with
 * g_v + |q - q_v| < c, the one closest to q; ties go to the lowest g, then the
 * lowest index (Sec. III-D); -1 when no vertex qualifies.
 *   tree      device SoA [dim+1][ld]: rows 0..dim-1 configuration, row dim g
 *   n_vertices  vertices 0..n_vertices-1 are scanned (n_vertices <= ld)
 *   queries   device SoA [dim][n_queries];  budgets device float [n_queries]
 *   out_idx   device int64 [n_queries]
 * dim <= MRPOP_MAX_LINKS.  Distances are FP32. */
mrpop_status mrpop_nearest(const float *tree, int64_t n_vertices, int64_t ld, int32_t dim,
                           const float *queries, const float *budgets, int64_t n_queries,
                           int64_t *out_idx, void *cuda_stream);

/* Filters of the large-batch NEAREST path (mrpop_nearest_ex).  Batches of
 * >= 2048 queries in dimensions 3, 6, 7, 14, 21 or 28 order the tree by g and
 * the queries by budget, then pass each (query, vertex) pair through an
 * expansion filter |q|^2 + |x|^2 - 2 q.x <= bound, whose rounding error is
 * bounded so that it never drops the nearest admissible vertex; every vertex
 * that passes is decided with the exact FP32 distance, so the indices do not
 * depend on the filter.
 *   MRPOP_NEAREST_FILTER_FP32    FP32 fused multiply-adds on the FMA pipe
 *                                (the default of mrpop_nearest)
 *   MRPOP_NEAREST_FILTER_TENSOR  the cross term on the tensor cores
 *                                (mma.sync: FP16 operands under an exact
 *                                power-of-two scaling for dim <= 14, TF32
 *                                above); a deliberate option beside the
 *                                FP32 path, faster on this GPU */
#define MRPOP_NEAREST_FILTER_FP32 0
#define MRPOP_NEAREST_FILTER_TENSOR 1

/* mrpop_nearest with an explicit large-batch filter (one of the two above;
 * EINVAL otherwise).  Other batches take the small-batch scan whatever the
 * filter.  Same arguments, results and errors as mrpop_nearest. */
mrpop_status mrpop_nearest_ex(const float *tree, int64_t n_vertices, int64_t ld, int32_t dim,
                              const float *queries, const float *budgets, int64_t n_queries,
                              int32_t filter, int64_t *out_idx, void *cuda_stream);

/* How many (query, vertex) pairs mrpop_nearest evaluates for these inputs
 * (a diagnostic for roofline accounting; no paper counterpart).  A vertex
 * with g_v >= c is never admissible, so for batches of >= 2048 queries in
 * dimensions 3, 6, 7, 14, 21 or 28 mrpop_nearest orders the tree by g and the
 * queries by budget and lets each block of 256 consecutive queries scan only
 * the vertices whose g bucket lies at or below its largest budget; other
 * batches scan all n_queries x n_vertices pairs.  Same arguments as
 * mrpop_nearest, with *pairs (host) receiving the count.  Synchronises the
 * stream.  Errors: as mrpop_nearest. */
mrpop_status mrpop_nearest_work(const float *tree, int64_t n_vertices, int64_t ld, int32_t dim,
                                const float *queries, const float *budgets, int64_t n_queries,
                                int64_t *pairs, void *cuda_stream);

/* Largest n_queries accepted by mrpop_nearest_noalloc. */
#define MRPOP_NEAREST_NOALLOC_MAX_QUERIES 65536

/* NEAREST with no device allocation.  The paper has no counterpart: this is a
 * library convenience for callers that cannot allocate device memory while
 * they plan -- a real-time replanning loop that must neither stall on the
 * allocator nor risk an out-of-memory failure mid-cycle, or a process whose
 * device memory is already reserved by another framework's caching allocator.
 * Same arguments, results and errors as mrpop_nearest (the caller still passes
 * every input and output), but the partial minima live in one fixed device
 * array of 2 * MRPOP_NEAREST_NOALLOC_MAX_QUERIES records (1.5 MiB) that every
 * GPU loading this library holds until the process exits.
 *   - n_queries > MRPOP_NEAREST_NOALLOC_MAX_QUERIES is rejected with
 *     MRPOP_EINVAL; nothing is launched.
 *   - Every call looks up the array's device address on the current device
 *     (an allocation-free query once the library's module is loaded there,
 *     which the first call on a device does); make that first call before
 *     any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (for example
 *     on two streams) race and must be serialised by the caller.  Each call
 *     writes every record it reads, so nothing needs clearing between calls.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
mrpop_status mrpop_nearest_noalloc(const float *tree, int64_t n_vertices, int64_t ld,
                                   int32_t dim, const float *queries, const float *budgets,
                                   int64_t n_queries, int64_t *out_idx, void *cuda_stream);

/* NEIGHBORS(V, q, delta) of Alg. 2: indices of the vertices with |q - q_v| <=
 * delta, in ascending index order.  The first k_max of them go to
 * out_idx[i * k_max + j] (device int64 [n_queries][k_max], unused slots -1);
 * out_cnt (device int64 [n_queries]) receives the full count, which may exceed
 * k_max.  tree rows 0..dim-1 are read (a g row, if any, is ignored). */
mrpop_status mrpop_neighbors(const float *tree, int64_t n_vertices, int64_t ld, int32_t dim,
                             const float *queries, int64_t n_queries, float delta,
                             int64_t k_max, int64_t *out_idx, int64_t *out_cnt,
                             void *cuda_stream);

/* C(sigma) = sum_j |q_{j+1} - q_j| (Sec. III-A) of a path of M vertices
 * (device [M][dim], row-major per vertex), segment lengths in FP32 summed in
 * FP64, written to cost_out (device double [1]). */
mrpop_status mrpop_path_cost(const float *path, int64_t M, int32_t dim, double *cost_out,
                             void *cuda_stream);

/* MR. POP's anytime planner (Alg. 1): ROADMAP, then the initial dRRT search,
 * then AO-X calls with the shrinking incumbent cost c_best (Alg. 2), until
 * time_budget_s seconds of wall time have passed.  The problem must have been
 * created with start and goal; both must be collision-free.  Planner state
 * (roadmaps, trees, incumbent) stays on the device in the handle, so a later
 * call continues where this one stopped.
 *   path      host float [path_cap][D]: the best path found, q_start first,
 *             q_goal last (may be NULL to query the length and cost only)
 *   path_len  vertices of that path;  cost  C(sigma) = sum of segment lengths
 *             (Sec. III-A) in FP64 from the returned FP32 vertices, +inf when
 *             none.
 * Every returned path has been re-checked at resolution / 4 with the
 * problem's margin; incumbents only ever decrease strictly.  A single-robot
 * problem (K = 1) skips roadmap construction and extends its trees directly
 * in configuration space by at most cfg.delta per step (Sec. V-C ablation).
 * Errors: EINVAL (no start/goal, or either in collision), ENOSOLUTION (no path
 * within the budget), ECAPACITY (path_cap too small; path_len is set). */
mrpop_status mrpop_plan(mrpop_problem *p, double time_budget_s, float *path, int64_t path_cap,
                        int64_t *path_len, double *cost);

/* Plans n problems at once (the batched form of mrpop_plan) in one
 * persistent kernel launch, captured in a CUDA graph.  CTAs resident on every
 * SM advance every problem through Alg. 1 on the device -- ROADMAP rounds
 * (Alg. 2), search steps of 256 iterations, the re-check of each incumbent at
 * resolution / 4 and the anytime bookkeeping -- each problem independently:
 * its phases are cut into chunks that any CTA may claim, and the CTA finishing
 * a phase starts the next one, so no problem waits for another and the host
 * takes part only before and after the launch.  An outer iteration of Alg. 1
 * (an optional ROADMAP round, then a search step) is one "step".  Runs until
 * time_budget_s of wall time (checked at step boundaries), or max_steps steps
 * per problem when max_steps > 0, or until every problem has reached
 * target_costs[i] (host [n], or NULL for none).  A problem's planner evolves
 * exactly as it would alone for the same number of steps (per-problem random
 * streams, fixed-position writes, ordered inserts), so results do not depend
 * on the mix.  statuses (host [n], may be NULL): MRPOP_OK, MRPOP_EINVAL for a
 * problem whose start or goal is in collision, MRPOP_ETIMEOUT for a problem
 * left unfinished when a bounded wait ran out (see
 * mrpop_set_persistent_limits).  Results: mrpop_plan_result, mrpop_plan_trace.
 * Errors: EINVAL (NULL, repeated or start/goal-less problems, tables too large
 * for the launch's shared memory), ENOMEM / ECUDA, ETIMEOUT (an idle CTA's
 * bounded wait for work ran out; results found until then are kept). */
mrpop_status mrpop_plan_batch(mrpop_problem *const *ps, int32_t n, double time_budget_s,
                              int64_t max_steps, const double *target_costs,
                              mrpop_status *statuses);

/* Batch forms of mrpop_plan_batch_ex. */
#define MRPOP_BATCH_PERSISTENT 0  /* one persistent launch (mrpop_plan_batch)        */
#define MRPOP_BATCH_STEPPED 1     /* every step a replay of a captured graph of 9
                                   * launches with a problem dimension, ROADMAP
                                   * rounds as launches with a robot dimension,
                                   * host bookkeeping between steps (the form
                                   * mrpop_plan runs one problem in)              */

/* mrpop_plan_batch in either form (EINVAL for another value).  Same
 * arguments, results and errors otherwise. */
mrpop_status mrpop_plan_batch_ex(mrpop_problem *const *ps, int32_t n, double time_budget_s,
                                 int64_t max_steps, const double *target_costs,
                                 mrpop_status *statuses, int32_t form);

/* Limits of the persistent launch, process-wide, for tests and diagnostics:
 * ctas > 0 sets the number of CTAs (0: as many as fit on every SM);
 * idle_polls > 0 lets a CTA that found no work give up after that many
 * consecutive polls (0: only after the budget plus a grace period), setting
 * the launch's timeout flag (mrpop_plan_batch then returns MRPOP_ETIMEOUT).
 * Errors: EINVAL for negative values. */
mrpop_status mrpop_set_persistent_limits(int32_t ctas, int64_t idle_polls);

/* Where the CTA time of the last persistent launch in this process went (a
 * diagnostic of the batched planner, Alg. 1/2).  Host int64 arrays of
 * MRPOP_PLAN_PHASES: ns[k] = summed time of the chunks of phase kind k (CTA
 * nanoseconds, from the device timer), chunks[k] = their number; ctas_wall
 * [2] = the launch's CTAs and its wall time (ns), so that sum(ns) /
 * (ctas * wall) is the fraction of CTA time spent in chunks.  Kinds:
 *    0 start              1 ROADMAP sample        2 ROADMAP candidate check
 *    3 ROADMAP append     4 ROADMAP NEIGHBORS     5 ROADMAP candidate edges
 *    6 ROADMAP edge check 7 ROADMAP link + BFS    8 search sample
 *    9 NEAREST (own tree) 10 direction oracle     11 extension check
 *   12 insert             13 NEAREST (other tree) 14 connection prep
 *   15 connection check   16 solution             17 res/4 re-check
 *   18 accept             19 phase transitions (no chunks: the time the
 *                            finishing CTA spends deciding the next phase)
 * Zeros before the first launch.  Errors: EINVAL for NULL. */
#define MRPOP_PLAN_PHASES 20
mrpop_status mrpop_plan_batch_phase_stats(int64_t *ns, int64_t *chunks, int64_t *ctas_wall);

/* Best path and cost found so far for p (same outputs and errors as
 * mrpop_plan, without planning). */
mrpop_status mrpop_plan_result(mrpop_problem *p, float *path, int64_t path_cap, int64_t *path_len,
                               double *cost);

/* ---------------------------------------------------------------------------
 * Serving (continuous batching).  A server owns one thread that keeps up to
 * max_slots requests on the device and advances every running request by one
 * planner iteration per loop, exactly as mrpop_plan_batch does; queued
 * requests are admitted in arrival order whenever a slot is free and their
 * estimated device memory fits in device_mem_budget bytes (<= 0: 80 % of the
 * free memory at creation; a request is always admitted when nothing else
 * runs).  A request's roadmaps and trees stay on the device until it
 * finishes, then its device state is released (results stay readable with
 * mrpop_plan_result / mrpop_plan_trace).  A problem handle belongs to the
 * server from submission until its request is done: do not use or destroy it
 * meanwhile.  The server uses the CUDA device current at creation.
 * ------------------------------------------------------------------------- */
typedef struct mrpop_server mrpop_server;

mrpop_status mrpop_server_create(int32_t max_slots, int64_t device_mem_budget,
                                 mrpop_server **out);

/* Queues a planning request.  It finishes when its incumbent reaches
 * target_cost (NaN: no target; +inf: the first solution), when budget_s
 * seconds have passed since admission, or after max_steps iterations when
 * max_steps > 0, whichever comes first.  *ticket identifies it.  Errors:
 * EINVAL, EBUSY (the problem is already queued or running). */
mrpop_status mrpop_server_submit(mrpop_server *s, mrpop_problem *p, double budget_s,
                                 int64_t max_steps, double target_cost, int64_t *ticket);

/* State of a request: *state 0 queued, 1 running, 2 done.  times (host
 * double [4], may be NULL): admission, first solution, target reached, done,
 * each in seconds since submission or -1 if not (yet) happened.  *cost: the
 * final incumbent once done (+inf if none).  A request that failed returns its
 * error status once done. */
mrpop_status mrpop_server_poll(mrpop_server *s, int64_t ticket, int32_t *state, double *times,
                               double *cost);

/* Counters (host int64 [6]): requests admitted, completed, peak concurrent
 * requests, peak admitted device memory (bytes), memory budget, queue length. */
mrpop_status mrpop_server_stats(mrpop_server *s, int64_t *stats);

/* Cancels a request: a queued one is dropped before admission, a running one
 * ends after the iteration in flight; either finishes with MRPOP_ECANCELLED
 * (reported by mrpop_server_poll once done), keeping any path it found.  A
 * request already done is left as it is.  Errors: EINVAL (unknown ticket). */
mrpop_status mrpop_server_cancel(mrpop_server *s, int64_t ticket);

/* Host-side fault injection for tests of the serving loop's failure paths
 * (nothing faults on the GPU):
 *   MRPOP_FAULT_ADMIT_ENOMEM  the next count admissions fail as if their
 *                             device allocation had been refused: each such
 *                             request finishes with MRPOP_ENOMEM and the
 *                             server carries on with the others;
 *   MRPOP_FAULT_STALL_MS      the server loop stalls once for count
 *                             milliseconds, outside its lock (submit, poll
 *                             and cancel stay responsive).
 * Errors: EINVAL (unknown fault, negative count). */
#define MRPOP_FAULT_ADMIT_ENOMEM 1
#define MRPOP_FAULT_STALL_MS 2
mrpop_status mrpop_server_inject(mrpop_server *s, int32_t fault, int64_t count);

/* Stops the server: running requests finish at once, queued ones are
 * dropped, the thread is joined.  NULL is accepted. */
mrpop_status mrpop_server_destroy(mrpop_server *s);

/* The index-th accepted incumbent path (0 = first solution; costs decrease
 * with the index), for use as seeds of a downstream optimiser (Sec. III-F
 * records every path of the optimisation for that).  Same outputs as
 * mrpop_plan_result; cost is that incumbent's cost.  Errors: EINVAL (index
 * outside [0, n) with n from mrpop_plan_trace), ECAPACITY. */
mrpop_status mrpop_plan_history(const mrpop_problem *p, int64_t index, float *path,
                                int64_t path_cap, int64_t *path_len, double *cost);

/* Measured FP32 FMA throughput of the current device in TFLOP/s, the
 * roofline denominator of this library's FP32 SIMT kernels (validation,
 * NEIGHBORS, path cost and the default NEAREST filter).  The paper
 * has no counterpart: this is a calibration utility.  It launches 8
 * independent FMA chains per thread of iters steps each on 2,048 threads per
 * SM, once to warm up and then 5 times timed with CUDA events on cuda_stream
 * (synchronises it).  packed 0 times scalar FFMA, 1 the packed two-lane
 * fma.rn.f32x2 form.  Errors: EINVAL (NULL tflops, packed not 0/1, iters
 * outside 1 .. 2^24), ECUDA. */
mrpop_status mrpop_fp32_peak(int32_t packed, int32_t iters, double *tflops, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Test hooks for the planner's internal NEAREST and NEIGHBORS kernels (the
 * search step and ROADMAP rounds run their own forms of Alg. 2's NEAREST and
 * NEIGHBORS on the device-resident trees and roadmaps).  Each hook runs one
 * pass of that kernel on caller-given device arrays and synchronises the
 * stream; results follow the primitives' definitions, so they can be
 * compared with an oracle directly.
 * ------------------------------------------------------------------------- */
#define MRPOP_PLANNER_STEP_ITERS 256   /* queries per planner NEAREST pass      */
#define MRPOP_ROADMAP_DEGREE_CAP 64    /* neighbours kept per roadmap vertex    */

/* NEAREST(V, q, c) of Alg. 2 as a planner search step runs it: pass 0 (the
 * expanded tree, q_rand and c_rand) or pass 1 (the opposite tree, q_new and
 * the budget c_best - g_new); same definition and tie rule as mrpop_nearest.
 *   tree     device SoA [dim+1][ld], row dim = g;  n_vertices <= ld
 *   queries  device SoA [dim][n_queries];  budgets device [n_queries]
 *   out_idx  device int64 [n_queries], -1 when no vertex qualifies
 * 1 <= n_queries <= MRPOP_PLANNER_STEP_ITERS, dim <= MRPOP_MAX_LINKS.
 * Errors: EINVAL, ENOMEM / ECUDA. */
mrpop_status mrpop_planner_nearest_pass(const float *tree, int64_t n_vertices, int64_t ld,
                                        int32_t dim, const float *queries, const float *budgets,
                                        int32_t n_queries, int32_t pass, int64_t *out_idx,
                                        void *cuda_stream);

/* NEIGHBORS(V_r, c, delta) of Alg. 2 as a ROADMAP round runs it on a robot's
 * roadmap: the first MRPOP_ROADMAP_DEGREE_CAP vertices (ascending index) with
 * |c - v| <= delta, the rest of each row -1, and the full count.
 *   V        device SoA [dof][ld] (roadmap vertices), n_vertices <= ld
 *   queries  device SoA [dof][n_queries]
 *   out_idx  device int64 [n_queries][MRPOP_ROADMAP_DEGREE_CAP]
 *   out_cnt  device int64 [n_queries]
 * dof <= MRPOP_MAX_DOF.  Errors: EINVAL, ENOMEM / ECUDA. */
mrpop_status mrpop_planner_neighbors_pass(const float *V, int64_t n_vertices, int64_t ld,
                                          int32_t dof, const float *queries, int64_t n_queries,
                                          float delta, int64_t *out_idx, int64_t *out_cnt,
                                          void *cuda_stream);

/* Incumbent history of the problem's planner: times[i] (seconds since the
 * start of the mrpop_plan call that found it) and costs[i], in order, at most
 * cap entries; *n receives the full count and *iterations the planner
 * iterations run so far (host arrays; any pointer may be NULL). */
mrpop_status mrpop_plan_trace(const mrpop_problem *p, double *times, double *costs, int64_t cap,
                              int64_t *n, int64_t *iterations);

#ifdef __cplusplus
}
#endif
#endif /* MRPOP_H */
