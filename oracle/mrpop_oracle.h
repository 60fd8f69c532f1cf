/*
 * mrpop_oracle.h -- plain FP64 CPU oracle for MR. POP's motion validation
 * and nearest-neighbour primitives.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the product path never calls it.
 *
 * Every floating-point quantity is computed in double from float32 inputs
 * (the conversion is exact).  The single exception is the number of
 * interpolation points of an edge, an integer that the GPU decides in FP32:
 * the oracle takes that decision in FP32 too, with the same operation order
 * (see orc_edge_npoints).
 */
#ifndef MRPOP_ORACLE_H
#define MRPOP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A scene: K serial arms with sphere sets, plus sphere and cuboid obstacles.
 * Layouts follow the shared synthetic-input conventions:
 *   dh           [sum dof][4]  (a, alpha, d, theta_offset) per joint
 *   sphere_link  [sum S]       link index of each sphere within its robot
 *   sphere_xyzr  [sum S][4]    centre in the link frame F_j' and radius
 *   base         [K][12]       row-major 3x4 [R | t]
 *   obs_spheres  [n][4]        cx, cy, cz, r
 *   obs_cuboids  [n][15]       c[3], half extents h[3], R[9] row-major       */
typedef struct {
    int32_t K;
    const int32_t *dof;
    const float *dh;
    const int32_t *n_spheres;
    const int32_t *sphere_link;
    const float *sphere_xyzr;
    const float *base;
    int32_t n_obs_spheres;
    const float *obs_spheres;
    int32_t n_obs_cuboids;
    const float *obs_cuboids;
    int32_t self_collision;  /* 1: also test link pairs of one robot (below)  */
    const uint16_t *self_mask; /* [sum dof] or NULL: bit i of row j (i < j) of a
                                * robot pairs its links i and j; NULL pairs
                                * every i, j with j >= i + 2                */
} orc_scene;

/* Forward kinematics of robot k at its joint vector q (length dof[k]):
 * writes world sphere centres and radii to out [n_spheres[k]][4]. */
void orc_fk_robot(const orc_scene *s, int32_t k, const double *q, double *out);

/* Link frames of robot k: frames[j] (row-major 4x4) is F_j', the frame of
 * joint j after its rotation.  Used by the tests' orthonormality pin. */
void orc_link_frames(const orc_scene *s, int32_t k, const double *q, double *frames);

/* Signed clearances: distance between surfaces (negative when overlapping). */
double orc_sphere_sphere_clearance(const double *c1, double r1, const double *c2, double r2);
double orc_sphere_cuboid_clearance(const double *c, double r, const float *cuboid);

/* Validity of one composite configuration q [D].  Returns 1 when no robot
 * sphere is in contact with an obstacle and no two spheres of different robots
 * are in contact (and, with self_collision, no two spheres of one robot on
 * a link pair of its adjacency mask); contact means clearance < margin.
 * *min_clear receives the smallest clearance of any tested pair (may be NULL). */
int32_t orc_config_valid(const orc_scene *s, const double *q, double margin, double *min_clear);

/* Number of interpolation intervals n = max(1, ceil(||qb - qa||_2 / res)),
 * decided in FP32 in the order fixed by the kernel (sequential fmaf sum). */
int32_t orc_edge_npoints(const float *qa, const float *qb, int64_t stride, int32_t D, float res);

/* Validity of the composite edge qa -> qb (float32, element i at qa[i*stride]):
 * every point q_k = qa + (k/n)(qb - qa), k = 0..n, must be valid.
 * With early_exit = 0 every point is evaluated and *min_clear is the minimum
 * over the whole edge; *first_hit receives the lowest colliding k or -1. */
int32_t orc_edge_valid(const orc_scene *s, const float *qa, const float *qb, int64_t stride,
                       float res, double margin, int32_t early_exit,
                       double *min_clear, int32_t *first_hit, int32_t *npoints);

/* Batched form over SoA edges qa, qb [D][ld], edges e0 .. e0+n-1. */
void orc_validate_edges(const orc_scene *s, const float *qa, const float *qb, int64_t ld,
                        int64_t e0, int64_t n, float res, double margin, int32_t early_exit,
                        uint8_t *valid, double *min_clear, int32_t *first_hit,
                        int32_t *npoints);

/* NEAREST(V, q, c) of Alg. 2: among tree vertices with g_v + ||q - q_v|| < c,
 * the one closest to q; ties by lowest g, then lowest index; -1 when empty.
 * tree is SoA [D+1][ld] with row D holding g.  Optional diagnostics: the best
 * and runner-up admissible distances and the smallest |g_v + d_v - c| over
 * all vertices (closeness to the filter boundary). */
int64_t orc_nearest(const float *tree, int64_t N, int64_t ld, int32_t D, const float *q,
                    float c, double *best_d, double *second_d, double *filter_gap);

/* NEIGHBORS(V, q, delta) of Alg. 2 (radius query): indices of all vertices
 * with ||q - q_v|| <= delta in ascending order; the first k_max go to out and
 * the total count is returned.  *gap receives min |d_v - delta|. */
int64_t orc_neighbors(const float *tree, int64_t N, int64_t ld, int32_t D, const float *q,
                      float delta, int64_t k_max, int64_t *out, double *gap);

/* C(sigma) = sum_j ||q_{j+1} - q_j|| over a path stored [M][D] (Sec. III-A). */
double orc_path_cost(const float *path, int64_t M, int32_t D);

/* 1 when every segment of the path [M][D] is a valid edge at resolution res. */
int32_t orc_path_valid(const orc_scene *s, const float *path, int64_t M, float res,
                       double margin, int64_t *bad_segment);

/* ------------------------------------------------------------------------- */
/* Work of the paper's two-stage check (Sec. III-E), for roofline accounting. */
/* ------------------------------------------------------------------------- */
/* Each checkpoint first runs FK with one conservative (coarse) sphere per
 * link and tests it against every obstacle and against every link of every
 * other robot (and, with self_collision, the link pairs of the adjacency
 * mask); only then the fine spheres of a link that a coarse test hit are
 * placed and tested, against the obstacles and links that its coarse sphere
 * hit.  A link's coarse sphere (the paper takes it from its sphere model) is
 * built here from the link's fine spheres: centre at the midpoint of the box
 * around their centres, radius max(|c - c_s| + r_s) + 1e-4.  Links without
 * spheres take part in no test.  Units counted (added to counts[]):        */
enum {
    ORC_WORK_CHECKPOINTS = 0,      /* checkpoints evaluated                  */
    ORC_WORK_JOINTS = 1,           /* joint transforms (FK of every robot)   */
    ORC_WORK_COARSE_POINTS = 2,    /* coarse centres placed (one per link)   */
    ORC_WORK_COARSE_SPHERE = 3,    /* coarse sphere vs obstacle sphere tests */
    ORC_WORK_COARSE_CUBOID = 4,    /* coarse sphere vs cuboid tests          */
    ORC_WORK_COARSE_PAIR = 5,      /* coarse sphere vs coarse sphere tests   */
    ORC_WORK_FINE_POINTS = 6,      /* fine centres placed (links with a hit) */
    ORC_WORK_FINE_SPHERE = 7,      /* fine sphere vs obstacle sphere tests   */
    ORC_WORK_FINE_CUBOID = 8,      /* fine sphere vs cuboid tests            */
    ORC_WORK_FINE_PAIR = 9,        /* fine sphere vs fine sphere tests       */
    ORC_WORK_UNITS = 10
};

/* Runs the two-stage check over the checkpoints of edge qa -> qb (as in
 * orc_edge_valid, k = 0..n in order), adds its units to counts
 * [ORC_WORK_UNITS] and returns the edge's validity (1 free, 0 colliding),
 * which equals orc_edge_valid's because the coarse spheres enclose the fine
 * ones.  With early_exit the checkpoints after the first colliding one are
 * not evaluated (the colliding one is). */
int32_t orc_edge_method_work(const orc_scene *s, const float *qa, const float *qb,
                             int64_t stride, float res, double margin, int32_t early_exit,
                             int64_t *counts);

/* Batched form over SoA edges qa, qb [D][ld], edges e0 .. e0+n-1; counts are
 * summed over the edges; valid (may be NULL) receives each verdict. */
void orc_method_work_edges(const orc_scene *s, const float *qa, const float *qb, int64_t ld,
                           int64_t e0, int64_t n, float res, double margin, int32_t early_exit,
                           int64_t *counts, uint8_t *valid);

/* ------------------------------------------------------------------------- */
/* FP64 reference planner (mrpop_ref_planner.c): Alg. 1 and Alg. 2 run one    */
/* iteration at a time on one host thread.                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    double resolution;    /* edge discretisation step (rad)                    */
    double margin;        /* contact inflation (m)                             */
    double delta;         /* per-robot roadmap connection radius (rad)         */
    int32_t n_per_round;  /* roadmap samples per robot per ROADMAP call        */
    int64_t max_iters;    /* iterations per dRRT / AO-X search call            */
    int64_t iter_budget;  /* total search iterations (<= 0: no limit)          */
    double time_budget_s; /* wall-clock budget (<= 0: no limit); a time or an
                           * iteration budget must be set                      */
    int64_t round_budget; /* total ROADMAP rounds (<= 0: no limit)            */
    double target_cost;   /* stop once the incumbent costs <= this (-1: never) */
    uint64_t seed;        /* SplitMix64 seed                                   */
} orc_plan_params;

/* Plans from start to goal (composite, double [D]) within the joint limits
 * q_lo, q_hi [D].  Returns 0 with a path (path [path_len][D] when path_len <=
 * path_cap; *cost = C(sigma) in FP64), 1 when no path was found within the
 * budget, -1 on invalid input, allocation failure, a start or goal in
 * collision, or a robot without free samples.  Every accepted incumbent is
 * recorded: trace_t (seconds since the call began), trace_c (its cost),
 * trace_it (iterations so far), at most trace_cap entries; *n_trace receives
 * the full count and *iterations the search iterations run. */
int32_t orc_plan(const orc_scene *s, const float *q_lo, const float *q_hi, const double *start,
                 const double *goal, const orc_plan_params *pp, double *path, int64_t path_cap,
                 int64_t *path_len, double *cost, double *trace_t, double *trace_c,
                 int64_t *trace_it, int64_t trace_cap, int64_t *n_trace, int64_t *iterations);

#ifdef __cplusplus
}
#endif
#endif
