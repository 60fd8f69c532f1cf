// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "mrpop.h"

namespace mrpop {

// ---------------------------------------------------------------------------
// Geometry tables.  Everything a validation kernel reads about a problem lives
// in one contiguous float4 blob that each block stages into shared memory:
//
//   base     K x 3 float4   rows of the 3x4 base pose [R | t]
//   link     L x 3 float4   (a, d, cos alpha, sin alpha)
//                           (theta_offset, first sphere, sphere count, robot)
//                           (coarse centre x, y, z in F_j', coarse radius)
//   sphere   S x 1 float4   (x, y, z in F_j', r), grouped by link
//   osphere  NS x 1 float4  (cx, cy, cz, r)
//   cuboid   NC x 5 float4  (cx, cy, cz, bounding radius |h|), (hx, hy, hz, 0),
//                           box axis 0, axis 1, axis 2 as (x, y, z, 0)
//
// Integer fields are stored as float bit patterns (__int_as_float).
// "Link" j of the composite chain is joint j: link index == q index.
// ---------------------------------------------------------------------------
struct Tables {
    int K = 0, L = 0, S = 0, NS = 0, NC = 0;
    int link0[MRPOP_MAX_ROBOTS + 1] = {0};  // first link of robot k; link0[K] = L
    int max_spheres_per_link = 0;
    int selfcol = 0;  // 1: also test links i, j >= i + 2 of one robot
    int off_base = 0, off_link = 0, off_sph = 0, off_os = 0, off_oc = 0, n_f4 = 0;
    // A corner below every point that a link's coarse sphere centre can reach
    // (each base origin minus its chain length, its farthest coarse centre and
    // 1 m): coordinates taken relative to it are >= 0, so their float bits
    // order like unsigned integers.
    float ws_lo[3] = {0.f, 0.f, 0.f};
};

constexpr int kLinkF4 = 3;
constexpr int kCuboidF4 = 5;
// Kept per stored link and checkpoint for later links' robot-robot tests: the
// link's coarse sphere centre (3 floats); the rare fine tests rebuild the
// link's frame along its chain instead of keeping it.
constexpr int kXcFloats = 3;
constexpr int kFrFloats = 12;  // a full frame, R (9) and t (3)

// Parameters of one validation launch (one problem, one batch of edges).
struct VParams {
    Tables t;
    const float4 *blob;
    const float *qa;
    const float *qb;
    int64_t E;
    float res;
    float margin;
    uint8_t *valid;
    float *length;
    int32_t *npoints;
    float *min_clear;
    unsigned long long *counters;
    int *work;  // [0] next edge, [1] finished warps; both return to 0 at exit
    int total_warps;
    int warp_floats;
    int dpad;
    int nstore;  // links of robots 0..K-2 (their frames and tile bounds are kept)
    int warps;   // warps of each block that take edges (the rest only stage tables)
    int order;   // checkpoints to lanes: 0 strided across the edge, 1 contiguous
    int fine;    // fine obstacle tests: 0 warp-union mask, 1 reassigned work items
};

// Per-warp shared scratch of the validation kernel (floats): q_a, q_b - q_a,
// tile bounds and frames of the stored links, and with reassigned fine tests
// one more link frame [12][32] plus 32 hit masks and 32 prefix sums.
inline int validate_warp_floats(const Tables &t, int fine) {
    const int dpad = (t.L + 3) & ~3;
    const int nstore = t.selfcol ? t.L : t.link0[t.K - 1];
    return 2 * dpad + 4 * nstore + nstore * kXcFloats * 32 + (fine ? kFrFloats * 32 + 64 : 0);
}

struct DeviceProblem {
    Tables t;
    float4 *blob = nullptr;       // device copy of the table blob
    float *q_lo = nullptr;        // device [D]
    float *q_hi = nullptr;        // device [D]
    int *edge_counter = nullptr;  // device work counter for persistent launches
};

}  // namespace mrpop

namespace mrpop {
struct HostRobot {
    int dof = 0;
    std::vector<float> dh, q_lo, q_hi, sphere_xyzr;
    std::vector<int32_t> sphere_link;
    float base[12] = {0};
};
struct Planner;  // device-resident planner state (planner.cu)
void destroy_planner(Planner *pl);
}  // namespace mrpop

struct mrpop_problem {
    mrpop::DeviceProblem dev;
    std::vector<mrpop::HostRobot> robots;     // host copies (planner sub-problems)
    std::vector<float> obs_spheres, obs_cuboids;
    mrpop::Planner *planner = nullptr;
    mrpop_config cfg{};
    int device = 0;
    int D = 0;
    std::vector<float> h_blob;  // host copy of the table blob
    std::vector<float> start, goal, q_lo, q_hi;
    int num_sms = 0;
    size_t smem_optin = 0;
    int tuned_warps = 0;  // autotuned warps per block (0: largest that fits)
    int tuned_order = 0;  // autotuned checkpoint order
    int tuned_fine = 0;   // autotuned fine-test mode (0 union, 1 reassigned)
    int tuned_regs = 0;   // autotuned register budget (0 compact: most warps, 1 wide)
};

namespace mrpop {

// Process-wide cache of tuned launch choices (capi.cu), keyed by a text key
// that names the kernel family, the GPU architecture and the shape of the
// work (e.g. "validate sm_103 K=2 L=14 ..."); values are small integer lists.
// Thread-safe.  Saved to and loaded from text files by mrpop_autotune_cache_*.
std::string tune_arch();
bool tune_lookup(const std::string &key, std::vector<int> *val);
void tune_store(const std::string &key, const std::vector<int> &val);
std::string validate_tune_key(const mrpop_problem *p);
int log2_bucket(int64_t n);

// Stream-ordered scratch from the library's memory pool on the current device
// (keeps freed memory across synchronisations); free with cudaFreeAsync.
cudaError_t scratch_alloc(void **ptr, size_t bytes, cudaStream_t st);

// Thread-local error reporting.
mrpop_status set_error(mrpop_status st, const char *fmt, ...);
mrpop_status cuda_error(cudaError_t e, const char *what);

#define MRPOP_CUDA_TRY(expr)                                          \
    do {                                                              \
        cudaError_t _e = (expr);                                      \
        if (_e != cudaSuccess) return ::mrpop::cuda_error(_e, #expr); \
    } while (0)

// Kernel launchers (defined in the kernel translation units).
mrpop_status launch_validate(mrpop_problem *p, const float *qa, const float *qb, int64_t n,
                             uint8_t *valid, float *length, int32_t *npoints,
                             float *min_clear, unsigned long long *counters,
                             cudaStream_t st);
mrpop_status autotune_validate(mrpop_problem *p, const float *qa, const float *qb, int64_t n,
                               uint8_t *valid, int reps, int32_t *out, float *ms_out,
                               cudaStream_t st);
// Fills V for validating n edges of problem p (warps per block and dynamic
// shared memory of the launch go to *warps_out / *smem_out).
mrpop_status make_vparams(mrpop_problem *p, const float *qa, const float *qb, int64_t n,
                          uint8_t *valid, VParams *V, size_t *smem_out, int *warps_out);
// Validates every problem's batch in one launch: d_params is a device array
// of nslots VParams whose total_warps equal blocks_per_slot * warps; fine
// selects the reassigned fine stage (every slot's scratch must provide it).
mrpop_status launch_validate_batch(const VParams *d_params, int nslots, int spl, int warps,
                                   int blocks_per_slot, size_t smem, bool fine,
                                   cudaStream_t st);
mrpop_status launch_fk(mrpop_problem *p, const float *q, int64_t n, float *out, cudaStream_t st);
mrpop_status launch_nearest(const float *tree, int64_t N, int64_t ld, int dim,
                            const float *queries, const float *budgets, int64_t Q,
                            int64_t *out_idx, cudaStream_t st,
                            int filter = MRPOP_NEAREST_FILTER_FP32, int waves = 0);
int nearest_tuned(int dim, int64_t N, int64_t Q, int filter);
int neighbors_tuned(int dim, int64_t N, int64_t Q);
mrpop_status autotune_nearest(const float *tree, int64_t N, int64_t ld, int dim,
                              const float *queries, const float *budgets, int64_t Q,
                              int filter, int64_t *out_idx, int32_t *waves_out, float *ms_out,
                              cudaStream_t st);
mrpop_status autotune_neighbors(const float *tree, int64_t N, int64_t ld, int dim,
                                const float *queries, int64_t Q, float delta, int64_t k_max,
                                int64_t *out_idx, int64_t *out_cnt, int32_t *target_out,
                                float *ms_out, cudaStream_t st);
// Number of (query, vertex) pairs launch_nearest scans for these inputs.
mrpop_status nearest_pairs(const float *tree, int64_t N, int64_t ld, int dim, const float *queries,
                           const float *budgets, int64_t Q, int64_t *pairs, cudaStream_t st);
mrpop_status launch_neighbors(const float *tree, int64_t N, int64_t ld, int dim,
                              const float *queries, int64_t Q, float delta, int64_t k_max,
                              int64_t *out_idx, int64_t *out_cnt, cudaStream_t st,
                              int warps_per_sm = 0);
mrpop_status launch_path_cost(const float *path, int64_t M, int dim, double *out,
                              cudaStream_t st);

}  // namespace mrpop
