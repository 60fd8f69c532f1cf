// MR. POP planner (Alg. 1, Alg. 2) on device-resident roadmaps and trees.
//
// Outer loop (Alg. 1): ROADMAP, then the initial dRRT search, then AO-X calls
// with a shrinking incumbent cost, until the time budget runs out.
//
// GB300 design: instead of one thread block per planner iteration, every
// search *step* runs kStepIters iterations for every problem in the batch at
// once, as a fixed sequence of launches whose grids have a problem ("slot")
// dimension: sample -> NEAREST on the expanded tree -> dRRT / AO-X direction
// oracle -> edge validation -> insert -> NEAREST on the opposite tree ->
// connection validation -> incumbent candidates.  The sequence has a fixed
// shape, so it is captured once in a CUDA graph and replayed; the host only
// rewrites a small control block per slot and reads it back.
//
// Roadmaps (Alg. 2 ROADMAP): per robot, batches of uniform samples are
// checked against the obstacles (a single-robot sub-problem), connected to
// their neighbours within delta (NEIGHBORS) by checked edges, and grown until
// start and goal are connected (a BFS on the device).  A round runs for every
// robot of every problem that needs one at once: each phase is one launch
// with a job dimension, and the round ends with one host synchronisation.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "mrpop_internal.cuh"
#include "validate_body.cuh"

namespace mrpop {

constexpr int kStepIters = 256;     // iterations per step and problem
constexpr int kKmax = 64;           // roadmap degree cap
constexpr int kOversample = 4;      // roadmap candidates per wanted sample
constexpr int kRoadmapEdgesPerWarp = 16;  // roadmap validation: edges per warp on average
constexpr int kInformedTries = 16;  // informed-sampling rejection limit

struct Ctrl {
    float c_best;                  // incumbent cost (+inf before the first solution)
    int mode;                      // 0 dRRT search, 1 AO-X, 2 idle
    int step;                      // RNG stream of the step
    int tree_a;                    // tree expanded this step (set on device)
    unsigned long long seed;
    unsigned long long best_key;   // min over (cost bits << 32 | iteration)
    int overflow;                  // a tree reached its capacity
    int pad;
};

struct Slot {
    int K, D, rcap, tcap;
    int direct;    // single robot: no roadmap, steer in configuration space
    float step;    // direct mode: extension length (rad)
    int dof[MRPOP_MAX_ROBOTS];
    int qoff[MRPOP_MAX_ROBOTS];
    const float *q_lo, *q_hi, *start, *goal, *centre, *axis;
    float c_min;
    float *rm_q[MRPOP_MAX_ROBOTS];  // [dof][rcap]
    int *rm_adj[MRPOP_MAX_ROBOTS];  // [rcap][kKmax]
    int *rm_deg[MRPOP_MAX_ROBOTS];  // [rcap]
    int *rm_n;                      // [K]
    float *tq[2];                   // [D+1][tcap], row D = g
    int *tpar[2];                   // [tcap]
    int *trmv[2];                   // [K][tcap] roadmap vertex of each robot
    int *tn;                        // [2]
    float *qrand, *crand, *qnear, *qnew, *gnew, *budget2, *qconn;
    int64_t *near, *conn;
    int *rmvnew, *newidx;
    uint8_t *valid1, *valid2;
    Ctrl *ctrl;
};

// ---------------------------------------------------------------------------
// counter-based random numbers (SplitMix64 finaliser)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Rng {
    unsigned long long key, ctr;
    __device__ __forceinline__ float uniform() {  // [0, 1)
        return (float)(mix64(key ^ mix64(ctr++)) >> 40) * (1.0f / 16777216.0f);
    }
    __device__ __forceinline__ float normal() {
        const float u1 = 1.0f - uniform(), u2 = uniform();
        return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
};

__device__ __forceinline__ float nanf_() { return __int_as_float(0x7fc00000); }

// ---------------------------------------------------------------------------
// search step kernels (grid.y = slot)
// ---------------------------------------------------------------------------

// q_rand (uniform, or informed in the prolate hyperspheroid of c_best) and the
// cost coordinate c_rand ~ U[g_lb(q_rand), c_best] (Alg. 2 AO-X).
__device__ __forceinline__ void sample_body(const Slot &S, int i) {
    const Ctrl &C = *S.ctrl;
    const int a = (S.tn[0] <= S.tn[1]) ? 0 : 1;  // expand the smaller tree
    if (i == 0) S.ctrl->tree_a = a;
    if (i >= kStepIters) return;
    const int D = S.D, B = kStepIters;
    if (C.mode == 2) {
        S.crand[i] = -INFINITY;
        return;
    }
    Rng rng{mix64(C.seed ^ 0x5851F42D4C957F2Dull), ((unsigned long long)C.step << 32) ^ (unsigned)i};
    rng.ctr *= 977ull;
    float x[MRPOP_MAX_LINKS];
    const bool informed = C.mode == 1 && C.c_best < INFINITY && C.c_best > S.c_min;
    bool ok = false;
    if (informed) {
        // Direct sampling of the prolate hyperspheroid (foci start and goal,
        // transverse diameter c_best): uniform in the unit ball, scaled by the
        // radii, reflected so that e1 maps to the start->goal axis, centred.
        const float r1 = 0.5f * C.c_best;
        const float r2 = 0.5f * sqrtf(fmaxf(C.c_best * C.c_best - S.c_min * S.c_min, 0.f));
        for (int tr = 0; tr < kInformedTries && !ok; ++tr) {
            float n2 = 0.f;
            for (int d = 0; d < D; ++d) {
                x[d] = rng.normal();
                n2 = fmaf(x[d], x[d], n2);
            }
            const float rad = powf(rng.uniform(), 1.0f / (float)D) / sqrtf(fmaxf(n2, 1e-30f));
            for (int d = 0; d < D; ++d) x[d] *= rad * (d == 0 ? r1 : r2);
            // Householder reflection with w = e1 - axis
            float ww = 0.f, wx = 0.f;
            for (int d = 0; d < D; ++d) {
                const float w = (d == 0 ? 1.f : 0.f) - S.axis[d];
                ww = fmaf(w, w, ww);
                wx = fmaf(w, x[d], wx);
            }
            const float f = ww > 1e-12f ? 2.f * wx / ww : 0.f;
            ok = true;
            for (int d = 0; d < D; ++d) {
                const float w = (d == 0 ? 1.f : 0.f) - S.axis[d];
                x[d] = S.centre[d] + x[d] - f * w;
                ok = ok && x[d] >= S.q_lo[d] && x[d] <= S.q_hi[d];
            }
        }
    }
    if (!ok)
        for (int d = 0; d < D; ++d) x[d] = S.q_lo[d] + rng.uniform() * (S.q_hi[d] - S.q_lo[d]);
    for (int d = 0; d < D; ++d) S.qrand[(size_t)d * B + i] = x[d];
    if (C.mode == 1) {
        const float *root = a == 0 ? S.start : S.goal;
        float g2 = 0.f;
        for (int d = 0; d < D; ++d) {
            const float t = x[d] - root[d];
            g2 = fmaf(t, t, g2);
        }
        const float glb = sqrtf(g2);
        S.crand[i] = glb < C.c_best ? glb + rng.uniform() * (C.c_best - glb) : glb;
    } else {
        S.crand[i] = INFINITY;
    }
}

__global__ void k_sample(const Slot *__restrict__ slots) {
    sample_body(slots[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

// NEAREST over one of the slot's trees (pass 0: expanded tree with q_rand and
// c_rand; pass 1: opposite tree with q_new and c_best - g_new).  Vertices
// across the block's threads, 16 queries per block in shared memory, key
// (d^2, g, index), warp-shuffle argmin then a cross-warp pass.
constexpr int kPQB = 16;
constexpr int kPThreads = 128;

struct PBest {
    float d2, g;
    int idx;
};
__device__ __forceinline__ bool pbetter(const PBest &a, const PBest &b) {
    if (a.d2 != b.d2) return a.d2 < b.d2;
    if (a.g != b.g) return a.g < b.g;
    return (unsigned)a.idx < (unsigned)b.idx;
}

// Shared memory of one NEAREST chunk (16 queries) for a block of THREADS.
template <int THREADS>
struct NnShared {
    float qs[kPQB][MRPOP_MAX_LINKS];
    float cs[kPQB];
    PBest wb[THREADS / 32][kPQB];
};

template <int PASS, int THREADS>
__device__ __forceinline__ void nearest_body(const Slot &S, int chunk, NnShared<THREADS> &sh) {
    const Ctrl &C = *S.ctrl;
    float(&qs)[kPQB][MRPOP_MAX_LINKS] = sh.qs;
    float(&cs)[kPQB] = sh.cs;
    PBest(&wb)[THREADS / 32][kPQB] = sh.wb;
    const int B = kStepIters, D = S.D;
    const int t = PASS == 0 ? C.tree_a : 1 - C.tree_a;
    const float *tree = S.tq[t];
    const int N = min(S.tn[t], S.tcap);
    const int q0 = chunk * kPQB;
    const float *Qs = PASS == 0 ? S.qrand : S.qnew;
    const float *Cs = PASS == 0 ? S.crand : S.budget2;
    for (int k = threadIdx.x; k < kPQB * D; k += blockDim.x) {
        const int j = k / D, d = k % D;
        qs[j][d] = Qs[(size_t)d * B + q0 + j];
    }
    if (threadIdx.x < kPQB) cs[threadIdx.x] = Cs[q0 + threadIdx.x];
    __syncthreads();
    PBest best[kPQB];
#pragma unroll
    for (int j = 0; j < kPQB; ++j) best[j] = PBest{INFINITY, INFINITY, -1};
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        float acc[kPQB];
#pragma unroll
        for (int j = 0; j < kPQB; ++j) acc[j] = 0.f;
        for (int d = 0; d < D; ++d) {
            const float xv = tree[(size_t)d * S.tcap + v];
#pragma unroll
            for (int j = 0; j < kPQB; ++j) {
                const float a = qs[j][d] - xv;
                acc[j] = fmaf(a, a, acc[j]);
            }
        }
        const float g = tree[(size_t)D * S.tcap + v];
#pragma unroll
        for (int j = 0; j < kPQB; ++j)
            if (acc[j] <= best[j].d2 && g + __fsqrt_rn(acc[j]) < cs[j] &&
                (acc[j] < best[j].d2 || g < best[j].g))
                best[j] = PBest{acc[j], g, v};
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kPQB; ++j) {
        PBest b = best[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            PBest o{__shfl_xor_sync(0xffffffffu, b.d2, off), __shfl_xor_sync(0xffffffffu, b.g, off),
                    __shfl_xor_sync(0xffffffffu, b.idx, off)};
            if (pbetter(o, b)) b = o;
        }
        if (lane == 0) wb[warp][j] = b;
    }
    __syncthreads();
    if (threadIdx.x < kPQB) {
        PBest b = wb[0][threadIdx.x];
        for (int w = 1; w < THREADS / 32; ++w)
            if (pbetter(wb[w][threadIdx.x], b)) b = wb[w][threadIdx.x];
        (PASS == 0 ? S.near : S.conn)[q0 + threadIdx.x] = b.idx;
    }
}

template <int PASS>
__global__ void __launch_bounds__(kPThreads) k_nearest(const Slot *__restrict__ slots) {
    __shared__ NnShared<kPThreads> sh;
    nearest_body<PASS, kPThreads>(slots[blockIdx.y], blockIdx.x, sh);
}

// Direction oracle.  dRRT (Solovey et al.): per robot, the roadmap neighbour v
// of q_near^r with the largest cos angle(v - q_near^r, q_rand^r - q_near^r);
// the robot stays put when no neighbour has a positive cosine.  AO-X: the same
// choice, kept only when the extension is admissible, g_near + |q_new - q_near|
// <= c_rand (Sec. III-D).
__device__ __forceinline__ void oracle_body(const Slot &S, int i) {
    const Ctrl &C = *S.ctrl;
    if (i >= kStepIters) return;
    const int B = kStepIters, D = S.D, a = C.tree_a;
    const int nr = (int)S.near[i];
    bool active = C.mode != 2 && nr >= 0;
    bool moved = false;
    float len2 = 0.f;
    if (active && S.direct) {
        // single-robot mode (Sec. V-C): extend from q_near toward q_rand by at
        // most `step` (the robot plans in its configuration space directly)
        float d2 = 0.f;
        for (int d = 0; d < D; ++d) {
            const float t = S.qrand[(size_t)d * B + i] - S.tq[a][(size_t)d * S.tcap + nr];
            d2 = fmaf(t, t, d2);
        }
        const float dist = sqrtf(d2);
        const float f = dist > S.step ? S.step / dist : 1.f;
        for (int d = 0; d < D; ++d) {
            const float qa = S.tq[a][(size_t)d * S.tcap + nr];
            const float qb = fmaf(f, S.qrand[(size_t)d * B + i] - qa, qa);
            S.qnear[(size_t)d * B + i] = qa;
            S.qnew[(size_t)d * B + i] = qb;
            const float t = qb - qa;
            len2 = fmaf(t, t, len2);
        }
        S.rmvnew[i] = 0;
        moved = len2 > 0.f;
    } else if (active) {
        for (int r = 0; r < S.K; ++r) {
            const int u = S.trmv[a][(size_t)r * S.tcap + nr];
            const int dof = S.dof[r], off = S.qoff[r];
            const float *V = S.rm_q[r];
            float dn = 0.f;
            for (int d = 0; d < dof; ++d) {
                const float t = S.qrand[(size_t)(off + d) * B + i] - V[(size_t)d * S.rcap + u];
                dn = fmaf(t, t, dn);
            }
            int bestv = u;
            float bestc = 0.f;
            const int deg = min(S.rm_deg[r][u], kKmax);
            for (int k = 0; k < deg; ++k) {
                const int v = S.rm_adj[r][(size_t)u * kKmax + k];
                float dot = 0.f, vn = 0.f;
                for (int d = 0; d < dof; ++d) {
                    const float e = V[(size_t)d * S.rcap + v] - V[(size_t)d * S.rcap + u];
                    const float t = S.qrand[(size_t)(off + d) * B + i] - V[(size_t)d * S.rcap + u];
                    dot = fmaf(e, t, dot);
                    vn = fmaf(e, e, vn);
                }
                if (vn <= 0.f || dn <= 0.f) continue;
                const float c = dot / sqrtf(vn * dn);
                if (c > bestc || (c == bestc && bestv != u && v < bestv)) {
                    bestc = c;
                    bestv = v;
                }
            }
            S.rmvnew[(size_t)r * B + i] = bestv;
            moved |= bestv != u;
            for (int d = 0; d < dof; ++d) {
                const float qa = V[(size_t)d * S.rcap + u], qb = V[(size_t)d * S.rcap + bestv];
                S.qnear[(size_t)(off + d) * B + i] = qa;
                S.qnew[(size_t)(off + d) * B + i] = qb;
                const float t = qb - qa;
                len2 = fmaf(t, t, len2);
            }
        }
    }
    float gnew = INFINITY;
    if (active && moved) {
        gnew = S.tq[a][(size_t)D * S.tcap + nr] + sqrtf(len2);
        if (C.mode == 1 && !(gnew <= S.crand[i])) active = false;
    }
    if (!(active && moved)) {
        // inactive iteration: a NaN edge is rejected by validation at once
        S.qnew[i] = nanf_();
        S.qnear[i] = 0.f;
        gnew = INFINITY;
    }
    S.gnew[i] = gnew;
}

__global__ void k_oracle(const Slot *__restrict__ slots) {
    oracle_body(slots[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

// Insert z_new = (q_new, g_near + |q_new - q_near|) into the expanded tree and
// prepare the connection budget c_best - g_new (AO-X) or +inf (dRRT).  One
// block per slot; new vertices get consecutive indices in iteration order (a
// block-wide prefix sum), so a slot's trees do not depend on thread timing.
__device__ __forceinline__ void insert_body(const Slot &S, int *wsum) {
    Ctrl &C = *S.ctrl;
    const int i = threadIdx.x;
    const int B = kStepIters, D = S.D, a = C.tree_a;
    const bool want = S.valid1[i] && S.gnew[i] < INFINITY;
    const int lane = i & 31, warp = i >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, want);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kStepIters / 32; ++w) {
        before += w < warp ? wsum[w] : 0;
        total += wsum[w];
    }
    const int base = S.tn[a];
    __syncthreads();
    int idx = -1;
    if (want) {
        const int pos = base + before + __popc(bal & ((1u << lane) - 1u));
        if (pos < S.tcap) {
            idx = pos;
            for (int d = 0; d < D; ++d)
                S.tq[a][(size_t)d * S.tcap + idx] = S.qnew[(size_t)d * B + i];
            S.tq[a][(size_t)D * S.tcap + idx] = S.gnew[i];
            S.tpar[a][idx] = (int)S.near[i];
            for (int r = 0; r < S.K; ++r)
                S.trmv[a][(size_t)r * S.tcap + idx] = S.rmvnew[(size_t)r * B + i];
        } else {
            C.overflow = 1;
        }
    }
    if (i == 0) S.tn[a] = min(base + total, S.tcap);
    S.newidx[i] = idx;
    S.budget2[i] = idx < 0 ? -INFINITY : (C.mode == 1 ? C.c_best - S.gnew[i] : INFINITY);
}

__global__ void __launch_bounds__(kStepIters) k_insert(const Slot *__restrict__ slots) {
    __shared__ int wsum[kStepIters / 32];
    insert_body(slots[blockIdx.y], wsum);
}

__device__ __forceinline__ void conn_prep_body(const Slot &S, int i) {
    if (i >= kStepIters) return;
    const int B = kStepIters, D = S.D, b = 1 - S.ctrl->tree_a;
    const int c = (int)S.conn[i];
    if (c >= 0 && S.newidx[i] >= 0) {
        for (int d = 0; d < D; ++d) S.qconn[(size_t)d * B + i] = S.tq[b][(size_t)d * S.tcap + c];
    } else {
        S.qconn[i] = nanf_();
    }
}

__global__ void k_conn_prep(const Slot *__restrict__ slots) {
    conn_prep_body(slots[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

// A checked connection closes a path start -> ... -> z_new -> z_conn -> ...
// -> goal; the cheapest of the step wins (packed cost | iteration key).
__device__ __forceinline__ void solution_body(const Slot &S, int i) {
    Ctrl &C = *S.ctrl;
    if (i >= kStepIters) return;
    const int B = kStepIters, D = S.D, b = 1 - C.tree_a;
    const int c = (int)S.conn[i];
    if (!S.valid2[i] || c < 0 || S.newidx[i] < 0) return;
    float s2 = 0.f;
    for (int d = 0; d < D; ++d) {
        const float t = S.qconn[(size_t)d * B + i] - S.qnew[(size_t)d * B + i];
        s2 = fmaf(t, t, s2);
    }
    const float cost = S.gnew[i] + sqrtf(s2) + S.tq[b][(size_t)D * S.tcap + c];
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)i;
    atomicMin(&C.best_key, key);
}

__global__ void k_solution(const Slot *__restrict__ slots) {
    solution_body(slots[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

// Path of the winning iteration: root_a .. z_new, then z_conn .. root_b.
// One thread follows the parents; the configurations are written to
// out_q [cap][D] in that order (reversed to start -> goal by the host when the
// expanded tree was the goal tree).
__device__ __forceinline__ void extract_body(const Slot &S, int it, int *scratch, float *out_q,
                                             int cap, int *len_out) {
    const int a = S.ctrl->tree_a, b = 1 - a, D = S.D;
    int na = 0;
    for (int v = S.newidx[it]; v >= 0 && na < cap; v = S.tpar[a][v]) scratch[na++] = v;
    int n = 0;
    for (int k = na - 1; k >= 0; --k, ++n)
        for (int d = 0; d < D; ++d) out_q[(size_t)n * D + d] = S.tq[a][(size_t)d * S.tcap + scratch[k]];
    for (int v = (int)S.conn[it]; v >= 0 && n < cap; v = S.tpar[b][v], ++n)
        for (int d = 0; d < D; ++d) out_q[(size_t)n * D + d] = S.tq[b][(size_t)d * S.tcap + v];
    *len_out = n;
}

__global__ void k_extract(const Slot *__restrict__ slots, int it, int *scratch, float *out_q,
                          int cap, int *len_out) {
    extract_body(slots[0], it, scratch, out_q, cap, len_out);
}

// ---------------------------------------------------------------------------
// roadmap building blocks (one robot of one slot)
// ---------------------------------------------------------------------------
// Append up to `want` valid candidates (in candidate order) to V_r: one
// block; a block-wide prefix count of the valid flags gives every candidate
// its slot, chunk after chunk.
constexpr int kAppendThreads = 256;
__device__ __forceinline__ void append_valid(const float *cand, const uint8_t *valid, int n,
                                             int dof, int want, float *V, int rcap, int *count) {
    __shared__ int warp_sum[kAppendThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = *count;
    const int room = max(0, min(want, rcap - c0));
    __syncthreads();  // every thread has read *count before thread 0 rewrites it
    int base = 0;     // valid candidates before the current chunk
    for (int i0 = 0; i0 < n && base < room; i0 += kAppendThreads) {
        const int i = i0 + threadIdx.x;
        const bool v = i < n && valid[i];
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) warp_sum[w] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < kAppendThreads / 32; ++k) {
            before += k < w ? warp_sum[k] : 0;
            total += warp_sum[k];
        }
        const int pos = base + before + __popc(bal & ((1u << lane) - 1u));
        if (v && pos < room)
            for (int d = 0; d < dof; ++d) V[(size_t)d * rcap + c0 + pos] = cand[(size_t)d * n + i];
        base += total;
        __syncthreads();  // warp_sum is rewritten by the next chunk
    }
    if (threadIdx.x == 0) *count = c0 + min(base, room);
}

// Roadmap edges in candidate order, one warp: edges go in chunks of 32; in a
// chunk the new-vertex ends are appended first, then the neighbour ends, and
// lanes with the same target vertex take consecutive slots in lane order
// (match + rank), so the adjacency lists (capped at kKmax) do not depend on
// thread timing.  The direction oracle's choice does not depend on the order
// within a list (ties go to the lowest vertex index).
__device__ __forceinline__ void link_edges(const uint8_t *valid, const int *ea, const int *eb,
                                           int E, int *adj, int *deg) {
    const int lane = threadIdx.x;
    for (int e0 = 0; e0 < E; e0 += 32) {
        const int e = e0 + lane;
        const bool ok = e < E && valid[e] && ea[e] >= 0;
        const int a = ok ? ea[e] : -1, b = ok ? eb[e] : -1;
        for (int side = 0; side < 2; ++side) {
            const int x = side == 0 ? a : b, y = side == 0 ? b : a;
            const unsigned grp = __match_any_sync(0xffffffffu, x);
            const int d0 = x >= 0 ? deg[x] : 0;
            __syncwarp();  // the whole group has read deg[x]
            if (x >= 0) {
                const int slot = d0 + __popc(grp & ((1u << lane) - 1u));
                if (slot < kKmax) adj[(size_t)x * kKmax + slot] = y;
                if (lane == __ffs(grp) - 1) deg[x] = min(d0 + __popc(grp), kKmax);
            }
            __syncwarp();  // deg[] is read again by the other side
        }
    }
}

// Start-goal connectivity of a roadmap: level-synchronous BFS from vertex 0
// in one block (at most n levels), writes whether vertex 1 was reached.
__device__ __forceinline__ void bfs_connected(const int *adj, const int *deg, int n, int *level,
                                              int *connected) {
    __shared__ int changed;
    for (int v = threadIdx.x; v < n; v += blockDim.x) level[v] = v == 0 ? 0 : -1;
    __syncthreads();
    for (int l = 0; l < n; ++l) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            if (level[v] != l) continue;
            const int dg = min(deg[v], kKmax);
            for (int k = 0; k < dg; ++k) {
                const int w = adj[(size_t)v * kKmax + k];
                if (w >= 0 && w < n && level[w] < 0) {
                    level[w] = l + 1;
                    changed = 1;
                }
            }
        }
        __syncthreads();
        const int c = changed;
        __syncthreads();
        if (!c) break;
    }
    if (threadIdx.x == 0) *connected = n > 1 && level[1] >= 0;
}

// ---------------------------------------------------------------------------
// batched ROADMAP rounds: one job per robot of every problem that needs a
// round; every kernel takes a job dimension (blockIdx.y), so a round costs a
// fixed number of launches however many robots and problems take part.
// ---------------------------------------------------------------------------
struct RmJob {
    float *q;               // V_r, SoA [dof][rcap]
    int *adj, *deg, *count;  // adjacency [rcap][kKmax], degrees, vertex count (device)
    int rcap, dof;
    float *cand;            // candidate samples [dof][nc]
    uint8_t *cvalid;
    float *gq;              // vertices whose neighbours are searched [dof][m]
    int64_t *nb, *cnt;      // neighbour lists [m][kKmax] and counts
    float *ea_q, *eb_q;     // candidate edges [dof][emax]
    uint8_t *evalid;
    int *ea, *eb;
    int *level, *conn;      // BFS levels [rcap], start-goal connected flag
    const float *lo, *hi;   // joint limits of this robot
    unsigned long long key, ctr;  // sampling stream
    int nc, want, n_old, emax;
    float delta;
    int m, first;           // written by k_rmb_gather
};

__device__ __forceinline__ void rmb_sample_body(const RmJob &J, int i) {
    if (i >= J.nc) return;
    Rng rng{J.key, J.ctr + (unsigned long long)i * 64ull};
    for (int d = 0; d < J.dof; ++d)
        J.cand[(size_t)d * J.nc + i] = J.lo[d] + rng.uniform() * (J.hi[d] - J.lo[d]);
}

__global__ void k_rmb_sample(const RmJob *__restrict__ jobs) {
    rmb_sample_body(jobs[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(kAppendThreads) k_rmb_append(const RmJob *__restrict__ jobs) {
    const RmJob &J = jobs[blockIdx.y];
    append_valid(J.cand, J.cvalid, J.nc, J.dof, J.want, J.q, J.rcap, J.count);
}

// The vertices whose neighbours are searched: the new ones, and on the first
// round also start and goal (vertices 0 and 1).
__device__ __forceinline__ void rmb_gather_body(RmJob &J, int i, bool lead) {
    const int n_new = *J.count;
    const int first = J.n_old == 2 && n_new > 2 ? 0 : J.n_old;
    const int m = n_new - first;
    if (lead) {
        J.m = m;
        J.first = first;
    }
    if (i >= m) return;
    for (int d = 0; d < J.dof; ++d) J.gq[(size_t)d * m + i] = J.q[(size_t)d * J.rcap + first + i];
}

__global__ void k_rmb_gather(RmJob *__restrict__ jobs) {
    rmb_gather_body(jobs[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x,
                    blockIdx.x == 0 && threadIdx.x == 0);
}

// NEIGHBORS(V_r, c, delta) of Alg. 2 for the gathered vertices: one warp per
// query scans V_r in index order (ballot + prefix count), keeping the first
// kKmax indices within delta; the same test as the NEIGHBORS primitive.
constexpr int kRmNbWarps = 8;
__device__ __forceinline__ void rmb_neighbors_body(const RmJob &J, int i) {
    const int lane = threadIdx.x & 31;
    const int m = J.m, n = *J.count, dof = J.dof;
    if (i >= m) return;
    float qv[MRPOP_MAX_DOF];
#pragma unroll
    for (int d = 0; d < MRPOP_MAX_DOF; ++d) qv[d] = d < dof ? J.gq[(size_t)d * m + i] : 0.f;
    int count = 0;
    for (int c = 0; c < n; c += 32) {
        const int v = c + lane;
        bool in = false;
        if (v < n) {
            float d2 = 0.f;
#pragma unroll
            for (int d = 0; d < MRPOP_MAX_DOF; ++d)
                if (d < dof) {
                    const float a = qv[d] - J.q[(size_t)d * J.rcap + v];
                    d2 = fmaf(a, a, d2);
                }
            in = __fsqrt_rn(d2) <= J.delta;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int pos = count + __popc(bal & ((1u << lane) - 1u));
            if (pos < kKmax) J.nb[(size_t)i * kKmax + pos] = v;
        }
        count += __popc(bal);
    }
    for (int pos = count + lane; pos < kKmax; pos += 32) J.nb[(size_t)i * kKmax + pos] = -1;
    if (lane == 0) J.cnt[i] = count;
}

__global__ void __launch_bounds__(kRmNbWarps * 32) k_rmb_neighbors(const RmJob *__restrict__ jobs) {
    rmb_neighbors_body(jobs[blockIdx.y], blockIdx.x * kRmNbWarps + (threadIdx.x >> 5));
}

// Candidate roadmap edges (gathered vertex, earlier neighbour within delta);
// unused slots up to emax get a NaN edge, which validation rejects unchecked.
__device__ __forceinline__ void rmb_edges_body(const RmJob &J, int e) {
    if (e >= J.emax) return;
    const int E = J.m * kKmax, j = e / kKmax, k = e % kKmax;
    int v = -1, self = -1;
    if (e < E) {
        self = J.first + j;
        const int64_t c = J.cnt[j] < (int64_t)kKmax ? J.cnt[j] : (int64_t)kKmax;
        v = k < c ? (int)J.nb[(size_t)j * kKmax + k] : -1;
    }
    if (v < 0 || v >= self) {
        for (int d = 0; d < J.dof; ++d) {
            J.ea_q[(size_t)d * J.emax + e] = 0.f;
            J.eb_q[(size_t)d * J.emax + e] = nanf_();
        }
        J.ea[e] = -1;
        J.eb[e] = -1;
        return;
    }
    for (int d = 0; d < J.dof; ++d) {
        J.ea_q[(size_t)d * J.emax + e] = J.q[(size_t)d * J.rcap + self];
        J.eb_q[(size_t)d * J.emax + e] = J.q[(size_t)d * J.rcap + v];
    }
    J.ea[e] = self;
    J.eb[e] = v;
}

__global__ void k_rmb_edges(const RmJob *__restrict__ jobs) {
    rmb_edges_body(jobs[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_rmb_link(const RmJob *__restrict__ jobs) {
    const RmJob &J = jobs[blockIdx.y];
    link_edges(J.evalid, J.ea, J.eb, J.m * kKmax, J.adj, J.deg);
}

__global__ void __launch_bounds__(1024) k_rmb_bfs(const RmJob *__restrict__ jobs) {
    const RmJob &J = jobs[blockIdx.y];
    bfs_connected(J.adj, J.deg, *J.count, J.level, J.conn);
}

// (vertex count, connected) of every job, for one copy to the host.
__global__ void k_rmb_collect(const RmJob *__restrict__ jobs, int nj, int *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nj) return;
    out[2 * j] = *jobs[j].count;
    out[2 * j + 1] = *jobs[j].conn;
}

__device__ __forceinline__ void tree_reset_body(const Slot &S) {
    const int D = S.D;
    for (int t = 0; t < 2; ++t) {
        const float *root = t == 0 ? S.start : S.goal;
        for (int d = threadIdx.x; d < D; d += blockDim.x) S.tq[t][(size_t)d * S.tcap] = root[d];
        if (threadIdx.x == 0) {
            S.tq[t][(size_t)D * S.tcap] = 0.f;
            S.tpar[t][0] = -1;
            for (int r = 0; r < S.K; ++r) S.trmv[t][(size_t)r * S.tcap] = t;  // roadmap vertex 0 / 1
            S.tn[t] = 1;
        }
    }
}

__global__ void k_tree_reset(const Slot *__restrict__ slots) { tree_reset_body(slots[blockIdx.x]); }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <class T>
static cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(n, 1));
}

struct RobotRoadmap {
    mrpop_problem *sub = nullptr;   // this robot alone with the obstacles
    float *q = nullptr;             // [dof][rcap]
    int *adj = nullptr, *deg = nullptr;
    int n = 0;                      // host mirror of the vertex count
    bool connected = false;
    // scratch
    float *cand = nullptr, *gq = nullptr, *ea_q = nullptr, *eb_q = nullptr;
    uint8_t *cvalid = nullptr, *evalid = nullptr;
    int64_t *nb = nullptr, *cnt = nullptr;
    int *ea = nullptr, *eb = nullptr;
    int *level = nullptr;  // BFS levels [rcap]
    int *d_conn = nullptr;
    VParams vp_c, vp_e;    // validation of the candidates and of the candidate edges
    int vw_c = 1, vw_e = 1;
    size_t vs_c = 0, vs_e = 0;
};

// Device buffers of the persistent form, per planner (allocated on first use).
struct PerBuffers {
    Slot *slot = nullptr;
    RmJob *jobs = nullptr;
    VParams *vp = nullptr;
    int *seg_parts = nullptr;
    float *best = nullptr;
    double *trace_c = nullptr;
    unsigned long long *trace_ns = nullptr;
    long long *trace_it = nullptr;
    float *hist = nullptr;
    int *hist_len = nullptr;
    int hist_floats = 0;
    VParams vfine{};
    int vfine_w = 1;
    size_t vfine_s = 0;
};

static void per_free(PerBuffers &b) {
    cudaFree(b.slot); cudaFree(b.jobs); cudaFree(b.vp); cudaFree(b.seg_parts); cudaFree(b.best);
    cudaFree(b.trace_c); cudaFree(b.trace_ns); cudaFree(b.trace_it); cudaFree(b.hist);
    cudaFree(b.hist_len);
    b = PerBuffers{};
}

struct Planner {
    mrpop_problem *p = nullptr;
    mrpop_problem *fine = nullptr;  // same scene at resolution / 4
    int K = 0, D = 0, rcap = 0, tcap = 0, n_per_round = 0;
    std::vector<RobotRoadmap> rm;
    int *rm_n = nullptr;
    float *tq[2] = {nullptr, nullptr};
    int *tpar[2] = {nullptr, nullptr}, *trmv[2] = {nullptr, nullptr}, *tn = nullptr;
    float *buf = nullptr;  // step buffers
    int64_t *near = nullptr, *conn = nullptr;
    int *rmvnew = nullptr, *newidx = nullptr;
    uint8_t *valid1 = nullptr, *valid2 = nullptr;
    float *d_lo = nullptr, *d_hi = nullptr, *d_start = nullptr, *d_goal = nullptr,
          *d_centre = nullptr, *d_axis = nullptr;
    Ctrl *ctrl = nullptr;
    Slot slot{};
    VParams vp[2];
    size_t vsmem = 0;
    int vwarps = 1;
    // incumbent
    bool initialised = false, roadmap_ready = false, first_solved = false;
    int mode = 0;  // 0 dRRT, 1 AO-X
    long long iters_in_call = 0, total_iters = 0;
    double c_best = INFINITY;
    std::vector<float> best_path;  // [M][D]
    std::vector<double> trace_t, trace_c;
    std::vector<std::vector<float>> history;  // every accepted incumbent path
    double trace_t0 = 0.0;
    bool released = false;  // device state freed (results kept on the host)
    bool direct = false;    // single robot: no roadmap (Sec. V-C)
    unsigned long long seed = 0;
    int step = 0;
    float *fine_qa = nullptr, *fine_qb = nullptr;  // path re-check buffers
    uint8_t *fine_v = nullptr;
    size_t fine_cap = 0;
    int *d_path = nullptr;
    float *d_pathq = nullptr;
    int *d_len = nullptr;
    PerBuffers per;  // persistent-form buffers (allocated on first use)
};

static mrpop_status make_sub(mrpop_problem *p, int k, float res, mrpop_problem **out) {
    const HostRobot &hr = p->robots[k];
    mrpop_robot r{};
    r.dof = hr.dof;
    r.n_spheres = (int)hr.sphere_link.size();
    r.dh = hr.dh.data();
    r.q_lo = hr.q_lo.data();
    r.q_hi = hr.q_hi.data();
    r.sphere_link = hr.sphere_link.data();
    r.sphere_xyzr = hr.sphere_xyzr.data();
    std::memcpy(r.base, hr.base, sizeof(r.base));
    mrpop_obstacles o{(int)(p->obs_spheres.size() / 4), p->obs_spheres.data(),
                      (int)(p->obs_cuboids.size() / 15), p->obs_cuboids.data()};
    mrpop_config c = p->cfg;
    c.resolution = res;
    return mrpop_create_problem(&r, 1, &o, nullptr, nullptr, &c, out);
}

static mrpop_status make_fine(mrpop_problem *p, mrpop_problem **out) {
    std::vector<mrpop_robot> rs(p->robots.size());
    for (size_t k = 0; k < rs.size(); ++k) {
        const HostRobot &hr = p->robots[k];
        rs[k].dof = hr.dof;
        rs[k].n_spheres = (int)hr.sphere_link.size();
        rs[k].dh = hr.dh.data();
        rs[k].q_lo = hr.q_lo.data();
        rs[k].q_hi = hr.q_hi.data();
        rs[k].sphere_link = hr.sphere_link.data();
        rs[k].sphere_xyzr = hr.sphere_xyzr.data();
        std::memcpy(rs[k].base, hr.base, sizeof(rs[k].base));
    }
    mrpop_obstacles o{(int)(p->obs_spheres.size() / 4), p->obs_spheres.data(),
                      (int)(p->obs_cuboids.size() / 15), p->obs_cuboids.data()};
    mrpop_config c = p->cfg;
    c.resolution = p->cfg.resolution * 0.25f;
    return mrpop_create_problem(rs.data(), (int)rs.size(), &o, nullptr, nullptr, &c, out);
}

static void free_device(Planner *pl);
static mrpop_status planner_init(mrpop_problem *p, Planner **out);

void destroy_planner(Planner *pl) {
    if (!pl) return;
    free_device(pl);
    delete pl;
}

// Frees every device buffer of the planner; host-side results stay.
static void free_device(Planner *pl) {
    for (auto &r : pl->rm) {
        mrpop_destroy_problem(r.sub);
        cudaFree(r.q); cudaFree(r.adj); cudaFree(r.deg); cudaFree(r.cand); cudaFree(r.gq);
        cudaFree(r.ea_q); cudaFree(r.eb_q); cudaFree(r.cvalid); cudaFree(r.evalid);
        cudaFree(r.nb); cudaFree(r.cnt); cudaFree(r.ea); cudaFree(r.eb);
        cudaFree(r.level); cudaFree(r.d_conn);
    }
    mrpop_destroy_problem(pl->fine);
    cudaFree(pl->rm_n);
    for (int t = 0; t < 2; ++t) {
        cudaFree(pl->tq[t]); cudaFree(pl->tpar[t]); cudaFree(pl->trmv[t]);
    }
    cudaFree(pl->tn); cudaFree(pl->buf); cudaFree(pl->near); cudaFree(pl->conn);
    cudaFree(pl->rmvnew); cudaFree(pl->newidx); cudaFree(pl->valid1); cudaFree(pl->valid2);
    cudaFree(pl->d_lo); cudaFree(pl->d_hi); cudaFree(pl->d_start); cudaFree(pl->d_goal);
    cudaFree(pl->d_centre); cudaFree(pl->d_axis); cudaFree(pl->ctrl); cudaFree(pl->d_path);
    cudaFree(pl->d_pathq);
    cudaFree(pl->d_len);
    cudaFree(pl->fine_qa);
    cudaFree(pl->fine_qb);
    cudaFree(pl->fine_v);
    per_free(pl->per);
    pl->fine_qa = pl->fine_qb = nullptr;
    pl->fine_v = nullptr;
    pl->fine_cap = 0;
    for (auto &r : pl->rm) r = RobotRoadmap{};
    pl->rm.clear();
    pl->fine = nullptr;
    pl->rm_n = nullptr;
    for (int t = 0; t < 2; ++t) pl->tq[t] = nullptr, pl->tpar[t] = nullptr, pl->trmv[t] = nullptr;
    pl->tn = nullptr; pl->buf = nullptr; pl->near = pl->conn = nullptr;
    pl->rmvnew = pl->newidx = nullptr; pl->valid1 = pl->valid2 = nullptr;
    pl->d_lo = pl->d_hi = pl->d_start = pl->d_goal = pl->d_centre = pl->d_axis = nullptr;
    pl->ctrl = nullptr; pl->d_path = nullptr; pl->d_pathq = nullptr; pl->d_len = nullptr;
    pl->released = true;
}

// (Re)creates the device state of p's planner; results of a released
// planner (incumbent, path, trace) carry over.
static mrpop_status ensure_planner(mrpop_problem *p) {
    if (p->planner && !p->planner->released) return MRPOP_OK;
    Planner *old = p->planner;
    p->planner = nullptr;
    Planner *pl = nullptr;
    mrpop_status s = planner_init(p, &pl);
    if (s != MRPOP_OK) {
        destroy_planner(pl);
        p->planner = old;
        return s;
    }
    if (old) {
        pl->c_best = old->c_best;
        pl->best_path.swap(old->best_path);
        pl->trace_t.swap(old->trace_t);
        pl->trace_c.swap(old->trace_c);
        pl->history.swap(old->history);
        pl->total_iters = old->total_iters;
        pl->mode = old->c_best < INFINITY ? 1 : 0;
        delete old;
    }
    p->planner = pl;
    return MRPOP_OK;
}

#define PL_TRY(expr)                                       \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_error(_e, #expr); \
    } while (0)
#define ST_TRY(expr)                       \
    do {                                   \
        mrpop_status _s = (expr);          \
        if (_s != MRPOP_OK) return _s;     \
    } while (0)

static mrpop_status planner_init(mrpop_problem *p, Planner **out) {
    if (p->start.empty() || p->goal.empty())
        return set_error(MRPOP_EINVAL, "mrpop_plan: the problem was created without start/goal");
    Planner *pl = new (std::nothrow) Planner();
    if (!pl) return set_error(MRPOP_ENOMEM, "host allocation failed");
    *out = pl;
    pl->p = p;
    pl->K = p->dev.t.K;
    pl->D = p->D;
    pl->rcap = (int)std::max<int64_t>(64, std::min<int64_t>(p->cfg.roadmap_cap, 1 << 20));
    pl->tcap = (int)std::max<int64_t>(1024, std::min<int64_t>(p->cfg.tree_cap, 1 << 22));
    pl->n_per_round = std::max(1, std::min(p->cfg.n_per_round, 4096));
    pl->seed = p->cfg.seed;
    const int K = pl->K, D = pl->D, B = kStepIters, rcap = pl->rcap, tcap = pl->tcap;
    ST_TRY(make_fine(p, &pl->fine));
    pl->rm.resize(K);
    int qoff = 0;
    for (int k = 0; k < K; ++k) {
        RobotRoadmap &r = pl->rm[k];
        const int dof = p->robots[k].dof;
        ST_TRY(make_sub(p, k, p->cfg.resolution, &r.sub));
        const int nc = kOversample * pl->n_per_round;
        const int E = pl->n_per_round * kKmax;
        PL_TRY(dalloc(&r.q, (size_t)dof * rcap));
        PL_TRY(dalloc(&r.adj, (size_t)rcap * kKmax));
        PL_TRY(dalloc(&r.deg, (size_t)rcap));
        PL_TRY(cudaMemset(r.deg, 0, sizeof(int) * rcap));
        PL_TRY(dalloc(&r.cand, (size_t)dof * nc));
        PL_TRY(dalloc(&r.cvalid, (size_t)nc));
        PL_TRY(dalloc(&r.gq, (size_t)dof * pl->n_per_round + 2 * dof));
        PL_TRY(dalloc(&r.nb, (size_t)(pl->n_per_round + 2) * kKmax));
        PL_TRY(dalloc(&r.cnt, (size_t)pl->n_per_round + 2));
        PL_TRY(dalloc(&r.ea_q, (size_t)dof * (E + 2 * kKmax)));
        PL_TRY(dalloc(&r.eb_q, (size_t)dof * (E + 2 * kKmax)));
        PL_TRY(dalloc(&r.evalid, (size_t)E + 2 * kKmax));
        PL_TRY(dalloc(&r.ea, (size_t)E + 2 * kKmax));
        PL_TRY(dalloc(&r.eb, (size_t)E + 2 * kKmax));
        PL_TRY(dalloc(&r.level, (size_t)rcap));
        PL_TRY(dalloc(&r.d_conn, 1));
        // vertices 0 and 1: the robot's start and goal
        for (int d = 0; d < dof; ++d) {
            PL_TRY(cudaMemcpy(r.q + (size_t)d * rcap, &p->start[qoff + d], sizeof(float),
                              cudaMemcpyHostToDevice));
            PL_TRY(cudaMemcpy(r.q + (size_t)d * rcap + 1, &p->goal[qoff + d], sizeof(float),
                              cudaMemcpyHostToDevice));
        }
        r.n = 2;
        ST_TRY(make_vparams(r.sub, r.cand, r.cand, nc, r.cvalid, &r.vp_c, &r.vs_c, &r.vw_c));
        ST_TRY(make_vparams(r.sub, r.ea_q, r.eb_q, E + 2 * kKmax, r.evalid, &r.vp_e, &r.vs_e,
                            &r.vw_e));
        pl->slot.dof[k] = dof;
        pl->slot.qoff[k] = qoff;
        pl->slot.rm_q[k] = r.q;
        pl->slot.rm_adj[k] = r.adj;
        pl->slot.rm_deg[k] = r.deg;
        qoff += dof;
    }
    PL_TRY(dalloc(&pl->rm_n, K));
    std::vector<int> twos(K, 2);
    PL_TRY(cudaMemcpy(pl->rm_n, twos.data(), sizeof(int) * K, cudaMemcpyHostToDevice));
    for (int t = 0; t < 2; ++t) {
        PL_TRY(dalloc(&pl->tq[t], (size_t)(D + 1) * tcap));
        PL_TRY(dalloc(&pl->tpar[t], (size_t)tcap));
        PL_TRY(dalloc(&pl->trmv[t], (size_t)K * tcap));
    }
    PL_TRY(dalloc(&pl->tn, 2));
    // step buffers: qrand, qnear, qnew, qconn [D][B]; crand, gnew, budget2 [B]
    PL_TRY(dalloc(&pl->buf, (size_t)4 * D * B + 3 * B));
    PL_TRY(dalloc(&pl->near, B));
    PL_TRY(dalloc(&pl->conn, B));
    PL_TRY(dalloc(&pl->rmvnew, (size_t)K * B));
    PL_TRY(dalloc(&pl->newidx, B));
    PL_TRY(dalloc(&pl->valid1, B));
    PL_TRY(dalloc(&pl->valid2, B));
    PL_TRY(dalloc(&pl->d_lo, D));
    PL_TRY(dalloc(&pl->d_hi, D));
    PL_TRY(dalloc(&pl->d_start, D));
    PL_TRY(dalloc(&pl->d_goal, D));
    PL_TRY(dalloc(&pl->d_centre, D));
    PL_TRY(dalloc(&pl->d_axis, D));
    PL_TRY(dalloc(&pl->ctrl, 1));
    PL_TRY(dalloc(&pl->d_path, (size_t)2 * tcap + 2));
    PL_TRY(dalloc(&pl->d_pathq, (size_t)(2 * tcap + 2) * D));
    PL_TRY(dalloc(&pl->d_len, 1));
    std::vector<float> centre(D), axis(D);
    double cmin2 = 0.0;
    for (int d = 0; d < D; ++d) {
        const double g = (double)p->goal[d] - p->start[d];
        cmin2 += g * g;
        centre[d] = (float)(0.5 * ((double)p->goal[d] + p->start[d]));
    }
    const double cmin = std::sqrt(cmin2);
    for (int d = 0; d < D; ++d)
        axis[d] = cmin > 0 ? (float)(((double)p->goal[d] - p->start[d]) / cmin) : (d == 0 ? 1.f : 0.f);
    PL_TRY(cudaMemcpy(pl->d_lo, p->q_lo.data(), sizeof(float) * D, cudaMemcpyHostToDevice));
    PL_TRY(cudaMemcpy(pl->d_hi, p->q_hi.data(), sizeof(float) * D, cudaMemcpyHostToDevice));
    PL_TRY(cudaMemcpy(pl->d_start, p->start.data(), sizeof(float) * D, cudaMemcpyHostToDevice));
    PL_TRY(cudaMemcpy(pl->d_goal, p->goal.data(), sizeof(float) * D, cudaMemcpyHostToDevice));
    PL_TRY(cudaMemcpy(pl->d_centre, centre.data(), sizeof(float) * D, cudaMemcpyHostToDevice));
    PL_TRY(cudaMemcpy(pl->d_axis, axis.data(), sizeof(float) * D, cudaMemcpyHostToDevice));

    Slot &S = pl->slot;
    S.K = K; S.D = D; S.rcap = rcap; S.tcap = tcap;
    S.direct = K == 1 ? 1 : 0;
    S.step = p->cfg.delta > 0.f ? p->cfg.delta : 0.5f;
    pl->direct = S.direct != 0;
    S.q_lo = pl->d_lo; S.q_hi = pl->d_hi; S.start = pl->d_start; S.goal = pl->d_goal;
    S.centre = pl->d_centre; S.axis = pl->d_axis; S.c_min = (float)cmin;
    S.rm_n = pl->rm_n;
    for (int t = 0; t < 2; ++t) {
        S.tq[t] = pl->tq[t]; S.tpar[t] = pl->tpar[t]; S.trmv[t] = pl->trmv[t];
    }
    S.tn = pl->tn;
    float *b = pl->buf;
    S.qrand = b; b += (size_t)D * B;
    S.qnear = b; b += (size_t)D * B;
    S.qnew = b; b += (size_t)D * B;
    S.qconn = b; b += (size_t)D * B;
    S.crand = b; b += B;
    S.gnew = b; b += B;
    S.budget2 = b;
    S.near = pl->near; S.conn = pl->conn; S.rmvnew = pl->rmvnew; S.newidx = pl->newidx;
    S.valid1 = pl->valid1; S.valid2 = pl->valid2; S.ctrl = pl->ctrl;
    ST_TRY(make_vparams(p, S.qnear, S.qnew, B, S.valid1, &pl->vp[0], &pl->vsmem, &pl->vwarps));
    ST_TRY(make_vparams(p, S.qnew, S.qconn, B, S.valid2, &pl->vp[1], &pl->vsmem, &pl->vwarps));
    pl->initialised = true;
    return MRPOP_OK;
}

// One common launch shape for a batched validation over several problems
// (blocks of up to 4 warps, the shared memory of the most demanding one;
// each then uses as many warps as its per-warp scratch fits, at least as many
// as it would alone) and the per-problem parameters that go with it.
// edges_per_warp sets the blocks per problem: each block first stages the
// problem's tables, so large batches share that cost among several edges per
// warp (the per-problem work counter still hands out edges one at a time).
static void common_validation(std::vector<VParams> &vps, const std::vector<int> &own_warps,
                              const std::vector<const mrpop_problem *> &probs, int64_t max_edges,
                              int edges_per_warp, int *warps, int *bps, size_t *smem, int *spl) {
    size_t sm = 0;
    int sp = 1;
    for (size_t j = 0; j < vps.size(); ++j) {
        const size_t tab = (size_t)probs[j]->dev.t.n_f4 * sizeof(float4);
        sm = std::max(sm, tab + (size_t)own_warps[j] * vps[j].warp_floats * sizeof(float));
        sp = std::max(sp, probs[j]->dev.t.max_spheres_per_link);
    }
    int wmax = 1;
    std::vector<int> w(vps.size());
    for (size_t j = 0; j < vps.size(); ++j) {
        const size_t tab = (size_t)probs[j]->dev.t.n_f4 * sizeof(float4);
        const size_t per = (size_t)vps[j].warp_floats * sizeof(float);
        w[j] = std::max(own_warps[j], (int)std::min<size_t>(4, (sm - tab) / per));
        wmax = std::max(wmax, w[j]);
    }
    const int64_t per_block = (int64_t)wmax * std::max(1, edges_per_warp);
    const int b = (int)std::max<int64_t>(1, (max_edges + per_block - 1) / per_block);
    for (size_t j = 0; j < vps.size(); ++j) {
        vps[j].warps = w[j];
        vps[j].total_warps = b * w[j];
    }
    *warps = wmax;
    *bps = b;
    *smem = sm;
    *spl = sp;
}

// One ROADMAP round (Alg. 2) for every robot of every listed problem: each
// robot samples n free configurations, links them to the vertices of V_r
// within delta whose edges are free for that robot, and a BFS decides
// whether its start and goal are connected.  All robots of all problems share
// every launch (a job dimension) and one host synchronisation; the vertex
// counts stay on the device between the phases.
static mrpop_status roadmap_round_jobs(const std::vector<Planner *> &pls, cudaStream_t st) {
    std::vector<RmJob> jobs;
    std::vector<VParams> vc, ve;
    std::vector<int> wc, we;
    std::vector<const mrpop_problem *> subs;
    int nc_max = 1, m_max = 1, e_max = 1;
    for (Planner *pl : pls) {
        mrpop_problem *p = pl->p;
        for (int k = 0; k < pl->K; ++k) {
            RobotRoadmap &r = pl->rm[k];
            const int dof = p->robots[k].dof, off = pl->slot.qoff[k];
            RmJob J{};
            J.q = r.q;
            J.adj = r.adj;
            J.deg = r.deg;
            J.count = pl->rm_n + k;
            J.rcap = pl->rcap;
            J.dof = dof;
            J.cand = r.cand;
            J.cvalid = r.cvalid;
            J.gq = r.gq;
            J.nb = r.nb;
            J.cnt = r.cnt;
            J.ea_q = r.ea_q;
            J.eb_q = r.eb_q;
            J.evalid = r.evalid;
            J.ea = r.ea;
            J.eb = r.eb;
            J.level = r.level;
            J.conn = r.d_conn;
            J.lo = pl->d_lo + off;
            J.hi = pl->d_hi + off;
            J.key = mix64(pl->seed * 31ull + 7ull * (unsigned long long)k + 1ull);
            J.ctr = (unsigned long long)(pl->step + 1) * 0x100000ull +
                    (unsigned long long)r.n * 4096ull;
            J.want = r.n >= pl->rcap ? 0 : std::min(pl->n_per_round, pl->rcap - r.n);
            J.nc = kOversample * pl->n_per_round;
            J.n_old = r.n;
            J.emax = (pl->n_per_round + 2) * kKmax;
            J.delta = p->cfg.delta;
            nc_max = std::max(nc_max, J.nc);
            m_max = std::max(m_max, pl->n_per_round + 2);
            e_max = std::max(e_max, J.emax);
            jobs.push_back(J);
            vc.push_back(r.vp_c);
            ve.push_back(r.vp_e);
            wc.push_back(r.vw_c);
            we.push_back(r.vw_e);
            subs.push_back(r.sub);
        }
    }
    const int nj = (int)jobs.size();
    if (nj == 0) return MRPOP_OK;
    int w_c, b_c, spl_c, w_e, b_e, spl_e;
    size_t s_c, s_e;
    common_validation(vc, wc, subs, nc_max, kRoadmapEdgesPerWarp, &w_c, &b_c, &s_c, &spl_c);
    common_validation(ve, we, subs, e_max, kRoadmapEdgesPerWarp, &w_e, &b_e, &s_e, &spl_e);

    RmJob *d_jobs = nullptr;
    VParams *d_vp = nullptr;
    int *d_out = nullptr;
    PL_TRY(scratch_alloc((void **)&d_jobs, sizeof(RmJob) * nj, st));
    PL_TRY(scratch_alloc((void **)&d_vp, sizeof(VParams) * 2 * nj, st));
    PL_TRY(scratch_alloc((void **)&d_out, sizeof(int) * 2 * nj, st));
    struct Release {
        void *a, *b, *c;
        cudaStream_t s;
        ~Release() {
            cudaFreeAsync(a, s);
            cudaFreeAsync(b, s);
            cudaFreeAsync(c, s);
        }
    } release{d_jobs, d_vp, d_out, st};
    PL_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(RmJob) * nj, cudaMemcpyHostToDevice, st));
    PL_TRY(cudaMemcpyAsync(d_vp, vc.data(), sizeof(VParams) * nj, cudaMemcpyHostToDevice, st));
    PL_TRY(cudaMemcpyAsync(d_vp + nj, ve.data(), sizeof(VParams) * nj, cudaMemcpyHostToDevice, st));

    k_rmb_sample<<<dim3((nc_max + 127) / 128, nj), 128, 0, st>>>(d_jobs);
    PL_TRY(cudaGetLastError());
    ST_TRY(launch_validate_batch(d_vp, nj, spl_c, w_c, b_c, s_c, false, st));
    k_rmb_append<<<dim3(1, nj), kAppendThreads, 0, st>>>(d_jobs);
    k_rmb_gather<<<dim3((m_max + 127) / 128, nj), 128, 0, st>>>(d_jobs);
    k_rmb_neighbors<<<dim3((m_max + kRmNbWarps - 1) / kRmNbWarps, nj), kRmNbWarps * 32, 0, st>>>(
        d_jobs);
    k_rmb_edges<<<dim3((e_max + 127) / 128, nj), 128, 0, st>>>(d_jobs);
    PL_TRY(cudaGetLastError());
    ST_TRY(launch_validate_batch(d_vp + nj, nj, spl_e, w_e, b_e, s_e, false, st));
    k_rmb_link<<<dim3(1, nj), 32, 0, st>>>(d_jobs);
    k_rmb_bfs<<<dim3(1, nj), 1024, 0, st>>>(d_jobs);
    k_rmb_collect<<<(nj + 127) / 128, 128, 0, st>>>(d_jobs, nj, d_out);
    PL_TRY(cudaGetLastError());
    std::vector<int> out(2 * (size_t)nj);
    PL_TRY(cudaMemcpyAsync(out.data(), d_out, sizeof(int) * 2 * nj, cudaMemcpyDeviceToHost, st));
    PL_TRY(cudaStreamSynchronize(st));
    int j = 0;
    for (Planner *pl : pls)
        for (int k = 0; k < pl->K; ++k, ++j) {
            pl->rm[k].n = out[2 * (size_t)j];
            pl->rm[k].connected = out[2 * (size_t)j + 1] != 0;
        }
    return MRPOP_OK;
}

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Accepts a candidate path if it is strictly cheaper (FP64 cost) and every
// segment is valid at a quarter of the resolution.
static mrpop_status try_incumbent(Planner *pl, const Slot *d_slot, int it, int tree_a,
                                  cudaStream_t st, double t_now, bool *accepted) {
    *accepted = false;
    const int cap = 2 * pl->tcap + 2, D = pl->D;
    k_extract<<<1, 1, 0, st>>>(d_slot, it, pl->d_path, pl->d_pathq, cap, pl->d_len);
    PL_TRY(cudaGetLastError());
    int len = 0;
    PL_TRY(cudaMemcpyAsync(&len, pl->d_len, sizeof(int), cudaMemcpyDeviceToHost, st));
    PL_TRY(cudaStreamSynchronize(st));
    std::vector<float> path((size_t)len * D);
    PL_TRY(cudaMemcpyAsync(path.data(), pl->d_pathq, sizeof(float) * path.size(),
                           cudaMemcpyDeviceToHost, st));
    PL_TRY(cudaStreamSynchronize(st));
    const int a = tree_a;
    if (a == 1) {  // expanded tree was the goal tree: reverse to start -> goal
        for (int j = 0; j < len / 2; ++j)
            for (int d = 0; d < D; ++d)
                std::swap(path[(size_t)j * D + d], path[(size_t)(len - 1 - j) * D + d]);
    }
    double cost = 0.0;
    for (int j = 0; j + 1 < len; ++j) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) {
            const double t = (double)path[(size_t)(j + 1) * D + d] - path[(size_t)j * D + d];
            s += t * t;
        }
        cost += std::sqrt(s);
    }
    if (!(cost < pl->c_best) || len < 2) return MRPOP_OK;
    // Re-validate every segment at resolution / 4.  A segment is cut into
    // equal sub-edges of at most 31 intervals at that resolution, so that the
    // check spreads over many warps (one warp per sub-edge) instead of a few
    // long edges walked tile after tile; the checkpoint density is the same.
    const double res4 = 0.25 * (double)pl->p->cfg.resolution;
    std::vector<int> parts(len > 1 ? len - 1 : 0);
    int M = 0;
    for (int j = 0; j + 1 < len; ++j) {
        double s2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double t = (double)path[(size_t)(j + 1) * D + d] - path[(size_t)j * D + d];
            s2 += t * t;
        }
        const double n = std::ceil(std::sqrt(s2) / res4);
        parts[j] = (int)std::min(4096.0, std::max(1.0, std::ceil(n / 31.0)));
        M += parts[j];
    }
    std::vector<float> qa((size_t)D * M), qb((size_t)D * M);
    for (int j = 0, e = 0; j + 1 < len; ++j)
        for (int i = 0; i < parts[j]; ++i, ++e) {
            const double t0 = (double)i / parts[j], t1 = (double)(i + 1) / parts[j];
            for (int d = 0; d < D; ++d) {
                const double a = path[(size_t)j * D + d], b = path[(size_t)(j + 1) * D + d];
                qa[(size_t)d * M + e] = i == 0 ? (float)a : (float)(a + t0 * (b - a));
                qb[(size_t)d * M + e] = i + 1 == parts[j] ? (float)b : (float)(a + t1 * (b - a));
            }
        }
    if ((size_t)M > pl->fine_cap) {  // grow-only buffers for the fine re-check
        cudaFree(pl->fine_qa);
        cudaFree(pl->fine_qb);
        cudaFree(pl->fine_v);
        pl->fine_qa = pl->fine_qb = nullptr;
        pl->fine_v = nullptr;
        pl->fine_cap = 0;
        const size_t cap = std::max<size_t>(256, 2 * (size_t)M);
        PL_TRY(cudaMalloc(&pl->fine_qa, sizeof(float) * D * cap));
        PL_TRY(cudaMalloc(&pl->fine_qb, sizeof(float) * D * cap));
        PL_TRY(cudaMalloc(&pl->fine_v, cap));
        pl->fine_cap = cap;
    }
    PL_TRY(cudaMemcpyAsync(pl->fine_qa, qa.data(), sizeof(float) * qa.size(), cudaMemcpyHostToDevice, st));
    PL_TRY(cudaMemcpyAsync(pl->fine_qb, qb.data(), sizeof(float) * qb.size(), cudaMemcpyHostToDevice, st));
    std::vector<uint8_t> v(M);
    ST_TRY(launch_validate(pl->fine, pl->fine_qa, pl->fine_qb, M, pl->fine_v, nullptr, nullptr,
                           nullptr, nullptr, st));
    PL_TRY(cudaMemcpyAsync(v.data(), pl->fine_v, M, cudaMemcpyDeviceToHost, st));
    PL_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < M; ++j)
        if (!v[j]) return MRPOP_OK;  // rejected at the finer resolution
    pl->c_best = cost;
    pl->history.push_back(path);
    pl->best_path.swap(path);
    pl->trace_t.push_back(t_now);
    pl->trace_c.push_back(cost);
    *accepted = true;
    return MRPOP_OK;
}

// One planning batch: slots (problems) that step together.  Every slot's
// Ctrl lives in one device array so that a step needs one copy each way.
struct Batch {
    int n = 0;
    std::vector<Planner *> pls;
    Slot *d_slots = nullptr;
    VParams *d_vp = nullptr;  // [2][n]: connection pass after the extension pass
    Ctrl *d_ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;   // pinned
    int spl = 4, warps = 1, bps = 1;
    bool fine = false;  // reassigned fine stage (only when every slot asks for it)
    size_t smem = 0;
    std::vector<int> slot_warps;  // warps per block that take edges, per slot
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    bool owns = true;  // false: a view over arrays owned by a server
    ~Batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (!owns) return;
        cudaFree(d_slots);
        cudaFree(d_vp);
        cudaFree(d_ctrl);
        if (h_ctrl) cudaFreeHost(h_ctrl);
    }
};

// One launch configuration for all slots of a validation launch: blocks of
// up to 4 warps and the shared memory of the most demanding slot; each slot
// then uses as many of the 4 warps as its per-warp scratch fits into that
// budget (at least the count it would use alone).
static mrpop_status batch_config(Batch &bt) {
    size_t smem = 0;
    int spl = 1;
    for (Planner *pl : bt.pls) {
        const size_t tab = (size_t)pl->p->dev.t.n_f4 * sizeof(float4);
        smem = std::max(smem, tab + (size_t)pl->vwarps * pl->vp[0].warp_floats * sizeof(float));
        spl = std::max(spl, pl->p->dev.t.max_spheres_per_link);
    }
    bt.slot_warps.assign(bt.pls.size(), 1);
    int wmax = 1;
    for (size_t i = 0; i < bt.pls.size(); ++i) {
        Planner *pl = bt.pls[i];
        const size_t tab = (size_t)pl->p->dev.t.n_f4 * sizeof(float4);
        const size_t per = (size_t)pl->vp[0].warp_floats * sizeof(float);
        int w = (int)std::min<size_t>(4, (smem - tab) / per);
        w = std::max(w, pl->vwarps);
        bt.slot_warps[i] = w;
        wmax = std::max(wmax, w);
    }
    bt.warps = wmax;
    bt.smem = smem;
    bt.spl = spl;
    bt.fine = !bt.pls.empty();
    for (Planner *pl : bt.pls) bt.fine = bt.fine && pl->vp[0].fine != 0;
    bt.bps = (kStepIters + wmax - 1) / wmax;
    return MRPOP_OK;
}

static mrpop_status enqueue_step(Batch &bt, cudaStream_t st) {
    const int n = bt.n;
    const dim3 g1((kStepIters + 127) / 128, n), gq(kStepIters / kPQB, n);
    k_sample<<<g1, 128, 0, st>>>(bt.d_slots);
    k_nearest<0><<<gq, kPThreads, 0, st>>>(bt.d_slots);
    k_oracle<<<g1, 128, 0, st>>>(bt.d_slots);
    PL_TRY(cudaGetLastError());
    ST_TRY(launch_validate_batch(bt.d_vp, n, bt.spl, bt.warps, bt.bps, bt.smem, bt.fine, st));
    k_insert<<<dim3(1, n), kStepIters, 0, st>>>(bt.d_slots);
    k_nearest<1><<<gq, kPThreads, 0, st>>>(bt.d_slots);
    k_conn_prep<<<g1, 128, 0, st>>>(bt.d_slots);
    PL_TRY(cudaGetLastError());
    ST_TRY(launch_validate_batch(bt.d_vp + n, n, bt.spl, bt.warps, bt.bps, bt.smem, bt.fine,
                                 st));
    k_solution<<<g1, 128, 0, st>>>(bt.d_slots);
    PL_TRY(cudaGetLastError());
    return MRPOP_OK;
}

static mrpop_status build_batch(Batch &bt, cudaStream_t st) {
    const int n = bt.n;
    PL_TRY(cudaMalloc(&bt.d_slots, sizeof(Slot) * n));
    PL_TRY(cudaMalloc(&bt.d_vp, sizeof(VParams) * 2 * n));
    PL_TRY(cudaMalloc(&bt.d_ctrl, sizeof(Ctrl) * n));
    PL_TRY(cudaMallocHost(&bt.h_ctrl, sizeof(Ctrl) * n));
    ST_TRY(batch_config(bt));
    std::vector<Slot> slots(n);
    std::vector<VParams> vps(2 * n);
    for (int i = 0; i < n; ++i) {
        Planner *pl = bt.pls[i];
        slots[i] = pl->slot;
        slots[i].ctrl = bt.d_ctrl + i;
        for (int k = 0; k < 2; ++k) {
            vps[(size_t)k * n + i] = pl->vp[k];
            vps[(size_t)k * n + i].warps = bt.slot_warps[i];
            vps[(size_t)k * n + i].total_warps = bt.bps * bt.slot_warps[i];
        }
    }
    PL_TRY(cudaMemcpy(bt.d_slots, slots.data(), sizeof(Slot) * n, cudaMemcpyHostToDevice));
    PL_TRY(cudaMemcpy(bt.d_vp, vps.data(), sizeof(VParams) * 2 * n, cudaMemcpyHostToDevice));
    std::vector<Ctrl> idle(n);
    for (auto &c : idle) {
        c = Ctrl{};
        c.mode = 2;
        c.c_best = INFINITY;
        c.best_key = ~0ull;
    }
    PL_TRY(cudaMemcpy(bt.d_ctrl, idle.data(), sizeof(Ctrl) * n, cudaMemcpyHostToDevice));
    // one uncaptured step (sets kernel attributes), then capture the step
    ST_TRY(enqueue_step(bt, st));
    PL_TRY(cudaStreamSynchronize(st));
    PL_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    mrpop_status s = enqueue_step(bt, st);
    cudaError_t e = cudaStreamEndCapture(st, &bt.graph);
    if (s != MRPOP_OK) return s;
    PL_TRY(e);
    PL_TRY(cudaGraphInstantiate(&bt.exec, bt.graph, 0));
    return MRPOP_OK;
}

// A target is reached by an actual solution only (a target of +inf means
// "the first solution").
static inline bool reached_target(double c_best, double target) {
    return c_best < INFINITY && c_best <= target;
}

struct SlotRun {
    bool active = false, need_roadmap = true, reset_trees = true, reached = false;
    double target = -INFINITY;
    mrpop_status status = MRPOP_OK;
};

// Part of one outer iteration before the step: one ROADMAP round (Alg. 2) for
// every listed slot that needs one, all robots of all those slots sharing two
// host synchronisations; a slot whose robots all connect start and goal
// rejoins the search, its trees restarted from the roots for AO-X.
static mrpop_status roadmap_rounds(const std::vector<Planner *> &pls, std::vector<SlotRun *> &runs,
                                   const Slot *d_slots, cudaStream_t st) {
    std::vector<int> todo;
    for (size_t i = 0; i < pls.size(); ++i) {
        if (!runs[i]->active || !runs[i]->need_roadmap) continue;
        if (pls[i]->direct) {  // single robot: no roadmap, start from the roots
            SlotRun &run = *runs[i];
            run.need_roadmap = false;
            pls[i]->roadmap_ready = true;
            pls[i]->iters_in_call = 0;
            if (pls[i]->mode == 1 || run.reset_trees) {
                k_tree_reset<<<1, 64, 0, st>>>(d_slots + i);
                PL_TRY(cudaGetLastError());
                run.reset_trees = false;
            }
            continue;
        }
        todo.push_back((int)i);
    }
    if (todo.empty()) return MRPOP_OK;
    std::vector<Planner *> round;
    for (int i : todo) round.push_back(pls[i]);
    ST_TRY(roadmap_round_jobs(round, st));
    for (int i : todo) {
        Planner *pl = pls[i];
        SlotRun &run = *runs[i];
        bool all = true;
        for (int k = 0; k < pl->K; ++k) all = all && pl->rm[k].connected;
        ++pl->step;
        if (!all) continue;
        pl->roadmap_ready = true;
        run.need_roadmap = false;
        pl->iters_in_call = 0;
        if (pl->mode == 1 || run.reset_trees) {
            k_tree_reset<<<1, 64, 0, st>>>(d_slots + i);
            PL_TRY(cudaGetLastError());
            run.reset_trees = false;
        }
    }
    return MRPOP_OK;
}

static void slot_ctrl(Planner *pl, const SlotRun &run, Ctrl &c) {
    c = Ctrl{};
    c.c_best = pl->c_best < INFINITY ? (float)pl->c_best : INFINITY;
    c.mode = run.active && !run.need_roadmap ? pl->mode : 2;
    c.step = pl->step++;
    c.seed = pl->seed;
    c.best_key = ~0ull;
}

// Per-slot part after the step: incumbent candidates and Alg. 1 transitions.
static mrpop_status slot_after(Planner *pl, SlotRun &run, const Ctrl &r, const Slot *d_slot,
                               cudaStream_t st, double t_rel) {
    if (!run.active || run.need_roadmap) return MRPOP_OK;
    pl->iters_in_call += kStepIters;
    pl->total_iters += kStepIters;
    bool accepted = false;
    if (r.best_key != ~0ull)
        ST_TRY(try_incumbent(pl, d_slot, (int)(r.best_key & 0xffffffffu), r.tree_a, st, t_rel,
                             &accepted));
    const long long max_iters = std::max<long long>(kStepIters, pl->p->cfg.max_iters);
    if (accepted) {
        pl->mode = 1;             // from now on: AO-X
        run.need_roadmap = true;  // Alg. 1: grow the roadmap, optimise again
        if (pl->direct) {         // single robot: no roadmap; AO-X restarts from the roots
            run.need_roadmap = false;
            pl->iters_in_call = 0;
            k_tree_reset<<<1, 64, 0, st>>>(d_slot);
            PL_TRY(cudaGetLastError());
        }
        if (reached_target(pl->c_best, run.target)) {
            run.active = false;
            run.reached = true;
        }
    } else if (pl->iters_in_call >= max_iters || r.overflow) {
        if (pl->direct) {
            // single robot: the search continues; AO-X and full trees restart
            if (pl->mode == 1 || r.overflow) {
                k_tree_reset<<<1, 64, 0, st>>>(d_slot);
                PL_TRY(cudaGetLastError());
            }
            pl->iters_in_call = 0;
        } else {
            run.need_roadmap = true;  // iteration cap: grow the roadmap (c14)
            if (r.overflow) run.reset_trees = true;
        }
    }
    return MRPOP_OK;
}

static mrpop_status check_endpoints(const std::vector<Planner *> &pls, std::vector<SlotRun> &run,
                                    cudaStream_t st) {
    const int n = (int)pls.size();
    uint8_t *dv = nullptr;
    PL_TRY(cudaMalloc(&dv, 2 * (size_t)n));
    std::vector<uint8_t> sv(2 * (size_t)n);
    mrpop_status s = MRPOP_OK;
    for (int i = 0; i < n && s == MRPOP_OK; ++i) {
        Planner *pl = pls[i];
        s = launch_validate(pl->p, pl->d_start, pl->d_start, 1, dv + 2 * i, nullptr, nullptr,
                            nullptr, nullptr, st);
        if (s == MRPOP_OK)
            s = launch_validate(pl->p, pl->d_goal, pl->d_goal, 1, dv + 2 * i + 1, nullptr, nullptr,
                                nullptr, nullptr, st);
    }
    cudaError_t e = cudaMemcpyAsync(sv.data(), dv, 2 * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dv);
    if (s != MRPOP_OK) return s;
    PL_TRY(e);
    for (int i = 0; i < n; ++i) {
        run[i].active = sv[2 * i] && sv[2 * i + 1];
        if (!run[i].active) run[i].status = MRPOP_EINVAL;
        if (reached_target(pls[i]->c_best, run[i].target)) {
            run[i].active = false;
            run[i].reached = true;
        }
    }
    return MRPOP_OK;
}

// Runs Alg. 1 on every problem of ps at once until the budget ends or every
// problem reached its target cost.
static mrpop_status plan_batch(mrpop_problem *const *ps, int n, double budget, int64_t max_steps,
                               const double *targets, mrpop_status *statuses) {
    const double t0 = now_s();
    cudaStream_t st;
    PL_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct Guard {
        cudaStream_t s;
        ~Guard() { cudaStreamDestroy(s); }
    } guard{st};
    Batch bt;
    bt.n = n;
    std::vector<SlotRun> run(n);
    for (int i = 0; i < n; ++i) {
        mrpop_problem *p = ps[i];
        ST_TRY(ensure_planner(p));
        bt.pls.push_back(p->planner);
        run[i].target = targets ? targets[i] : -INFINITY;
        run[i].reset_trees = !p->planner->roadmap_ready;
    }
    ST_TRY(check_endpoints(bt.pls, run, st));
    ST_TRY(build_batch(bt, st));
    for (int64_t outer = 0; now_s() - t0 < budget && (max_steps <= 0 || outer < max_steps); ++outer) {
        bool any = false;
        std::vector<SlotRun *> rp;
        for (int i = 0; i < n; ++i) {
            any = any || run[i].active;
            rp.push_back(&run[i]);
        }
        if (!any) break;
        ST_TRY(roadmap_rounds(bt.pls, rp, bt.d_slots, st));
        for (int i = 0; i < n; ++i) slot_ctrl(bt.pls[i], run[i], bt.h_ctrl[i]);
        PL_TRY(cudaMemcpyAsync(bt.d_ctrl, bt.h_ctrl, sizeof(Ctrl) * n, cudaMemcpyHostToDevice, st));
        PL_TRY(cudaGraphLaunch(bt.exec, st));
        PL_TRY(cudaMemcpyAsync(bt.h_ctrl, bt.d_ctrl, sizeof(Ctrl) * n, cudaMemcpyDeviceToHost, st));
        PL_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i)
            ST_TRY(slot_after(bt.pls[i], run[i], bt.h_ctrl[i], bt.d_slots + i, st, now_s() - t0));
    }
    if (statuses)
        for (int i = 0; i < n; ++i) statuses[i] = run[i].status;
    return MRPOP_OK;
}


// ---------------------------------------------------------------------------
// Persistent batched planner.  One launch of CTAs resident on every SM runs
// Alg. 1 for every problem of the batch until each is done (time budget,
// step budget or target cost).  Every problem carries a state machine of
// phases -- a ROADMAP round is sample, candidate validation, append,
// NEIGHBORS, candidate edges, edge validation and link + BFS for each robot
// in turn; a search step is the nine phases of the stepped form; an
// incumbent candidate is re-checked at a quarter of the resolution -- and
// each phase is cut into chunks (256 samples or iterations, 16 NEAREST
// queries, 32 edges, 8 NEIGHBORS queries).  CTAs claim chunks of any problem
// with one atomic add on the problem's phase word, which carries the phase
// itself (kind, robot, chunk count) beside the next chunk, so a claim always
// names the phase it belongs to.  The CTA that finishes a phase's last chunk
// runs the transition (Alg. 1 bookkeeping on the device, in the stepped
// form's order) and publishes the next phase.  No CTA waits for another: a
// CTA that finds no chunk polls again after a short sleep, and gives up (a
// timeout flag) only past a hard deadline or an optional poll limit.  Every
// phase of a problem writes fixed positions, and its sequential parts run in
// single-chunk phases, so a problem evolves the same alone or in a mix.
// ---------------------------------------------------------------------------
enum PKind : int {
    PK_BEGIN = 0,
    PK_RM_SAMPLE, PK_RM_VALC, PK_RM_APPEND, PK_RM_NB, PK_RM_EDGES, PK_RM_VALE, PK_RM_LINK,
    PK_ST_SAMPLE, PK_ST_NN0, PK_ST_ORACLE, PK_ST_VAL1, PK_ST_INSERT, PK_ST_NN1, PK_ST_CONN,
    PK_ST_VAL2, PK_ST_SOLUTION, PK_FINE_VAL, PK_FINE_ACCEPT,
    PK_DONE
};
constexpr int kPerThreads = 256;          // threads per persistent CTA (= kStepIters)
constexpr int kPerWarps = kPerThreads / 32;
constexpr int kPerEdges = 32;             // edges per validation chunk
constexpr int kFineCap = 16384;           // sub-edges per fine re-check window
constexpr int kTraceCap = 256;            // incumbents recorded per problem
constexpr int kHistCap = 64;              // incumbent paths kept per problem
static_assert(kPerThreads == kStepIters, "one search-step iteration per thread");

// Phase word: kind (6 bits) | robot (6) | chunk count (20) | next chunk (32).
__host__ __device__ __forceinline__ unsigned long long phase_word(int kind, int robot, int total) {
    return ((unsigned long long)kind << 58) | ((unsigned long long)(robot & 63) << 52) |
           ((unsigned long long)(total & 0xFFFFF) << 32);
}

struct PState {
    unsigned long long claim;  // phase word
    int done;                  // chunks of the current phase finished
    int finished;              // 1 once the problem reached PK_DONE
    // Alg. 1 control (the stepped form keeps these on the host)
    int mode, step, need_roadmap, reset_trees, roadmap_ready, active, reached, direct, K, D;
    int timed_out;             // stopped by the time budget
    long long iters_in_call, total_iters, max_iters, steps_done, max_steps;
    double c_best, target;
    unsigned long long seed;
    int n_per_round, rcap;
    float res4;                // resolution / 4 (fine re-check)
    // incumbent candidate of the current step
    int cand_len, fine_M, fine_done, fine_cnt, fine_bad, accepted;
    double cand_cost;
    // results
    int best_len, n_trace, n_hist, hist_used;
    // device buffers
    Slot *slot;
    RmJob *jobs;               // [K]
    VParams *vp;               // [0] extension, [1] connection, [2] fine re-check,
                               // [3 + k] candidates, [3 + K + k] roadmap edges of robot k
    int *scratch;              // [path_cap] path indices, then segment offsets
    int *seg_parts;            // [path_cap]
    float *cand_path, *best_path;  // [path_cap][D]
    int path_cap;
    float *fine_qa, *fine_qb;  // [D][kFineCap]
    uint8_t *fine_v;           // [kFineCap]
    double *trace_c;           // [kTraceCap]
    unsigned long long *trace_ns;
    long long *trace_it;
    float *hist;               // arena of hist_floats
    int *hist_len;             // [kHistCap] (-1: did not fit)
    int hist_floats;
};

struct PLaunch {
    PState *states;
    int n;
    unsigned long long budget_ns, hard_ns;  // per problem budget; give-up horizon
    long long idle_poll_limit;              // consecutive empty polls before giving up (0: none)
    unsigned long long *t_start;            // earliest CTA start (globaltimer)
    int *finished;                          // problems done
    int *timeout;                           // an idle CTA gave up
    // CTA time (ns) and chunks per phase kind; slot PK_DONE holds the phase
    // transitions (decide)
    unsigned long long *phase_ns, *phase_chunks;
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int chunks_of(int n, int per) { return n <= 0 ? 0 : (n + per - 1) / per; }

// Validation of edges [chunk * 32, chunk * 32 + 32) of vp (count edges in all).
__device__ __noinline__ void val_chunk(const VParams &vp, int chunk, int count, float4 *sm4,
                                       int *s_next) {
    if (threadIdx.x == 0) *s_next = 0;
    const int e0 = chunk * kPerEdges, e1 = min(count, e0 + kPerEdges);
    vb::validate_body<vb::kVerdict, false, true>(vp, sm4, e0, e1, s_next);
    __syncthreads();
}

// Sub-edges [w0, w1) of the candidate path (segments cut into equal parts of
// at most 31 intervals at resolution / 4, as in the stepped form) into the
// fine re-check buffers, positions e - w0.
__device__ void fine_window(PState &ps, int w0, int w1) {
    const int len = ps.cand_len, D = ps.D;
    const float *path = ps.cand_path;
    for (int j = threadIdx.x; j + 1 < len; j += blockDim.x) {
        const int off = ps.scratch[j], parts = ps.seg_parts[j];
        for (int i = max(0, w0 - off); i < parts && off + i < w1; ++i) {
            const int e = off + i - w0;
            const double t0 = (double)i / parts, t1 = (double)(i + 1) / parts;
            for (int d = 0; d < D; ++d) {
                const double a = path[(size_t)j * D + d], b = path[(size_t)(j + 1) * D + d];
                ps.fine_qa[(size_t)d * kFineCap + e] = i == 0 ? (float)a : (float)(a + t0 * (b - a));
                ps.fine_qb[(size_t)d * kFineCap + e] =
                    i + 1 == parts ? (float)b : (float)(a + t1 * (b - a));
            }
        }
    }
}

// PK_ST_SOLUTION after k_solution's body: the cheapest connection of the step,
// if any, is extracted, put in start -> goal order and costed in FP64 (fixed
// summation order); a strictly cheaper one gets its fine re-check windows set up.
__device__ void solution_candidate(PState &ps, double *red) {
    const Slot &S = *ps.slot;
    const int tid = threadIdx.x;
    __syncthreads();
    const unsigned long long key = S.ctrl->best_key;
    if (tid == 0) ps.fine_M = 0;
    if (key == ~0ull) return;
    if (tid == 0)
        extract_body(S, (int)(key & 0xffffffffu), ps.scratch, ps.cand_path, ps.path_cap,
                     &ps.cand_len);
    __syncthreads();
    const int len = ps.cand_len, D = ps.D;
    if (S.ctrl->tree_a == 1)  // the expanded tree was the goal tree: reverse
        for (int k = tid; k < (len / 2) * D; k += blockDim.x) {
            const int j = k / D, d = k % D;
            float *x = ps.cand_path + (size_t)j * D + d, *y = ps.cand_path + (size_t)(len - 1 - j) * D + d;
            const float t = *x;
            *x = *y;
            *y = t;
        }
    __syncthreads();
    double c = 0.0;
    for (int j = tid; j + 1 < len; j += blockDim.x) {
        double s2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double t = (double)ps.cand_path[(size_t)(j + 1) * D + d] - ps.cand_path[(size_t)j * D + d];
            s2 += t * t;
        }
        c += sqrt(s2);
        const double n = ceil(sqrt(s2) / (double)ps.res4);
        ps.seg_parts[j] = (int)fmin(4096.0, fmax(1.0, ceil(n / 31.0)));
    }
    red[tid] = c;
    __syncthreads();
    if (tid == 0) {
        double cost = 0.0;
        for (int k = 0; k < blockDim.x; ++k) cost += red[k];
        ps.cand_cost = cost;
        if (cost < ps.c_best && len >= 2) {
            int M = 0;
            for (int j = 0; j + 1 < len; ++j) {
                ps.scratch[j] = M;  // the path indices are no longer needed
                M += ps.seg_parts[j];
            }
            ps.fine_M = M;
            ps.fine_done = 0;
            ps.fine_bad = 0;
            ps.accepted = 0;
            ps.fine_cnt = min(M, kFineCap);
        }
    }
    __syncthreads();
    if (ps.fine_M > 0) fine_window(ps, 0, ps.fine_cnt);
}

// PK_FINE_ACCEPT: the window just checked; the next window, a rejection, or
// the accepted incumbent (best path, trace entry, history entry).
__device__ void fine_accept(PState &ps) {
    const int tid = threadIdx.x;
    bool bad = false;
    for (int e = tid; e < ps.fine_cnt; e += blockDim.x) bad |= ps.fine_v[e] == 0;
    bad = __syncthreads_or(bad);
    if (bad) {
        if (tid == 0) {
            ps.fine_bad = 1;
            ps.accepted = 0;
        }
        return;
    }
    const int done = ps.fine_done + ps.fine_cnt;
    if (done < ps.fine_M) {
        const int cnt = min(kFineCap, ps.fine_M - done);
        __syncthreads();
        if (tid == 0) {
            ps.fine_done = done;
            ps.fine_cnt = cnt;
        }
        fine_window(ps, done, done + cnt);
        return;
    }
    // accepted: every window valid at resolution / 4
    const int len = ps.cand_len, D = ps.D;
    for (int k = tid; k < len * D; k += blockDim.x) ps.best_path[k] = ps.cand_path[k];
    const int h = ps.n_hist;
    const bool keep = h < kHistCap && ps.hist_used + len * D <= ps.hist_floats;
    if (keep)
        for (int k = tid; k < len * D; k += blockDim.x) ps.hist[ps.hist_used + k] = ps.cand_path[k];
    __syncthreads();
    if (tid == 0) {
        ps.fine_done = done;
        ps.accepted = 1;
        ps.c_best = ps.cand_cost;
        ps.best_len = len;
        const int t = ps.n_trace;
        if (t < kTraceCap) {
            ps.trace_c[t] = ps.cand_cost;
            ps.trace_ns[t] = gtimer();
            ps.trace_it[t] = ps.total_iters + kStepIters;  // this step's iterations included
        }
        ps.n_trace = t + 1;
        if (h < kHistCap) {
            ps.hist_len[h] = keep ? len : -1;
            if (keep) ps.hist_used += len * D;
            ps.n_hist = h + 1;
        }
    }
}

__device__ void run_chunk(PState &ps, int kind, int r, int c, float4 *sm4, NnShared<kPerThreads> &nn,
                          int *wsum, int *s_next, double *red) {
    const Slot &S = *ps.slot;
    const int tid = threadIdx.x;
    switch (kind) {
        case PK_RM_SAMPLE: rmb_sample_body(ps.jobs[r], c * kPerThreads + tid); break;
        case PK_RM_VALC: val_chunk(ps.vp[3 + r], c, ps.jobs[r].nc, sm4, s_next); break;
        case PK_RM_APPEND: {
            RmJob &J = ps.jobs[r];
            append_valid(J.cand, J.cvalid, J.nc, J.dof, J.want, J.q, J.rcap, J.count);
            __syncthreads();
            const int n_new = *J.count;
            const int first = J.n_old == 2 && n_new > 2 ? 0 : J.n_old;
            for (int i = tid; i < max(n_new - first, 1); i += blockDim.x)
                rmb_gather_body(J, i, i == 0);
            break;
        }
        case PK_RM_NB: rmb_neighbors_body(ps.jobs[r], c * kPerWarps + (tid >> 5)); break;
        case PK_RM_EDGES: rmb_edges_body(ps.jobs[r], c * kPerThreads + tid); break;
        case PK_RM_VALE: val_chunk(ps.vp[3 + ps.K + r], c, ps.jobs[r].emax, sm4, s_next); break;
        case PK_RM_LINK: {
            const RmJob &J = ps.jobs[r];
            if (tid < 32) link_edges(J.evalid, J.ea, J.eb, J.m * kKmax, J.adj, J.deg);
            __syncthreads();
            bfs_connected(J.adj, J.deg, *J.count, J.level, J.conn);
            break;
        }
        case PK_ST_SAMPLE: sample_body(S, tid); break;
        case PK_ST_NN0: nearest_body<0, kPerThreads>(S, c, nn); break;
        case PK_ST_ORACLE: oracle_body(S, tid); break;
        case PK_ST_VAL1: val_chunk(ps.vp[0], c, kStepIters, sm4, s_next); break;
        case PK_ST_INSERT: insert_body(S, wsum); break;
        case PK_ST_NN1: nearest_body<1, kPerThreads>(S, c, nn); break;
        case PK_ST_CONN: conn_prep_body(S, tid); break;
        case PK_ST_VAL2: val_chunk(ps.vp[1], c, kStepIters, sm4, s_next); break;
        case PK_ST_SOLUTION:
            solution_body(S, tid);
            solution_candidate(ps, red);
            break;
        case PK_FINE_VAL: val_chunk(ps.vp[2], c, ps.fine_cnt, sm4, s_next); break;
        case PK_FINE_ACCEPT: fine_accept(ps); break;
        default: break;
    }
}

// Alg. 1 bookkeeping between phases (thread 0), in the stepped form's order;
// returns the next phase word.  *reset asks the block for a tree reset.
struct PDecision {
    unsigned long long word;
    int reset;
};

__device__ unsigned long long round_setup(PState &ps, int k) {
    RmJob &J = ps.jobs[k];
    const int n = *J.count;
    J.ctr = (unsigned long long)(ps.step + 1) * 0x100000ull + (unsigned long long)n * 4096ull;
    J.want = n >= ps.rcap ? 0 : min(ps.n_per_round, ps.rcap - n);
    J.n_old = n;
    return phase_word(PK_RM_SAMPLE, k, chunks_of(J.nc, kPerThreads));
}

__device__ unsigned long long start_step(PState &ps) {
    Ctrl &C = *ps.slot->ctrl;
    C.c_best = ps.c_best < INFINITY ? (float)ps.c_best : INFINITY;
    C.mode = ps.active && !ps.need_roadmap ? ps.mode : 2;
    C.step = ps.step++;
    C.seed = ps.seed;
    C.tree_a = 0;
    C.best_key = ~0ull;
    C.overflow = 0;
    if (C.mode == 2) return 0ull;  // an idle step changes nothing: the outer iteration ends
    return phase_word(PK_ST_SAMPLE, 0, 1);
}

__device__ PDecision begin_outer(PState &ps, unsigned long long now, unsigned long long deadline);

__device__ PDecision end_outer(PState &ps, unsigned long long now, unsigned long long deadline) {
    ps.steps_done++;
    return begin_outer(ps, now, deadline);
}

__device__ PDecision begin_outer(PState &ps, unsigned long long now, unsigned long long deadline) {
    PDecision d{phase_word(PK_DONE, 0, 0), 0};
    if (!ps.active) return d;
    if (now >= deadline) {
        ps.timed_out = 1;
        return d;
    }
    if (ps.max_steps > 0 && ps.steps_done >= ps.max_steps) return d;
    if (ps.need_roadmap && !ps.direct) {
        d.word = round_setup(ps, 0);
        return d;
    }
    if (ps.need_roadmap) {  // single robot: no roadmap, start from the roots
        ps.need_roadmap = 0;
        ps.roadmap_ready = 1;
        ps.iters_in_call = 0;
        if (ps.mode == 1 || ps.reset_trees) {
            d.reset = 1;
            ps.reset_trees = 0;
        }
    }
    const unsigned long long w = start_step(ps);
    if (w == 0ull) {
        const PDecision e = end_outer(ps, now, deadline);
        return PDecision{e.word, d.reset | e.reset};
    }
    d.word = w;
    return d;
}

__device__ PDecision after_step(PState &ps, bool accepted, unsigned long long now,
                                unsigned long long deadline) {
    PDecision d{0ull, 0};
    ps.iters_in_call += kStepIters;
    ps.total_iters += kStepIters;
    const long long max_it = ps.max_iters > kStepIters ? ps.max_iters : kStepIters;
    const int overflow = ps.slot->ctrl->overflow;
    if (accepted) {
        ps.mode = 1;  // from now on: AO-X
        ps.need_roadmap = 1;
        if (ps.direct) {
            ps.need_roadmap = 0;
            ps.iters_in_call = 0;
            d.reset = 1;
        }
        if (ps.c_best < INFINITY && ps.c_best <= ps.target) {
            ps.active = 0;
            ps.reached = 1;
        }
    } else if (ps.iters_in_call >= max_it || overflow) {
        if (ps.direct) {
            if (ps.mode == 1 || overflow) d.reset = 1;
            ps.iters_in_call = 0;
        } else {
            ps.need_roadmap = 1;
            if (overflow) ps.reset_trees = 1;
        }
    }
    const PDecision e = end_outer(ps, now, deadline);
    return PDecision{e.word, d.reset | e.reset};
}

__device__ PDecision decide(PState &ps, int kind, int r, unsigned long long now,
                            unsigned long long deadline) {
    switch (kind) {
        case PK_BEGIN: return begin_outer(ps, now, deadline);
        case PK_RM_SAMPLE: return {phase_word(PK_RM_VALC, r, chunks_of(ps.jobs[r].nc, kPerEdges)), 0};
        case PK_RM_VALC: return {phase_word(PK_RM_APPEND, r, 1), 0};
        case PK_RM_APPEND: return {phase_word(PK_RM_NB, r, chunks_of(ps.jobs[r].m, kPerWarps)), 0};
        case PK_RM_NB: return {phase_word(PK_RM_EDGES, r, chunks_of(ps.jobs[r].emax, kPerThreads)), 0};
        case PK_RM_EDGES: return {phase_word(PK_RM_VALE, r, chunks_of(ps.jobs[r].emax, kPerEdges)), 0};
        case PK_RM_VALE: return {phase_word(PK_RM_LINK, r, 1), 0};
        case PK_RM_LINK: {
            if (r + 1 < ps.K) return {round_setup(ps, r + 1), 0};
            // the round is over for every robot (Alg. 2 ROADMAP)
            bool all = true;
            for (int k = 0; k < ps.K; ++k) all = all && *ps.jobs[k].conn != 0;
            ps.step++;
            PDecision d{0ull, 0};
            if (all) {
                ps.roadmap_ready = 1;
                ps.need_roadmap = 0;
                ps.iters_in_call = 0;
                if (ps.mode == 1 || ps.reset_trees) {
                    d.reset = 1;
                    ps.reset_trees = 0;
                }
            }
            const unsigned long long w = start_step(ps);
            if (w != 0ull) {
                d.word = w;
                return d;
            }
            const PDecision e = end_outer(ps, now, deadline);
            return {e.word, d.reset | e.reset};
        }
        case PK_ST_SAMPLE: return {phase_word(PK_ST_NN0, 0, kStepIters / kPQB), 0};
        case PK_ST_NN0: return {phase_word(PK_ST_ORACLE, 0, 1), 0};
        case PK_ST_ORACLE: return {phase_word(PK_ST_VAL1, 0, kStepIters / kPerEdges), 0};
        case PK_ST_VAL1: return {phase_word(PK_ST_INSERT, 0, 1), 0};
        case PK_ST_INSERT: return {phase_word(PK_ST_NN1, 0, kStepIters / kPQB), 0};
        case PK_ST_NN1: return {phase_word(PK_ST_CONN, 0, 1), 0};
        case PK_ST_CONN: return {phase_word(PK_ST_VAL2, 0, kStepIters / kPerEdges), 0};
        case PK_ST_VAL2: return {phase_word(PK_ST_SOLUTION, 0, 1), 0};
        case PK_ST_SOLUTION:
            if (ps.fine_M > 0) return {phase_word(PK_FINE_VAL, 0, chunks_of(ps.fine_cnt, kPerEdges)), 0};
            return after_step(ps, false, now, deadline);
        case PK_FINE_VAL: return {phase_word(PK_FINE_ACCEPT, 0, 1), 0};
        case PK_FINE_ACCEPT:
            if (ps.fine_bad) return after_step(ps, false, now, deadline);
            if (!ps.accepted) return {phase_word(PK_FINE_VAL, 0, chunks_of(ps.fine_cnt, kPerEdges)), 0};
            return after_step(ps, true, now, deadline);
        default: return {phase_word(PK_DONE, 0, 0), 0};
    }
}

__global__ void __launch_bounds__(kPerThreads) k_persistent(const PLaunch L) {
    extern __shared__ float4 per_sm4[];
    __shared__ NnShared<kPerThreads> nn;
    __shared__ int wsum[kPerWarps];
    __shared__ double red[kPerThreads];
    __shared__ int s_q, s_kind, s_robot, s_chunk, s_total, s_last, s_exit, s_next, s_reset;
    __shared__ unsigned long long s_t0, s_word;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const unsigned long long now = gtimer();
        const unsigned long long prev = atomicMin(L.t_start, now);
        s_t0 = prev < now ? prev : now;
    }
    __syncthreads();
    const unsigned long long t0 = s_t0, deadline = t0 + L.budget_ns, hard = t0 + L.hard_ns;
    int scan = blockIdx.x % max(L.n, 1);
    long long idle = 0;
    for (;;) {
        if (tid == 0) {
            s_q = -1;
            s_exit = 0;
            for (int j = 0; j < L.n && s_q < 0; ++j) {
                const int q = (scan + j) % L.n;
                PState &ps = L.states[q];
                const unsigned long long w = *(volatile unsigned long long *)&ps.claim;
                if ((unsigned)(w & 0xffffffffull) >= (unsigned)((w >> 32) & 0xFFFFF)) continue;
                const unsigned long long got = atomicAdd(&ps.claim, 1ull);
                const int tot = (int)((got >> 32) & 0xFFFFF), c = (int)(got & 0xffffffffull);
                if (c >= tot) continue;
                s_q = q;
                s_kind = (int)(got >> 58);
                s_robot = (int)((got >> 52) & 63);
                s_total = tot;
                s_chunk = c;
                // the next claim starts at the next problem: the CTAs spread
                // over the problems, so a phase with many chunks (a many-arm
                // problem's long edges) runs on many CTAs at once
                scan = (q + 1) % L.n;
            }
            if (s_q < 0) {
                if (*(volatile int *)L.finished >= L.n) {
                    s_exit = 1;
                } else if (gtimer() > hard || (L.idle_poll_limit > 0 && ++idle > L.idle_poll_limit)) {
                    atomicExch(L.timeout, 1);  // bounded wait ran out
                    s_exit = 1;
                } else {
                    scan = (scan + 1) % L.n;
                    __nanosleep(2000);
                }
            } else {
                idle = 0;
            }
        }
        __syncthreads();
        if (s_exit) break;
        if (s_q < 0) continue;
        __threadfence();  // acquire: the phase's inputs, written by other CTAs
        PState &ps = L.states[s_q];
        const unsigned long long tc0 = tid == 0 ? gtimer() : 0ull;
        run_chunk(ps, s_kind, s_robot, s_chunk, per_sm4, nn, wsum, &s_next, red);
        __threadfence();  // release: this chunk's results
        __syncthreads();
        if (tid == 0) {
            atomicAdd(L.phase_ns + s_kind, gtimer() - tc0);
            atomicAdd(L.phase_chunks + s_kind, 1ull);
        }
        if (tid == 0) s_last = atomicAdd(&ps.done, 1) == s_total - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            const unsigned long long td0 = tid == 0 ? gtimer() : 0ull;
            if (tid == 0) {
                const unsigned long long now = gtimer();
                PDecision d = decide(ps, s_kind, s_robot, now, deadline);
                // a phase without chunks (no new roadmap vertex to search
                // around) is complete at once
                for (int g = 0; g < 16; ++g) {
                    const int k2 = (int)(d.word >> 58);
                    if (k2 == PK_DONE || ((d.word >> 32) & 0xFFFFF) != 0) break;
                    const PDecision d2 = decide(ps, k2, (int)((d.word >> 52) & 63), now, deadline);
                    d = PDecision{d2.word, d.reset | d2.reset};
                }
                s_word = d.word;
                s_reset = d.reset;
            }
            __syncthreads();
            if (s_reset) tree_reset_body(*ps.slot);
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                ps.done = 0;
                const bool fin = (int)(s_word >> 58) == PK_DONE;
                if (fin) ps.finished = 1;
                __threadfence();
                atomicExch(&ps.claim, s_word);  // publish the next phase
                if (fin) atomicAdd(L.finished, 1);
                atomicAdd(L.phase_ns + PK_DONE, gtimer() - td0);
                atomicAdd(L.phase_chunks + PK_DONE, 1ull);
            }
        }
        __syncthreads();
    }
}

// Where the last persistent launch's CTA time went, per phase kind
// (mrpop_plan_batch_phase_stats).
constexpr int kPhaseKinds = PK_DONE + 1;
static_assert(kPhaseKinds == MRPOP_PLAN_PHASES, "phase kinds of the header");
static std::mutex g_phase_mu;
static int64_t g_phase_ns[kPhaseKinds] = {};
static int64_t g_phase_chunks[kPhaseKinds] = {};
static int64_t g_phase_ctas = 0, g_phase_wall_ns = 0;

// Test and diagnostic limits of the persistent launch (mrpop_set_persistent_limits).
static std::atomic<int> g_per_ctas{0};
static std::atomic<long long> g_per_idle_polls{0};

// Static per-robot fields of the roadmap jobs (the round-dependent ones are
// set on the device before each round).
static RmJob make_job(Planner *pl, int k) {
    mrpop_problem *p = pl->p;
    RobotRoadmap &r = pl->rm[k];
    const int off = pl->slot.qoff[k];
    RmJob J{};
    J.q = r.q; J.adj = r.adj; J.deg = r.deg; J.count = pl->rm_n + k;
    J.rcap = pl->rcap; J.dof = p->robots[k].dof;
    J.cand = r.cand; J.cvalid = r.cvalid; J.gq = r.gq; J.nb = r.nb; J.cnt = r.cnt;
    J.ea_q = r.ea_q; J.eb_q = r.eb_q; J.evalid = r.evalid; J.ea = r.ea; J.eb = r.eb;
    J.level = r.level; J.conn = r.d_conn;
    J.lo = pl->d_lo + off; J.hi = pl->d_hi + off;
    J.key = mix64(pl->seed * 31ull + 7ull * (unsigned long long)k + 1ull);
    J.nc = kOversample * pl->n_per_round;
    J.n_old = r.n;
    J.emax = (pl->n_per_round + 2) * kKmax;
    J.delta = p->cfg.delta;
    return J;
}

// Allocates the planner's persistent-form buffers (once) and returns the
// VParams of its validations: extension, connection, fine re-check, then the
// robots' candidates and roadmap edges.
static mrpop_status per_buffers(Planner *pl, std::vector<VParams> &vps) {
    PerBuffers &b = pl->per;
    const int K = pl->K, D = pl->D, cap = 2 * pl->tcap + 2;
    if (!b.slot) {
        PL_TRY(dalloc(&b.slot, 1));
        PL_TRY(dalloc(&b.jobs, K));
        PL_TRY(dalloc(&b.vp, 3 + 2 * K));
        PL_TRY(dalloc(&b.seg_parts, cap));
        PL_TRY(dalloc(&b.best, (size_t)cap * D));
        PL_TRY(dalloc(&b.trace_c, kTraceCap));
        PL_TRY(dalloc(&b.trace_ns, kTraceCap));
        PL_TRY(dalloc(&b.trace_it, kTraceCap));
        b.hist_floats = kHistCap * std::min(cap, 512) * D;
        PL_TRY(dalloc(&b.hist, (size_t)b.hist_floats));
        PL_TRY(dalloc(&b.hist_len, kHistCap));
        if (pl->fine_cap < (size_t)kFineCap) {  // grow the fine re-check buffers
            cudaFree(pl->fine_qa);
            cudaFree(pl->fine_qb);
            cudaFree(pl->fine_v);
            pl->fine_qa = pl->fine_qb = nullptr;
            pl->fine_v = nullptr;
            pl->fine_cap = 0;
            PL_TRY(cudaMalloc(&pl->fine_qa, sizeof(float) * D * kFineCap));
            PL_TRY(cudaMalloc(&pl->fine_qb, sizeof(float) * D * kFineCap));
            PL_TRY(cudaMalloc(&pl->fine_v, kFineCap));
            pl->fine_cap = kFineCap;
        }
        std::vector<RmJob> jobs(K);
        for (int k = 0; k < K; ++k) jobs[k] = make_job(pl, k);
        PL_TRY(cudaMemcpy(b.jobs, jobs.data(), sizeof(RmJob) * K, cudaMemcpyHostToDevice));
        PL_TRY(cudaMemcpy(b.slot, &pl->slot, sizeof(Slot), cudaMemcpyHostToDevice));
    }
    // (the stepped form may have grown the fine re-check buffers since)
    ST_TRY(make_vparams(pl->fine, pl->fine_qa, pl->fine_qb, kFineCap, pl->fine_v, &b.vfine,
                        &b.vfine_s, &b.vfine_w));
    vps.clear();
    vps.push_back(pl->vp[0]);
    vps.push_back(pl->vp[1]);
    vps.push_back(b.vfine);
    for (int k = 0; k < K; ++k) vps.push_back(pl->rm[k].vp_c);
    for (int k = 0; k < K; ++k) vps.push_back(pl->rm[k].vp_e);
    for (VParams &v : vps) v.fine = 0;  // the persistent form takes the union fine stage
    return MRPOP_OK;
}

static const mrpop_problem *vp_problem(Planner *pl, int j) {
    if (j < 2) return pl->p;
    if (j == 2) return pl->fine;
    return pl->rm[(j - 3) % pl->K].sub;
}

// Runs Alg. 1 on every problem of ps in one persistent launch until the
// budget ends, the step budget is used or every problem reached its target.
static mrpop_status plan_batch_persistent(mrpop_problem *const *ps, int n, double budget,
                                          int64_t max_steps, const double *targets,
                                          mrpop_status *statuses) {
    const double t0 = now_s();
    cudaStream_t st;
    PL_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct Guard {
        cudaStream_t s;
        ~Guard() { cudaStreamDestroy(s); }
    } guard{st};
    std::vector<Planner *> pls;
    std::vector<SlotRun> run(n);
    for (int i = 0; i < n; ++i) {
        mrpop_problem *p = ps[i];
        ST_TRY(ensure_planner(p));
        pls.push_back(p->planner);
        run[i].target = targets ? targets[i] : -INFINITY;
        run[i].reset_trees = !p->planner->roadmap_ready;
    }
    ST_TRY(check_endpoints(pls, run, st));
    // one shared-memory budget for every validation of the launch: as many
    // of the 8 warps as fit in about 100 KB (two CTAs per SM), at least one
    std::vector<std::vector<VParams>> vps(n);
    size_t need1 = 0, need8 = 0;
    for (int i = 0; i < n; ++i) {
        ST_TRY(per_buffers(pls[i], vps[i]));
        for (size_t j = 0; j < vps[i].size(); ++j) {
            const size_t tab = (size_t)vp_problem(pls[i], (int)j)->dev.t.n_f4 * sizeof(float4);
            const size_t per = (size_t)vps[i][j].warp_floats * sizeof(float);
            need1 = std::max(need1, tab + per);
            need8 = std::max(need8, tab + kPerWarps * per);
        }
    }
    int dev = 0, optin = 0, sms = 1;
    PL_TRY(cudaGetDevice(&dev));
    PL_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    PL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaFuncAttributes fa{};
    PL_TRY(cudaFuncGetAttributes(&fa, k_persistent));
    const size_t smem = std::max(need1, std::min(need8, (size_t)100 * 1024));
    if (smem + fa.sharedSizeBytes > (size_t)optin)
        return set_error(MRPOP_EINVAL, "plan_batch: a problem's tables exceed the persistent "
                                       "kernel's shared memory (%zu bytes)", smem);
    PL_TRY(cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
    int bps = 0;
    PL_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_persistent, kPerThreads, smem));
    if (bps < 1) return set_error(MRPOP_EINVAL, "plan_batch: persistent kernel does not fit an SM");
    const int ctas = g_per_ctas.load() > 0 ? g_per_ctas.load() : sms * bps;

    // per-problem state from the host mirrors (each call starts with a
    // roadmap round, as Alg. 1 does)
    std::vector<PState> hs(n);
    int finished0 = 0;
    const int64_t msteps = max_steps > 0 ? max_steps : 0;
    for (int i = 0; i < n; ++i) {
        Planner *pl = pls[i];
        PerBuffers &b = pl->per;
        for (size_t j = 0; j < vps[i].size(); ++j) {
            const size_t tab = (size_t)vp_problem(pl, (int)j)->dev.t.n_f4 * sizeof(float4);
            const size_t per = (size_t)vps[i][j].warp_floats * sizeof(float);
            vps[i][j].warps = (int)std::max<size_t>(1, std::min<size_t>(kPerWarps, (smem - tab) / per));
        }
        PL_TRY(cudaMemcpyAsync(b.vp, vps[i].data(), sizeof(VParams) * vps[i].size(),
                               cudaMemcpyHostToDevice, st));
        PState &s = hs[i];
        s = PState{};
        const bool act = run[i].active;
        s.claim = act ? phase_word(PK_BEGIN, 0, 1) : phase_word(PK_DONE, 0, 0);
        s.finished = act ? 0 : 1;
        finished0 += act ? 0 : 1;
        s.mode = pl->mode;
        s.step = pl->step;
        s.need_roadmap = 1;
        s.reset_trees = run[i].reset_trees ? 1 : 0;
        s.roadmap_ready = pl->roadmap_ready ? 1 : 0;
        s.active = act ? 1 : 0;
        s.reached = run[i].reached ? 1 : 0;
        s.direct = pl->direct ? 1 : 0;
        s.K = pl->K;
        s.D = pl->D;
        s.iters_in_call = pl->iters_in_call;
        s.total_iters = pl->total_iters;
        s.max_iters = pl->p->cfg.max_iters;
        s.max_steps = msteps;
        s.c_best = pl->c_best;
        s.target = run[i].target;
        s.seed = pl->seed;
        s.n_per_round = pl->n_per_round;
        s.rcap = pl->rcap;
        s.res4 = 0.25f * pl->p->cfg.resolution;
        s.slot = b.slot;
        s.jobs = b.jobs;
        s.vp = b.vp;
        s.scratch = pl->d_path;
        s.seg_parts = b.seg_parts;
        s.cand_path = pl->d_pathq;
        s.best_path = b.best;
        s.path_cap = 2 * pl->tcap + 2;
        s.fine_qa = pl->fine_qa;
        s.fine_qb = pl->fine_qb;
        s.fine_v = pl->fine_v;
        s.trace_c = b.trace_c;
        s.trace_ns = b.trace_ns;
        s.trace_it = b.trace_it;
        s.hist = b.hist;
        s.hist_len = b.hist_len;
        s.hist_floats = b.hist_floats;
    }
    PState *d_states = nullptr;
    // [0] start time, [1] finished | timeout << 32, then CTA time and chunks
    // per phase kind
    unsigned long long *d_aux = nullptr;
    constexpr int kAux = 2 + 2 * kPhaseKinds;
    PL_TRY(scratch_alloc((void **)&d_states, sizeof(PState) * n, st));
    PL_TRY(scratch_alloc((void **)&d_aux, sizeof(unsigned long long) * kAux, st));
    struct Release {
        void *a, *b;
        cudaStream_t s;
        ~Release() {
            cudaFreeAsync(a, s);
            cudaFreeAsync(b, s);
        }
    } release{d_states, d_aux, st};
    PL_TRY(cudaMemcpyAsync(d_states, hs.data(), sizeof(PState) * n, cudaMemcpyHostToDevice, st));
    unsigned long long aux0[kAux] = {~0ull, (unsigned long long)finished0};
    PL_TRY(cudaMemcpyAsync(d_aux, aux0, sizeof(aux0), cudaMemcpyHostToDevice, st));
    PLaunch L{};
    L.states = d_states;
    L.n = n;
    const double left = std::max(0.0, budget - (now_s() - t0));
    L.budget_ns = (unsigned long long)(std::min(left, 1e6) * 1e9);
    L.hard_ns = L.budget_ns + (unsigned long long)(std::min(30.0 + left, 1e6) * 1e9);
    L.idle_poll_limit = g_per_idle_polls.load();
    L.t_start = d_aux;
    L.finished = reinterpret_cast<int *>(d_aux + 1);
    L.timeout = reinterpret_cast<int *>(d_aux + 1) + 1;
    L.phase_ns = d_aux + 2;
    L.phase_chunks = d_aux + 2 + kPhaseKinds;
    // the launch, captured in a CUDA graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    PL_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    k_persistent<<<ctas, kPerThreads, smem, st>>>(L);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    PL_TRY(le);
    PL_TRY(ce);
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    const double t_launch = now_s() - t0;
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    PL_TRY(e);
    unsigned long long aux[kAux];
    const double t_wall = now_s() - t0 - t_launch;
    PL_TRY(cudaMemcpy(hs.data(), d_states, sizeof(PState) * n, cudaMemcpyDeviceToHost));
    PL_TRY(cudaMemcpy(aux, d_aux, sizeof(aux), cudaMemcpyDeviceToHost));
    {
        std::lock_guard<std::mutex> lock(g_phase_mu);
        for (int k = 0; k < kPhaseKinds; ++k) {
            g_phase_ns[k] = (int64_t)aux[2 + k];
            g_phase_chunks[k] = (int64_t)aux[2 + kPhaseKinds + k];
        }
        g_phase_ctas = ctas;
        g_phase_wall_ns = (int64_t)(t_wall * 1e9);
    }
    const bool timeout = (aux[1] >> 32) != 0;
    // results and mirrors back to the host planners
    for (int i = 0; i < n; ++i) {
        Planner *pl = pls[i];
        PerBuffers &b = pl->per;
        const PState &s = hs[i];
        const int D = pl->D;
        const int nt = std::min(s.n_trace, kTraceCap), nh = std::min(s.n_hist, kHistCap);
        if (nt > 0) {
            std::vector<double> tc(nt);
            std::vector<unsigned long long> tn(nt);
            PL_TRY(cudaMemcpy(tc.data(), b.trace_c, sizeof(double) * nt, cudaMemcpyDeviceToHost));
            PL_TRY(cudaMemcpy(tn.data(), b.trace_ns, sizeof(unsigned long long) * nt,
                              cudaMemcpyDeviceToHost));
            for (int k = 0; k < nt; ++k) {
                pl->trace_t.push_back(t_launch + (double)(tn[k] - aux[0]) * 1e-9);
                pl->trace_c.push_back(tc[k]);
            }
            std::vector<int> hl(std::max(nh, 1));
            if (nh > 0)
                PL_TRY(cudaMemcpy(hl.data(), b.hist_len, sizeof(int) * nh, cudaMemcpyDeviceToHost));
            size_t off = 0;
            for (int k = 0; k < nh; ++k) {
                std::vector<float> path;
                if (hl[k] > 0) {
                    path.resize((size_t)hl[k] * D);
                    PL_TRY(cudaMemcpy(path.data(), b.hist + off, sizeof(float) * path.size(),
                                      cudaMemcpyDeviceToHost));
                    off += path.size();
                }
                pl->history.push_back(std::move(path));
            }
            for (int k = nh; k < nt; ++k) pl->history.emplace_back();  // did not fit
            pl->best_path.resize((size_t)s.best_len * D);
            PL_TRY(cudaMemcpy(pl->best_path.data(), b.best, sizeof(float) * pl->best_path.size(),
                              cudaMemcpyDeviceToHost));
            pl->c_best = s.c_best;
        }
        pl->mode = s.mode;
        pl->step = s.step;
        pl->iters_in_call = s.iters_in_call;
        pl->total_iters = s.total_iters;
        const bool clean = s.finished != 0;
        pl->roadmap_ready = clean && s.roadmap_ready != 0;
        std::vector<int> counts(pl->K);
        PL_TRY(cudaMemcpy(counts.data(), pl->rm_n, sizeof(int) * pl->K, cudaMemcpyDeviceToHost));
        for (int k = 0; k < pl->K; ++k) {
            int c = 0;
            PL_TRY(cudaMemcpy(&c, pl->rm[k].d_conn, sizeof(int), cudaMemcpyDeviceToHost));
            pl->rm[k].n = counts[k];
            pl->rm[k].connected = c != 0;
        }
        if (!clean) {
            // stopped mid-phase (an idle CTA gave up): the next call starts
            // from fresh trees and a new roadmap round
            pl->roadmap_ready = false;
            if (run[i].status == MRPOP_OK) run[i].status = MRPOP_ETIMEOUT;
        }
    }
    if (statuses)
        for (int i = 0; i < n; ++i) statuses[i] = run[i].status;
    if (timeout)
        return set_error(MRPOP_ETIMEOUT, "plan_batch: a bounded wait of the persistent launch ran "
                                         "out before every problem finished");
    return MRPOP_OK;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching.  A server thread keeps up to max_slots
// requests on the device and advances all of them by one planner iteration
// per loop (the same per-slot logic as mrpop_plan_batch, direct launches
// instead of a graph because membership changes between iterations).  Queued
// requests are admitted in arrival order when a slot and enough device memory
// are free; a finished request releases its device state at once.
// ---------------------------------------------------------------------------
static size_t planner_bytes(const mrpop_problem *p) {
    const int K = p->dev.t.K, D = p->D;
    const size_t rcap = (size_t)std::max<int64_t>(64, std::min<int64_t>(p->cfg.roadmap_cap, 1 << 20));
    const size_t tcap = (size_t)std::max<int64_t>(1024, std::min<int64_t>(p->cfg.tree_cap, 1 << 22));
    const size_t npr = (size_t)std::max(1, std::min(p->cfg.n_per_round, 4096));
    size_t b = 2 * ((size_t)D + 3 + K) * tcap * 4;            // trees
    b += ((size_t)2 * tcap + 2) * ((size_t)D + 1) * 4;         // path extraction
    b += ((size_t)4 * D + 8 + K) * kStepIters * 8;             // step buffers
    for (const HostRobot &r : p->robots) {
        b += rcap * ((size_t)r.dof + kKmax + 1) * 4;           // roadmap
        b += npr * ((size_t)r.dof * (kOversample + 1) + (size_t)kKmax * (2 * r.dof + 12)) * 4;
    }
    b += (size_t)p->dev.t.n_f4 * 16 * (K + 2) + (1 << 16);     // sub-problem tables
    return b;
}

struct Request {
    int64_t ticket = 0;
    mrpop_problem *p = nullptr;
    double budget = 0.0, target = -INFINITY;
    int64_t max_steps = 0, steps = 0;
    double t_submit = 0.0, t_admit = -1.0, t_first = -1.0, t_target = -1.0, t_done = -1.0;
    int state = 0;  // 0 queued, 1 running, 2 done
    mrpop_status status = MRPOP_OK;
    SlotRun run;
    size_t mem = 0;
    bool cancel = false;  // set by mrpop_server_cancel (under the server's lock)
};

}  // namespace mrpop

struct mrpop_server {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<mrpop::Request *> queue;
    std::vector<mrpop::Request *> active;  // server thread only
    std::map<int64_t, std::unique_ptr<mrpop::Request>> all;
    int max_slots = 64;
    size_t mem_budget = 0, mem_used = 0;
    int device = 0;
    bool stop = false;
    int64_t next_ticket = 1;
    double t0 = 0.0;
    mrpop_status fatal = MRPOP_OK;
    int64_t admitted = 0, completed = 0, peak_active = 0;
    size_t peak_mem = 0;
    mrpop::Slot *d_slots = nullptr;
    mrpop::VParams *d_vp = nullptr;
    mrpop::Ctrl *d_ctrl = nullptr, *h_ctrl = nullptr;
    std::thread th;
    // host-side fault injection (mrpop_server_inject)
    int64_t inject_admit_enomem = 0;  // admissions still to refuse
    int64_t inject_stall_ms = 0;      // one stall of the loop, then 0
    int64_t cancelled = 0;
};

namespace mrpop {

static mrpop_status server_rebuild(mrpop_server *sv, Batch &bt, cudaStream_t st) {
    const int n = (int)sv->active.size();
    bt.n = n;
    bt.pls.clear();
    if (n == 0) return MRPOP_OK;
    for (Request *r : sv->active) bt.pls.push_back(r->p->planner);
    ST_TRY(batch_config(bt));
    std::vector<Slot> slots(n);
    std::vector<VParams> vps(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        slots[i] = bt.pls[i]->slot;
        slots[i].ctrl = sv->d_ctrl + i;
        for (int k = 0; k < 2; ++k) {
            vps[(size_t)k * n + i] = bt.pls[i]->vp[k];
            vps[(size_t)k * n + i].warps = bt.slot_warps[i];
            vps[(size_t)k * n + i].total_warps = bt.bps * bt.slot_warps[i];
        }
    }
    // (the previous iteration's work on these arrays has completed: every
    // iteration ends with a stream synchronisation)
    PL_TRY(cudaMemcpyAsync(sv->d_slots, slots.data(), sizeof(Slot) * n, cudaMemcpyHostToDevice, st));
    PL_TRY(cudaMemcpyAsync(sv->d_vp, vps.data(), sizeof(VParams) * 2 * n, cudaMemcpyHostToDevice, st));
    bt.d_vp = sv->d_vp;
    return MRPOP_OK;
}

static void server_finish(mrpop_server *sv, Request *r, double now) {
    std::lock_guard<std::mutex> lock(sv->mu);
    r->state = 2;
    r->t_done = now - r->t_submit;
    if (r->p->planner) free_device(r->p->planner);
    sv->mem_used -= r->mem;
    ++sv->completed;
}

static void server_loop(mrpop_server *sv) {
    cudaSetDevice(sv->device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->fatal = MRPOP_ECUDA;
        return;
    }
    Batch bt;
    bt.owns = false;
    bt.d_slots = sv->d_slots;
    bt.d_ctrl = sv->d_ctrl;
    bt.h_ctrl = sv->h_ctrl;
    bool changed = true;
    auto fail = [&](mrpop_status s) {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->fatal = s;
    };
    for (;;) {
        std::vector<Request *> admit;
        std::vector<bool> refuse;
        int64_t stall = 0;
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (sv->stop) break;
            stall = sv->inject_stall_ms;
            sv->inject_stall_ms = 0;
            // cancelled requests leave the queue before admission
            for (auto it = sv->queue.begin(); it != sv->queue.end();) {
                if ((*it)->cancel) {
                    Request *r = *it;
                    it = sv->queue.erase(it);
                    r->state = 2;
                    r->status = MRPOP_ECANCELLED;
                    r->t_done = now_s() - r->t_submit;
                    ++sv->completed;
                    ++sv->cancelled;
                } else {
                    ++it;
                }
            }
            while ((int)(sv->active.size() + admit.size()) < sv->max_slots && !sv->queue.empty()) {
                Request *r = sv->queue.front();
                const size_t need = planner_bytes(r->p);
                // memory admission: wait for room unless nothing else runs
                if (sv->mem_used + need > sv->mem_budget && !(sv->active.empty() && admit.empty()))
                    break;
                sv->queue.pop_front();
                r->mem = need;
                sv->mem_used += need;
                sv->peak_mem = std::max(sv->peak_mem, sv->mem_used);
                admit.push_back(r);
                refuse.push_back(sv->inject_admit_enomem > 0);
                if (sv->inject_admit_enomem > 0) --sv->inject_admit_enomem;
            }
            if (sv->active.empty() && admit.empty() && stall == 0) {
                sv->cv.wait_for(lock, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (stall > 0)  // injected stall, outside the lock: submit and poll stay responsive
            std::this_thread::sleep_for(std::chrono::milliseconds(stall));
        for (size_t ai = 0; ai < admit.size(); ++ai) {
            Request *r = admit[ai];
            // an injected refusal stands in for a failed device allocation
            mrpop_status s = refuse[ai] ? set_error(MRPOP_ENOMEM, "injected allocation failure")
                                        : ensure_planner(r->p);
            std::vector<Planner *> one{r->p->planner};
            std::vector<SlotRun> run(1);
            run[0].target = r->target;
            run[0].reset_trees = s == MRPOP_OK && !r->p->planner->roadmap_ready;
            if (s != MRPOP_OK) one.clear();
            if (s == MRPOP_OK) s = check_endpoints(one, run, st);
            if (s == MRPOP_OK) s = run[0].status;
            const double now = now_s();
            if (s != MRPOP_OK || !run[0].active) {
                r->status = s;
                server_finish(sv, r, now);
                continue;
            }
            r->run = run[0];
            r->t_admit = now - r->t_submit;
            r->p->planner->trace_t0 = now;
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                r->state = 1;
                ++sv->admitted;
            }
            sv->active.push_back(r);
            changed = true;
        }
        sv->peak_active = std::max<int64_t>(sv->peak_active, (int64_t)sv->active.size());
        if (sv->active.empty()) continue;
        if (changed) {
            mrpop_status s = server_rebuild(sv, bt, st);
            if (s != MRPOP_OK) return fail(s);
            changed = false;
        }
        const int n = bt.n;
        std::vector<SlotRun *> rp;
        for (Request *r : sv->active) rp.push_back(&r->run);
        mrpop_status s = roadmap_rounds(bt.pls, rp, bt.d_slots, st);
        for (int i = 0; i < n; ++i) slot_ctrl(bt.pls[i], sv->active[i]->run, bt.h_ctrl[i]);
        cudaError_t e = cudaSuccess;
        if (s == MRPOP_OK)
            e = cudaMemcpyAsync(bt.d_ctrl, bt.h_ctrl, sizeof(Ctrl) * n, cudaMemcpyHostToDevice, st);
        if (s == MRPOP_OK && e == cudaSuccess) s = enqueue_step(bt, st);
        if (s == MRPOP_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(bt.h_ctrl, bt.d_ctrl, sizeof(Ctrl) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(cuda_error(e, "server step"));
        if (s != MRPOP_OK) return fail(s);
        const double now = now_s();
        std::vector<Request *> keep;
        for (int i = 0; i < n; ++i) {
            Request *r = sv->active[i];
            Planner *pl = bt.pls[i];
            s = slot_after(pl, r->run, bt.h_ctrl[i], bt.d_slots + i, st, now - pl->trace_t0);
            if (s != MRPOP_OK) return fail(s);
            ++r->steps;
            const double t = now - r->t_submit;
            if (r->t_first < 0 && !pl->trace_c.empty()) r->t_first = t;
            if (r->t_target < 0 && reached_target(pl->c_best, r->target)) r->t_target = t;
            bool cancel;
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                cancel = r->cancel;
            }
            const bool done = cancel || r->run.reached || !r->run.active ||
                              now - (r->t_submit + r->t_admit) >= r->budget ||
                              (r->max_steps > 0 && r->steps >= r->max_steps);
            if (done) {
                if (cancel) {
                    r->status = MRPOP_ECANCELLED;
                    std::lock_guard<std::mutex> lock(sv->mu);
                    ++sv->cancelled;
                }
                server_finish(sv, r, now);
                changed = true;
            } else {
                keep.push_back(r);
            }
        }
        sv->active.swap(keep);
    }
    // shutdown: running requests end now
    const double now = now_s();
    for (Request *r : sv->active) server_finish(sv, r, now);
    sv->active.clear();
    cudaStreamDestroy(st);
}

}  // namespace mrpop

using namespace mrpop;

static mrpop_status result(mrpop_problem *p, float *path, int64_t path_cap, int64_t *path_len,
                           double *cost) {
    Planner *pl = p->planner;
    const int64_t M = pl ? (int64_t)(pl->best_path.size() / std::max(1, pl->D)) : 0;
    if (path_len) *path_len = M;
    if (cost) *cost = pl && M > 0 ? pl->c_best : INFINITY;
    if (M == 0) return set_error(MRPOP_ENOSOLUTION, "no path found within the budget");
    if (path) {
        if (path_cap < M)
            return set_error(MRPOP_ECAPACITY, "path needs %lld vertices, cap %lld", (long long)M,
                             (long long)path_cap);
        std::memcpy(path, pl->best_path.data(), sizeof(float) * pl->best_path.size());
    }
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_plan(mrpop_problem *p, double time_budget_s, float *path,
                                   int64_t path_cap, int64_t *path_len, double *cost) {
    if (!p) return set_error(MRPOP_EINVAL, "mrpop_plan: problem is NULL");
    if (!(time_budget_s >= 0.0)) return set_error(MRPOP_EINVAL, "mrpop_plan: negative budget");
    if (p->start.empty() || p->goal.empty())
        return set_error(MRPOP_EINVAL, "mrpop_plan: the problem was created without start/goal");
    mrpop_status st = MRPOP_OK;
    mrpop_status s = plan_batch(&p, 1, time_budget_s, 0, nullptr, &st);
    if (s != MRPOP_OK) return s;
    if (st != MRPOP_OK) return set_error(st, "mrpop_plan: start or goal is in collision");
    return result(p, path, path_cap, path_len, cost);
}

extern "C" mrpop_status mrpop_plan_batch(mrpop_problem *const *ps, int32_t n, double time_budget_s,
                                         int64_t max_steps, const double *target_costs,
                                         mrpop_status *statuses) {
    if (!ps || n < 1) return set_error(MRPOP_EINVAL, "mrpop_plan_batch: no problems");
    if (!(time_budget_s >= 0.0)) return set_error(MRPOP_EINVAL, "mrpop_plan_batch: negative budget");
    for (int i = 0; i < n; ++i) {
        if (!ps[i]) return set_error(MRPOP_EINVAL, "mrpop_plan_batch: problem %d is NULL", i);
        if (ps[i]->start.empty() || ps[i]->goal.empty())
            return set_error(MRPOP_EINVAL, "mrpop_plan_batch: problem %d has no start/goal", i);
        for (int j = 0; j < i; ++j)
            if (ps[j] == ps[i]) return set_error(MRPOP_EINVAL, "mrpop_plan_batch: problem %d repeated", i);
    }
    return plan_batch_persistent(ps, n, time_budget_s, max_steps, target_costs, statuses);
}

extern "C" mrpop_status mrpop_plan_batch_ex(mrpop_problem *const *ps, int32_t n,
                                            double time_budget_s, int64_t max_steps,
                                            const double *target_costs, mrpop_status *statuses,
                                            int32_t form) {
    if (form != MRPOP_BATCH_PERSISTENT && form != MRPOP_BATCH_STEPPED)
        return set_error(MRPOP_EINVAL, "mrpop_plan_batch_ex: form=%d is not a batch form", form);
    if (form == MRPOP_BATCH_PERSISTENT)
        return mrpop_plan_batch(ps, n, time_budget_s, max_steps, target_costs, statuses);
    if (!ps || n < 1) return set_error(MRPOP_EINVAL, "mrpop_plan_batch_ex: no problems");
    if (!(time_budget_s >= 0.0)) return set_error(MRPOP_EINVAL, "mrpop_plan_batch_ex: negative budget");
    for (int i = 0; i < n; ++i) {
        if (!ps[i]) return set_error(MRPOP_EINVAL, "mrpop_plan_batch_ex: problem %d is NULL", i);
        if (ps[i]->start.empty() || ps[i]->goal.empty())
            return set_error(MRPOP_EINVAL, "mrpop_plan_batch_ex: problem %d has no start/goal", i);
        for (int j = 0; j < i; ++j)
            if (ps[j] == ps[i])
                return set_error(MRPOP_EINVAL, "mrpop_plan_batch_ex: problem %d repeated", i);
    }
    return plan_batch(ps, n, time_budget_s, max_steps, target_costs, statuses);
}

extern "C" mrpop_status mrpop_set_persistent_limits(int32_t ctas, int64_t idle_polls) {
    if (ctas < 0 || idle_polls < 0)
        return set_error(MRPOP_EINVAL, "mrpop_set_persistent_limits: negative limit");
    mrpop::g_per_ctas.store(ctas);
    mrpop::g_per_idle_polls.store(idle_polls);
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_plan_batch_phase_stats(int64_t *ns, int64_t *chunks,
                                                    int64_t *ctas_wall) {
    if (!ns || !chunks || !ctas_wall)
        return set_error(MRPOP_EINVAL, "mrpop_plan_batch_phase_stats: NULL argument");
    std::lock_guard<std::mutex> lock(g_phase_mu);
    for (int k = 0; k < kPhaseKinds; ++k) {
        ns[k] = g_phase_ns[k];
        chunks[k] = g_phase_chunks[k];
    }
    ctas_wall[0] = g_phase_ctas;
    ctas_wall[1] = g_phase_wall_ns;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_plan_result(mrpop_problem *p, float *path, int64_t path_cap,
                                          int64_t *path_len, double *cost) {
    if (!p) return set_error(MRPOP_EINVAL, "mrpop_plan_result: problem is NULL");
    return result(p, path, path_cap, path_len, cost);
}

extern "C" mrpop_status mrpop_plan_trace(const mrpop_problem *p, double *times, double *costs,
                                         int64_t cap, int64_t *n, int64_t *iterations) {
    if (!p) return set_error(MRPOP_EINVAL, "mrpop_plan_trace: problem is NULL");
    const Planner *pl = p->planner;
    const int64_t m = pl ? (int64_t)pl->trace_c.size() : 0;
    if (n) *n = m;
    if (iterations) *iterations = pl ? pl->total_iters : 0;
    for (int64_t i = 0; i < std::min(m, cap); ++i) {
        if (times) times[i] = pl->trace_t[i];
        if (costs) costs[i] = pl->trace_c[i];
    }
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_create(int32_t max_slots, int64_t device_mem_budget,
                                            mrpop_server **out) {
    if (!out) return set_error(MRPOP_EINVAL, "mrpop_server_create: out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 4096)
        return set_error(MRPOP_EINVAL, "mrpop_server_create: max_slots=%d outside [1, 4096]", max_slots);
    mrpop_server *sv = new (std::nothrow) mrpop_server();
    if (!sv) return set_error(MRPOP_ENOMEM, "host allocation failed");
    sv->max_slots = max_slots;
    cudaError_t e = cudaGetDevice(&sv->device);
    size_t fr = 0, tot = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_slots, sizeof(Slot) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_vp, sizeof(VParams) * 2 * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_ctrl, sizeof(Ctrl) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&sv->h_ctrl, sizeof(Ctrl) * max_slots);
    if (e != cudaSuccess) {
        mrpop_status s = cuda_error(e, "mrpop_server_create");
        cudaFree(sv->d_slots); cudaFree(sv->d_vp); cudaFree(sv->d_ctrl);
        if (sv->h_ctrl) cudaFreeHost(sv->h_ctrl);
        delete sv;
        return s;
    }
    sv->mem_budget = device_mem_budget > 0 ? (size_t)device_mem_budget : (size_t)(0.8 * (double)fr);
    sv->t0 = now_s();
    sv->th = std::thread(server_loop, sv);
    *out = sv;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_submit(mrpop_server *sv, mrpop_problem *p, double budget_s,
                                            int64_t max_steps, double target_cost,
                                            int64_t *ticket) {
    if (!sv || !p) return set_error(MRPOP_EINVAL, "mrpop_server_submit: NULL argument");
    if (!(budget_s >= 0.0)) return set_error(MRPOP_EINVAL, "mrpop_server_submit: negative budget");
    if (p->start.empty() || p->goal.empty())
        return set_error(MRPOP_EINVAL, "mrpop_server_submit: problem has no start/goal");
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->fatal != MRPOP_OK) return set_error(sv->fatal, "mrpop_server_submit: server stopped on an error");
    for (auto &kv : sv->all)
        if (kv.second->p == p && kv.second->state != 2)
            return set_error(MRPOP_EBUSY, "mrpop_server_submit: problem already queued or running");
    auto r = std::make_unique<Request>();
    r->ticket = sv->next_ticket++;
    r->p = p;
    r->budget = budget_s;
    r->max_steps = max_steps;
    r->target = std::isnan(target_cost) ? -INFINITY : target_cost;
    r->t_submit = now_s();
    if (ticket) *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->all[r->ticket] = std::move(r);
    sv->cv.notify_one();
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_poll(mrpop_server *sv, int64_t ticket, int32_t *state,
                                          double *times, double *cost) {
    if (!sv) return set_error(MRPOP_EINVAL, "mrpop_server_poll: server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return set_error(MRPOP_EINVAL, "mrpop_server_poll: unknown ticket");
    const Request &r = *it->second;
    if (state) *state = r.state;
    if (times) {
        times[0] = r.t_admit;
        times[1] = r.t_first;
        times[2] = r.t_target;
        times[3] = r.t_done;
    }
    if (cost) *cost = (r.state == 2 && r.p->planner) ? r.p->planner->c_best : INFINITY;
    if (r.state == 2 && r.status != MRPOP_OK) return set_error(r.status, "request failed");
    if (sv->fatal != MRPOP_OK) return set_error(sv->fatal, "server stopped on an error");
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_cancel(mrpop_server *sv, int64_t ticket) {
    if (!sv) return set_error(MRPOP_EINVAL, "mrpop_server_cancel: server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return set_error(MRPOP_EINVAL, "mrpop_server_cancel: unknown ticket");
    if (it->second->state != 2) it->second->cancel = true;
    sv->cv.notify_all();
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_inject(mrpop_server *sv, int32_t fault, int64_t count) {
    if (!sv) return set_error(MRPOP_EINVAL, "mrpop_server_inject: server is NULL");
    if (count < 0) return set_error(MRPOP_EINVAL, "mrpop_server_inject: negative count");
    std::lock_guard<std::mutex> lock(sv->mu);
    if (fault == MRPOP_FAULT_ADMIT_ENOMEM)
        sv->inject_admit_enomem = count;
    else if (fault == MRPOP_FAULT_STALL_MS)
        sv->inject_stall_ms = count;
    else
        return set_error(MRPOP_EINVAL, "mrpop_server_inject: fault=%d is not a fault", fault);
    sv->cv.notify_all();
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_stats(mrpop_server *sv, int64_t *stats) {
    if (!sv || !stats) return set_error(MRPOP_EINVAL, "mrpop_server_stats: NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    stats[0] = sv->admitted;
    stats[1] = sv->completed;
    stats[2] = sv->peak_active;
    stats[3] = (int64_t)sv->peak_mem;
    stats[4] = (int64_t)sv->mem_budget;
    stats[5] = (int64_t)sv->queue.size();
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_server_destroy(mrpop_server *sv) {
    if (!sv) return MRPOP_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->th.joinable()) sv->th.join();
    cudaFree(sv->d_slots);
    cudaFree(sv->d_vp);
    cudaFree(sv->d_ctrl);
    if (sv->h_ctrl) cudaFreeHost(sv->h_ctrl);
    delete sv;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_plan_history(const mrpop_problem *p, int64_t index, float *path,
                                           int64_t path_cap, int64_t *path_len, double *cost) {
    if (!p) return set_error(MRPOP_EINVAL, "mrpop_plan_history: problem is NULL");
    const Planner *pl = p->planner;
    const int64_t n = pl ? (int64_t)pl->history.size() : 0;
    if (index < 0 || index >= n)
        return set_error(MRPOP_EINVAL, "mrpop_plan_history: index %lld outside [0, %lld)",
                         (long long)index, (long long)n);
    const std::vector<float> &h = pl->history[(size_t)index];
    const int64_t M = (int64_t)(h.size() / std::max(1, pl->D));
    if (path_len) *path_len = M;
    if (cost) *cost = pl->trace_c[(size_t)index];
    if (path) {
        if (path_cap < M)
            return set_error(MRPOP_ECAPACITY, "mrpop_plan_history: path needs %lld vertices",
                             (long long)M);
        std::memcpy(path, h.data(), sizeof(float) * h.size());
    }
    return MRPOP_OK;
}

// ---------------------------------------------------------------------------
// Test hooks: one pass of the planner's own NEAREST kernel (k_nearest, both
// passes of a search step) and roadmap NEIGHBORS kernel (k_rmb_neighbors) on
// caller-given arrays, through a minimal slot / job built on the device, so
// that these kernels can be compared with the oracle directly.
// ---------------------------------------------------------------------------
extern "C" mrpop_status mrpop_planner_nearest_pass(const float *tree, int64_t n_vertices,
                                                   int64_t ld, int32_t dim, const float *queries,
                                                   const float *budgets, int32_t n_queries,
                                                   int32_t pass, int64_t *out_idx, void *stream) {
    using namespace mrpop;
    if (dim < 1 || dim > MRPOP_MAX_LINKS || n_vertices < 0 || ld < n_vertices ||
        ld > (int64_t)INT32_MAX || n_queries < 1 || n_queries > kStepIters ||
        (pass != 0 && pass != 1))
        return set_error(MRPOP_EINVAL,
                         "mrpop_planner_nearest_pass: dim=%d n_vertices=%lld ld=%lld "
                         "n_queries=%d pass=%d out of range", dim, (long long)n_vertices,
                         (long long)ld, n_queries, pass);
    if (!queries || !budgets || !out_idx || (n_vertices > 0 && !tree))
        return set_error(MRPOP_EINVAL, "mrpop_planner_nearest_pass: NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    // one arena: slot, control block, counts, padded queries [dim][256],
    // budgets [256] (padding admits nothing), results [256]
    const size_t b_slot = 256 * ((sizeof(Slot) + 255) / 256);
    const size_t b_ctrl = 256 * ((sizeof(Ctrl) + 255) / 256);
    const size_t b_q = sizeof(float) * (size_t)dim * kStepIters;
    const size_t b_c = sizeof(float) * kStepIters;
    char *arena = nullptr;
    PL_TRY(scratch_alloc((void **)&arena, b_slot + b_ctrl + 256 + b_q + b_c +
                                                sizeof(int64_t) * kStepIters, st));
    Slot *d_slot = (Slot *)arena;
    Ctrl *d_ctrl = (Ctrl *)(arena + b_slot);
    int *d_tn = (int *)(arena + b_slot + b_ctrl);
    float *d_q = (float *)(arena + b_slot + b_ctrl + 256);
    float *d_c = (float *)((char *)d_q + b_q);
    int64_t *d_out = (int64_t *)((char *)d_c + b_c);
    Slot S{};
    S.D = dim;
    S.tcap = (int)ld;
    S.tq[0] = S.tq[1] = const_cast<float *>(tree);
    S.tn = d_tn;
    S.qrand = S.qnew = d_q;
    S.crand = S.budget2 = d_c;
    S.near = S.conn = d_out;
    S.ctrl = d_ctrl;
    Ctrl C{};
    C.tree_a = 0;  // pass 0 reads tree tree_a, pass 1 tree 1 - tree_a: both are `tree`
    const int tn[2] = {(int)n_vertices, (int)n_vertices};
    std::vector<float> pad_c(kStepIters, -FLT_MAX);
    cudaError_t e = cudaMemcpyAsync(d_slot, &S, sizeof(Slot), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ctrl, &C, sizeof(Ctrl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tn, tn, sizeof(tn), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_q, 0, b_q, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_c, pad_c.data(), b_c, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_q, sizeof(float) * kStepIters, queries, sizeof(float) * n_queries,
                              sizeof(float) * n_queries, dim, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_c, budgets, sizeof(float) * n_queries, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        const dim3 grid(kStepIters / kPQB, 1);
        if (pass == 0)
            k_nearest<0><<<grid, kPThreads, 0, st>>>(d_slot);
        else
            k_nearest<1><<<grid, kPThreads, 0, st>>>(d_slot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_idx, d_out, sizeof(int64_t) * n_queries, cudaMemcpyDeviceToDevice,
                            st);
    // the host-side copies above read stack memory: finish before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(arena, st);
    if (e != cudaSuccess) return cuda_error(e, "mrpop_planner_nearest_pass");
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_planner_neighbors_pass(const float *V, int64_t n_vertices,
                                                     int64_t ld, int32_t dof,
                                                     const float *queries, int64_t n_queries,
                                                     float delta, int64_t *out_idx,
                                                     int64_t *out_cnt, void *stream) {
    using namespace mrpop;
    if (dof < 1 || dof > MRPOP_MAX_DOF || n_vertices < 0 || ld < n_vertices ||
        ld > (int64_t)INT32_MAX || n_queries < 0 || n_queries > (int64_t)INT32_MAX / kKmax)
        return set_error(MRPOP_EINVAL,
                         "mrpop_planner_neighbors_pass: dof=%d n_vertices=%lld ld=%lld "
                         "n_queries=%lld out of range", dof, (long long)n_vertices, (long long)ld,
                         (long long)n_queries);
    if (n_queries == 0) return MRPOP_OK;
    if (!queries || !out_idx || !out_cnt || (n_vertices > 0 && !V))
        return set_error(MRPOP_EINVAL, "mrpop_planner_neighbors_pass: NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    char *arena = nullptr;
    const size_t b_job = 256 * ((sizeof(RmJob) + 255) / 256);
    PL_TRY(scratch_alloc((void **)&arena, b_job + 256, st));
    RmJob *d_job = (RmJob *)arena;
    int *d_count = (int *)(arena + b_job);
    RmJob J{};
    J.q = const_cast<float *>(V);
    J.rcap = (int)ld;
    J.dof = dof;
    J.count = d_count;
    J.gq = const_cast<float *>(queries);
    J.m = (int)n_queries;
    J.nb = out_idx;
    J.cnt = out_cnt;
    J.delta = delta;
    const int n = (int)n_vertices;
    cudaError_t e = cudaMemcpyAsync(d_job, &J, sizeof(RmJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_count, &n, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)((n_queries + kRmNbWarps - 1) / kRmNbWarps), 1);
        k_rmb_neighbors<<<grid, kRmNbWarps * 32, 0, st>>>(d_job);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host copies read stack memory
    cudaFreeAsync(arena, st);
    if (e != cudaSuccess) return cuda_error(e, "mrpop_planner_neighbors_pass");
    return MRPOP_OK;
}
