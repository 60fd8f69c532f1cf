// Motion validation of composite edges (Sec. III-E) and forward kinematics.
//
// Design (sm_103a, FP32 SIMT; not a dense contraction, so no tensor cores):
//  * One warp per edge, fetched dynamically from a self-resetting work
//    counter.  The edge's q_a and q_b - q_a are staged in shared memory and the
//    interval count n is computed once per warp.
//  * Checkpoints across lanes: tile t of an edge with n+1 points and
//    T = ceil((n+1)/32) tiles assigns point k = t + T*lane to each lane, so
//    every tile samples the whole edge and a collision anywhere ends the edge
//    after few tiles (early exit with __any_sync).
//  * Per link, forward kinematics in registers (Rz, then the d/a/alpha
//    offsets), then three levels of culling:
//      1. tile level: the warp bounds the link's coarse spheres at its 32
//         checkpoints by one sphere (around the exact box of the centres, from
//         order-preserving integer min/max warp reductions); lane i tests
//         obstacle i (and the tile bound of earlier links i) against it, and a
//         ballot gives the candidate set -- when it is empty, nothing below
//         runs for that obstacle group;
//      2. checkpoint level ("coarse" stage of the paper): each lane tests its
//         own link sphere against the candidates only;
//      3. sphere level ("fine" stage): the warp-wide OR of the lanes' hit
//         masks (__reduce_or_sync) selects the obstacles / links whose spheres
//         are tested, on a register cache of the link's world spheres.
//    Culling never changes a verdict: each bound encloses what it replaces
//    with a slack above FP32 rounding.
//  * The paper's own design (4 threads per motion, then threads reassigned in
//    proportion to the fine-test load) balances work across motions; here the
//    warp-uniform union mask keeps all 32 lanes busy on the same tests instead.
//  * Geometry tables are staged once per block into shared memory; the
//    coarse centres of robots 0..K-2 go to a per-warp shared scratch
//    [link][3][lane] (lane-contiguous, conflict-free) for the robot-robot
//    tests, whose rare fine stage rebuilds the other link's frame.
#include <cfloat>
#include <cmath>
#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "mrpop_internal.cuh"
#include "validate_body.cuh"

namespace mrpop {
namespace {

using namespace vb;

template <int MODE, bool RA>
__global__ void __launch_bounds__(kWarpsMax * 32) validate_kernel(const VParams P) {
    extern __shared__ float4 sm4[];
    validate_body<MODE, RA>(P, sm4);
}

// The same kernel with a wide register budget (up to 128 registers: four
// blocks of four warps per SM): fewer warps, no spills in the robot-robot
// fine stage, which many-arm scenes reach often.  An autotuner dimension.
template <int MODE, bool RA>
__global__ void __launch_bounds__(kWarpsMax * 32, 4) validate_kernel_wide(const VParams P) {
    extern __shared__ float4 sm4[];
    validate_body<MODE, RA>(P, sm4);
}

// Many problems in one launch: block row y serves problem y (its parameters
// are staged in shared memory once per block).
template <bool RA>
__global__ void __launch_bounds__(kWarpsMax * 32) validate_batch_kernel(const VParams *Ps) {
    extern __shared__ float4 sm4[];
    __shared__ VParams sP;
    if (threadIdx.x == 0) sP = Ps[blockIdx.y];
    __syncthreads();
    validate_body<kVerdict, RA>(sP, sm4);
}

// Resident blocks per SM of a validation kernel for a launch shape.  The
// kernel's dynamic shared-memory limit is raised to the device maximum once,
// and occupancies are cached per (kernel, device, threads, bytes): the
// planner issues thousands of small validation launches, and these host
// queries would otherwise cost more than the launches themselves.
static mrpop_status cached_occupancy(const void *kern, int device, int smem_optin, int threads,
                                     size_t smem, int *bps) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> occ;
    static std::set<std::pair<const void *, int>> raised;
    std::lock_guard<std::mutex> lock(mu);
    if (!raised.count({kern, device})) {
        cudaFuncAttributes fa{};
        MRPOP_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        const int limit = smem_optin - (int)fa.sharedSizeBytes;  // static shared memory counts too
        MRPOP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            limit));
        raised.insert({kern, device});
    }
    const auto key = std::make_tuple(kern, device, threads, smem);
    auto it = occ.find(key);
    if (it == occ.end()) {
        int b = 0;
        MRPOP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem));
        it = occ.emplace(key, b).first;
    }
    *bps = it->second;
    return MRPOP_OK;
}

template <int MODE, bool RA>
mrpop_status launch_mode(mrpop_problem *p, VParams &V, int warps, size_t smem,
                         cudaStream_t st) {
    auto kern = MODE == kVerdict && p->tuned_regs ? validate_kernel_wide<MODE, RA>
                                                  : validate_kernel<MODE, RA>;
    int bps = 0;
    const mrpop_status os = cached_occupancy((const void *)kern, p->device, (int)p->smem_optin,
                                             warps * 32, smem, &bps);
    if (os != MRPOP_OK) return os;
    if (bps < 1) return set_error(MRPOP_EINVAL, "validation kernel does not fit on an SM");
    const int64_t want = (V.E + warps - 1) / warps;
    const int grid = (int)std::min<int64_t>((int64_t)p->num_sms * bps, want);
    V.total_warps = grid * warps;
    V.warps = warps;
    kern<<<grid, warps * 32, smem, st>>>(V);
    MRPOP_CUDA_TRY(cudaGetLastError());
    return MRPOP_OK;
}

// The reassigned fine stage exists for verdicts only; the clearance and
// work-count modes always take the union form.
template <int MODE>
mrpop_status launch_spl(mrpop_problem *p, VParams &V, int warps, size_t smem,
                        cudaStream_t st) {
    if (MODE == kVerdict && V.fine) return launch_mode<MODE, true>(p, V, warps, smem, st);
    return launch_mode<MODE, false>(p, V, warps, smem, st);
}

// ---------------------------------------------------------------------------
// Forward kinematics of a batch of configurations: one thread per config.
// ---------------------------------------------------------------------------
__global__ void fk_kernel(const float4 *__restrict__ tab, const Tables t,
                          const float *__restrict__ q, int64_t n, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t S = t.S;
    for (int b = 0; b < t.K; ++b) {
        Frame Tm = load_base(tab, t, b);
        for (int l = t.link0[b]; l < t.link0[b + 1]; ++l) {
            const float4 LA = tab[t.off_link + kLinkF4 * l];
            const float4 LB = tab[t.off_link + kLinkF4 * l + 1];
            float sn, cs;
            joint_sincos(q[(size_t)l * n + i] + LB.x, &sn, &cs);
            const Frame F = rotz(Tm, cs, sn);
            const int sf = __float_as_int(LB.y), ns = __float_as_int(LB.z);
            for (int s = 0; s < ns; ++s) {
                const float4 sp = tab[t.off_sph + sf + s];
                const float3 pw = apply(F, sp.x, sp.y, sp.z);
                out[((size_t)0 * S + sf + s) * n + i] = pw.x;
                out[((size_t)1 * S + sf + s) * n + i] = pw.y;
                out[((size_t)2 * S + sf + s) * n + i] = pw.z;
            }
            Tm = advance(F, LA.x, LA.y, LA.z, LA.w);
        }
    }
}

}  // namespace

mrpop_status launch_validate(mrpop_problem *p, const float *qa, const float *qb, int64_t n,
                             uint8_t *valid, float *length, int32_t *npoints,
                             float *min_clear, unsigned long long *counters,
                             cudaStream_t st) {
    const Tables &t = p->dev.t;
    VParams V;
    V.t = t;
    V.blob = p->dev.blob;
    V.qa = qa;
    V.qb = qb;
    V.E = n;
    V.res = p->cfg.resolution;
    V.margin = p->cfg.margin;
    V.valid = valid;
    V.length = length;
    V.npoints = npoints;
    V.min_clear = min_clear;
    V.counters = counters;
    V.work = p->dev.edge_counter;
    V.dpad = (t.L + 3) & ~3;
    V.nstore = t.selfcol ? t.L : t.link0[t.K - 1];
    V.fine = p->tuned_fine;
    V.warp_floats = validate_warp_floats(t, V.fine);
    const size_t tab_bytes = (size_t)t.n_f4 * sizeof(float4);
    int warps = p->tuned_warps > 0 ? p->tuned_warps : kWarpsMax;
    size_t smem = 0;
    for (; warps >= 1; warps >>= 1) {
        smem = tab_bytes + (size_t)warps * V.warp_floats * sizeof(float);
        if (smem <= p->smem_optin) break;
    }
    V.order = p->tuned_order;
    if (warps < 1)
        return set_error(MRPOP_EINVAL,
                         "problem too large for the validation kernel's shared memory "
                         "(%zu bytes of tables + %d bytes per warp)",
                         tab_bytes, V.warp_floats * 4);
    if (min_clear) return launch_spl<kClearance>(p, V, warps, smem, st);
    if (counters) return launch_spl<kCount>(p, V, warps, smem, st);
    return launch_spl<kVerdict>(p, V, warps, smem, st);
}

mrpop_status make_vparams(mrpop_problem *p, const float *qa, const float *qb, int64_t n,
                          uint8_t *valid, VParams *V, size_t *smem_out, int *warps_out) {
    const Tables &t = p->dev.t;
    *V = VParams{};
    V->t = t;
    V->blob = p->dev.blob;
    V->qa = qa;
    V->qb = qb;
    V->E = n;
    V->res = p->cfg.resolution;
    V->margin = p->cfg.margin;
    V->valid = valid;
    V->work = p->dev.edge_counter;
    V->dpad = (t.L + 3) & ~3;
    V->nstore = t.selfcol ? t.L : t.link0[t.K - 1];
    V->fine = p->tuned_fine;
    V->warp_floats = validate_warp_floats(t, V->fine);
    const size_t tab_bytes = (size_t)t.n_f4 * sizeof(float4);
    int warps = p->tuned_warps > 0 ? p->tuned_warps : kWarpsMax;
    size_t smem = 0;
    for (; warps >= 1; warps >>= 1) {
        smem = tab_bytes + (size_t)warps * V->warp_floats * sizeof(float);
        if (smem + sizeof(VParams) + 1024 <= p->smem_optin) break;
    }
    V->order = p->tuned_order;
    if (warps < 1)
        return set_error(MRPOP_EINVAL, "problem too large for the validation kernel's shared memory");
    *smem_out = smem;
    *warps_out = warps;
    V->warps = warps;
    return MRPOP_OK;
}

template <bool RA>
static mrpop_status batch_ra(const VParams *d_params, int nslots, int warps, int blocks_per_slot,
                             size_t smem, cudaStream_t st) {
    auto kern = validate_batch_kernel<RA>;
    int dev = 0, optin = 0, bps = 0;
    MRPOP_CUDA_TRY(cudaGetDevice(&dev));
    MRPOP_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const mrpop_status os = cached_occupancy((const void *)kern, dev, optin, warps * 32, smem, &bps);
    if (os != MRPOP_OK) return os;
    dim3 grid(blocks_per_slot, nslots);
    kern<<<grid, warps * 32, smem, st>>>(d_params);
    MRPOP_CUDA_TRY(cudaGetLastError());
    return MRPOP_OK;
}

mrpop_status launch_validate_batch(const VParams *d_params, int nslots, int /*spl*/, int warps,
                                   int blocks_per_slot, size_t smem, bool fine,
                                   cudaStream_t st) {
    if (fine) return batch_ra<true>(d_params, nslots, warps, blocks_per_slot, smem, st);
    return batch_ra<false>(d_params, nslots, warps, blocks_per_slot, smem, st);
}

// Times the validation kernel on the caller's edges for every candidate
// launch (warps per block 1, 2, 4 that fit; strided or contiguous checkpoint
// order; union or reassigned fine tests; compact or wide register budget),
// keeps the fastest in the problem and in the tuned-launch cache under the
// problem's shape, and reports it.
mrpop_status autotune_validate(mrpop_problem *p, const float *qa, const float *qb, int64_t n,
                               uint8_t *valid, int reps, int32_t *out, float *ms_out,
                               cudaStream_t st) {
    cudaEvent_t a, b;
    MRPOP_CUDA_TRY(cudaEventCreate(&a));
    MRPOP_CUDA_TRY(cudaEventCreate(&b));
    float best = INFINITY;
    int bw = 0, bo = 0, bf = 0, br = 0;
    const int save_w = p->tuned_warps, save_o = p->tuned_order, save_f = p->tuned_fine,
              save_r = p->tuned_regs;
    mrpop_status s = MRPOP_OK;
    for (int w = 1; w <= kWarpsMax && s == MRPOP_OK; w *= 2)
        for (int o = 0; o < 2 && s == MRPOP_OK; ++o)
        for (int f = 0; f < 2 && s == MRPOP_OK; ++f)
        for (int rg = 0; rg < 2 && s == MRPOP_OK; ++rg) {
            const size_t need = (size_t)p->dev.t.n_f4 * sizeof(float4) +
                                (size_t)w * validate_warp_floats(p->dev.t, f) * sizeof(float);
            if (need + sizeof(VParams) + 1024 > p->smem_optin) continue;
            p->tuned_warps = w;
            p->tuned_order = o;
            p->tuned_fine = f;
            p->tuned_regs = rg;
            s = launch_validate(p, qa, qb, n, valid, nullptr, nullptr, nullptr, nullptr, st);  // warm
            float tot = 0.f;
            for (int r = 0; r < reps && s == MRPOP_OK; ++r) {
                cudaEventRecord(a, st);
                s = launch_validate(p, qa, qb, n, valid, nullptr, nullptr, nullptr, nullptr, st);
                cudaEventRecord(b, st);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                tot += ms;
            }
            if (s == MRPOP_OK && tot < best) {
                best = tot;
                bw = w;
                bo = o;
                bf = f;
                br = rg;
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != MRPOP_OK || bw == 0) {
        p->tuned_warps = save_w;
        p->tuned_order = save_o;
        p->tuned_fine = save_f;
        p->tuned_regs = save_r;
        return s != MRPOP_OK ? s : set_error(MRPOP_EINVAL, "no launch configuration fits");
    }
    p->tuned_warps = bw;
    p->tuned_order = bo;
    p->tuned_fine = bf;
    p->tuned_regs = br;
    tune_store(validate_tune_key(p), {bw, bo, bf, br});
    if (out) {
        out[0] = bw;
        out[1] = bo;
        out[2] = bf;
    }
    if (ms_out) *ms_out = best / std::max(1, reps);
    return MRPOP_OK;
}

mrpop_status launch_fk(mrpop_problem *p, const float *q, int64_t n, float *out, cudaStream_t st) {
    const int threads = 128;
    const int64_t blocks = (n + threads - 1) / threads;
    fk_kernel<<<(unsigned)blocks, threads, 0, st>>>(p->dev.blob, p->dev.t, q, n, out);
    MRPOP_CUDA_TRY(cudaGetLastError());
    return MRPOP_OK;
}

}  // namespace mrpop
