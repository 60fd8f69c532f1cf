// Validation body shared by the validation kernels (validate.cu) and the
// planner's persistent kernel (planner.cu): one warp per edge, checkpoints
// across lanes, per-link FK with tile / checkpoint / sphere culling and
// early exit.  See validate.cu for the design.
#pragma once
#include <cfloat>

#include "mrpop_internal.cuh"

namespace mrpop {
namespace vb {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsMax = 4;
constexpr int kCounters = MRPOP_WORK_COUNTERS;
// Absolute slack (m) added to tile bounds: covers FP32 rounding of the box
// centre and half extents (a few ulps of workspace coordinates), so the tile
// test never drops a candidate that a checkpoint's own link-level test keeps.
constexpr float kTileSlack = 4e-4f;


enum Mode { kVerdict = 0, kClearance = 1, kCount = 2 };



struct Frame {
    float r[9];  // row-major rotation
    float t[3];
};

// F = T * Rz(theta): columns 0 and 1 rotate, column 2 and t are unchanged.
__device__ __forceinline__ Frame rotz(const Frame &T, float c, float s) {
    Frame F;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float a = T.r[3 * i], b = T.r[3 * i + 1];
        F.r[3 * i] = fmaf(c, a, s * b);
        F.r[3 * i + 1] = fmaf(c, b, -s * a);
        F.r[3 * i + 2] = T.r[3 * i + 2];
        F.t[i] = T.t[i];
    }
    return F;
}

// T = F * Tz(d) * Tx(a) * Rx(alpha)
__device__ __forceinline__ Frame advance(const Frame &F, float a, float d, float ca, float sa) {
    Frame T;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float c0 = F.r[3 * i], c1 = F.r[3 * i + 1], c2 = F.r[3 * i + 2];
        T.t[i] = fmaf(a, c0, fmaf(d, c2, F.t[i]));
        T.r[3 * i] = c0;
        T.r[3 * i + 1] = fmaf(ca, c1, sa * c2);
        T.r[3 * i + 2] = fmaf(ca, c2, -sa * c1);
    }
    return T;
}

__device__ __forceinline__ float3 apply(const Frame &F, float x, float y, float z) {
    return make_float3(fmaf(F.r[0], x, fmaf(F.r[1], y, fmaf(F.r[2], z, F.t[0]))),
                       fmaf(F.r[3], x, fmaf(F.r[4], y, fmaf(F.r[5], z, F.t[1]))),
                       fmaf(F.r[6], x, fmaf(F.r[7], y, fmaf(F.r[8], z, F.t[2]))));
}

__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by,
                                       float bz) {
    const float dx = ax - bx, dy = ay - by, dz = az - bz;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Squared distance from point p to an oriented box (centre C, half extents H,
// unit axes A0..A2 as columns): |max(|A^T (p - C)| - h, 0)|^2.
__device__ __forceinline__ float box_dist2(float px, float py, float pz, const float4 &C,
                                           const float4 &H, const float4 &A0, const float4 &A1,
                                           const float4 &A2) {
    const float vx = px - C.x, vy = py - C.y, vz = pz - C.z;
    const float p0 = fmaf(A0.x, vx, fmaf(A0.y, vy, A0.z * vz));
    const float p1 = fmaf(A1.x, vx, fmaf(A1.y, vy, A1.z * vz));
    const float p2 = fmaf(A2.x, vx, fmaf(A2.y, vy, A2.z * vz));
    const float u0 = fmaxf(fabsf(p0) - H.x, 0.f);
    const float u1 = fmaxf(fabsf(p1) - H.y, 0.f);
    const float u2 = fmaxf(fabsf(p2) - H.z, 0.f);
    return fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
}

__device__ __forceinline__ Frame load_base(const float4 *tab, const Tables &t, int b) {
    const float4 r0 = tab[t.off_base + 3 * b], r1 = tab[t.off_base + 3 * b + 1],
                 r2 = tab[t.off_base + 3 * b + 2];
    Frame T;
    T.r[0] = r0.x; T.r[1] = r0.y; T.r[2] = r0.z; T.t[0] = r0.w;
    T.r[3] = r1.x; T.r[4] = r1.y; T.r[5] = r1.z; T.t[1] = r1.w;
    T.r[6] = r2.x; T.r[7] = r2.y; T.r[8] = r2.z; T.t[2] = r2.w;
    return T;
}

// Frame F_i' of link i at the lane's checkpoint (parameter tk), rebuilt along
// its robot's chain from the base with the same operations, in the same order,
// as the main forward-kinematics loop.  Used only by fine robot-robot tests,
// which are rare; the coarse tests read the stored coarse centres.
__device__ __forceinline__ Frame link_frame(const float4 *tab, const Tables &t, const float *qa_s,
                                            const float *dq_s, int i, float tk);

// Joint-angle sine and cosine: reduce the angle to [-pi, pi] with one fused
// multiply-add, then the hardware approximation __sincosf (absolute error
// about 2^-21 on that interval; over a 7-joint chain with a 1.2 m reach it
// moves a sphere by a few micrometres, far inside the 1e-4 m contact band
// and the 1e-5 relative distance tolerance).
__device__ __forceinline__ void joint_sincos(float th, float *s, float *c) {
    const float k = rintf(th * 0.15915494f);        // th / (2 pi), nearest integer
    __sincosf(fmaf(-6.28318548f, k, th), s, c);
}

__device__ __forceinline__ unsigned low_mask(int n) { return n >= 32 ? kFull : ((1u << n) - 1u); }

// Second stage with load-proportional reassignment (Sec. III-E): the fine
// tests that the lanes' own coarse hits call for -- (checkpoint k, obstacle o
// hit by k's link sphere, fine sphere s of the link) -- are numbered by a warp
// prefix sum of the per-lane counts and dealt out to all 32 lanes in turn, so
// the warp spends ceil(total / 32) passes on them instead of one pass of
// every lane over every obstacle that any lane hit.  A lane rebuilds its
// item's fine sphere from the owning checkpoint's link frame, which every lane
// puts in the warp's shared scratch fr ([12][32] floats, then 32 hit masks and
// 32 prefix sums).  A fine hit implies a coarse hit (the coarse sphere encloses
// the fine ones with slack), so the verdict equals the union form's.
template <bool CUBOID>
__device__ __forceinline__ bool fine_reassigned(unsigned own, int c0, int ns, int sf,
                                                const Frame &F, float m, const float4 *tab,
                                                const Tables &t, float *fr, int lane) {
    if (!__any_sync(kFull, own != 0u)) return false;  // the common case: no fine work
    const int mine = __popc(own) * ns;
    int incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return false;
    unsigned *own_s = reinterpret_cast<unsigned *>(fr + kFrFloats * 32);
    int *pre_s = reinterpret_cast<int *>(own_s + 32);
#pragma unroll
    for (int c = 0; c < 9; ++c) fr[c * 32 + lane] = F.r[c];
    fr[9 * 32 + lane] = F.t[0];
    fr[10 * 32 + lane] = F.t[1];
    fr[11 * 32 + lane] = F.t[2];
    own_s[lane] = own;
    pre_s[lane] = incl - mine;
    __syncwarp();
    const float inv_ns = 1.f / (float)ns;
    bool hit = false;
    for (int b = 0; b < total; b += 32) {
        const int item = b + lane;
        if (item < total) {
            int k = 0;  // owner: the last lane whose first item is <= item
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (pre_s[k + step] <= item) k += step;
            const int r = item - pre_s[k];
            int jo = (int)((float)r * inv_ns);  // r / ns, corrected below
            if (jo * ns > r) --jo;
            if ((jo + 1) * ns <= r) ++jo;
            const int s = r - jo * ns;
            unsigned mm = own_s[k];
            for (int q = 0; q < jo; ++q) mm &= mm - 1;  // jo-th set bit of k's mask
            const int o = __ffs(mm) - 1;
            Frame Fk;
#pragma unroll
            for (int c = 0; c < 9; ++c) Fk.r[c] = fr[c * 32 + k];
            Fk.t[0] = fr[9 * 32 + k];
            Fk.t[1] = fr[10 * 32 + k];
            Fk.t[2] = fr[11 * 32 + k];
            const float4 sp = tab[t.off_sph + sf + s];
            const float3 p = apply(Fk, sp.x, sp.y, sp.z);
            if (CUBOID) {
                const float4 *cbp = tab + t.off_oc + kCuboidF4 * (c0 + o);
                const float d2 = box_dist2(p.x, p.y, p.z, cbp[0], cbp[1], cbp[2], cbp[3], cbp[4]);
                const float th2 = sp.w + m;
                hit |= d2 < th2 * th2;
            } else {
                const float4 ob = tab[t.off_os + c0 + o];
                const float d2 = dist2(p.x, p.y, p.z, ob.x, ob.y, ob.z);
                const float th2 = sp.w + ob.w + m;
                hit |= d2 < th2 * th2;
            }
        }
    }
    __syncwarp();  // the scratch is rewritten by the next call
    return hit;
}

__device__ __forceinline__ Frame link_frame(const float4 *tab, const Tables &t, const float *qa_s,
                                            const float *dq_s, int i, float tk) {
    int b = 0;
    while (t.link0[b + 1] <= i) ++b;
    Frame Tm = load_base(tab, t, b);
    for (int l = t.link0[b];; ++l) {
        const float4 LA = tab[t.off_link + kLinkF4 * l];
        const float4 LB = tab[t.off_link + kLinkF4 * l + 1];
        const float th = __fmaf_rn(tk, dq_s[l], qa_s[l]) + LB.x;
        float sn, cs;
        joint_sincos(th, &sn, &cs);
        const Frame F = rotz(Tm, cs, sn);
        if (l == i) return F;
        Tm = advance(F, LA.x, LA.y, LA.z, LA.w);
    }
}

// Interval count n = max(1, ceil(|dq|_2 / res)) in FP32 with a sequential
// fused multiply-add sum (the oracle takes the same integer decision in FP32).
__device__ __forceinline__ int interval_count(const float *dq, int D, float res, float *len_out) {
    float acc = 0.f;
    for (int i = 0; i < D; ++i) acc = __fmaf_rn(dq[i], dq[i], acc);
    const float len = __fsqrt_rn(acc);
    const float nf = ceilf(__fdiv_rn(len, res));
    *len_out = len;
    if (!(nf >= 1.f)) return 1;
    return nf > 1073741824.f ? 1073741824 : (int)nf;
}

// LOCAL: the edges [e0, e1) are handed out to the block's warps through the
// shared-memory counter *s_next (zeroed by the caller before the call) instead
// of the problem's global work counter, which is then left untouched.
template <int MODE, bool RA, bool LOCAL = false>
__device__ __forceinline__ void validate_body(const VParams &P, float4 *sm4, int e0 = 0,
                                              int e1 = 0, int *s_next = nullptr) {
    float4 *tab = sm4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *ws = reinterpret_cast<float *>(sm4 + P.t.n_f4) + (size_t)warp * P.warp_floats;
    float *qa_s = ws, *dq_s = ws + P.dpad;
    float4 *tb = reinterpret_cast<float4 *>(ws + 2 * P.dpad);      // tile bounds [nstore]
    float *xc = ws + 2 * P.dpad + 4 * P.nstore;                     // [nstore][3][32]
    float *fr = xc + P.nstore * kXcFloats * 32;                     // reassignment scratch
    constexpr bool ra = MODE == kVerdict && RA;  // reassigned fine obstacle tests

    for (int i = threadIdx.x; i < P.t.n_f4; i += blockDim.x) tab[i] = P.blob[i];
    __syncthreads();
    if (warp >= P.warps) return;  // spare warps of a shared multi-problem launch

    const Tables &t = P.t;
    // table offsets and the workspace corner read once (the loops below would
    // otherwise reload them from the launch parameters at every use)
    const int o_link = t.off_link, o_os = t.off_os, o_oc = t.off_oc, o_sph = t.off_sph;
    const float wlx = t.ws_lo[0], wly = t.ws_lo[1], wlz = t.ws_lo[2];
    const int K = t.K, D = t.L, NS = t.NS, NC = t.NC;
    const float m = P.margin;
    unsigned long long cnt[kCounters];
#pragma unroll
    for (int c = 0; c < kCounters; ++c) cnt[c] = 0ull;

    for (;;) {
        int e = 0;
        if (lane == 0) e = LOCAL ? e0 + atomicAdd(s_next, 1) : atomicAdd(&P.work[0], 1);
        e = __shfl_sync(kFull, e, 0);
        if (e >= (LOCAL ? e1 : P.E)) break;
        __syncwarp();
        for (int i = lane; i < D; i += 32) {
            // (the persistent planner rewrites its edge buffers within one
            // launch: there the loads bypass the non-coherent cache)
            const float a = LOCAL ? __ldcg(P.qa + (size_t)i * P.E + e) : __ldg(P.qa + (size_t)i * P.E + e);
            const float b = LOCAL ? __ldcg(P.qb + (size_t)i * P.E + e) : __ldg(P.qb + (size_t)i * P.E + e);
            qa_s[i] = a;
            dq_s[i] = __fsub_rn(b, a);
        }
        __syncwarp();
        float len;
        const int n = interval_count(dq_s, D, P.res, &len);
        // Edges beyond MRPOP_MAX_EDGE_INTERVALS intervals (or with non-finite
        // coordinates) are reported invalid without being checked.
        const bool too_long = !(len <= P.res * (float)MRPOP_MAX_EDGE_INTERVALS);
        const int T = too_long ? 0 : (n >> 5) + 1;  // ceil((n + 1) / 32)
        bool edge_hit = too_long;
        float minc = too_long ? -FLT_MAX : FLT_MAX;

        for (int tile = 0; tile < T; ++tile) {
            int k = P.order ? tile * 32 + lane : tile + T * lane;
            const bool active = k <= n;
            if (!active) k = n;
            const float tk = __fdiv_rn((float)k, (float)n);
            bool hit = false;
            if (MODE == kCount && active) cnt[0] += 1;
            // joint angles' sine and cosine one link ahead, so that the
            // special-function latency overlaps the previous link's tests
            float sn_next, cs_next;
            joint_sincos(__fmaf_rn(tk, dq_s[0], qa_s[0]) + tab[o_link + 1].x, &sn_next,
                         &cs_next);

            for (int b = 0; b < K; ++b) {
                const int l0 = t.link0[b], l1 = t.link0[b + 1];
                const bool store = b < K - 1 || t.selfcol;
                Frame Tm = load_base(tab, t, b);
                for (int l = l0; l < l1; ++l) {
                    const float4 LA = tab[o_link + kLinkF4 * l];
                    const float4 LB = tab[o_link + kLinkF4 * l + 1];
                    const float4 LC = tab[o_link + kLinkF4 * l + 2];
                    const float sn = sn_next, cs = cs_next;
                    if (l + 1 < D)
                        joint_sincos(__fmaf_rn(tk, dq_s[l + 1], qa_s[l + 1]) +
                                         tab[o_link + kLinkF4 * (l + 1) + 1].x,
                                     &sn_next, &cs_next);
                    const Frame F = rotz(Tm, cs, sn);
                    const float3 cc = apply(F, LC.x, LC.y, LC.z);
                    const int sf = __float_as_int(LB.y), ns = __float_as_int(LB.z);
                    if (MODE == kCount && active) cnt[1] += 1;

                    // Tile bound: one sphere around this link's coarse spheres at
                    // all 32 checkpoints of the tile (warp-uniform), built from the
                    // exact axis-aligned box of the coarse centres.  Taken relative
                    // to the workspace corner ws_lo the coordinates are >= 0, so
                    // their float bits order like unsigned integers and min and max
                    // are single-instruction warp reductions.
                    float4 bnd = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (MODE != kClearance) {
                        const unsigned ux = __float_as_uint(cc.x - wlx);
                        const unsigned uy = __float_as_uint(cc.y - wly);
                        const unsigned uz = __float_as_uint(cc.z - wlz);
                        const float x0 = __uint_as_float(__reduce_min_sync(kFull, ux));
                        const float x1 = __uint_as_float(__reduce_max_sync(kFull, ux));
                        const float y0 = __uint_as_float(__reduce_min_sync(kFull, uy));
                        const float y1 = __uint_as_float(__reduce_max_sync(kFull, uy));
                        const float z0 = __uint_as_float(__reduce_min_sync(kFull, uz));
                        const float z1 = __uint_as_float(__reduce_max_sync(kFull, uz));
                        const float ex = 0.5f * (x1 - x0), ey = 0.5f * (y1 - y0),
                                    ez = 0.5f * (z1 - z0);
                        bnd.x = wlx + 0.5f * (x0 + x1);
                        bnd.y = wly + 0.5f * (y0 + y1);
                        bnd.z = wlz + 0.5f * (z0 + z1);
                        // the hardware's approximate square root (an error of a few
                        // ulps), padded by 2^-16 relative; kTileSlack covers the rest
                        float rbox;
                        asm("sqrt.approx.f32 %0, %1;"
                            : "=f"(rbox)
                            : "f"(fmaf(ex, ex, fmaf(ey, ey, ez * ez))));
                        bnd.w = fmaf(rbox, 1.0000153f, LC.w + kTileSlack);
                        if (!(bnd.w < FLT_MAX)) bnd.w = FLT_MAX * 2.f;  // never for finite inputs
                        if (MODE == kCount && lane == 0) cnt[9] += 1;
                    }
                    if (store) {
                        float *x = xc + (size_t)l * kXcFloats * 32 + lane;
                        x[0] = cc.x;
                        x[32] = cc.y;
                        x[64] = cc.z;
                        if (lane == 0) tb[l] = bnd;
                        __syncwarp();
                    }
                    bool vote = false;  // a fine stage ran: the early-exit vote is due
                    if (ns > 0) {
                        bool own_any = false;
                        if (MODE == kCount && active) cnt[7] += 1;  // coarse centre
                        const float rc = LC.w + m;

                        // ---- robot vs obstacle spheres
                        for (int c0 = 0; c0 < NS; c0 += 32) {
                            const int cn = min(32, NS - c0);
                            unsigned own = 0, cand = 0;
                            if (MODE == kClearance) {
                                own = low_mask(cn);
                            } else {
                                bool h = false;
                                if (lane < cn) {
                                    const float4 ob = tab[o_os + c0 + lane];
                                    const float d2 = dist2(bnd.x, bnd.y, bnd.z, ob.x, ob.y, ob.z);
                                    const float th2 = bnd.w + ob.w + m;
                                    h = d2 < th2 * th2;
                                }
                                cand = __ballot_sync(kFull, h);
                                unsigned cm = cand;
                                while (cm) {
                                    const int o = __ffs(cm) - 1;
                                    cm &= cm - 1;
                                    const float4 ob = tab[o_os + c0 + o];
                                    const float d2 = dist2(cc.x, cc.y, cc.z, ob.x, ob.y, ob.z);
                                    const float th2 = rc + ob.w;
                                    own |= (d2 < th2 * th2) ? (1u << o) : 0u;
                                }
                                if (MODE == kCount) {
                                    if (lane == 0) cnt[8] += cn;
                                    if (active) cnt[2] += __popc(cand);
                                }
                            }
                            if (MODE != kClearance && cand == 0u) continue;  // nothing near
                            vote = true;
                            if (ra) {
                                hit |= fine_reassigned<false>(own, c0, ns, sf, F, m, tab, t, fr,
                                                              lane);
                                continue;
                            }
                            const unsigned wm =
                                MODE == kClearance ? own : __reduce_or_sync(kFull, own);
                            if (MODE == kCount && active) {
                                cnt[4] += (unsigned long long)__popc(own) * ns;
                                own_any |= own != 0;
                            }
                            // fine stage: each of the link's spheres is placed once and
                            // tested against every obstacle of the warp's union mask
                            for (int s = 0; wm && s < ns; ++s) {
                                const float4 sp = tab[o_sph + sf + s];
                                const float3 p = apply(F, sp.x, sp.y, sp.z);
                                unsigned mm = wm;
                                while (mm) {
                                    const int o = __ffs(mm) - 1;
                                    mm &= mm - 1;
                                    const float4 ob = tab[o_os + c0 + o];
                                    const float d2 = dist2(p.x, p.y, p.z, ob.x, ob.y, ob.z);
                                    if (MODE == kClearance) {
                                        minc = fminf(minc, __fsqrt_rn(d2) - sp.w - ob.w);
                                    } else {
                                        const float th2 = sp.w + ob.w + m;
                                        hit |= d2 < th2 * th2;
                                    }
                                }
                            }
                        }

                        // ---- robot vs obstacle cuboids (oriented boxes); the tile and
                        // checkpoint levels test their bounding spheres against the box
                        // itself (distance to a convex set is 1-Lipschitz, so a sphere
                        // that encloses the fine spheres stays conservative)
                        for (int c0 = 0; c0 < NC; c0 += 32) {
                            const int cn = min(32, NC - c0);
                            unsigned own = 0, cand = 0;
                            if (MODE == kClearance) {
                                own = low_mask(cn);
                            } else {
                                // the box's bounding sphere first (the box lies within
                                // it), its exact distance only when the sphere is near
                                bool h = false, exact = false;
                                if (lane < cn) {
                                    const float4 *cbp = tab + o_oc + kCuboidF4 * (c0 + lane);
                                    const float4 cb0 = cbp[0];
                                    const float dc2 = dist2(bnd.x, bnd.y, bnd.z, cb0.x, cb0.y, cb0.z);
                                    const float reach = cb0.w + bnd.w + m;
                                    exact = dc2 < reach * reach;
                                    if (exact) {
                                        const float d2 = box_dist2(bnd.x, bnd.y, bnd.z, cb0, cbp[1],
                                                                   cbp[2], cbp[3], cbp[4]);
                                        const float th2 = bnd.w + m;
                                        h = d2 < th2 * th2;
                                    }
                                }
                                cand = __ballot_sync(kFull, h);
                                unsigned cm = cand;
                                while (cm) {
                                    const int o = __ffs(cm) - 1;
                                    cm &= cm - 1;
                                    const float4 *cbp = tab + o_oc + kCuboidF4 * (c0 + o);
                                    const float d2 = box_dist2(cc.x, cc.y, cc.z, cbp[0], cbp[1],
                                                               cbp[2], cbp[3], cbp[4]);
                                    own |= (d2 < rc * rc) ? (1u << o) : 0u;
                                }
                                if (MODE == kCount) {
                                    if (lane == 0) cnt[8] += cn;  // the bounding-sphere tests
                                    if (exact) cnt[11] += 1;
                                    if (active) cnt[10] += __popc(cand);
                                }
                            }
                            if (MODE != kClearance && cand == 0u) continue;  // nothing near
                            vote = true;
                            if (ra) {
                                hit |= fine_reassigned<true>(own, c0, ns, sf, F, m, tab, t, fr,
                                                             lane);
                                continue;
                            }
                            const unsigned wm =
                                MODE == kClearance ? own : __reduce_or_sync(kFull, own);
                            if (MODE == kCount && active) {
                                cnt[5] += (unsigned long long)__popc(own) * ns;
                                own_any |= own != 0;
                            }
                            for (int s = 0; wm && s < ns; ++s) {
                                const float4 sp = tab[o_sph + sf + s];
                                const float3 p = apply(F, sp.x, sp.y, sp.z);
                                unsigned mm = wm;
                                while (mm) {
                                    const int o = __ffs(mm) - 1;
                                    mm &= mm - 1;
                                    const float4 *cbp = tab + o_oc + kCuboidF4 * (c0 + o);
                                    const float d2 = box_dist2(p.x, p.y, p.z, cbp[0], cbp[1], cbp[2],
                                                               cbp[3], cbp[4]);
                                    if (MODE == kClearance) {
                                        minc = fminf(minc, __fsqrt_rn(d2) - sp.w);
                                    } else {
                                        const float th2 = sp.w + m;
                                        hit |= d2 < th2 * th2;
                                    }
                                }
                            }
                        }

                        // ---- robot vs earlier robots (links 0 .. l0-1) and, with
                        // self-collision, vs the links of this robot that its
                        // adjacency mask pairs with link l (bit i: link l0 + i)
                        const unsigned long long pm =
                            (l0 > 0 ? ~0ull >> (64 - l0) : 0ull) |
                            ((unsigned long long)(unsigned)__float_as_int(LB.w) << l0);
                        const unsigned pm0 = (unsigned)pm, pm1 = (unsigned)(pm >> 32);
                        if (pm) {
                            unsigned own0 = 0, own1 = 0, candp = 0;
                            if (MODE == kClearance) {
                                own0 = pm0;
                                own1 = pm1;
                            } else {
                                // tile-level candidates: lane i tests link i (and i + 32)
                                bool h0 = false, h1 = false;
                                if ((pm0 >> lane) & 1u) {
                                    const float4 o = tb[lane];
                                    const float d2 = dist2(bnd.x, bnd.y, bnd.z, o.x, o.y, o.z);
                                    const float th2 = bnd.w + o.w + m;
                                    h0 = d2 < th2 * th2;
                                }
                                if ((pm1 >> lane) & 1u) {
                                    const float4 o = tb[lane + 32];
                                    const float d2 = dist2(bnd.x, bnd.y, bnd.z, o.x, o.y, o.z);
                                    const float th2 = bnd.w + o.w + m;
                                    h1 = d2 < th2 * th2;
                                }
                                const unsigned cand0 = __ballot_sync(kFull, h0);
                                const unsigned cand1 = __ballot_sync(kFull, h1);
                                for (int w = 0; w < 2; ++w) {
                                    unsigned cm = w == 0 ? cand0 : cand1;
                                    unsigned own = 0;
                                    while (cm) {
                                        const int bit = __ffs(cm) - 1;
                                        cm &= cm - 1;
                                        const int i = bit + 32 * w;
                                        const float4 LCi = tab[o_link + kLinkF4 * i + 2];
                                        const float *x = xc + (size_t)i * kXcFloats * 32 + lane;
                                        const float d2 = dist2(cc.x, cc.y, cc.z, x[0], x[32], x[64]);
                                        const float th2 = LC.w + LCi.w + m;
                                        own |= (d2 < th2 * th2) ? (1u << bit) : 0u;
                                    }
                                    if (w == 0)
                                        own0 = own;
                                    else
                                        own1 = own;
                                }
                                if (MODE == kCount) {
                                    if (lane == 0) cnt[8] += __popcll(pm);
                                    if (active) cnt[3] += __popc(cand0) + __popc(cand1);
                                }
                                candp = cand0 | cand1;
                            }
                            if (MODE == kClearance || candp != 0u) {
                            vote = true;
                            const unsigned w0 = MODE == kClearance ? own0 : __reduce_or_sync(kFull, own0);
                            const unsigned w1 = MODE == kClearance ? own1 : __reduce_or_sync(kFull, own1);
                            if (MODE == kCount && active) {
                                own_any |= (own0 | own1) != 0;
                                for (int w = 0; w < 2; ++w) {
                                    unsigned mm = w == 0 ? own0 : own1;
                                    while (mm) {
                                        const int i = __ffs(mm) - 1 + 32 * w;
                                        mm &= mm - 1;
                                        const int nsi =
                                            __float_as_int(tab[o_link + kLinkF4 * i + 1].z);
                                        cnt[6] += (unsigned long long)nsi * ns;
                                        cnt[7] += nsi;
                                    }
                                }
                            }
                            for (int w = 0; w < 2; ++w) {
                                unsigned mm = w == 0 ? w0 : w1;
                                while (mm) {
                                    const int i = __ffs(mm) - 1 + 32 * w;
                                    mm &= mm - 1;
                                    const Frame Fi = link_frame(tab, t, qa_s, dq_s, i, tk);
                                    const float4 LBi = tab[o_link + kLinkF4 * i + 1];
                                    const int sfi = __float_as_int(LBi.y), nsi = __float_as_int(LBi.z);
                                    // the other link's spheres four at a time, this
                                    // link's placed once per group of four
                                    for (int g0 = 0; g0 < nsi; g0 += 4) {
                                        float4 pa[4];
#pragma unroll
                                        for (int j = 0; j < 4; ++j) {
                                            const float4 sp2 = tab[o_sph + sfi + min(g0 + j, nsi - 1)];
                                            const float3 q3 = apply(Fi, sp2.x, sp2.y, sp2.z);
                                            pa[j] = make_float4(q3.x, q3.y, q3.z, sp2.w);
                                        }
                                        const int gn = min(4, nsi - g0);
                                        for (int s = 0; s < ns; ++s) {
                                            const float4 sp = tab[o_sph + sf + s];
                                            const float3 p = apply(F, sp.x, sp.y, sp.z);
#pragma unroll
                                            for (int j = 0; j < 4; ++j) {
                                                if (j >= gn) break;
                                                const float d2 =
                                                    dist2(p.x, p.y, p.z, pa[j].x, pa[j].y, pa[j].z);
                                                if (MODE == kClearance) {
                                                    minc = fminf(minc,
                                                                 __fsqrt_rn(d2) - sp.w - pa[j].w);
                                                } else {
                                                    const float th2 = sp.w + pa[j].w + m;
                                                    hit |= d2 < th2 * th2;
                                                }
                                            }
                                        }
                                    }
                                }
                            }
                            }  // candidates near link l
                        }
                        if (MODE == kCount && active && own_any) cnt[7] += ns;
                    }
                    Tm = advance(F, LA.x, LA.y, LA.z, LA.w);
                    // a hit can only come from a fine stage of this link
                    if (MODE != kClearance && vote && __any_sync(kFull, hit)) goto tile_done;
                }
            }
        tile_done:
            if (MODE != kClearance && __any_sync(kFull, hit)) {
                edge_hit = true;
                break;
            }
        }

        if (MODE == kClearance) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                minc = fminf(minc, __shfl_xor_sync(kFull, minc, off));
            if (lane == 0) P.min_clear[e] = minc;
        } else if (MODE == kVerdict) {
            if (lane == 0) {
                P.valid[e] = edge_hit ? 0 : 1;
                if (P.length) P.length[e] = len;
                if (P.npoints) P.npoints[e] = n;
            }
        }
    }

    if (MODE == kCount) {
#pragma unroll
        for (int c = 0; c < kCounters; ++c) {
            unsigned long long v = cnt[c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
            if (lane == 0 && v) atomicAdd(P.counters + c, v);
        }
    }
    // The last warp to leave resets the work counter for the next launch on
    // this problem (every warp has made its final fetch before counting out).
    if (!LOCAL && lane == 0) {
        __threadfence();
        if (atomicAdd(&P.work[1], 1) == P.total_warps - 1) {
            atomicExch(&P.work[0], 0);
            atomicExch(&P.work[1], 0);
        }
    }
}

}  // namespace vb
}  // namespace mrpop
