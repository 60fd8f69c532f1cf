// C ABI entry points: problem creation (geometry tables), argument checking
// and dispatch to the kernel launchers.  Every entry point returns a status
// and records a message for mrpop_last_error(); nothing here aborts.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>

#include "mrpop_internal.cuh"

namespace mrpop {

static thread_local char g_err[512] = "";

mrpop_status set_error(mrpop_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

mrpop_status cuda_error(cudaError_t e, const char *what) {
    return set_error(e == cudaErrorMemoryAllocation ? MRPOP_ENOMEM : MRPOP_ECUDA,
                     "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Tuned launch cache
// ---------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::string, std::vector<int>> g_tune;

std::string tune_arch() {
    static std::string arch;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, ma = 0, mi = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess)
            arch = "sm_" + std::to_string(ma) + std::to_string(mi);
        else
            arch = "sm_unknown";
    });
    return arch;
}

bool tune_lookup(const std::string &key, std::vector<int> *val) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *val = it->second;
    return true;
}

void tune_store(const std::string &key, const std::vector<int> &val) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = val;
}

int log2_bucket(int64_t n) {
    int b = 0;
    while (n > 1) {
        n >>= 1;
        ++b;
    }
    return b;
}

// Shape of a problem's validation work (robots, links, spheres, obstacles,
// largest spheres per link, self-collision): problems of one shape share a
// tuned launch.
std::string validate_tune_key(const mrpop_problem *p) {
    const Tables &t = p->dev.t;
    std::ostringstream k;
    k << "validate " << tune_arch() << " K=" << t.K << " L=" << t.L << " S=" << t.S
      << " NS=" << t.NS << " NC=" << t.NC << " spl=" << t.max_spheres_per_link
      << " self=" << t.selfcol;
    return k.str();
}

// ---------------------------------------------------------------------------
// Stream-ordered scratch from a library-owned memory pool per device.  The
// device's default pool returns freed memory to the system at every
// synchronisation, so a call that follows one would map its scratch again
// (about 0.1 ms for a NEAREST batch); this pool keeps up to 1 GiB of it.
// ---------------------------------------------------------------------------
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaError_t scratch_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        unsigned long long keep = 1ull << 30;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) !=
            cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

cudaError_t scratch_alloc(void **ptr, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = scratch_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

static bool finite_all(const float *v, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

static float f_of_i(int v) {
    float f;
    std::memcpy(&f, &v, sizeof(f));
    return f;
}

}  // namespace mrpop

using namespace mrpop;

extern "C" const char *mrpop_last_error(void) { return g_err; }

// Coarse sphere of one link, in the link frame F_j': centre at the midpoint of
// the axis-aligned box around the link's fine spheres, radius the largest
// |centre - c_s| + r_s plus a slack that absorbs FP32 rounding of both the
// coarse and the fine sphere positions (coarse culling never changes a
// verdict, Sec. III-E two-stage check).
static void coarse_sphere(const float *xyzr, int n, float out[4]) {
    if (n == 0) {
        out[0] = out[1] = out[2] = 0.f;
        out[3] = 0.f;
        return;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int s = 0; s < n; ++s)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::fmin(lo[a], (double)xyzr[4 * s + a] - xyzr[4 * s + 3]);
            hi[a] = std::fmax(hi[a], (double)xyzr[4 * s + a] + xyzr[4 * s + 3]);
        }
    double c[3], r = 0.0;
    for (int a = 0; a < 3; ++a) c[a] = 0.5 * (lo[a] + hi[a]);
    for (int s = 0; s < n; ++s) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double d = (double)xyzr[4 * s + a] - c[a];
            d2 += d * d;
        }
        r = std::fmax(r, std::sqrt(d2) + xyzr[4 * s + 3]);
    }
    for (int a = 0; a < 3; ++a) out[a] = (float)c[a];
    out[3] = (float)(r + 1e-4);
}

extern "C" mrpop_status mrpop_create_problem(const mrpop_robot *robots, int32_t K,
                                             const mrpop_obstacles *obs, const float *start,
                                             const float *goal, const mrpop_config *cfg,
                                             mrpop_problem **out) {
    if (!out) return set_error(MRPOP_EINVAL, "mrpop_create_problem: out is NULL");
    *out = nullptr;
    if (!robots || !obs || !cfg)
        return set_error(MRPOP_EINVAL, "mrpop_create_problem: robots, obs and cfg are required");
    if (K < 1 || K > MRPOP_MAX_ROBOTS)
        return set_error(MRPOP_EINVAL, "K=%d outside [1, %d]", K, MRPOP_MAX_ROBOTS);
    if (!(cfg->resolution > 0.f) || !std::isfinite(cfg->resolution))
        return set_error(MRPOP_EINVAL, "resolution must be positive and finite");
    if (!(cfg->margin >= 0.f) || !std::isfinite(cfg->margin))
        return set_error(MRPOP_EINVAL, "margin must be >= 0 and finite");

    if (cfg->self_collision != 0 && cfg->self_collision != 1)
        return set_error(MRPOP_EINVAL, "self_collision must be 0 or 1");
    Tables t;
    t.K = K;
    t.selfcol = cfg->self_collision;
    int L = 0, S = 0;
    for (int k = 0; k < K; ++k) {
        const mrpop_robot &r = robots[k];
        if (r.dof < 1 || r.dof > MRPOP_MAX_DOF)
            return set_error(MRPOP_EINVAL, "robot %d: dof=%d outside [1, %d]", k, r.dof,
                             MRPOP_MAX_DOF);
        if (r.n_spheres < 0) return set_error(MRPOP_EINVAL, "robot %d: n_spheres < 0", k);
        if (!r.dh || !r.q_lo || !r.q_hi || (r.n_spheres > 0 && (!r.sphere_link || !r.sphere_xyzr)))
            return set_error(MRPOP_EINVAL, "robot %d: missing table pointer", k);
        if (!finite_all(r.dh, 4 * r.dof) || !finite_all(r.q_lo, r.dof) ||
            !finite_all(r.q_hi, r.dof) || !finite_all(r.base, 12) ||
            (r.n_spheres > 0 && !finite_all(r.sphere_xyzr, 4 * (int64_t)r.n_spheres)))
            return set_error(MRPOP_EINVAL, "robot %d: non-finite table entry", k);
        for (int j = 0; j < r.dof; ++j)
            if (!(r.q_lo[j] <= r.q_hi[j]))
                return set_error(MRPOP_EINVAL, "robot %d joint %d: q_lo > q_hi", k, j);
        {   // the base rotation must be proper: R^T R = I within 1e-3, det R > 0
            const float *b = r.base;
            double worst = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double dot = 0.0;
                    for (int m = 0; m < 3; ++m) dot += (double)b[4 * m + i] * b[4 * m + j];
                    worst = std::max(worst, std::fabs(dot - (i == j ? 1.0 : 0.0)));
                }
            const double det = (double)b[0] * ((double)b[5] * b[10] - (double)b[6] * b[9]) -
                               (double)b[1] * ((double)b[4] * b[10] - (double)b[6] * b[8]) +
                               (double)b[2] * ((double)b[4] * b[9] - (double)b[5] * b[8]);
            if (!(worst <= 1e-3) || !(det > 0.0))
                return set_error(MRPOP_EINVAL, "robot %d: base is not a proper rotation", k);
        }
        int prev = 0;
        for (int s = 0; s < r.n_spheres; ++s) {
            const int l = r.sphere_link[s];
            if (l < prev || l >= r.dof)
                return set_error(MRPOP_EINVAL,
                                 "robot %d sphere %d: link %d not non-decreasing in [0, %d)",
                                 k, s, l, r.dof);
            if (r.sphere_xyzr[4 * s + 3] < 0.f)
                return set_error(MRPOP_EINVAL, "robot %d sphere %d: negative radius", k, s);
            prev = l;
        }
        t.link0[k] = L;
        L += r.dof;
        S += r.n_spheres;
    }
    if (L > MRPOP_MAX_LINKS)
        return set_error(MRPOP_EINVAL, "total dof %d exceeds %d", L, MRPOP_MAX_LINKS);
    t.link0[K] = L;
    t.L = L;
    t.S = S;
    if (obs->n_spheres < 0 || obs->n_cuboids < 0 ||
        obs->n_spheres + (int64_t)obs->n_cuboids > MRPOP_MAX_OBSTACLES)
        return set_error(MRPOP_EINVAL, "obstacle counts (%d spheres, %d cuboids) outside [0, %d]",
                         obs->n_spheres, obs->n_cuboids, MRPOP_MAX_OBSTACLES);
    if ((obs->n_spheres > 0 && !obs->spheres) || (obs->n_cuboids > 0 && !obs->cuboids))
        return set_error(MRPOP_EINVAL, "missing obstacle table pointer");
    if ((obs->n_spheres > 0 && !finite_all(obs->spheres, 4 * (int64_t)obs->n_spheres)) ||
        (obs->n_cuboids > 0 && !finite_all(obs->cuboids, 15 * (int64_t)obs->n_cuboids)))
        return set_error(MRPOP_EINVAL, "non-finite obstacle entry");
    for (int o = 0; o < obs->n_spheres; ++o)
        if (obs->spheres[4 * o + 3] < 0.f)
            return set_error(MRPOP_EINVAL, "obstacle sphere %d: negative radius", o);
    for (int o = 0; o < obs->n_cuboids; ++o)
        for (int a = 0; a < 3; ++a)
            if (obs->cuboids[15 * o + 3 + a] < 0.f)
                return set_error(MRPOP_EINVAL, "cuboid %d: negative half extent", o);
    t.NS = obs->n_spheres;
    t.NC = obs->n_cuboids;

    // --- pack the blob ---------------------------------------------------
    t.off_base = 0;
    t.off_link = t.off_base + 3 * K;
    t.off_sph = t.off_link + kLinkF4 * L;
    t.off_os = t.off_sph + S;
    t.off_oc = t.off_os + t.NS;
    t.n_f4 = t.off_oc + kCuboidF4 * t.NC;
    std::vector<float> blob(4 * (size_t)t.n_f4, 0.f);
    auto f4 = [&](int i) { return blob.data() + 4 * (size_t)i; };
    int s_glob = 0;
    for (int k = 0; k < K; ++k) {
        const mrpop_robot &r = robots[k];
        std::memcpy(f4(t.off_base + 3 * k), r.base, 12 * sizeof(float));
        int s = 0;
        for (int j = 0; j < r.dof; ++j) {
            const int l = t.link0[k] + j;
            const int first = s;
            while (s < r.n_spheres && r.sphere_link[s] == j) ++s;
            const int cnt = s - first;
            if (cnt > MRPOP_MAX_SPHERES_PER_LINK)
                return set_error(MRPOP_EINVAL, "robot %d link %d: %d spheres exceed %d", k, j,
                                 cnt, MRPOP_MAX_SPHERES_PER_LINK);
            t.max_spheres_per_link = cnt > t.max_spheres_per_link ? cnt : t.max_spheres_per_link;
            const float *dh = r.dh + 4 * j;  // a, alpha, d, theta_offset
            float *A = f4(t.off_link + kLinkF4 * l);
            A[0] = dh[0];
            A[1] = dh[2];
            A[2] = (float)std::cos((double)dh[1]);
            A[3] = (float)std::sin((double)dh[1]);
            A[4] = dh[3];
            A[5] = f_of_i(s_glob + first);
            A[6] = f_of_i(cnt);
            // same-robot partner links of link j (bit i: link i < j), or 0
            // when self-collision is off
            uint32_t sm = 0;
            if (t.selfcol) sm = r.self_mask ? r.self_mask[j] : (j >= 2 ? (1u << (j - 1)) - 1u : 0u);
            if (sm >> j)
                return set_error(MRPOP_EINVAL, "robot %d: self_mask[%d] has bits at or above %d", k,
                                 j, j);
            A[7] = f_of_i((int)sm);
            coarse_sphere(r.sphere_xyzr + 4 * first, cnt, A + 8);
        }
        std::memcpy(f4(t.off_sph + s_glob), r.sphere_xyzr, 4 * sizeof(float) * r.n_spheres);
        s_glob += r.n_spheres;
    }
    // workspace corner below every reachable coarse centre: |origin_j - base|
    // <= sum_i |(a_i, 0, d_i)| along the chain, |coarse centre - origin_j| <=
    // the largest coarse-centre offset of the robot
    {
        double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL};
        for (int k = 0; k < K; ++k) {
            const mrpop_robot &r = robots[k];
            double reach = 1.0, off = 0.0;
            for (int j = 0; j < r.dof; ++j) {
                const double a = r.dh[4 * j], d = r.dh[4 * j + 2];
                reach += std::sqrt(a * a + d * d);
                const float *A = f4(t.off_link + kLinkF4 * (t.link0[k] + j)) + 8;
                off = std::max(off, std::sqrt((double)A[0] * A[0] + (double)A[1] * A[1] +
                                              (double)A[2] * A[2]));
            }
            for (int a = 0; a < 3; ++a)
                lo[a] = std::min(lo[a], (double)r.base[4 * a + 3] - reach - off);
        }
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(lo[a]))
                return set_error(MRPOP_EINVAL, "robot chain or base is not finite");
            t.ws_lo[a] = std::nextafter((float)lo[a], -HUGE_VALF);
        }
    }
    if (t.NS > 0) std::memcpy(f4(t.off_os), obs->spheres, 4 * sizeof(float) * t.NS);
    for (int o = 0; o < t.NC; ++o) {
        const float *c = obs->cuboids + 15 * o;
        float *B = f4(t.off_oc + kCuboidF4 * o);
        const double hb = std::sqrt((double)c[3] * c[3] + (double)c[4] * c[4] + (double)c[5] * c[5]);
        B[0] = c[0]; B[1] = c[1]; B[2] = c[2]; B[3] = (float)(hb + 1e-4);
        B[4] = c[3]; B[5] = c[4]; B[6] = c[5]; B[7] = 0.f;
        for (int a = 0; a < 3; ++a) {  // axis a = column a of the row-major R
            B[8 + 4 * a + 0] = c[6 + 0 * 3 + a];
            B[8 + 4 * a + 1] = c[6 + 1 * 3 + a];
            B[8 + 4 * a + 2] = c[6 + 2 * 3 + a];
            B[8 + 4 * a + 3] = 0.f;
        }
    }

    mrpop_problem *p = new (std::nothrow) mrpop_problem();
    if (!p) return set_error(MRPOP_ENOMEM, "host allocation failed");
    p->dev.t = t;
    p->cfg = *cfg;
    p->D = L;
    p->h_blob.swap(blob);
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < robots[k].dof; ++j) {
            p->q_lo.push_back(robots[k].q_lo[j]);
            p->q_hi.push_back(robots[k].q_hi[j]);
        }
    if (start) p->start.assign(start, start + L);
    if (goal) p->goal.assign(goal, goal + L);
    for (int k = 0; k < K; ++k) {
        const mrpop_robot &r = robots[k];
        HostRobot hr;
        hr.dof = r.dof;
        hr.dh.assign(r.dh, r.dh + 4 * r.dof);
        hr.q_lo.assign(r.q_lo, r.q_lo + r.dof);
        hr.q_hi.assign(r.q_hi, r.q_hi + r.dof);
        if (r.n_spheres > 0) {
            hr.sphere_xyzr.assign(r.sphere_xyzr, r.sphere_xyzr + 4 * r.n_spheres);
            hr.sphere_link.assign(r.sphere_link, r.sphere_link + r.n_spheres);
        }
        std::memcpy(hr.base, r.base, sizeof(hr.base));
        p->robots.push_back(std::move(hr));
    }
    if (obs->n_spheres > 0) p->obs_spheres.assign(obs->spheres, obs->spheres + 4 * obs->n_spheres);
    if (obs->n_cuboids > 0)
        p->obs_cuboids.assign(obs->cuboids, obs->cuboids + 15 * obs->n_cuboids);

    auto fail = [&](mrpop_status st) {
        mrpop_destroy_problem(p);
        return st;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaGetDevice"));
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, p->device);
    p->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    p->smem_optin = (size_t)v;
    if ((e = cudaMalloc(&p->dev.blob, p->h_blob.size() * sizeof(float))) != cudaSuccess)
        return fail(cuda_error(e, "cudaMalloc(tables)"));
    if ((e = cudaMemcpy(p->dev.blob, p->h_blob.data(), p->h_blob.size() * sizeof(float),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(cuda_error(e, "cudaMemcpy(tables)"));
    if ((e = cudaMalloc(&p->dev.q_lo, sizeof(float) * L)) != cudaSuccess ||
        (e = cudaMalloc(&p->dev.q_hi, sizeof(float) * L)) != cudaSuccess)
        return fail(cuda_error(e, "cudaMalloc(limits)"));
    cudaMemcpy(p->dev.q_lo, p->q_lo.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
    if ((e = cudaMemcpy(p->dev.q_hi, p->q_hi.data(), sizeof(float) * L,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(cuda_error(e, "cudaMemcpy(limits)"));
    if ((e = cudaMalloc(&p->dev.edge_counter, sizeof(int) * 4)) != cudaSuccess)
        return fail(cuda_error(e, "cudaMalloc(counter)"));
    if ((e = cudaMemset(p->dev.edge_counter, 0, sizeof(int) * 4)) != cudaSuccess)
        return fail(cuda_error(e, "cudaMemset(counter)"));
    // a launch tuned earlier for a problem of this shape (mrpop_autotune)
    std::vector<int> tuned;
    if (tune_lookup(validate_tune_key(p), &tuned) && tuned.size() >= 4) {
        p->tuned_warps = tuned[0];
        p->tuned_order = tuned[1];
        p->tuned_fine = tuned[2];
        p->tuned_regs = tuned[3];
    }
    *out = p;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_destroy_problem(mrpop_problem *p) {
    if (!p) return MRPOP_OK;
    if (p->dev.blob || p->dev.edge_counter) cudaDeviceSynchronize();
    destroy_planner(p->planner);
    p->planner = nullptr;
    cudaFree(p->dev.blob);
    cudaFree(p->dev.q_lo);
    cudaFree(p->dev.q_hi);
    cudaFree(p->dev.edge_counter);
    delete p;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_problem_dims(const mrpop_problem *p, int32_t *D, int32_t *K,
                                           int32_t *S) {
    if (!p) return set_error(MRPOP_EINVAL, "problem is NULL");
    if (D) *D = p->D;
    if (K) *K = p->dev.t.K;
    if (S) *S = p->dev.t.S;
    return MRPOP_OK;
}

static mrpop_status check_edges(mrpop_problem *p, const float *qa, const float *qb,
                                int64_t n, const void *out, const char *fn) {
    if (!p) return set_error(MRPOP_EINVAL, "%s: problem is NULL", fn);
    if (n < 0) return set_error(MRPOP_EINVAL, "%s: n_edges < 0", fn);
    if (n > (int64_t)INT32_MAX)
        return set_error(MRPOP_EINVAL, "%s: n_edges exceeds %d", fn, INT32_MAX);
    if (n > 0 && (!qa || !qb || !out))
        return set_error(MRPOP_EINVAL, "%s: NULL buffer", fn);
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_fk(mrpop_problem *p, const float *q, int64_t n, float *out,
                                 void *stream) {
    mrpop_status st = check_edges(p, q, q, n, out, "mrpop_fk");
    if (st != MRPOP_OK || n == 0) return st;
    return launch_fk(p, q, n, out, (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_validate_edges_ex(mrpop_problem *p, const float *qa,
                                                const float *qb, int64_t n, uint8_t *valid,
                                                float *length, int32_t *npoints,
                                                void *stream) {
    mrpop_status st = check_edges(p, qa, qb, n, valid, "mrpop_validate_edges");
    if (st != MRPOP_OK || n == 0) return st;
    return launch_validate(p, qa, qb, n, valid, length, npoints, nullptr, nullptr,
                           (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_validate_edges(mrpop_problem *p, const float *qa,
                                             const float *qb, int64_t n, uint8_t *valid,
                                             void *stream) {
    return mrpop_validate_edges_ex(p, qa, qb, n, valid, nullptr, nullptr, stream);
}

extern "C" mrpop_status mrpop_edge_clearance(mrpop_problem *p, const float *qa,
                                             const float *qb, int64_t n, float *min_clear,
                                             void *stream) {
    mrpop_status st = check_edges(p, qa, qb, n, min_clear, "mrpop_edge_clearance");
    if (st != MRPOP_OK || n == 0) return st;
    return launch_validate(p, qa, qb, n, nullptr, nullptr, nullptr, min_clear, nullptr,
                           (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_validate_work(mrpop_problem *p, const float *qa, const float *qb,
                                            int64_t n, int64_t *counters, void *stream) {
    mrpop_status st = check_edges(p, qa, qb, n, counters, "mrpop_validate_work");
    if (st != MRPOP_OK) return st;
    if (!counters) return set_error(MRPOP_EINVAL, "mrpop_validate_work: counters is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    MRPOP_CUDA_TRY(cudaMemsetAsync(counters, 0, MRPOP_WORK_COUNTERS * sizeof(int64_t), s));
    if (n == 0) return MRPOP_OK;
    return launch_validate(p, qa, qb, n, nullptr, nullptr, nullptr, nullptr,
                           (unsigned long long *)counters, s);
}

extern "C" mrpop_status mrpop_nearest_ex(const float *tree, int64_t N, int64_t ld, int32_t dim,
                                         const float *queries, const float *budgets, int64_t Q,
                                         int32_t filter, int64_t *out_idx, void *stream) {
    if (dim < 1 || dim > MRPOP_MAX_LINKS)
        return set_error(MRPOP_EINVAL, "mrpop_nearest: dim=%d outside [1, %d]", dim,
                         MRPOP_MAX_LINKS);
    if (N < 0 || Q < 0 || ld < N || N > (int64_t)INT32_MAX || Q > (int64_t)INT32_MAX)
        return set_error(MRPOP_EINVAL, "mrpop_nearest: bad sizes N=%lld ld=%lld Q=%lld",
                         (long long)N, (long long)ld, (long long)Q);
    if (filter != MRPOP_NEAREST_FILTER_FP32 && filter != MRPOP_NEAREST_FILTER_TENSOR)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_ex: filter=%d is not a filter", filter);
    if (Q == 0) return MRPOP_OK;
    if (!queries || !budgets || !out_idx || (N > 0 && !tree))
        return set_error(MRPOP_EINVAL, "mrpop_nearest: NULL buffer");
    return launch_nearest(tree, N, ld, dim, queries, budgets, Q, out_idx, (cudaStream_t)stream,
                          filter);
}

extern "C" mrpop_status mrpop_nearest(const float *tree, int64_t N, int64_t ld, int32_t dim,
                                      const float *queries, const float *budgets, int64_t Q,
                                      int64_t *out_idx, void *stream) {
    return mrpop_nearest_ex(tree, N, ld, dim, queries, budgets, Q, MRPOP_NEAREST_FILTER_FP32,
                            out_idx, stream);
}

extern "C" mrpop_status mrpop_nearest_work(const float *tree, int64_t N, int64_t ld, int32_t dim,
                                           const float *queries, const float *budgets, int64_t Q,
                                           int64_t *pairs, void *stream) {
    if (!pairs) return set_error(MRPOP_EINVAL, "mrpop_nearest_work: pairs is NULL");
    *pairs = 0;
    if (dim < 1 || dim > MRPOP_MAX_LINKS)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_work: dim=%d outside [1, %d]", dim,
                         MRPOP_MAX_LINKS);
    if (N < 0 || Q < 0 || ld < N || N > (int64_t)INT32_MAX || Q > (int64_t)INT32_MAX)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_work: bad sizes");
    if (Q == 0 || N == 0) return MRPOP_OK;
    if (!queries || !budgets || !tree) return set_error(MRPOP_EINVAL, "mrpop_nearest_work: NULL buffer");
    return nearest_pairs(tree, N, ld, dim, queries, budgets, Q, pairs, (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_neighbors(const float *tree, int64_t N, int64_t ld, int32_t dim,
                                        const float *queries, int64_t Q, float delta,
                                        int64_t k_max, int64_t *out_idx, int64_t *out_cnt,
                                        void *stream) {
    if (dim < 1 || dim > MRPOP_MAX_LINKS)
        return set_error(MRPOP_EINVAL, "mrpop_neighbors: dim=%d outside [1, %d]", dim,
                         MRPOP_MAX_LINKS);
    if (N < 0 || Q < 0 || ld < N || k_max < 0 || N > (int64_t)INT32_MAX ||
        Q > (int64_t)INT32_MAX)
        return set_error(MRPOP_EINVAL, "mrpop_neighbors: bad sizes");
    if (!std::isfinite(delta)) return set_error(MRPOP_EINVAL, "mrpop_neighbors: delta not finite");
    if (Q == 0) return MRPOP_OK;
    if (!queries || !out_cnt || (k_max > 0 && !out_idx) || (N > 0 && !tree))
        return set_error(MRPOP_EINVAL, "mrpop_neighbors: NULL buffer");
    return launch_neighbors(tree, N, ld, dim, queries, Q, delta, k_max, out_idx, out_cnt,
                            (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_nearest_autotune(const float *tree, int64_t N, int64_t ld,
                                               int32_t dim, const float *queries,
                                               const float *budgets, int64_t Q, int32_t filter,
                                               int64_t *out_idx, int32_t *waves,
                                               float *ms_per_call, void *stream) {
    if (dim < 1 || dim > MRPOP_MAX_LINKS || N < 0 || Q < 1 || ld < N || N > (int64_t)INT32_MAX ||
        Q > (int64_t)INT32_MAX)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_autotune: bad sizes");
    if (filter != MRPOP_NEAREST_FILTER_FP32 && filter != MRPOP_NEAREST_FILTER_TENSOR)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_autotune: filter=%d is not a filter", filter);
    if (!queries || !budgets || !out_idx || (N > 0 && !tree))
        return set_error(MRPOP_EINVAL, "mrpop_nearest_autotune: NULL buffer");
    return autotune_nearest(tree, N, ld, dim, queries, budgets, Q, filter, out_idx, waves,
                            ms_per_call, (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_neighbors_autotune(const float *tree, int64_t N, int64_t ld,
                                                 int32_t dim, const float *queries, int64_t Q,
                                                 float delta, int64_t k_max, int64_t *out_idx,
                                                 int64_t *out_cnt, int32_t *warps_per_sm,
                                                 float *ms_per_call, void *stream) {
    if (dim < 1 || dim > MRPOP_MAX_LINKS || N < 0 || Q < 1 || ld < N || k_max < 0 ||
        N > (int64_t)INT32_MAX || Q > (int64_t)INT32_MAX || !std::isfinite(delta))
        return set_error(MRPOP_EINVAL, "mrpop_neighbors_autotune: bad arguments");
    if (!queries || !out_cnt || (k_max > 0 && !out_idx) || (N > 0 && !tree))
        return set_error(MRPOP_EINVAL, "mrpop_neighbors_autotune: NULL buffer");
    return autotune_neighbors(tree, N, ld, dim, queries, Q, delta, k_max, out_idx, out_cnt,
                              warps_per_sm, ms_per_call, (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_path_cost(const float *path, int64_t M, int32_t dim,
                                        double *cost_out, void *stream) {
    if (dim < 1 || M < 0) return set_error(MRPOP_EINVAL, "mrpop_path_cost: bad sizes");
    if (!cost_out || (M > 0 && !path)) return set_error(MRPOP_EINVAL, "mrpop_path_cost: NULL buffer");
    return launch_path_cost(path, M, dim, cost_out, (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_autotune(mrpop_problem *p, const float *qa, const float *qb,
                                      int64_t n_edges, uint8_t *valid, int32_t *config,
                                      float *ms_per_launch, void *stream) {
    mrpop_status st = check_edges(p, qa, qb, n_edges, valid, "mrpop_autotune");
    if (st != MRPOP_OK) return st;
    if (n_edges == 0) return set_error(MRPOP_EINVAL, "mrpop_autotune: no edges to time");
    return autotune_validate(p, qa, qb, n_edges, valid, 3, config, ms_per_launch,
                             (cudaStream_t)stream);
}

extern "C" mrpop_status mrpop_set_launch(mrpop_problem *p, int32_t warps_per_block,
                                        int32_t order, int32_t fine_stage) {
    if (!p) return set_error(MRPOP_EINVAL, "mrpop_set_launch: problem is NULL");
    if (warps_per_block != 0 && warps_per_block != 1 && warps_per_block != 2 &&
        warps_per_block != 4)
        return set_error(MRPOP_EINVAL, "mrpop_set_launch: warps_per_block must be 0, 1, 2 or 4");
    if (order != 0 && order != 1) return set_error(MRPOP_EINVAL, "mrpop_set_launch: order must be 0 or 1");
    if (fine_stage != 0 && fine_stage != 1)
        return set_error(MRPOP_EINVAL, "mrpop_set_launch: fine_stage must be 0 or 1");
    p->tuned_warps = warps_per_block;
    p->tuned_order = order;
    p->tuned_fine = fine_stage;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_set_launch_ex(mrpop_problem *p, int32_t warps_per_block,
                                           int32_t order, int32_t fine_stage,
                                           int32_t registers) {
    if (registers != 0 && registers != 1)
        return set_error(MRPOP_EINVAL, "mrpop_set_launch_ex: registers must be 0 or 1");
    const mrpop_status s = mrpop_set_launch(p, warps_per_block, order, fine_stage);
    if (s != MRPOP_OK) return s;
    p->tuned_regs = registers;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_get_launch(const mrpop_problem *p, int32_t *config) {
    if (!p || !config) return set_error(MRPOP_EINVAL, "mrpop_get_launch: NULL argument");
    config[0] = p->tuned_warps;
    config[1] = p->tuned_order;
    config[2] = p->tuned_fine;
    config[3] = p->tuned_regs;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_autotune_cache_save(const char *path) {
    if (!path) return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_save: path is NULL");
    std::ofstream f(path);
    if (!f) return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_save: cannot write %s", path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    f << "# mrpop tuned launches: <key> = <values>\n";
    for (const auto &kv : g_tune) {
        f << kv.first << " =";
        for (int v : kv.second) f << ' ' << v;
        f << '\n';
    }
    return f ? MRPOP_OK : set_error(MRPOP_EINVAL, "mrpop_autotune_cache_save: write failed");
}

extern "C" mrpop_status mrpop_autotune_cache_load(const char *path) {
    if (!path) return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_load: path is NULL");
    std::ifstream f(path);
    if (!f) return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_load: cannot read %s", path);
    std::string line;
    std::map<std::string, std::vector<int>> add;
    int no = 0;
    while (std::getline(f, line)) {
        ++no;
        if (line.empty() || line[0] == '#') continue;
        const size_t eq = line.rfind(" = ");
        if (eq == std::string::npos || eq == 0)
            return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_load: %s:%d: no ' = '", path, no);
        std::istringstream vs(line.substr(eq + 3));
        std::vector<int> v;
        long long x;
        while (vs >> x) {
            if (x < -(1ll << 30) || x > (1ll << 30))
                return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_load: %s:%d: value out of range",
                                 path, no);
            v.push_back((int)x);
        }
        if (!vs.eof() || v.empty())
            return set_error(MRPOP_EINVAL, "mrpop_autotune_cache_load: %s:%d: bad values", path, no);
        add[line.substr(0, eq)] = v;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto &kv : add) g_tune[kv.first] = kv.second;
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_scratch_stats(int32_t reset_high, int64_t *stats) {
    if (!stats) return set_error(MRPOP_EINVAL, "mrpop_scratch_stats: stats is NULL");
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(&pool);
    if (e != cudaSuccess) return cuda_error(e, "mrpop_scratch_stats");
    unsigned long long v[3] = {0, 0, 0};
    if ((e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v[0])) != cudaSuccess ||
        (e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v[1])) != cudaSuccess ||
        (e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v[2])) != cudaSuccess)
        return cuda_error(e, "mrpop_scratch_stats");
    for (int i = 0; i < 3; ++i) stats[i] = (int64_t)v[i];
    if (reset_high) {
        unsigned long long zero = 0;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero)) != cudaSuccess)
            return cuda_error(e, "mrpop_scratch_stats");
    }
    return MRPOP_OK;
}

extern "C" mrpop_status mrpop_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
    return MRPOP_OK;
}
