/*
 * mrpop_oracle.c -- plain, slow FP64 CPU oracle (test infrastructure only).
 *
 * Written from the definitions in the paper:
 *   Sec. III-A   composite configuration q = (q^1..q^K); composite free space
 *                excludes robot-obstacle and robot-robot collisions; path cost
 *                C(sigma) = sum_j ||q_{j+1} - q_j||.
 *   Sec. III-E   robots are approximated by collision spheres; an edge is
 *                discretised into motions and every checkpoint is checked.
 *   Alg. 2       NEAREST(V, q, c) = argmin over {g_v + ||q - q_v|| < c} of
 *                ||q - q_v||; NEIGHBORS(V, c, delta) = vertices within delta.
 *   Sec. III-D   ties between vertices at one configuration go to lowest cost.
 *
 * No culling, blocking, early reordering or fusion: every sphere is tested
 * against every obstacle and every sphere of every other robot, with explicit
 * 4x4 homogeneous transforms.  Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg may load this library.
 */
#include "mrpop_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* 4x4 homogeneous transforms, row-major                                      */
/* ------------------------------------------------------------------------- */

static void m4_identity(double M[16]) {
    memset(M, 0, 16 * sizeof(double));
    M[0] = M[5] = M[10] = M[15] = 1.0;
}

static void m4_mul(const double A[16], const double B[16], double C[16]) {
    double T[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) acc += A[4 * i + k] * B[4 * k + j];
            T[4 * i + j] = acc;
        }
    memcpy(C, T, sizeof(T));
}

static void m4_rotz(double th, double M[16]) {
    m4_identity(M);
    M[0] = cos(th); M[1] = -sin(th);
    M[4] = sin(th); M[5] = cos(th);
}

static void m4_rotx(double al, double M[16]) {
    m4_identity(M);
    M[5] = cos(al); M[6] = -sin(al);
    M[9] = sin(al); M[10] = cos(al);
}

static void m4_trans(double x, double y, double z, double M[16]) {
    m4_identity(M);
    M[3] = x; M[7] = y; M[11] = z;
}

static void m4_apply(const double M[16], const double p[3], double out[3]) {
    for (int i = 0; i < 3; ++i)
        out[i] = M[4 * i + 0] * p[0] + M[4 * i + 1] * p[1] + M[4 * i + 2] * p[2] + M[4 * i + 3];
}

/* offsets of robot k's rows in the concatenated tables */
static int32_t joint_offset(const orc_scene *s, int32_t k) {
    int32_t o = 0;
    for (int32_t i = 0; i < k; ++i) o += s->dof[i];
    return o;
}

static int32_t sphere_offset(const orc_scene *s, int32_t k) {
    int32_t o = 0;
    for (int32_t i = 0; i < k; ++i) o += s->n_spheres[i];
    return o;
}

static int32_t total_dof(const orc_scene *s) { return joint_offset(s, s->K); }

/* ------------------------------------------------------------------------- */
/* Forward kinematics (serial chain, standard DH)                             */
/* ------------------------------------------------------------------------- */

void orc_link_frames(const orc_scene *s, int32_t k, const double *q, double *frames) {
    const int32_t j0 = joint_offset(s, k);
    const float *b = s->base + 12 * k;
    double T[16];
    m4_identity(T);
    for (int i = 0; i < 12; ++i) T[i] = b[i];
    for (int32_t j = 0; j < s->dof[k]; ++j) {
        const float *row = s->dh + 4 * (j0 + j); /* a, alpha, d, theta_offset */
        double R[16], Tz[16], Tx[16], Rx[16];
        m4_rotz(q[j] + (double)row[3], R);
        m4_mul(T, R, T);                       /* F_j' = F_{j-1} Rz(theta)   */
        memcpy(frames + 16 * j, T, sizeof(T));
        m4_trans(0.0, 0.0, row[2], Tz);
        m4_trans(row[0], 0.0, 0.0, Tx);
        m4_rotx(row[1], Rx);
        m4_mul(T, Tz, T);
        m4_mul(T, Tx, T);
        m4_mul(T, Rx, T);                      /* next frame                 */
    }
}

void orc_fk_robot(const orc_scene *s, int32_t k, const double *q, double *out) {
    const int32_t dof = s->dof[k];
    const int32_t s0 = sphere_offset(s, k);
    double *frames = (double *)malloc(sizeof(double) * 16 * (size_t)(dof > 0 ? dof : 1));
    orc_link_frames(s, k, q, frames);
    for (int32_t i = 0; i < s->n_spheres[k]; ++i) {
        const int32_t link = s->sphere_link[s0 + i];
        const float *sp = s->sphere_xyzr + 4 * (s0 + i);
        const double p[3] = {sp[0], sp[1], sp[2]};
        m4_apply(frames + 16 * link, p, out + 4 * i);
        out[4 * i + 3] = sp[3];
    }
    free(frames);
}

/* ------------------------------------------------------------------------- */
/* Distances                                                                  */
/* ------------------------------------------------------------------------- */

double orc_sphere_sphere_clearance(const double *c1, double r1, const double *c2, double r2) {
    const double dx = c1[0] - c2[0], dy = c1[1] - c2[1], dz = c1[2] - c2[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - r1 - r2;
}

/* Oriented box: p = R^T (c - centre) in box coordinates; the closest box
 * point is clamp(p, -h, h); clearance = |p - clamp(p)| - r. */
double orc_sphere_cuboid_clearance(const double *c, double r, const float *cub) {
    const double v[3] = {c[0] - cub[0], c[1] - cub[1], c[2] - cub[2]};
    double acc = 0.0;
    for (int a = 0; a < 3; ++a) {
        /* column a of R is box axis a */
        const double p = cub[6 + 0 * 3 + a] * v[0] + cub[6 + 1 * 3 + a] * v[1] +
                         cub[6 + 2 * 3 + a] * v[2];
        const double h = cub[3 + a];
        const double cl = p < -h ? -h : (p > h ? h : p);
        acc += (p - cl) * (p - cl);
    }
    return sqrt(acc) - r;
}

/* ------------------------------------------------------------------------- */
/* Configuration validity (composite free space, Sec. III-A)                  */
/* ------------------------------------------------------------------------- */

int32_t orc_config_valid(const orc_scene *s, const double *q, double margin, double *min_clear) {
    int32_t total_s = sphere_offset(s, s->K);
    double *w = (double *)malloc(sizeof(double) * 4 * (size_t)(total_s > 0 ? total_s : 1));
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total_s > 0 ? total_s : 1));
    for (int32_t k = 0; k < s->K; ++k) {
        const int32_t s0 = sphere_offset(s, k);
        orc_fk_robot(s, k, q + joint_offset(s, k), w + 4 * s0);
        for (int32_t i = 0; i < s->n_spheres[k]; ++i) owner[s0 + i] = k;
    }
    const int32_t *link = s->sphere_link;  /* link of each sphere within its robot */
    double mc = DBL_MAX;
    int32_t valid = 1;
    for (int32_t i = 0; i < total_s; ++i) {
        const double *ci = w + 4 * i;
        for (int32_t o = 0; o < s->n_obs_spheres; ++o) {
            const float *ob = s->obs_spheres + 4 * o;
            const double oc[3] = {ob[0], ob[1], ob[2]};
            const double cl = orc_sphere_sphere_clearance(ci, ci[3], oc, ob[3]);
            if (cl < mc) mc = cl;
            if (cl < margin) valid = 0;
        }
        for (int32_t o = 0; o < s->n_obs_cuboids; ++o) {
            const double cl = orc_sphere_cuboid_clearance(ci, ci[3], s->obs_cuboids + 15 * o);
            if (cl < mc) mc = cl;
            if (cl < margin) valid = 0;
        }
        /* robot-robot: spheres of two different robots; with self-collision
         * also spheres of one robot on a link pair of its adjacency mask */
        for (int32_t j = i + 1; j < total_s; ++j) {
            if (owner[j] == owner[i]) {
                if (!s->self_collision) continue;
                const int32_t hi = link[j] > link[i] ? link[j] : link[i];
                const int32_t lo = link[j] > link[i] ? link[i] : link[j];
                const int32_t paired = s->self_mask
                    ? (s->self_mask[joint_offset(s, owner[i]) + hi] >> lo) & 1
                    : hi - lo >= 2;
                if (hi == lo || !paired) continue;
            }
            const double *cj = w + 4 * j;
            const double cl = orc_sphere_sphere_clearance(ci, ci[3], cj, cj[3]);
            if (cl < mc) mc = cl;
            if (cl < margin) valid = 0;
        }
    }
    free(w);
    free(owner);
    if (min_clear) *min_clear = mc;
    return valid;
}

/* ------------------------------------------------------------------------- */
/* Edges (Sec. III-E: discretise, check every checkpoint)                     */
/* ------------------------------------------------------------------------- */

int32_t orc_edge_npoints(const float *qa, const float *qb, int64_t stride, int32_t D, float res) {
    /* FP32 on purpose: the interval count is an integer decided in the
     * kernel's precision.  Order: sequential fused multiply-add over i. */
    float acc = 0.0f;
    for (int32_t i = 0; i < D; ++i) {
        const float d = qb[i * stride] - qa[i * stride];
        acc = fmaf(d, d, acc);
    }
    const float len = sqrtf(acc);
    const float nf = ceilf(len / res);
    int32_t n = (nf >= 1.0f) ? (int32_t)nf : 1;
    return n;
}

int32_t orc_edge_valid(const orc_scene *s, const float *qa, const float *qb, int64_t stride,
                       float res, double margin, int32_t early_exit,
                       double *min_clear, int32_t *first_hit, int32_t *npoints) {
    const int32_t D = total_dof(s);
    const int32_t n = orc_edge_npoints(qa, qb, stride, D, res);
    double *q = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
    double mc = DBL_MAX;
    int32_t hit = -1;
    for (int32_t k = 0; k <= n; ++k) {
        const double t = (double)k / (double)n;
        for (int32_t i = 0; i < D; ++i) {
            const double a = qa[i * stride], b = qb[i * stride];
            q[i] = a + t * (b - a);
        }
        double c;
        const int32_t ok = orc_config_valid(s, q, margin, &c);
        if (c < mc) mc = c;
        if (!ok && hit < 0) {
            hit = k;
            if (early_exit) break;
        }
    }
    free(q);
    if (min_clear) *min_clear = mc;
    if (first_hit) *first_hit = hit;
    if (npoints) *npoints = n;
    return hit < 0;
}

void orc_validate_edges(const orc_scene *s, const float *qa, const float *qb, int64_t ld,
                        int64_t e0, int64_t n, float res, double margin, int32_t early_exit,
                        uint8_t *valid, double *min_clear, int32_t *first_hit,
                        int32_t *npoints) {
    for (int64_t e = 0; e < n; ++e) {
        double mc;
        int32_t fh, np;
        const int32_t ok = orc_edge_valid(s, qa + e0 + e, qb + e0 + e, ld, res, margin,
                                          early_exit, &mc, &fh, &np);
        if (valid) valid[e] = (uint8_t)ok;
        if (min_clear) min_clear[e] = mc;
        if (first_hit) first_hit[e] = fh;
        if (npoints) npoints[e] = np;
    }
}

/* ------------------------------------------------------------------------- */
/* Nearest / neighbours over a state-cost tree (Alg. 2)                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double d, g;
    int64_t idx;
} orc_cand;

static int cand_cmp(const void *pa, const void *pb) {
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static double vertex_distance(const float *tree, int64_t v, int64_t ld, int32_t D,
                              const float *q) {
    double acc = 0.0;
    for (int32_t i = 0; i < D; ++i) {
        const double diff = (double)q[i] - (double)tree[i * ld + v];
        acc += diff * diff;
    }
    return sqrt(acc);
}

int64_t orc_nearest(const float *tree, int64_t N, int64_t ld, int32_t D, const float *q,
                    float c, double *best_d, double *second_d, double *filter_gap) {
    orc_cand *A = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(N > 0 ? N : 1));
    int64_t na = 0;
    double gap = DBL_MAX;
    for (int64_t v = 0; v < N; ++v) {
        const double d = vertex_distance(tree, v, ld, D, q);
        const double g = tree[(int64_t)D * ld + v];
        const double slack = fabs(g + d - (double)c);
        if (slack < gap) gap = slack;
        if (g + d < (double)c) {
            A[na].d = d;
            A[na].g = g;
            A[na].idx = v;
            ++na;
        }
    }
    qsort(A, (size_t)na, sizeof(orc_cand), cand_cmp);
    const int64_t out = na > 0 ? A[0].idx : -1;
    if (best_d) *best_d = na > 0 ? A[0].d : INFINITY;
    if (second_d) *second_d = na > 1 ? A[1].d : INFINITY;
    if (filter_gap) *filter_gap = gap;
    free(A);
    return out;
}

int64_t orc_neighbors(const float *tree, int64_t N, int64_t ld, int32_t D, const float *q,
                      float delta, int64_t k_max, int64_t *out, double *gap) {
    int64_t cnt = 0;
    double gp = DBL_MAX;
    for (int64_t v = 0; v < N; ++v) {
        const double d = vertex_distance(tree, v, ld, D, q);
        const double sl = fabs(d - (double)delta);
        if (sl < gp) gp = sl;
        if (d <= (double)delta) {
            if (cnt < k_max && out) out[cnt] = v;
            ++cnt;
        }
    }
    if (gap) *gap = gp;
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Paths (Sec. III-A)                                                         */
/* ------------------------------------------------------------------------- */

double orc_path_cost(const float *path, int64_t M, int32_t D) {
    double c = 0.0;
    for (int64_t j = 0; j + 1 < M; ++j) {
        double acc = 0.0;
        for (int32_t i = 0; i < D; ++i) {
            const double diff = (double)path[(j + 1) * D + i] - (double)path[j * D + i];
            acc += diff * diff;
        }
        c += sqrt(acc);
    }
    return c;
}

int32_t orc_path_valid(const orc_scene *s, const float *path, int64_t M, float res,
                       double margin, int64_t *bad_segment) {
    const int32_t D = total_dof(s);
    for (int64_t j = 0; j + 1 < M; ++j) {
        if (!orc_edge_valid(s, path + j * D, path + (j + 1) * D, 1, res, margin, 1,
                            NULL, NULL, NULL)) {
            if (bad_segment) *bad_segment = j;
            return 0;
        }
    }
    if (M == 1 && !orc_edge_valid(s, path, path, 1, res, margin, 1, NULL, NULL, NULL)) {
        if (bad_segment) *bad_segment = 0;
        return 0;
    }
    if (bad_segment) *bad_segment = -1;
    return 1;
}
