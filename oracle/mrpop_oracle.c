/*
 * mrpop_oracle.c -- plain, slow FP64 CPU oracle (test infrastructure only).
 *
 * Written from the definitions in the paper:
 *   Sec. III-A   composite configuration q = (q^1..q^K); composite free space
 *                excludes robot-obstacle and robot-robot collisions; path cost
 *                C(sigma) = sum_j ||q_{j+1} - q_j||.
 *   Sec. III-E   robots are approximated by collision spheres; an edge is
 *                discretised into motions and every checkpoint is checked;
 *                the two-stage check (one conservative sphere per link, then
 *                the fine spheres of the links it hit) only for counting its
 *                work (orc_edge_method_work).
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

/* ------------------------------------------------------------------------- */
/* Work of the two-stage check (Sec. III-E)                                   */
/* ------------------------------------------------------------------------- */

/* Coarse sphere of every link of every robot, in its link frame: centre and
 * radius [4] per link (radius < 0: the link has no sphere). */
static void coarse_spheres(const orc_scene *s, double *coarse) {
    for (int32_t k = 0; k < s->K; ++k) {
        const int32_t j0 = joint_offset(s, k), s0 = sphere_offset(s, k);
        for (int32_t j = 0; j < s->dof[k]; ++j) {
            double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
            int32_t any = 0;
            for (int32_t i = 0; i < s->n_spheres[k]; ++i) {
                if (s->sphere_link[s0 + i] != j) continue;
                const float *sp = s->sphere_xyzr + 4 * (s0 + i);
                for (int a = 0; a < 3; ++a) {
                    if (sp[a] < lo[a]) lo[a] = sp[a];
                    if (sp[a] > hi[a]) hi[a] = sp[a];
                }
                any = 1;
            }
            double *c = coarse + 4 * (j0 + j);
            if (!any) {
                c[0] = c[1] = c[2] = 0.0;
                c[3] = -1.0;
                continue;
            }
            for (int a = 0; a < 3; ++a) c[a] = 0.5 * (lo[a] + hi[a]);
            double r = 0.0;
            for (int32_t i = 0; i < s->n_spheres[k]; ++i) {
                if (s->sphere_link[s0 + i] != j) continue;
                const float *sp = s->sphere_xyzr + 4 * (s0 + i);
                const double dx = sp[0] - c[0], dy = sp[1] - c[1], dz = sp[2] - c[2];
                const double e = sqrt(dx * dx + dy * dy + dz * dz) + sp[3];
                if (e > r) r = e;
            }
            c[3] = r + 1e-4;
        }
    }
}

/* Do links (global joint rows) a < b belong to a pair that is tested? */
static int32_t link_pair_tested(const orc_scene *s, const int32_t *robot_of, const int32_t *link_of,
                                int32_t a, int32_t b) {
    if (robot_of[a] != robot_of[b]) return 1;
    if (!s->self_collision) return 0;
    const int32_t lo = link_of[a] < link_of[b] ? link_of[a] : link_of[b];
    const int32_t hi = link_of[a] < link_of[b] ? link_of[b] : link_of[a];
    if (hi == lo) return 0;
    return s->self_mask ? (s->self_mask[joint_offset(s, robot_of[a]) + hi] >> lo) & 1
                        : hi - lo >= 2;
}

/* Two-stage check of one configuration q; returns validity, adds units. */
static int32_t method_config(const orc_scene *s, const double *coarse, const int32_t *robot_of,
                             const int32_t *link_of, const double *q, double margin,
                             double *frames, double *cw, int32_t *hit_link, int64_t *counts) {
    const int32_t L = total_dof(s);
    const int32_t NS = s->n_obs_spheres, NC = s->n_obs_cuboids;
    counts[ORC_WORK_CHECKPOINTS] += 1;
    /* stage 1: FK and a coarse centre per link */
    for (int32_t k = 0; k < s->K; ++k) {
        const int32_t j0 = joint_offset(s, k);
        orc_link_frames(s, k, q + j0, frames + 16 * j0);
        counts[ORC_WORK_JOINTS] += s->dof[k];
    }
    for (int32_t l = 0; l < L; ++l) {
        hit_link[l] = 0;
        if (coarse[4 * l + 3] < 0.0) continue;
        m4_apply(frames + 16 * l, coarse + 4 * l, cw + 4 * l);
        cw[4 * l + 3] = coarse[4 * l + 3];
        counts[ORC_WORK_COARSE_POINTS] += 1;
    }
    /* coarse tests; the hits are kept for stage 2 */
    uint8_t *hs = (uint8_t *)calloc((size_t)L * (size_t)(NS > 0 ? NS : 1), 1);
    uint8_t *hc = (uint8_t *)calloc((size_t)L * (size_t)(NC > 0 ? NC : 1), 1);
    uint8_t *hp = (uint8_t *)calloc((size_t)L * (size_t)L, 1);
    for (int32_t l = 0; l < L; ++l) {
        if (coarse[4 * l + 3] < 0.0) continue;
        const double *c = cw + 4 * l;
        for (int32_t o = 0; o < NS; ++o) {
            const float *ob = s->obs_spheres + 4 * o;
            const double oc[3] = {ob[0], ob[1], ob[2]};
            counts[ORC_WORK_COARSE_SPHERE] += 1;
            if (orc_sphere_sphere_clearance(c, c[3], oc, ob[3]) < margin) {
                hs[(size_t)l * NS + o] = 1;
                hit_link[l] = 1;
            }
        }
        for (int32_t o = 0; o < NC; ++o) {
            counts[ORC_WORK_COARSE_CUBOID] += 1;
            if (orc_sphere_cuboid_clearance(c, c[3], s->obs_cuboids + 15 * o) < margin) {
                hc[(size_t)l * NC + o] = 1;
                hit_link[l] = 1;
            }
        }
        for (int32_t m = l + 1; m < L; ++m) {
            if (coarse[4 * m + 3] < 0.0 || !link_pair_tested(s, robot_of, link_of, l, m)) continue;
            counts[ORC_WORK_COARSE_PAIR] += 1;
            if (orc_sphere_sphere_clearance(c, c[3], cw + 4 * m, cw[4 * m + 3]) < margin) {
                hp[(size_t)l * L + m] = 1;
                hit_link[l] = hit_link[m] = 1;
            }
        }
    }
    /* stage 2: fine spheres of the links that a coarse test hit */
    int32_t valid = 1;
    int32_t total_s = sphere_offset(s, s->K);
    double *fw = (double *)malloc(sizeof(double) * 4 * (size_t)(total_s > 0 ? total_s : 1));
    int32_t *first = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L + 1));
    int32_t *cnt = (int32_t *)calloc((size_t)(L > 0 ? L : 1), sizeof(int32_t));
    for (int32_t k = 0; k < s->K; ++k) {
        const int32_t j0 = joint_offset(s, k), s0 = sphere_offset(s, k);
        for (int32_t j = 0; j < s->dof[k]; ++j) first[j0 + j] = -1;
        for (int32_t i = 0; i < s->n_spheres[k]; ++i) {
            const int32_t l = j0 + s->sphere_link[s0 + i];
            if (first[l] < 0) first[l] = s0 + i;
            cnt[l] += 1;
        }
    }
    for (int32_t l = 0; l < L; ++l) {
        if (!hit_link[l]) continue;
        for (int32_t i = first[l]; i < first[l] + cnt[l]; ++i) {
            const float *sp = s->sphere_xyzr + 4 * i;
            const double p[3] = {sp[0], sp[1], sp[2]};
            m4_apply(frames + 16 * l, p, fw + 4 * i);
            fw[4 * i + 3] = sp[3];
        }
        counts[ORC_WORK_FINE_POINTS] += cnt[l];
    }
    for (int32_t l = 0; l < L; ++l) {
        if (!hit_link[l]) continue;
        for (int32_t o = 0; o < NS; ++o) {
            if (!hs[(size_t)l * NS + o]) continue;
            const float *ob = s->obs_spheres + 4 * o;
            const double oc[3] = {ob[0], ob[1], ob[2]};
            for (int32_t i = first[l]; i < first[l] + cnt[l]; ++i) {
                counts[ORC_WORK_FINE_SPHERE] += 1;
                if (orc_sphere_sphere_clearance(fw + 4 * i, fw[4 * i + 3], oc, ob[3]) < margin)
                    valid = 0;
            }
        }
        for (int32_t o = 0; o < NC; ++o) {
            if (!hc[(size_t)l * NC + o]) continue;
            for (int32_t i = first[l]; i < first[l] + cnt[l]; ++i) {
                counts[ORC_WORK_FINE_CUBOID] += 1;
                if (orc_sphere_cuboid_clearance(fw + 4 * i, fw[4 * i + 3],
                                                s->obs_cuboids + 15 * o) < margin)
                    valid = 0;
            }
        }
        for (int32_t m = l + 1; m < L; ++m) {
            if (!hp[(size_t)l * L + m]) continue;
            for (int32_t i = first[l]; i < first[l] + cnt[l]; ++i)
                for (int32_t j = first[m]; j < first[m] + cnt[m]; ++j) {
                    counts[ORC_WORK_FINE_PAIR] += 1;
                    if (orc_sphere_sphere_clearance(fw + 4 * i, fw[4 * i + 3], fw + 4 * j,
                                                    fw[4 * j + 3]) < margin)
                        valid = 0;
                }
        }
    }
    free(fw);
    free(first);
    free(cnt);
    free(hs);
    free(hc);
    free(hp);
    return valid;
}

int32_t orc_edge_method_work(const orc_scene *s, const float *qa, const float *qb,
                             int64_t stride, float res, double margin, int32_t early_exit,
                             int64_t *counts) {
    const int32_t D = total_dof(s);
    const int32_t n = orc_edge_npoints(qa, qb, stride, D, res);
    const size_t LL = (size_t)(D > 0 ? D : 1);
    double *coarse = (double *)malloc(sizeof(double) * 4 * LL);
    double *frames = (double *)malloc(sizeof(double) * 16 * LL);
    double *cw = (double *)malloc(sizeof(double) * 4 * LL);
    double *q = (double *)malloc(sizeof(double) * LL);
    int32_t *robot_of = (int32_t *)malloc(sizeof(int32_t) * LL);
    int32_t *link_of = (int32_t *)malloc(sizeof(int32_t) * LL);
    int32_t *hit_link = (int32_t *)malloc(sizeof(int32_t) * LL);
    coarse_spheres(s, coarse);
    for (int32_t k = 0; k < s->K; ++k)
        for (int32_t j = 0; j < s->dof[k]; ++j) {
            robot_of[joint_offset(s, k) + j] = k;
            link_of[joint_offset(s, k) + j] = j;
        }
    int32_t valid = 1;
    for (int32_t k = 0; k <= n; ++k) {
        const double t = (double)k / (double)n;
        for (int32_t i = 0; i < D; ++i) {
            const double a = qa[i * stride], b = qb[i * stride];
            q[i] = a + t * (b - a);
        }
        if (!method_config(s, coarse, robot_of, link_of, q, margin, frames, cw, hit_link,
                           counts)) {
            valid = 0;
            if (early_exit) break;
        }
    }
    free(coarse);
    free(frames);
    free(cw);
    free(q);
    free(robot_of);
    free(link_of);
    free(hit_link);
    return valid;
}

void orc_method_work_edges(const orc_scene *s, const float *qa, const float *qb, int64_t ld,
                           int64_t e0, int64_t n, float res, double margin, int32_t early_exit,
                           int64_t *counts, uint8_t *valid) {
    for (int64_t e = 0; e < n; ++e) {
        const int32_t ok = orc_edge_method_work(s, qa + e0 + e, qb + e0 + e, ld, res, margin,
                                                early_exit, counts);
        if (valid) valid[e] = (uint8_t)ok;
    }
}
