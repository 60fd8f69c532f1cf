/*
 * mrpop_ref_planner.c -- slow, sequential FP64 reference planner.
 *
 * TEST AND CPU-BASELINE INFRASTRUCTURE ONLY (see mrpop_oracle.h).  It runs the
 * MR. POP main loop (Alg. 1) and its subroutines ROADMAP, AO-X and NEAREST
 * (Alg. 2) one iteration at a time on one host thread, in double precision,
 * with plain data structures: linear scans for every nearest and radius query,
 * an all-pairs collision test per configuration (orc_config_valid) and an
 * FP64 discretisation of every edge.  It shares nothing with the CUDA planner:
 * random numbers come from its own SplitMix64 stream, so its trajectories are
 * not those of the GPU; it serves as a CPU baseline and as an independent
 * source of solution costs.
 *
 * Readings where the paper is silent:
 *   - the dRRT initial solve is the AO-X iteration with c_best = +inf
 *     (uniform samples, no cost budget), the solve keeps its trees across
 *     ROADMAP rounds, an AO-X call starts from fresh trees rooted at
 *     (q_start, 0) and (q_goal, 0);
 *   - a search call ends at a solution or after max_iters iterations; either
 *     way the main loop then grows every roadmap by one round of n samples;
 *   - the direction oracle moves robot r from its roadmap vertex u to the
 *     neighbour v maximising cos(v - u, q_rand^r - u), ties to the lowest
 *     vertex index, and keeps r in place unless that cosine is positive; the
 *     composite step is kept iff g_near + |q_new - q_near| <= c_rand;
 *   - informed samples: Gaussian direction, radius U^(1/D), radii c_best / 2
 *     and sqrt(c_best^2 - c_min^2) / 2, a Householder reflection taking e_1
 *     to the start-goal axis; samples outside the joint limits are redrawn up
 *     to 16 times, then drawn uniformly in the limits;
 *   - c_rand ~ U[|q_rand - root_a|, c_best], root_a the root of the tree
 *     being extended;
 *   - a candidate path is accepted only when its FP64 cost C(sigma) is
 *     strictly below c_best and each segment is free at resolution / 4.
 */
#define _POSIX_C_SOURCE 199309L /* clock_gettime */
#include "mrpop_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)                            */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint64_t state;
} rp_rng;

static uint64_t rp_next(rp_rng *r) {
    uint64_t z = (r->state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* uniform in [0, 1) with 53 random bits */
static double rp_unif(rp_rng *r) { return (double)(rp_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* standard normal by the Box-Muller transform */
static double rp_gauss(rp_rng *r) {
    const double u1 = 1.0 - rp_unif(r); /* (0, 1] */
    const double u2 = rp_unif(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static double dist_d(const double *a, const double *b, int32_t n) {
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) acc += (a[i] - b[i]) * (a[i] - b[i]);
    return sqrt(acc);
}

/* grow *p (elements of size elt) to hold at least need elements */
static int grow(void **p, int64_t *cap, int64_t need, size_t elt) {
    if (need <= *cap) return 1;
    int64_t c = *cap > 0 ? *cap : 16;
    while (c < need) c *= 2;
    void *q = realloc(*p, (size_t)c * elt);
    if (!q) return 0;
    *p = q;
    *cap = c;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Scene views and FP64 edge checks                                           */
/* ------------------------------------------------------------------------- */

/* robot r alone with the obstacles: its own free space C^f_r (Sec. III-A) */
static orc_scene robot_scene(const orc_scene *s, int32_t r) {
    int32_t j0 = 0, s0 = 0;
    for (int32_t i = 0; i < r; ++i) {
        j0 += s->dof[i];
        s0 += s->n_spheres[i];
    }
    orc_scene o = *s;
    o.K = 1;
    o.dof = s->dof + r;
    o.dh = s->dh + 4 * j0;
    o.n_spheres = s->n_spheres + r;
    o.sphere_link = s->sphere_link + s0;
    o.sphere_xyzr = s->sphere_xyzr + 4 * s0;
    o.base = s->base + 12 * r;
    o.self_mask = s->self_mask ? s->self_mask + j0 : NULL;
    return o;
}

/* The edge qa -> qb is free when every q_k = qa + (k/n)(qb - qa), k = 0..n,
 * n = max(1, ceil(|qb - qa| / res)), is valid (Sec. III-E), all in FP64.
 * work holds n coordinates. */
static int edge_free(const orc_scene *s, const double *qa, const double *qb, int32_t n,
                     double res, double margin, double *work) {
    const double len = dist_d(qa, qb, n);
    double steps = ceil(len / res);
    if (!(steps >= 1.0)) steps = 1.0;
    if (steps > 1e7) return 0; /* absurdly long edge: treated as blocked */
    const int64_t m = (int64_t)steps;
    for (int64_t k = 0; k <= m; ++k) {
        const double t = (double)k / (double)m;
        for (int32_t i = 0; i < n; ++i) work[i] = qa[i] + t * (qb[i] - qa[i]);
        if (!orc_config_valid(s, work, margin, NULL)) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Per-robot roadmaps R_r = (V_r, E_r)                                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t dof;
    double *v; /* [n][dof] */
    int64_t n, cap_v;
    int32_t **adj; /* adjacency lists */
    int64_t *deg, *cap_adj;
    int64_t cap_lists, cap_deg, cap_caps;
    int connected;
} rp_roadmap;

static void roadmap_free(rp_roadmap *R) {
    for (int64_t i = 0; i < R->n; ++i) free(R->adj[i]);
    free(R->adj);
    free(R->deg);
    free(R->cap_adj);
    free(R->v);
    memset(R, 0, sizeof(*R));
}

static int64_t roadmap_add_vertex(rp_roadmap *R, const double *q) {
    if (!grow((void **)&R->v, &R->cap_v, R->n + 1, sizeof(double) * (size_t)R->dof) ||
        !grow((void **)&R->adj, &R->cap_lists, R->n + 1, sizeof(int32_t *)) ||
        !grow((void **)&R->deg, &R->cap_deg, R->n + 1, sizeof(int64_t)) ||
        !grow((void **)&R->cap_adj, &R->cap_caps, R->n + 1, sizeof(int64_t)))
        return -1;
    memcpy(R->v + (size_t)R->n * R->dof, q, sizeof(double) * (size_t)R->dof);
    R->adj[R->n] = NULL;
    R->deg[R->n] = 0;
    R->cap_adj[R->n] = 0;
    return R->n++;
}

static int roadmap_link(rp_roadmap *R, int64_t a, int64_t b) {
    const int64_t ends[2][2] = {{a, b}, {b, a}};
    for (int e = 0; e < 2; ++e) {
        const int64_t u = ends[e][0];
        if (!grow((void **)&R->adj[u], &R->cap_adj[u], R->deg[u] + 1, sizeof(int32_t))) return 0;
        R->adj[u][R->deg[u]++] = (int32_t)ends[e][1];
    }
    return 1;
}

/* BFS over E_r from vertex 0 (q_start^r) to vertex 1 (q_goal^r) */
static int roadmap_connected(const rp_roadmap *R) {
    if (R->n < 2) return 0;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)R->n);
    char *seen = (char *)calloc((size_t)R->n, 1);
    if (!queue || !seen) {
        free(queue);
        free(seen);
        return -1;
    }
    int64_t head = 0, tail = 0;
    queue[tail++] = 0;
    seen[0] = 1;
    int found = 0;
    while (head < tail && !found) {
        const int64_t u = queue[head++];
        for (int64_t k = 0; k < R->deg[u]; ++k) {
            const int64_t w = R->adj[u][k];
            if (!seen[w]) {
                seen[w] = 1;
                if (w == 1) found = 1;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    free(seen);
    return found;
}

/* ------------------------------------------------------------------------- */
/* State-cost trees T = (V, E) with vertices z = (q, g)                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double *q; /* [n][D] */
    double *g;
    int64_t *parent;
    int32_t *rm; /* [n][K]: roadmap vertex of each robot */
    int64_t n, cap_q, cap_g, cap_p, cap_rm;
    int root_is_start;
} rp_tree;

static void tree_free(rp_tree *T) {
    free(T->q);
    free(T->g);
    free(T->parent);
    free(T->rm);
    memset(T, 0, sizeof(*T));
}

static int64_t tree_add(rp_tree *T, int32_t D, int32_t K, const double *q, double g,
                        int64_t parent, const int32_t *rm) {
    if (!grow((void **)&T->q, &T->cap_q, T->n + 1, sizeof(double) * (size_t)D) ||
        !grow((void **)&T->g, &T->cap_g, T->n + 1, sizeof(double)) ||
        !grow((void **)&T->parent, &T->cap_p, T->n + 1, sizeof(int64_t)) ||
        !grow((void **)&T->rm, &T->cap_rm, T->n + 1, sizeof(int32_t) * (size_t)K))
        return -1;
    memcpy(T->q + (size_t)T->n * D, q, sizeof(double) * (size_t)D);
    T->g[T->n] = g;
    T->parent[T->n] = parent;
    memcpy(T->rm + (size_t)T->n * K, rm, sizeof(int32_t) * (size_t)K);
    return T->n++;
}

/* NEAREST(V, q, c) of Alg. 2: the vertex closest to q among those with
 * g_v + |q - q_v| < c; equal distances go to the lower g, then to the lower
 * index (Sec. III-D); -1 when none qualifies. */
static int64_t tree_nearest(const rp_tree *T, int32_t D, const double *q, double c) {
    int64_t best = -1;
    double bd = 0.0, bg = 0.0;
    for (int64_t v = 0; v < T->n; ++v) {
        const double d = dist_d(q, T->q + (size_t)v * D, D);
        const double g = T->g[v];
        if (!(g + d < c)) continue;
        if (best < 0 || d < bd || (d == bd && g < bg)) {
            best = v;
            bd = d;
            bg = g;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Planner state                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    const orc_scene *s;
    orc_scene *robot; /* [K] per-robot views */
    int32_t K, D;
    int32_t *j0; /* [K + 1] joint offsets */
    const double *lo, *hi, *start, *goal;
    orc_plan_params pp;
    rp_rng rng;
    rp_roadmap *R; /* [K] */
    double *work;  /* scratch [D] */
    double t0;
    int64_t iters, rounds;
    double c_best;
    double *best_path; /* [best_len][D] */
    int64_t best_len, cap_best;
    double *trace_t, *trace_c;
    int64_t *trace_it;
    int64_t trace_cap, n_trace;
} rp_planner;

static int out_of_budget(const rp_planner *P) {
    if (P->pp.time_budget_s > 0.0 && now_s() - P->t0 >= P->pp.time_budget_s) return 1;
    if (P->pp.iter_budget > 0 && P->iters >= P->pp.iter_budget) return 1;
    if (P->pp.round_budget > 0 && P->rounds >= P->pp.round_budget) return 1;
    if (P->c_best < INFINITY && P->c_best <= P->pp.target_cost) return 1;
    return 0;
}

/* SAMPLE_FREE(r): uniform in robot r's joint limits until it is collision
 * free for robot r alone; 0 when 100,000 draws found none. */
static int sample_free(rp_planner *P, int32_t r, double *c) {
    const int32_t o = P->j0[r], d = P->j0[r + 1] - o;
    for (int tries = 0; tries < 100000; ++tries) {
        for (int32_t i = 0; i < d; ++i)
            c[i] = P->lo[o + i] + (P->hi[o + i] - P->lo[o + i]) * rp_unif(&P->rng);
        if (orc_config_valid(&P->robot[r], c, P->pp.margin, NULL)) return 1;
    }
    return 0;
}

/* ROADMAP(q_start, q_goal, phi, delta, n) of Alg. 2, sequentially: every
 * robot whose roadmap is not (yet) re-connected adds n free samples, each
 * linked to the vertices of V_r within delta whose edges are free for robot
 * r; a BFS then marks connectivity of q_start^r and q_goal^r.  Every round
 * counts against the round budget.  Returns 1, 0 when a budget ran out, -1
 * on failure. */
static int roadmap_round(rp_planner *P, int phi) {
    double c[64];
    for (int32_t r = 0; r < P->K; ++r) {
        P->R[r].connected = 0;
        if (phi && P->R[r].n == 0) {
            if (roadmap_add_vertex(&P->R[r], P->start + P->j0[r]) < 0 ||
                roadmap_add_vertex(&P->R[r], P->goal + P->j0[r]) < 0)
                return -1;
        }
    }
    for (;;) {
        int all = 1;
        for (int32_t r = 0; r < P->K; ++r) all &= P->R[r].connected;
        if (all) return 1;
        if (P->pp.round_budget > 0 && P->rounds >= P->pp.round_budget) return 0;
        ++P->rounds;
        for (int32_t r = 0; r < P->K; ++r) {
            rp_roadmap *R = &P->R[r];
            if (R->connected) continue;
            const int32_t d = R->dof;
            for (int32_t i = 0; i < P->pp.n_per_round; ++i) {
                if (P->pp.time_budget_s > 0.0 && now_s() - P->t0 >= P->pp.time_budget_s) return 0;
                if (!sample_free(P, r, c)) return -1;
                const int64_t nv = roadmap_add_vertex(R, c);
                if (nv < 0) return -1;
                for (int64_t u = 0; u < nv; ++u) {
                    const double *cu = R->v + (size_t)u * d;
                    if (dist_d(c, cu, d) > P->pp.delta) continue;
                    if (edge_free(&P->robot[r], R->v + (size_t)nv * d, cu, d, P->pp.resolution,
                                  P->pp.margin, P->work))
                        if (!roadmap_link(R, nv, u)) return -1;
                }
            }
        }
        for (int32_t r = 0; r < P->K; ++r) {
            const int cn = roadmap_connected(&P->R[r]);
            if (cn < 0) return -1;
            P->R[r].connected = cn;
        }
    }
}

/* INFORMED_SAMPLE(c_best): uniform in the prolate hyperspheroid with foci
 * q_start, q_goal and transverse diameter c_best (Gammell et al. 2014),
 * clipped to the joint limits by redrawing. */
static void informed_sample(rp_planner *P, double *q) {
    const int32_t D = P->D;
    if (!(P->c_best < INFINITY)) {
        for (int32_t i = 0; i < D; ++i) q[i] = P->lo[i] + (P->hi[i] - P->lo[i]) * rp_unif(&P->rng);
        return;
    }
    const double cmin = dist_d(P->start, P->goal, D);
    const double r1 = 0.5 * P->c_best;
    const double r2 = 0.5 * sqrt(fmax(P->c_best * P->c_best - cmin * cmin, 0.0));
    for (int attempt = 0; attempt < 16; ++attempt) {
        /* x uniform in the unit D-ball */
        double nrm = 0.0;
        for (int32_t i = 0; i < D; ++i) {
            q[i] = rp_gauss(&P->rng);
            nrm += q[i] * q[i];
        }
        nrm = sqrt(nrm);
        const double rad = pow(rp_unif(&P->rng), 1.0 / (double)D);
        for (int32_t i = 0; i < D; ++i) q[i] *= rad / (nrm > 0.0 ? nrm : 1.0);
        /* scale to the hyperspheroid's radii */
        q[0] *= r1;
        for (int32_t i = 1; i < D; ++i) q[i] *= r2;
        /* Householder reflection H = I - 2 w w^T / (w^T w), w = e_1 - a_1,
         * maps e_1 to the axis a_1 = (q_goal - q_start) / c_min */
        if (cmin > 0.0) {
            double ww = 0.0, wy = 0.0;
            for (int32_t i = 0; i < D; ++i) {
                const double a = (P->goal[i] - P->start[i]) / cmin;
                const double w = (i == 0 ? 1.0 : 0.0) - a;
                ww += w * w;
                wy += w * q[i];
            }
            if (ww > 1e-24) {
                const double f = 2.0 * wy / ww;
                for (int32_t i = 0; i < D; ++i) {
                    const double a = (P->goal[i] - P->start[i]) / cmin;
                    q[i] -= f * ((i == 0 ? 1.0 : 0.0) - a);
                }
            }
        }
        int inside = 1;
        for (int32_t i = 0; i < D; ++i) {
            q[i] += 0.5 * (P->start[i] + P->goal[i]);
            inside &= q[i] >= P->lo[i] && q[i] <= P->hi[i];
        }
        if (inside) return;
    }
    for (int32_t i = 0; i < D; ++i) q[i] = P->lo[i] + (P->hi[i] - P->lo[i]) * rp_unif(&P->rng);
}

/* ORACLE_AOX: per robot, the roadmap neighbour of q_near^r best aligned with
 * q_rand^r (positive cosine required, ties to the lowest index), else stay.
 * Writes q_new and its roadmap vertices; returns 0 when every robot stays. */
static int direction_oracle(rp_planner *P, const rp_tree *T, int64_t near, const double *q_rand,
                            double *q_new, int32_t *rm_new) {
    int moved = 0;
    for (int32_t r = 0; r < P->K; ++r) {
        const rp_roadmap *R = &P->R[r];
        const int32_t o = P->j0[r], d = R->dof;
        const int32_t u = T->rm[(size_t)near * P->K + r];
        const double *qu = R->v + (size_t)u * d;
        double tn = 0.0;
        for (int32_t i = 0; i < d; ++i) tn += (q_rand[o + i] - qu[i]) * (q_rand[o + i] - qu[i]);
        tn = sqrt(tn);
        int32_t best = -1;
        double bcos = 0.0;
        if (tn > 0.0) {
            for (int64_t k = 0; k < R->deg[u]; ++k) {
                const int32_t v = R->adj[u][k];
                const double *qv = R->v + (size_t)v * d;
                double dot = 0.0, vn = 0.0;
                for (int32_t i = 0; i < d; ++i) {
                    dot += (qv[i] - qu[i]) * (q_rand[o + i] - qu[i]);
                    vn += (qv[i] - qu[i]) * (qv[i] - qu[i]);
                }
                if (vn <= 0.0) continue;
                const double cs = dot / (sqrt(vn) * tn);
                if (cs > bcos || (cs == bcos && best >= 0 && v < best)) {
                    bcos = cs;
                    best = v;
                }
            }
        }
        const int32_t pick = best >= 0 ? best : u;
        moved |= pick != u;
        rm_new[r] = pick;
        memcpy(q_new + o, R->v + (size_t)pick * d, sizeof(double) * (size_t)d);
    }
    return moved;
}

/* EXTRACT_PATH(T_a, T_b): the start tree's branch to its vertex, then the
 * goal tree's branch from its vertex back to q_goal. */
static int extract_path(rp_planner *P, const rp_tree *Ts, int64_t vs, const rp_tree *Tg,
                        int64_t vg, double **out, int64_t *len) {
    int64_t ns = 0, ng = 0;
    for (int64_t v = vs; v >= 0; v = Ts->parent[v]) ++ns;
    for (int64_t v = vg; v >= 0; v = Tg->parent[v]) ++ng;
    const int32_t D = P->D;
    double *p = (double *)malloc(sizeof(double) * (size_t)(ns + ng) * D);
    if (!p) return 0;
    int64_t i = ns - 1;
    for (int64_t v = vs; v >= 0; v = Ts->parent[v], --i)
        memcpy(p + (size_t)i * D, Ts->q + (size_t)v * D, sizeof(double) * (size_t)D);
    i = ns;
    for (int64_t v = vg; v >= 0; v = Tg->parent[v], ++i)
        memcpy(p + (size_t)i * D, Tg->q + (size_t)v * D, sizeof(double) * (size_t)D);
    *out = p;
    *len = ns + ng;
    return 1;
}

static double path_cost_d(const double *p, int64_t M, int32_t D) {
    double c = 0.0;
    for (int64_t j = 0; j + 1 < M; ++j) c += dist_d(p + (size_t)j * D, p + (size_t)(j + 1) * D, D);
    return c;
}

static void tree_reset(rp_planner *P, rp_tree *T, int at_start) {
    T->n = 0;
    T->root_is_start = at_start;
    int32_t rm[64];
    for (int32_t r = 0; r < P->K; ++r) rm[r] = at_start ? 0 : 1;
    tree_add(T, P->D, P->K, at_start ? P->start : P->goal, 0.0, -1, rm);
}

/* One search call: the dRRT initial solve when c_best = +inf, else AO-X
 * (Alg. 2).  Returns 1 with a new incumbent, 0 without one, -1 on failure. */
static int search(rp_planner *P, rp_tree *Ta, rp_tree *Tb) {
    const int32_t D = P->D, K = P->K;
    double *q_rand = (double *)malloc(sizeof(double) * (size_t)D * 2);
    int32_t rm_new[64];
    if (!q_rand) return -1;
    double *q_new = q_rand + D;
    int result = 0;
    for (int64_t it = 0; it < P->pp.max_iters && !out_of_budget(P); ++it) {
        ++P->iters;
        if (Ta->n > Tb->n) { /* extend the smaller tree */
            rp_tree *t = Ta;
            Ta = Tb;
            Tb = t;
        }
        informed_sample(P, q_rand);
        double c_rand = INFINITY;
        if (P->c_best < INFINITY) {
            const double lower = dist_d(q_rand, Ta->root_is_start ? P->start : P->goal, D);
            if (!(lower < P->c_best)) continue;
            c_rand = lower + (P->c_best - lower) * rp_unif(&P->rng);
        }
        const int64_t near = tree_nearest(Ta, D, q_rand, c_rand);
        if (near < 0) continue;
        if (!direction_oracle(P, Ta, near, q_rand, q_new, rm_new)) continue;
        const double *q_near = Ta->q + (size_t)near * D;
        const double g_new = Ta->g[near] + dist_d(q_new, q_near, D);
        if (!(g_new <= c_rand)) continue;
        if (!edge_free(P->s, q_near, q_new, D, P->pp.resolution, P->pp.margin, P->work)) continue;
        const int64_t vn = tree_add(Ta, D, K, q_new, g_new, near, rm_new);
        if (vn < 0) {
            result = -1;
            break;
        }
        const int64_t conn = tree_nearest(Tb, D, q_new, P->c_best - g_new);
        if (conn < 0) continue;
        if (!edge_free(P->s, q_new, Tb->q + (size_t)conn * D, D, P->pp.resolution, P->pp.margin,
                       P->work))
            continue;
        double *path = NULL;
        int64_t len = 0;
        const int ok = Ta->root_is_start ? extract_path(P, Ta, vn, Tb, conn, &path, &len)
                                         : extract_path(P, Tb, conn, Ta, vn, &path, &len);
        if (!ok) {
            result = -1;
            break;
        }
        const double cost = path_cost_d(path, len, D);
        int accept = cost < P->c_best;
        for (int64_t j = 0; accept && j + 1 < len; ++j)
            accept = edge_free(P->s, path + (size_t)j * D, path + (size_t)(j + 1) * D, D,
                               0.25 * P->pp.resolution, P->pp.margin, P->work);
        if (!accept) {
            free(path);
            continue;
        }
        free(P->best_path);
        P->best_path = path;
        P->best_len = len;
        P->c_best = cost;
        if (P->n_trace < P->trace_cap) {
            if (P->trace_t) P->trace_t[P->n_trace] = now_s() - P->t0;
            if (P->trace_c) P->trace_c[P->n_trace] = cost;
            if (P->trace_it) P->trace_it[P->n_trace] = P->iters;
        }
        ++P->n_trace;
        result = 1;
        break;
    }
    free(q_rand);
    return result;
}

int32_t orc_plan(const orc_scene *s, const float *q_lo, const float *q_hi, const double *start,
                 const double *goal, const orc_plan_params *pp, double *path, int64_t path_cap,
                 int64_t *path_len, double *cost, double *trace_t, double *trace_c,
                 int64_t *trace_it, int64_t trace_cap, int64_t *n_trace, int64_t *iterations) {
    if (path_len) *path_len = 0;
    if (cost) *cost = INFINITY;
    if (n_trace) *n_trace = 0;
    if (iterations) *iterations = 0;
    if (!s || !q_lo || !q_hi || !start || !goal || !pp || s->K < 1 || s->K > 64) return -1;
    if (!(pp->resolution > 0.0) || !(pp->delta > 0.0) || pp->n_per_round < 1 ||
        pp->max_iters < 1 || !(pp->time_budget_s > 0.0 || pp->iter_budget > 0))
        return -1;
    rp_planner P;
    memset(&P, 0, sizeof(P));
    P.s = s;
    P.K = s->K;
    P.pp = *pp;
    P.rng.state = pp->seed;
    P.j0 = (int32_t *)calloc((size_t)P.K + 1, sizeof(int32_t));
    P.robot = (orc_scene *)calloc((size_t)P.K, sizeof(orc_scene));
    P.R = (rp_roadmap *)calloc((size_t)P.K, sizeof(rp_roadmap));
    if (!P.j0 || !P.robot || !P.R) {
        free(P.j0);
        free(P.robot);
        free(P.R);
        return -1;
    }
    for (int32_t r = 0; r < P.K; ++r) {
        if (s->dof[r] < 1 || s->dof[r] > 64) {
            free(P.j0);
            free(P.robot);
            free(P.R);
            return -1;
        }
        P.j0[r + 1] = P.j0[r] + s->dof[r];
        P.robot[r] = robot_scene(s, r);
        P.R[r].dof = s->dof[r];
    }
    P.D = P.j0[P.K];
    double *lo = (double *)malloc(sizeof(double) * (size_t)P.D * 3);
    P.work = lo ? lo + 2 * P.D : NULL;
    int32_t status = -1;
    rp_tree Ts, Tg, As, Ag;
    memset(&Ts, 0, sizeof(Ts));
    memset(&Tg, 0, sizeof(Tg));
    memset(&As, 0, sizeof(As));
    memset(&Ag, 0, sizeof(Ag));
    if (!lo) goto done;
    for (int32_t i = 0; i < P.D; ++i) {
        lo[i] = q_lo[i];
        lo[P.D + i] = q_hi[i];
    }
    P.lo = lo;
    P.hi = lo + P.D;
    P.start = start;
    P.goal = goal;
    P.c_best = INFINITY;
    P.trace_t = trace_t;
    P.trace_c = trace_c;
    P.trace_it = trace_it;
    P.trace_cap = trace_t || trace_c || trace_it ? trace_cap : 0;
    P.t0 = now_s();
    if (!orc_config_valid(s, start, pp->margin, NULL) || !orc_config_valid(s, goal, pp->margin, NULL))
        goto done;
    tree_reset(&P, &Ts, 1);
    tree_reset(&P, &Tg, 0);
    if (Ts.n != 1 || Tg.n != 1) goto done;
    {
        /* Alg. 1: ROADMAP, then the dRRT solve until a first solution (phi),
         * then AO-X calls, growing the roadmaps before every call */
        int phi = 1;
        while (!out_of_budget(&P)) {
            const int rr = roadmap_round(&P, phi);
            if (rr < 0) goto done;
            if (rr == 0) break;
            if (phi) {
                const int sr = search(&P, &Ts, &Tg);
                if (sr < 0) goto done;
                if (sr > 0) phi = 0;
            } else {
                tree_reset(&P, &As, 1);
                tree_reset(&P, &Ag, 0);
                if (As.n != 1 || Ag.n != 1) goto done;
                if (search(&P, &As, &Ag) < 0) goto done;
            }
        }
    }
    status = P.best_len > 0 ? 0 : 1;
    if (status == 0) {
        if (path_len) *path_len = P.best_len;
        if (cost) *cost = P.c_best;
        if (path && P.best_len <= path_cap)
            memcpy(path, P.best_path, sizeof(double) * (size_t)P.best_len * P.D);
    }
done:
    if (n_trace) *n_trace = P.n_trace;
    if (iterations) *iterations = P.iters;
    tree_free(&Ts);
    tree_free(&Tg);
    tree_free(&As);
    tree_free(&Ag);
    for (int32_t r = 0; r < P.K; ++r) roadmap_free(&P.R[r]);
    free(P.R);
    free(P.robot);
    free(P.j0);
    free(P.best_path);
    free(lo);
    return status;
}
