/*
 * sa_oracle.c -- plain FP64 CPU oracle for shadow accumulation.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes is the plain definition the paper's accrual schemes reach exactly
 * (Sec. 3.1 for the two measures; Theorem 1 in Sec. 4 for "the same as one shadow map
 * per step"):
 *
 *   shadow(r, j) = 1  iff  the ray o_r + t * d_j, t > t_min, meets any triangle.
 *   gross(r)      = sum_j shadow(r, j)                       (gross shadow, Sec. 3.1)
 *   continuous(r) = max over days of the longest run of 1s   (continuous shadow, Sec. 3.1)
 *
 * d_j points toward the sun (the sun is a directional light, Sec. 3.2).  Receivers:
 *   ground receiver  (no normal):  o = p,               t_min = 1e-3 m
 *   facade receiver  (normal n):   o = p + 1e-2 m * n,  t_min = 0
 * Ray/triangle: Moller-Trumbore (1997) in double with inclusive barycentric bounds, so a
 * ray through an edge shared by two triangles hits.  Zero-area triangles are skipped and
 * a ray lying in a triangle's plane (det == 0) does not hit it.  The only culling is a
 * per-building axis-aligned box slab test, padded so it can never reject a ray that hits
 * one of the building's triangles (result-preserving; checked against the pure loop).
 *
 * Also here: the near-boundary classification used by the parity bar (a step is near a
 * shadow boundary if rotating d_j by +-eps along the sun arc changes its status), the
 * inverse-accrual-map algorithm of Sec. 5 in FP64 (an approximation, so it is given in
 * the paper's own steps), and the continuous-time shadow integral used for finite
 * differences of the height gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GROUND_TMIN 1e-3
#define FACADE_OFFSET 1e-2

typedef struct {
    double v0[3], e1[3], e2[3];
    int degenerate;
} otri;

typedef struct {
    int64_t T;
    otri* tri;
    int32_t G;          /* groups (buildings) */
    int64_t* goff;      /* CSR offsets [G+1] into gtri */
    int64_t* gtri;      /* triangle indices grouped by building */
    double* gbox;       /* [G][6] padded AABB lo.xyz hi.xyz */
} oscene;

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static int scene_init(oscene* s, const float* tri9, const int32_t* tri_building, int64_t T) {
    memset(s, 0, sizeof(*s));
    s->T = T;
    s->tri = (otri*)malloc(sizeof(otri) * (size_t)(T > 0 ? T : 1));
    if (!s->tri) return -3;
    for (int64_t t = 0; t < T; ++t) {
        const float* f = tri9 + 9 * t;
        otri* o = &s->tri[t];
        for (int k = 0; k < 3; ++k) {
            o->v0[k] = (double)f[k];
            o->e1[k] = (double)f[3 + k] - (double)f[k];
            o->e2[k] = (double)f[6 + k] - (double)f[k];
        }
        double n[3];
        cross3(o->e1, o->e2, n);
        o->degenerate = (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0);
    }
    int32_t G = 1;
    if (tri_building) {
        G = 0;
        for (int64_t t = 0; t < T; ++t) if (tri_building[t] + 1 > G) G = tri_building[t] + 1;
        if (G < 1) G = 1;
    }
    s->G = G;
    s->goff = (int64_t*)calloc((size_t)G + 1, sizeof(int64_t));
    s->gtri = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
    s->gbox = (double*)malloc(sizeof(double) * 6 * (size_t)G);
    if (!s->goff || !s->gtri || !s->gbox) return -3;
    for (int64_t t = 0; t < T; ++t) s->goff[(tri_building ? tri_building[t] : 0) + 1]++;
    for (int32_t g = 0; g < G; ++g) s->goff[g + 1] += s->goff[g];
    int64_t* fill = (int64_t*)calloc((size_t)G, sizeof(int64_t));
    if (!fill) return -3;
    for (int64_t t = 0; t < T; ++t) {
        int32_t g = tri_building ? tri_building[t] : 0;
        s->gtri[s->goff[g] + fill[g]++] = t;
    }
    free(fill);
    for (int32_t g = 0; g < G; ++g) {
        double* b = s->gbox + 6 * g;
        for (int k = 0; k < 3; ++k) { b[k] = INFINITY; b[3 + k] = -INFINITY; }
        for (int64_t i = s->goff[g]; i < s->goff[g + 1]; ++i) {
            const float* f = tri9 + 9 * s->gtri[i];
            for (int v = 0; v < 3; ++v)
                for (int k = 0; k < 3; ++k) {
                    double x = (double)f[3 * v + k];
                    if (x < b[k]) b[k] = x;
                    if (x > b[3 + k]) b[3 + k] = x;
                }
        }
        for (int k = 0; k < 3; ++k) {
            double pad = 1e-6 + 1e-9 * fmax(fabs(b[k]), fabs(b[3 + k]));
            b[k] -= pad;
            b[3 + k] += pad;
        }
    }
    return 0;
}

static void scene_free(oscene* s) {
    free(s->tri); free(s->goff); free(s->gtri); free(s->gbox);
    memset(s, 0, sizeof(*s));
}

/* slab test of the ray o + t d, t >= 0, against a padded box */
static int ray_box(const double* o, const double* d, const double* b) {
    double t0 = 0.0, t1 = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < b[k] || o[k] > b[3 + k]) return 0;
            continue;
        }
        double ta = (b[k] - o[k]) / d[k], tb = (b[3 + k] - o[k]) / d[k];
        double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
        if (lo > t0) t0 = lo;
        if (hi < t1) t1 = hi;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* Moller-Trumbore in double; returns 1 and the distance if hit with t > tmin */
static int ray_tri(const double* o, const double* d, const otri* tr, double tmin, double* t_out) {
    if (tr->degenerate) return 0;
    double p[3], q[3], s[3];
    cross3(d, tr->e2, p);
    double det = dot3(tr->e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    for (int k = 0; k < 3; ++k) s[k] = o[k] - tr->v0[k];
    double u = dot3(s, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    cross3(s, tr->e1, q);
    double v = dot3(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    double t = dot3(tr->e2, q) * inv;
    if (!(t > tmin)) return 0;
    if (t_out) *t_out = t;
    return 1;
}

static int any_hit(const oscene* s, const double* o, const double* d, double tmin) {
    for (int32_t g = 0; g < s->G; ++g) {
        if (!ray_box(o, d, s->gbox + 6 * g)) continue;
        for (int64_t i = s->goff[g]; i < s->goff[g + 1]; ++i)
            if (ray_tri(o, d, &s->tri[s->gtri[i]], tmin, NULL)) return 1;
    }
    return 0;
}

static void receiver_origin(const float* pos, const float* nrm, int64_t r, double* o, double* tmin) {
    for (int k = 0; k < 3; ++k) o[k] = (double)pos[3 * r + k];
    if (nrm) {
        for (int k = 0; k < 3; ++k) o[k] += FACADE_OFFSET * (double)nrm[3 * r + k];
        *tmin = 0.0;
    } else {
        *tmin = GROUND_TMIN;
    }
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* shadow(r, j) for every receiver and step: out[r * S + j] in {0, 1} */
int sao_shadow_bits(const float* tri9, const int32_t* tri_building, int64_t T,
                    const float* pos, const float* nrm, int64_t R,
                    const float* dirs, int32_t S, uint8_t* out, int nthreads) {
    if (T < 0 || R < 0 || S < 0 || (R > 0 && (!pos || !out)) || (S > 0 && !dirs)) return -1;
    oscene sc;
    if (scene_init(&sc, tri9, tri_building, T) != 0) { scene_free(&sc); return -3; }
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < R; ++r) {
        double o[3], tmin;
        receiver_origin(pos, nrm, r, o, &tmin);
        for (int32_t j = 0; j < S; ++j) {
            double d[3] = {(double)dirs[3 * j], (double)dirs[3 * j + 1], (double)dirs[3 * j + 2]};
            out[r * S + j] = (uint8_t)any_hit(&sc, o, d, tmin);
        }
    }
    scene_free(&sc);
    return 0;
}

/* Unit tangent of the sun arc at step j (within its day), or 0 if the day has one step. */
static int arc_tangent(const float* dirs, int32_t j, int32_t lo, int32_t hi, double* tan_out) {
    int32_t a = j > lo ? j - 1 : j, b = j < hi - 1 ? j + 1 : j;
    if (a == b) return 0;
    double d[3], v[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = dirs[3 * j + k];
        v[k] = (double)dirs[3 * b + k] - (double)dirs[3 * a + k];
    }
    double dn = sqrt(dot3(d, d));
    for (int k = 0; k < 3; ++k) d[k] /= dn;
    double p = dot3(v, d);
    for (int k = 0; k < 3; ++k) v[k] -= p * d[k];
    double n = sqrt(dot3(v, v));
    if (n == 0.0) return 0;
    for (int k = 0; k < 3; ++k) tan_out[k] = v[k] / n;
    return 1;
}

/* near[r * S + j] = 1 if rotating d_j by +eps or -eps (radians) along the sun arc flips
 * shadow(r, j).  Steps are grouped into days by day_start[0..D]. */
int sao_near_boundary(const float* tri9, const int32_t* tri_building, int64_t T,
                      const float* pos, const float* nrm, int64_t R,
                      const float* dirs, const int32_t* day_start, int32_t D, double eps,
                      const uint8_t* status, uint8_t* near, int nthreads) {
    if (T < 0 || R < 0 || D < 0) return -1;
    int32_t S = D > 0 ? day_start[D] : 0;
    oscene sc;
    if (scene_init(&sc, tri9, tri_building, T) != 0) { scene_free(&sc); return -3; }
    set_threads(nthreads);
    double* rot = (double*)malloc(sizeof(double) * 6 * (size_t)(S > 0 ? S : 1));
    uint8_t* has = (uint8_t*)malloc((size_t)(S > 0 ? S : 1));
    for (int32_t k = 0; k < D; ++k)
        for (int32_t j = day_start[k]; j < day_start[k + 1]; ++j) {
            double t[3], d[3];
            has[j] = (uint8_t)arc_tangent(dirs, j, day_start[k], day_start[k + 1], t);
            for (int c = 0; c < 3; ++c) d[c] = dirs[3 * j + c];
            double dn = sqrt(dot3(d, d));
            for (int c = 0; c < 3; ++c) {
                rot[6 * j + c] = cos(eps) * d[c] / dn + sin(eps) * (has[j] ? t[c] : 0.0);
                rot[6 * j + 3 + c] = cos(eps) * d[c] / dn - sin(eps) * (has[j] ? t[c] : 0.0);
            }
        }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < R; ++r) {
        double o[3], tmin;
        receiver_origin(pos, nrm, r, o, &tmin);
        for (int32_t j = 0; j < S; ++j) {
            uint8_t c = status[r * S + j];
            uint8_t nb = 0;
            if (has[j]) {
                nb = (uint8_t)(any_hit(&sc, o, rot + 6 * j, tmin) != c ||
                               any_hit(&sc, o, rot + 6 * j + 3, tmin) != c);
            }
            near[r * S + j] = nb;
        }
    }
    free(rot); free(has);
    scene_free(&sc);
    return 0;
}

/* gross and continuous shadow (in steps) from per-step bits (Sec. 3.1): the gross value is
 * the count over all days; the continuous value is the longest run of consecutive shadowed
 * steps within a day, maximised over days (runs never cross days). */
int sao_reduce(const uint8_t* bits, int64_t R, const int32_t* day_start, int32_t D,
               int32_t* gross, int32_t* continuous) {
    if (R < 0 || D < 0) return -1;
    int32_t S = D > 0 ? day_start[D] : 0;
    for (int64_t r = 0; r < R; ++r) {
        int32_t g = 0, best = 0;
        for (int32_t k = 0; k < D; ++k) {
            int32_t run = 0;
            for (int32_t j = day_start[k]; j < day_start[k + 1]; ++j) {
                if (bits[r * S + j]) {
                    ++g;
                    ++run;
                    if (run > best) best = run;
                } else {
                    run = 0;
                }
            }
        }
        gross[r] = g;
        if (continuous) continuous[r] = best;
    }
    return 0;
}
