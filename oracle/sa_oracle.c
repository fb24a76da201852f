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

/* ------------------------------------------------------------------------------------
 * Inverse accrual map (Sec. 5), in the paper's steps, FP64.  An approximation by design.
 *
 * For each block of steps [j0, j0 + K) and each ground cell centre p of the grid:
 *   1. Forward map (t_1 -> t_n): cast the ray from p toward the sun at the block's first
 *      step; each intersection farther than `tmin_src` (the paper's 100 cm) is a source
 *      of shadow; keep the L closest (source levels l = 1..L).
 *   2. For each source s, its shadow at step k is q_k, the projection of s along d_k onto
 *      the ground.  The shadow line from p (= q_0) to q_{K-1} is cut into K - 1 pieces
 *      [q_k, q_{k+1}]; bit k of every cell the piece touches is set, and bit K-1 of the
 *      cell(s) of q_{K-1}.
 *   3. Reverse map (t_n -> t_1): the same from the block's last step, the pieces running
 *      backwards: [q_k, q_{k-1}] sets bit k, and bit 0 is set at q_0.
 * Cells are closed squares of side dx around the centres ("touches" includes edges and
 * corners).  Gross and continuous shadow then follow from the bits as in Sec. 3.1.
 * ------------------------------------------------------------------------------------ */

typedef struct { double t; } ohit;

/* all hits with t > tmin along o + t d; keeps the L smallest t in ascending order */
static int nearest_hits(const oscene* s, const double* o, const double* d, double tmin, int L,
                        double* best) {
    int n = 0;
    for (int32_t g = 0; g < s->G; ++g) {
        if (!ray_box(o, d, s->gbox + 6 * g)) continue;
        for (int64_t i = s->goff[g]; i < s->goff[g + 1]; ++i) {
            double t;
            if (!ray_tri(o, d, &s->tri[s->gtri[i]], tmin, &t)) continue;
            if (n < L) {
                int k = n++;
                while (k > 0 && best[k - 1] > t) { best[k] = best[k - 1]; --k; }
                best[k] = t;
            } else if (t < best[L - 1]) {
                int k = L - 1;
                while (k > 0 && best[k - 1] > t) { best[k] = best[k - 1]; --k; }
                best[k] = t;
            }
        }
    }
    return n;
}

typedef struct {
    double x0, y0, dx;
    int32_t nx, ny;
} ogrid;

static void set_bit_cell(uint8_t* blk, int32_t K, int64_t cell, int32_t k) {
    uint8_t* b = blk + cell * K + k;
#pragma omp atomic write
    *b = 1;
}

/* thin line: m = ceil(max(|dx|, |dy|) / cell) + 1 equally spaced samples from P to Q
 * (both ends included); the cell holding each sample (half-open cells) gets bit k */
static void draw_thin(const ogrid* g, double px, double py, double qx, double qy,
                      uint8_t* blk, int32_t K, int32_t k) {
    const double len = fmax(fabs(qx - px), fabs(qy - py)) / g->dx;
    const int64_t m = (int64_t)ceil(len) + 1;
    for (int64_t i = 0; i < m; ++i) {
        const double a = m > 1 ? (double)i / (double)(m - 1) : 0.0;
        const double x = px + a * (qx - px), y = py + a * (qy - py);
        const double fx = floor((x - g->x0) / g->dx), fy = floor((y - g->y0) / g->dx);
        if (fx < 0 || fy < 0 || fx >= g->nx || fy >= g->ny) continue;
        set_bit_cell(blk, K, (int64_t)fy * g->nx + (int64_t)fx, k);
    }
}

/* every closed cell touched by the segment P -> Q gets bit k.  With eps != 0 each cell is
 * taken as its square grown by eps on every side (eps > 0) or shrunk by |eps| (eps < 0):
 * the first touches every cell a copy of the segment moved by up to eps in x and y can
 * touch, the second only cells every such copy touches (bounds for rounded endpoints). */
static void draw_segment_eps(const ogrid* g, double px, double py, double qx, double qy,
                             double eps, uint8_t* blk, int32_t K, int32_t k) {
    const double ymin = fmin(py, qy), ymax = fmax(py, qy);
    int64_t iy0 = (int64_t)ceil((ymin - eps - g->y0) / g->dx) - 1;
    int64_t iy1 = (int64_t)floor((ymax + eps - g->y0) / g->dx);
    if (iy0 < 0) iy0 = 0;
    if (iy1 > g->ny - 1) iy1 = g->ny - 1;
    for (int64_t iy = iy0; iy <= iy1; ++iy) {
        const double c0 = g->y0 + (double)iy * g->dx;
        const double b0 = c0 - eps, b1 = c0 + g->dx + eps;
        if (b0 > b1) continue;
        double xa, xb;
        if (py == qy) {
            if (py < b0 || py > b1) continue;
            xa = fmin(px, qx); xb = fmax(px, qx);
        } else {
            double ta = (b0 - py) / (qy - py), tb = (b1 - py) / (qy - py);
            double lo = fmax(fmin(ta, tb), 0.0), hi = fmin(fmax(ta, tb), 1.0);
            if (lo > hi) continue;
            double x1 = px + lo * (qx - px), x2 = px + hi * (qx - px);
            xa = fmin(x1, x2); xb = fmax(x1, x2);
        }
        int64_t ix0 = (int64_t)ceil((xa - eps - g->x0) / g->dx) - 1;
        int64_t ix1 = (int64_t)floor((xb + eps - g->x0) / g->dx);
        if (ix0 < 0) ix0 = 0;
        if (ix1 > g->nx - 1) ix1 = g->nx - 1;
        for (int64_t ix = ix0; ix <= ix1; ++ix) set_bit_cell(blk, K, iy * g->nx + ix, k);
    }
}

static void draw_segment(const ogrid* g, double px, double py, double qx, double qy,
                         uint8_t* blk, int32_t K, int32_t k) {
    draw_segment_eps(g, px, py, qx, qy, 0.0, blk, K, k);
}

/* One segment drawn on its own (for the drawer's pins): out[cell] = 1 on every cell of the
 * nx x ny grid that draw_segment_eps marks. */
int sao_draw_segment(double x0, double y0, double dx, int32_t nx, int32_t ny, double px,
                     double py, double qx, double qy, double eps, uint8_t* out) {
    if (nx < 0 || ny < 0 || !(dx > 0.0) || !out || fabs(eps) * 2.0 >= dx) return -1;
    ogrid g = {x0, y0, dx, nx, ny};
    draw_segment_eps(&g, px, py, qx, qy, eps, out, 1, 0);
    return 0;
}

int sao_iam(const float* tri9, const int32_t* tri_building, int64_t T,
            float x0, float y0, float dx, int32_t nx, int32_t ny,
            const float* dirs, const int32_t* block_j0, const int32_t* block_K, int32_t n_blocks,
            int32_t L, double tmin_src, int32_t line_mode, int32_t S, uint8_t* out, int nthreads) {
    if (T < 0 || nx < 0 || ny < 0 || L < 1 || L > 16 || n_blocks < 0) return -1;
    void (*draw)(const ogrid*, double, double, double, double, uint8_t*, int32_t, int32_t) =
        line_mode == 1 ? draw_thin : draw_segment;
    oscene sc;
    if (scene_init(&sc, tri9, tri_building, T) != 0) { scene_free(&sc); return -3; }
    set_threads(nthreads);
    const int64_t R = (int64_t)nx * ny;
    ogrid g = {(double)x0, (double)y0, (double)dx, nx, ny};
    int32_t Kmax = 1;
    for (int32_t b = 0; b < n_blocks; ++b) if (block_K[b] > Kmax) Kmax = block_K[b];
    uint8_t* blk = (uint8_t*)malloc((size_t)(R > 0 ? R : 1) * (size_t)Kmax);
    if (!blk) { scene_free(&sc); return -3; }
    for (int32_t b = 0; b < n_blocks; ++b) {
        const int32_t j0 = block_j0[b], K = block_K[b];
        memset(blk, 0, (size_t)R * (size_t)K);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t r = 0; r < R; ++r) {
            const int64_t ix = r % nx, iy = r / nx;
            /* cell centre rounded in FP32 exactly as the receivers are defined */
            const float cxf = x0 + ((float)ix + 0.5f) * dx;
            const float cyf = y0 + ((float)iy + 0.5f) * dx;
            const double o[3] = {(double)cxf, (double)cyf, 0.0};
            for (int dir = 0; dir < 2; ++dir) {
                const int32_t js = dir == 0 ? j0 : j0 + K - 1;
                double d[3] = {dirs[3 * js], dirs[3 * js + 1], dirs[3 * js + 2]};
                double best[16];
                const int n = nearest_hits(&sc, o, d, tmin_src, L, best);
                for (int l = 0; l < n; ++l) {
                    const double s[3] = {o[0] + best[l] * d[0], o[1] + best[l] * d[1], o[2] + best[l] * d[2]};
                    double qx[64], qy[64];
                    for (int32_t k = 0; k < K; ++k) {
                        const double dk[3] = {dirs[3 * (j0 + k)], dirs[3 * (j0 + k) + 1], dirs[3 * (j0 + k) + 2]};
                        qx[k] = s[0] - s[2] * dk[0] / dk[2];
                        qy[k] = s[1] - s[2] * dk[1] / dk[2];
                    }
                    if (dir == 0) {
                        for (int32_t k = 0; k + 1 < K; ++k)
                            draw(&g, qx[k], qy[k], qx[k + 1], qy[k + 1], blk, K, k);
                        draw(&g, qx[K - 1], qy[K - 1], qx[K - 1], qy[K - 1], blk, K, K - 1);
                    } else {
                        for (int32_t k = K - 1; k >= 1; --k)
                            draw(&g, qx[k], qy[k], qx[k - 1], qy[k - 1], blk, K, k);
                        draw(&g, qx[0], qy[0], qx[0], qy[0], blk, K, 0);
                    }
                }
            }
        }
        for (int64_t r = 0; r < R; ++r)
            for (int32_t k = 0; k < K; ++k) out[r * S + j0 + k] = blk[r * K + k];
    }
    free(blk);
    scene_free(&sc);
    return 0;
}

/* Clearance of the ray o + t d through triangle tr: the perpendicular distance (metres)
 * from the ray's line to the nearest of the three edge lines, positive when the ray
 * passes inside the triangle, negative outside; *t_out is the distance along the ray to
 * the triangle's plane.  Returns 0 for a zero-area triangle, a triangle seen edge-on, or
 * an edge parallel to the ray (no clearance is defined then). */
static int ray_tri_clearance(const double* o, const double* d, const otri* tr, double* margin,
                             double* t_out) {
    if (tr->degenerate) return 0;
    double v[3][3], e[3][3];
    for (int k = 0; k < 3; ++k) {
        v[0][k] = tr->v0[k];
        v[1][k] = tr->v0[k] + tr->e1[k];
        v[2][k] = tr->v0[k] + tr->e2[k];
    }
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) e[i][k] = v[(i + 1) % 3][k] - v[i][k];
    double sv[3], nv[3], sum = 0.0;
    for (int i = 0; i < 3; ++i) {
        double c[3], w[3];
        cross3(d, e[i], c);
        for (int k = 0; k < 3; ++k) w[k] = v[i][k] - o[k];
        sv[i] = dot3(w, c);
        nv[i] = sqrt(dot3(c, c));
        if (nv[i] == 0.0) return 0;
        sum += sv[i];
    }
    if (sum == 0.0) return 0;
    const double sg = sum > 0.0 ? 1.0 : -1.0;
    double m = INFINITY;
    for (int i = 0; i < 3; ++i) m = fmin(m, sg * sv[i] / nv[i]);
    double n[3], w0[3];
    cross3(tr->e1, tr->e2, n);
    const double dn = dot3(d, n);
    if (dn == 0.0) return 0;
    for (int k = 0; k < 3; ++k) w0[k] = tr->v0[k] - o[k];
    *margin = m;
    *t_out = dot3(w0, n) / dn;
    return 1;
}

typedef struct { double t, margin; } ocand;

#define IAM_MAX_CANDIDATES 1024

/* Every triangle the ray may hit within the tolerances: clearance >= -eps_src and plane
 * distance t > tmin - eps_t; sorted by t.  Returns the count, or -1 if there are more
 * than `cap`. */
static int candidate_hits(const oscene* s, const double* o, const double* d, double tmin,
                          double eps_src, double eps_t, ocand* out, int cap) {
    int n = 0;
    for (int32_t g = 0; g < s->G; ++g) {
        /* the padded box pre-test, widened by eps_src so that near misses are kept */
        double b[6];
        for (int k = 0; k < 3; ++k) {
            b[k] = s->gbox[6 * g + k] - eps_src;
            b[3 + k] = s->gbox[6 * g + 3 + k] + eps_src;
        }
        if (!ray_box(o, d, b)) continue;
        for (int64_t i = s->goff[g]; i < s->goff[g + 1]; ++i) {
            double m, t;
            if (!ray_tri_clearance(o, d, &s->tri[s->gtri[i]], &m, &t)) continue;
            if (m < -eps_src || !(t > tmin - eps_t)) continue;
            if (n == cap) return -1;
            int k = n++;
            while (k > 0 && out[k - 1].t > t) { out[k] = out[k - 1]; --k; }
            out[k].t = t;
            out[k].margin = m;
        }
    }
    return n;
}

/* Bounds of the inverse accrual map (the supercover reading, as sao_iam with line_mode 0)
 * under small perturbations of its geometry, for comparing an implementation that rounds
 * differently (e.g. FP32):
 *   a hit is SURE if the ray passes at least eps_src inside the triangle and t > tmin_src
 *   + eps_t, POSSIBLE if it passes no more than eps_src outside and t > tmin_src - eps_t;
 *   a sure hit is a source for certain if fewer than L possible hits lie before t + eps_t;
 *   a possible hit may be a source if fewer than L sure hits lie before t - eps_t;
 *   `must` draws the certain sources' lines on cells shrunk by eps_cell, `may` draws the
 *   possible sources' lines on cells grown by eps_cell (draw_segment_eps).
 * An implementation whose sources and shadow-line ends stay within these tolerances of
 * the FP64 ones sets every bit of `must` and no bit outside `may`.  out arrays are [R, S]
 * like sao_iam's.  Returns -4 if a ray has more than IAM_MAX_CANDIDATES candidates. */
int sao_iam_bounds(const float* tri9, const int32_t* tri_building, int64_t T,
                   float x0, float y0, float dx, int32_t nx, int32_t ny,
                   const float* dirs, const int32_t* block_j0, const int32_t* block_K,
                   int32_t n_blocks, int32_t L, double tmin_src, double eps_cell, double eps_src,
                   double eps_t, int32_t S, uint8_t* must, uint8_t* may, int nthreads) {
    if (T < 0 || nx < 0 || ny < 0 || L < 1 || L > 16 || n_blocks < 0) return -1;
    if (eps_cell < 0.0 || eps_src < 0.0 || eps_t < 0.0 || 2.0 * eps_cell >= (double)dx) return -1;
    oscene sc;
    if (scene_init(&sc, tri9, tri_building, T) != 0) { scene_free(&sc); return -3; }
    set_threads(nthreads);
    const int64_t R = (int64_t)nx * ny;
    ogrid g = {(double)x0, (double)y0, (double)dx, nx, ny};
    int32_t Kmax = 1;
    for (int32_t b = 0; b < n_blocks; ++b) if (block_K[b] > Kmax) Kmax = block_K[b];
    uint8_t* bm = (uint8_t*)malloc((size_t)(R > 0 ? R : 1) * (size_t)Kmax);
    uint8_t* bp = (uint8_t*)malloc((size_t)(R > 0 ? R : 1) * (size_t)Kmax);
    if (!bm || !bp) { free(bm); free(bp); scene_free(&sc); return -3; }
    int overflow = 0;
    for (int32_t b = 0; b < n_blocks; ++b) {
        const int32_t j0 = block_j0[b], K = block_K[b];
        memset(bm, 0, (size_t)R * (size_t)K);
        memset(bp, 0, (size_t)R * (size_t)K);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t r = 0; r < R; ++r) {
            const int64_t ix = r % nx, iy = r / nx;
            const float cxf = x0 + ((float)ix + 0.5f) * dx;
            const float cyf = y0 + ((float)iy + 0.5f) * dx;
            const double o[3] = {(double)cxf, (double)cyf, 0.0};
            ocand c[IAM_MAX_CANDIDATES];
            for (int dir = 0; dir < 2; ++dir) {
                const int32_t js = dir == 0 ? j0 : j0 + K - 1;
                double d[3] = {dirs[3 * js], dirs[3 * js + 1], dirs[3 * js + 2]};
                const int n = candidate_hits(&sc, o, d, tmin_src, eps_src, eps_t, c,
                                             IAM_MAX_CANDIDATES);
                if (n < 0) {
#pragma omp atomic write
                    overflow = 1;
                    continue;
                }
                for (int h = 0; h < n; ++h) {
                    const int sure = c[h].margin >= eps_src && c[h].t > tmin_src + eps_t;
                    int before_possible = 0, before_sure = 0;
                    for (int q = 0; q < n; ++q) {
                        if (q == h) continue;
                        if (c[q].t < c[h].t + eps_t) ++before_possible;
                        if (c[q].t < c[h].t - eps_t && c[q].margin >= eps_src &&
                            c[q].t > tmin_src + eps_t) ++before_sure;
                    }
                    const int certain = sure && before_possible < L;
                    const int maybe = before_sure < L;
                    if (!certain && !maybe) continue;
                    const double s[3] = {o[0] + c[h].t * d[0], o[1] + c[h].t * d[1], o[2] + c[h].t * d[2]};
                    double qx[64], qy[64];
                    for (int32_t k = 0; k < K; ++k) {
                        const double dk[3] = {dirs[3 * (j0 + k)], dirs[3 * (j0 + k) + 1], dirs[3 * (j0 + k) + 2]};
                        qx[k] = s[0] - s[2] * dk[0] / dk[2];
                        qy[k] = s[1] - s[2] * dk[1] / dk[2];
                    }
                    for (int pass = 0; pass < 2; ++pass) {
                        if (pass == 0 && !certain) continue;
                        if (pass == 1 && !maybe) continue;
                        uint8_t* blk = pass == 0 ? bm : bp;
                        const double e = pass == 0 ? -eps_cell : eps_cell;
                        if (dir == 0) {
                            for (int32_t k = 0; k + 1 < K; ++k)
                                draw_segment_eps(&g, qx[k], qy[k], qx[k + 1], qy[k + 1], e, blk, K, k);
                            draw_segment_eps(&g, qx[K - 1], qy[K - 1], qx[K - 1], qy[K - 1], e, blk, K, K - 1);
                        } else {
                            for (int32_t k = K - 1; k >= 1; --k)
                                draw_segment_eps(&g, qx[k], qy[k], qx[k - 1], qy[k - 1], e, blk, K, k);
                            draw_segment_eps(&g, qx[0], qy[0], qx[0], qy[0], e, blk, K, 0);
                        }
                    }
                }
            }
        }
        for (int64_t r = 0; r < R; ++r)
            for (int32_t k = 0; k < K; ++k) {
                must[r * S + j0 + k] = bm[r * K + k];
                may[r * S + j0 + k] = bp[r * K + k];
            }
    }
    free(bm); free(bp);
    scene_free(&sc);
    return overflow ? -4 : 0;
}

/* ------------------------------------------------------------------------------------
 * Continuous-time shadow integral (the objective of the height gradient; the paper
 * motivates height trade-offs but gives no formula, so this is the stated reading).
 *
 * Between consecutive steps j, j+1 of a day the sun direction is the great-circle
 * interpolation d(a) = slerp(d_j, d_{j+1}, a), a in [0, 1], and time runs linearly over
 * the step length.  A receiver's shadow time over the interval is
 *     chi(0)                                  if chi(0) == chi(1)
 *     a*        (shadow -> lit at a*)         otherwise, a* the status flip, found by
 *     1 - a*    (lit -> shadow at a*)         bisection on the exact ray test
 * (a second flip inside one interval is not looked for).  S = sum_r w_r * step_minutes *
 * sum over intervals -- shadow-minutes of the region, weighted per receiver.
 * ------------------------------------------------------------------------------------ */
static void slerp_dir(const double* a, const double* b, double theta, double alpha, double* out) {
    if (theta < 1e-12) {
        for (int k = 0; k < 3; ++k) out[k] = a[k] + alpha * (b[k] - a[k]);
    } else {
        const double s = sin(theta), wa = sin((1.0 - alpha) * theta) / s, wb = sin(alpha * theta) / s;
        for (int k = 0; k < 3; ++k) out[k] = wa * a[k] + wb * b[k];
    }
    const double n = sqrt(dot3(out, out));
    for (int k = 0; k < 3; ++k) out[k] /= n;
}

int sao_shadow_integral(const float* tri9, const int32_t* tri_building, int64_t T,
                        const float* pos, int64_t R, const float* dirs,
                        const int32_t* day_start, int32_t D, double step_minutes,
                        const double* weights, int32_t bisect_iters, double* S_out,
                        double* per_receiver, int nthreads) {
    if (T < 0 || R < 0 || D < 0 || !S_out) return -1;
    oscene sc;
    if (scene_init(&sc, tri9, tri_building, T) != 0) { scene_free(&sc); return -3; }
    set_threads(nthreads);
    double total = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t r = 0; r < R; ++r) {
        double o[3], tmin;
        receiver_origin(pos, NULL, r, o, &tmin);
        double acc = 0.0;
        for (int32_t k = 0; k < D; ++k) {
            int prev = -1;
            for (int32_t j = day_start[k]; j + 1 < day_start[k + 1]; ++j) {
                double a[3] = {dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2]};
                double b[3] = {dirs[3 * j + 3], dirs[3 * j + 4], dirs[3 * j + 5]};
                const double na = sqrt(dot3(a, a)), nb = sqrt(dot3(b, b));
                for (int q = 0; q < 3; ++q) { a[q] /= na; b[q] /= nb; }
                const int c0 = prev >= 0 ? prev : any_hit(&sc, o, a, tmin);
                const int c1 = any_hit(&sc, o, b, tmin);
                prev = c1;
                if (c0 == c1) {
                    acc += c0;
                    continue;
                }
                double cd = dot3(a, b);
                if (cd > 1.0) cd = 1.0;
                const double theta = acos(cd);
                double lo = 0.0, hi = 1.0;
                for (int it = 0; it < bisect_iters; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    double d[3];
                    slerp_dir(a, b, theta, mid, d);
                    if (any_hit(&sc, o, d, tmin) == c0) lo = mid; else hi = mid;
                }
                const double astar = 0.5 * (lo + hi);
                acc += c0 ? astar : 1.0 - astar;
            }
        }
        const double v = acc * step_minutes * (weights ? weights[r] : 1.0);
        if (per_receiver) per_receiver[r] = v;
        total += v;
    }
    *S_out = total;
    scene_free(&sc);
    return 0;
}

/* ---------------------------------------------------------------- building contribution
 * Sec. 7.2 ("Building contribution"): the shadow that results from each building.  For a
 * receiver and step, building g casts the shadow when the ray meets one of g's triangles
 * beyond t_min; the nearest caster is the building of the nearest such hit.  Summed over
 * the given receivers and all steps:
 *   casting[g]    pairs (receiver, step) whose ray meets building g
 *   nearest[g]    pairs whose nearest hit lies on building g
 *   unstable[g]   pairs where rotating d_j by +-eps along the sun arc changes whether the
 *                 ray meets g (the parity bar's near-boundary rule, per building)
 *   *unstable_any pairs where that happens for some building
 * Buildings are the tri_building groups; n_buildings must exceed every id. */
static int building_hit(const oscene* s, int32_t g, const double* o, const double* d,
                        double tmin, double* t_best) {
    if (!ray_box(o, d, s->gbox + 6 * g)) return 0;
    int hit = 0;
    for (int64_t i = s->goff[g]; i < s->goff[g + 1]; ++i) {
        double t;
        if (ray_tri(o, d, &s->tri[s->gtri[i]], tmin, &t)) {
            if (!hit || t < *t_best) *t_best = t;
            hit = 1;
        }
    }
    return hit;
}

int sao_building_steps(const float* tri9, const int32_t* tri_building, int64_t T,
                       const float* pos, const float* nrm, int64_t R,
                       const float* dirs, const int32_t* day_start, int32_t D, double eps,
                       int32_t n_buildings, int64_t* casting, int64_t* nearest,
                       int64_t* unstable, int64_t* unstable_any, int nthreads) {
    if (T < 0 || R < 0 || D < 0 || n_buildings < 1) return -1;
    int32_t S = D > 0 ? day_start[D] : 0;
    oscene sc;
    if (scene_init(&sc, tri9, tri_building, T) != 0) { scene_free(&sc); return -3; }
    if (sc.G > n_buildings) { scene_free(&sc); return -1; }
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
    for (int32_t g = 0; g < n_buildings; ++g) casting[g] = nearest[g] = unstable[g] = 0;
    int64_t any_total = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : any_total)
    for (int64_t r = 0; r < R; ++r) {
        double o[3], tmin;
        receiver_origin(pos, nrm, r, o, &tmin);
        for (int32_t j = 0; j < S; ++j) {
            double d[3] = {(double)dirs[3 * j], (double)dirs[3 * j + 1], (double)dirs[3 * j + 2]};
            int32_t best_g = -1;
            double best_t = INFINITY;
            int any_flip = 0;
            for (int32_t g = 0; g < sc.G; ++g) {
                double t = INFINITY;
                const int h = building_hit(&sc, g, o, d, tmin, &t);
                if (h) {
#pragma omp atomic
                    casting[g]++;
                    if (t < best_t) { best_t = t; best_g = g; }
                }
                if (has[j]) {
                    double tp, tm;
                    const int flip = building_hit(&sc, g, o, rot + 6 * j, tmin, &tp) != h ||
                                     building_hit(&sc, g, o, rot + 6 * j + 3, tmin, &tm) != h;
                    if (flip) {
#pragma omp atomic
                        unstable[g]++;
                        any_flip = 1;
                    }
                }
            }
            if (best_g >= 0) {
#pragma omp atomic
                nearest[best_g]++;
            }
            any_total += any_flip;
        }
    }
    *unstable_any = any_total;
    free(rot); free(has);
    scene_free(&sc);
    return 0;
}
