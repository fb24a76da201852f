// sa_internal.cuh -- shared device structures and helpers of libshadowaccrual.
//
// Geometry conventions follow the paper's statement of the problem (Sec. 3): the sun is a
// directional light, each step j has a unit direction d_j toward the sun, and a receiver
// is in shadow at step j when the ray from it toward the sun meets a triangle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "shadowaccrual.h"

namespace sa {

// ------------------------------------------------------------- bounds-checked build
// Built with -DSA_CHECKED, the kernels range-check every index they take from data (a
// BVH leaf's triangle, an escape link, a binned triangle or receiver, a permutation
// entry, a tile cell) before using it.  The first index out of range is recorded in a
// device word of its translation unit -- the site, the index and its bound -- and replaced
// by an index in range (an escape link by the end of the list), so that no access leaves
// its buffer and no loop runs on; the public calls then return SA_ERR_INTERNAL.  Without
// the flag the checks compile to nothing.
enum CheckSite {
    CK_NONE = 0, CK_TRACE_LEAF, CK_TRACE_ESCAPE, CK_RASTER_BIN, CK_RASTER_CELL, CK_BIN_SLOT,
    CK_POINTS_TRI, CK_POINTS_RECV, CK_POINTS_PERM, CK_POINTS_MASK, CK_CONTRIB_LEAF,
    CK_CONTRIB_ESCAPE, CK_CONTRIB_BUILDING, CK_CONTRIB_CELL, CK_IAM_LEAF, CK_IAM_ESCAPE, CK_ADJ_LEAF,
    CK_ADJ_ESCAPE, CK_SITES
};
const char* check_site_name(int site);
// Reader of one translation unit's word: copies [site, index, bound] into w and, if a
// violation is recorded and reset != 0, clears it.
typedef cudaError_t (*CheckReader)(unsigned long long* w, int reset);
int register_check_reader(CheckReader r);
// The first recorded violation over all translation units (w[0] = 0: none); clears them.
cudaError_t read_check_words(unsigned long long* w);

}  // namespace sa

#ifdef SA_CHECKED
namespace {
__device__ unsigned long long g_sa_check[3];
__device__ __forceinline__ long long sa_checked_index(long long i, long long n, int site) {
    if (i >= 0 && i < n) return i;
    if (atomicCAS(&g_sa_check[0], 0ull, (unsigned long long)site) == 0ull) {
        g_sa_check[1] = (unsigned long long)i;
        g_sa_check[2] = (unsigned long long)n;
    }
    return 0;
}
__device__ __forceinline__ int sa_checked_escape(int esc, int i, int n, int site) {
    if (esc > i && esc <= n) return esc;
    if (atomicCAS(&g_sa_check[0], 0ull, (unsigned long long)site) == 0ull) {
        g_sa_check[1] = (unsigned long long)(long long)esc;
        g_sa_check[2] = (unsigned long long)(long long)n;
    }
    return n;
}
cudaError_t sa_read_check_tu(unsigned long long* w, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(w, g_sa_check, sizeof(unsigned long long) * 3);
    if (e == cudaSuccess && reset && w[0]) {
        const unsigned long long z[3] = {0ull, 0ull, 0ull};
        e = cudaMemcpyToSymbol(g_sa_check, z, sizeof(z));
    }
    return e;
}
const int g_sa_check_registered = sa::register_check_reader(&sa_read_check_tu);
}  // namespace
// index i checked against [0, n); an escape link checked against (i, n]
#define SA_CHK(i, n, site) sa_checked_index((long long)(i), (long long)(n), (int)(site))
#define SA_ESC(esc, i, n, site) sa_checked_escape((esc), (i), (n), (int)(site))
#else
#define SA_CHK(i, n, site) (i)
#define SA_ESC(esc, i, n, site) (esc)
#endif
// a node's triangle: -1 for an inner node, else checked against [0, T)
#define SA_LEAF(tri, T, site) ((tri) < 0 ? (tri) : (int)SA_CHK((tri), (T), (site)))

namespace sa {

// Stream-ordered scratch from the library's own memory pool (one per device, created on
// first use).  The pool keeps up to 4 GiB reserved across synchronisations, so calls that
// repeat do not map and unmap their scratch every time; free with cudaFreeAsync.
cudaError_t scratch_alloc_bytes(void** p, size_t bytes, cudaStream_t st);
template <class T>
inline cudaError_t scratch_alloc(T** p, size_t bytes, cudaStream_t st) {
    return scratch_alloc_bytes(reinterpret_cast<void**>(p), bytes, st);
}

// Two FP32 values in one 64-bit register.  The packed multiply-add and multiply of sm_100
// and later (fma.rn.f32x2, mul.rn.f32x2) round each half exactly as the scalar instruction
// does, so code may pair two independent steps per instruction without changing a result.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// three-input minimum and maximum (one instruction on sm_100 and later; no NaN reaches
// them here)
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

constexpr float kGroundTmin = 1e-3f;     // ground receivers: hits closer than 1 mm ignored
constexpr float kFacadeOffset = 1e-2f;   // facade receivers start 1 cm along their normal
constexpr int kMaxBlock = 64;            // steps per accrual block (one uint64 mask)

// ---------------------------------------------------------------------------- sun
// Per-step constants (one sun direction), read warp-uniformly.
struct StepConst {
    float dx, dy, dz;   // unit direction toward the sun
    float ux, uy;       // ground slope: d_xy / d_z (a point at height z shadows p - z * u)
    float ix, iy, iz;   // 1 / d (safe against zero components)
    float Sx, Sy, Sz;   // watertight shear for the major axis kz (Woop et al. 2013)
    int kz;             // major axis of |d|
    int pad0, pad1, pad2, pad3;
};

// Per-block constants: a block is <= 64 consecutive steps of one day.
// The block's rays from one origin form a thin fan ("wedge") around the plane through
// its first and last directions: n is that plane's unit normal, s_off bounds |n . d_j|,
// and g1, g2 are in-plane normals of the two half-spaces that bound the in-plane angles
// of the block's directions.  psi[k] is the in-plane angle of step j0 + k measured in the
// orthonormal basis (e1, e2) of the plane, relative to the middle of the block.
struct BlockConst {
    int j0, K;              // first step, number of steps
    int new_day;            // 1 if the block is the first of its day (runs restart)
    int monotone;           // 1 if psi is non-decreasing over the block
    int mask_block;         // block of the requested partition that holds these steps
    int mask_bit;           // bit of step j0 within that block's mask
    int pad_i0, pad_i1;
    float uxlo, uxhi, uylo, uyhi;   // slope box of the block's steps
    float nx, ny, nz, s_off;
    float g1x, g1y, g1z, wedge_ok;  // wedge_ok = 0: fall back to the slope box only
    float g2x, g2y, g2z, psi_eps;
    float e1x, e1y, e1z, pad_f0;
    float e2x, e2y, e2z, pad_f1;
    float dlo[3], dhi[3];           // component-wise box of the block's directions
    float psi[kMaxBlock];
};

// Can some ray of the block (directions inside [dlo, dhi]) from o meet the plane of the
// triangle (a, b, c) at t > 0?  If o lies strictly on one side and every direction in the
// box points away from the plane, no ray of the block can hit the triangle.
__device__ __forceinline__ bool plane_reachable(const float3& o, const float4& a, const float4& b,
                                                const float4& c, const BlockConst& bc) {
    const float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
    const float vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
    const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    const float s0 = nx * (o.x - a.x) + ny * (o.y - a.y) + nz * (o.z - a.z);
    const float lo = fminf(nx * bc.dlo[0], nx * bc.dhi[0]) + fminf(ny * bc.dlo[1], ny * bc.dhi[1]) +
                     fminf(nz * bc.dlo[2], nz * bc.dhi[2]);
    const float hi = fmaxf(nx * bc.dlo[0], nx * bc.dhi[0]) + fmaxf(ny * bc.dlo[1], ny * bc.dhi[1]) +
                     fmaxf(nz * bc.dlo[2], nz * bc.dhi[2]);
    // relative slack for rounding of s0 and of the bounds
    const float tol = 1e-5f * (fabsf(nx) + fabsf(ny) + fabsf(nz)) *
                      (1.f + fabsf(o.x - a.x) + fabsf(o.y - a.y) + fabsf(o.z - a.z));
    if (s0 > tol && lo > tol) return false;
    if (s0 < -tol && hi < -tol) return false;
    return true;
}

// ------------------------------------------------------------- fan of a block's rays
// Conservative test of a box against the block's ray fan from origin o (see BlockConst).
// front: the receiver's normal nf has nf . d > 0 for every direction of the block, so all
// rays stay in front of the receiver's wall plane and boxes wholly behind it are skipped.
__device__ __forceinline__ bool fan_box(const float3& o, const BlockConst& bc, const float4& lo,
                                        const float4& hi, bool front = false,
                                        const float3& nf = float3{0.f, 0.f, 0.f}) {
    if (hi.z < o.z) return false;                       // every ray climbs
    const float cx = 0.5f * (lo.x + hi.x) - o.x, cy = 0.5f * (lo.y + hi.y) - o.y,
                cz = 0.5f * (lo.z + hi.z) - o.z;
    const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
    if (front && nf.x * cx + nf.y * cy + nf.z * cz + fabsf(nf.x) * hx + fabsf(nf.y) * hy +
                     fabsf(nf.z) * hz < -1e-4f)
        return false;
    const float R = sqrtf(cx * cx + cy * cy + cz * cz) + sqrtf(hx * hx + hy * hy + hz * hz);
    const float slack = 1e-5f * R + 1e-4f;
    // in-plane half-spaces
    const float g1 = bc.g1x * cx + bc.g1y * cy + bc.g1z * cz +
                     fabsf(bc.g1x) * hx + fabsf(bc.g1y) * hy + fabsf(bc.g1z) * hz;
    const float g2 = bc.g2x * cx + bc.g2y * cy + bc.g2z * cz +
                     fabsf(bc.g2x) * hx + fabsf(bc.g2y) * hy + fabsf(bc.g2z) * hz;
    if (g1 < -slack || g2 < -slack) return false;
    // out of plane: |n . x| <= s_off |x| on the fan
    const float nc = bc.nx * cx + bc.ny * cy + bc.nz * cz;
    const float rn = fabsf(bc.nx) * hx + fabsf(bc.ny) * hy + fabsf(bc.nz) * hz;
    const float lim = bc.s_off * R + slack;
    return (nc - rn <= lim) && (nc + rn >= -lim);
}

// Slope-box version (used when the block's wedge is degenerate): a point at height z above
// o on one of the rays lies at o.xy + (z - o.z) * u with u in the block's slope box.
__device__ __forceinline__ bool slope_box(const float3& o, const BlockConst& bc, const float4& lo,
                                          const float4& hi) {
    const float h1 = hi.z - o.z;
    if (h1 < 0.f) return false;
    const float h0 = fmaxf(lo.z - o.z, 0.f);
    const float xa = fminf(h0 * bc.uxlo, h1 * bc.uxlo), xb = fmaxf(h0 * bc.uxhi, h1 * bc.uxhi);
    const float ya = fminf(h0 * bc.uylo, h1 * bc.uylo), yb = fmaxf(h0 * bc.uyhi, h1 * bc.uyhi);
    const float sl = 1e-4f + 1e-6f * (fabsf(o.x) + fabsf(o.y) + h1);
    return (o.x + xa <= hi.x + sl) && (o.x + xb >= lo.x - sl) && (o.y + ya <= hi.y + sl) &&
           (o.y + yb >= lo.y - sl);
}

// Steps of the block whose in-plane angle can meet the triangle: [*ka, *kb] (inclusive).
__device__ __forceinline__ void candidate_steps(const float3& o, const BlockConst& bc,
                                                const float* psi, const float4& a,
                                                const float4& b, const float4& c, int* ka,
                                                int* kb) {
    *ka = 0;
    *kb = bc.K - 1;
    if (bc.wedge_ok == 0.f || !bc.monotone) return;
    float ang[3];
    const float4* v[3] = {&a, &b, &c};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float x = v[q]->x - o.x, y = v[q]->y - o.y, z = v[q]->z - o.z;
        const float p = bc.e1x * x + bc.e1y * y + bc.e1z * z;
        const float s = bc.e2x * x + bc.e2y * y + bc.e2z * z;
        if (p * p + s * s < 1e-12f) return;             // vertex on the fan's axis line
        ang[q] = atan2f(s, p);
    }
    const float amin = fminf(ang[0], fminf(ang[1], ang[2]));
    const float amax = fmaxf(ang[0], fmaxf(ang[1], ang[2]));
    if (amax - amin >= 3.1f) return;                    // may surround the origin: all steps
    const float lo = amin - bc.psi_eps, hi = amax + bc.psi_eps;
    // first k with psi[k] >= lo, last k with psi[k] <= hi
    int l = 0, r = bc.K;
    while (l < r) { int m = (l + r) >> 1; if (psi[m] >= lo) r = m; else l = m + 1; }
    *ka = l;
    l = 0; r = bc.K;
    while (l < r) { int m = (l + r) >> 1; if (psi[m] > hi) r = m; else l = m + 1; }
    *kb = l - 1;
}

// ---------------------------------------------------------------------------- scene
// BVH nodes in depth-first order, two float4 each:
//   n0 = (lo.x, lo.y, lo.z, escape as int)   escape = index of the next node after the subtree
//   n1 = (hi.x, hi.y, hi.z, tri as int)      tri = leaf triangle (leaf order) or -1
// Triangles in leaf order, three float4 each: (v0, building), (v1, original index), (v2, 0).
struct DevScene {
    const float4* nodes;
    const float4* tris;
    int n_nodes;
    int T;
    int closed;     // every building is a closed, outward-oriented solid
};

// ------------------------------------------------------------------- reduction state
// Running gross / continuous state of one receiver (Sec. 3.1 and the prefix/max/suffix
// stitching of Sec. 6 applied to consecutive blocks of a day).
struct RunState {
    int gross, run, best;
};

__device__ __forceinline__ int longest_run64(uint64_t m) {
    int n = 0;
    while (m) { m &= m << 1; ++n; }
    return n;
}

// Fold the mask of one block (bits 0..K-1 = its steps in order) into the state.
__device__ __forceinline__ void stitch(RunState& s, uint64_t m, int K, int new_day) {
    if (new_day) s.run = 0;
    const uint64_t full = (K >= 64) ? ~0ull : ((1ull << K) - 1ull);
    m &= full;
    s.gross += __popcll(m);
    if (m == full) {
        s.run += K;
        s.best = max(s.best, s.run);
        return;
    }
    const int prefix = __ffsll((long long)~m) - 1;              // ones from bit 0 upward
    const uint64_t zeros = (~m) & full;                         // the block's unshadowed steps
    const int suffix = K - 1 - (63 - __clzll((long long)zeros));  // ones below bit K-1
    s.best = max(s.best, s.run + prefix);
    s.best = max(s.best, longest_run64(m));
    s.run = suffix;
}

// ------------------------------------------------------------------ float helpers
template <int A> __device__ __forceinline__ float comp(const float4& v);
template <> __device__ __forceinline__ float comp<0>(const float4& v) { return v.x; }
template <> __device__ __forceinline__ float comp<1>(const float4& v) { return v.y; }
template <> __device__ __forceinline__ float comp<2>(const float4& v) { return v.z; }
template <int A> __device__ __forceinline__ float comp3(const float3& v);
template <> __device__ __forceinline__ float comp3<0>(const float3& v) { return v.x; }
template <> __device__ __forceinline__ float comp3<1>(const float3& v) { return v.y; }
template <> __device__ __forceinline__ float comp3<2>(const float3& v) { return v.z; }

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013) specialised for the
// major axis KZ.  The edge functions use explicit round-to-nearest products and
// differences (no contraction), so the value computed for an edge shared by two
// triangles is the exact negation in the other and a ray through the edge hits at
// least one of them.  Zero edge values count as inside (inclusive, like the oracle).
// woop_td: false when the ray's line misses the triangle or lies in its plane; otherwise
// T and det, the hit distance being T / det in units of |d|.
template <int KZ>
__device__ __forceinline__ bool woop_td(const float3& o, const float4& a, const float4& b,
                                        const float4& c, float Sx, float Sy, float Sz,
                                        float& T, float& det) {
    constexpr int KX = (KZ + 1) % 3, KY = (KZ + 2) % 3;
    const float az = comp<KZ>(a) - comp3<KZ>(o);
    const float bz = comp<KZ>(b) - comp3<KZ>(o);
    const float cz = comp<KZ>(c) - comp3<KZ>(o);
    const float ax = fmaf(-Sx, az, comp<KX>(a) - comp3<KX>(o));
    const float ay = fmaf(-Sy, az, comp<KY>(a) - comp3<KY>(o));
    const float bx = fmaf(-Sx, bz, comp<KX>(b) - comp3<KX>(o));
    const float by = fmaf(-Sy, bz, comp<KY>(b) - comp3<KY>(o));
    const float cx = fmaf(-Sx, cz, comp<KX>(c) - comp3<KX>(o));
    const float cy = fmaf(-Sy, cz, comp<KY>(c) - comp3<KY>(o));
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    det = U + V + W;
    if (det == 0.f) return false;
    T = U * (Sz * az) + V * (Sz * bz) + W * (Sz * cz);
    return true;
}

// the watertight test: does the ray meet the triangle beyond tmin?
template <int KZ>
__device__ __forceinline__ bool hit_tri(const float3& o, const float4& a, const float4& b,
                                        const float4& c, float Sx, float Sy, float Sz,
                                        float tmin) {
    float T, det;
    if (!woop_td<KZ>(o, a, b, c, Sx, Sy, Sz, T, det)) return false;
    return det > 0.f ? (T > tmin * det) : (T < tmin * det);
}

// the same decision, returning the hit distance T / det (in units of |d|), or -1
template <int KZ>
__device__ __forceinline__ float hit_tri_dist(const float3& o, const float4& a, const float4& b,
                                              const float4& c, float Sx, float Sy, float Sz,
                                              float tmin) {
    float T, det;
    if (!woop_td<KZ>(o, a, b, c, Sx, Sy, Sz, T, det)) return -1.f;
    const bool ahead = det > 0.f ? (T > tmin * det) : (T < tmin * det);
    return ahead ? T / det : -1.f;
}

__device__ __forceinline__ bool hit_tri_any(int kz, const float3& o, const float4& a,
                                            const float4& b, const float4& c,
                                            const StepConst& s, float tmin) {
    if (kz == 2) return hit_tri<2>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
    if (kz == 0) return hit_tri<0>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
    return hit_tri<1>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
}

__device__ __forceinline__ float hit_dist_any(int kz, const float3& o, const float4& a,
                                              const float4& b, const float4& c,
                                              const StepConst& s, float tmin) {
    if (kz == 2) return hit_tri_dist<2>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
    if (kz == 0) return hit_tri_dist<0>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
    return hit_tri_dist<1>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
}

// Slab test of the ray o + t d, t in [0, inf), against a (padded) box.
__device__ __forceinline__ bool hit_box(const float3& o, float ix, float iy, float iz,
                                        const float4& lo, const float4& hi) {
    float tx0 = (lo.x - o.x) * ix, tx1 = (hi.x - o.x) * ix;
    float ty0 = (lo.y - o.y) * iy, ty1 = (hi.y - o.y) * iy;
    float tz0 = (lo.z - o.z) * iz, tz1 = (hi.z - o.z) * iz;
    float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    return tn <= tf * 1.0000005f;
}

// Plücker form of the exact ray/triangle test for one origin and many steps.  For the
// line through o along d, the side of edge v -> v' is  d . ((v - o) x (v' - o)):  the
// moment m_e = (v - o) x (v' - o) depends only on the origin and the edge, so a triangle
// is set up once per receiver and each step costs three dot products.  The cross product
// is formed from correctly rounded products and differences, so the reversed edge gives
// exactly the negated moment (up to the sign of zero): a line through an edge shared by
// two triangles sees exactly negated values and is inside at least one (watertight; zero
// counts as inside on both sides).  The hit distance t = ((a - o) . n) / (d . n) must
// exceed t_min.  Every quantity is formed with explicit roundings, so all kernels that use
// these helpers take identical decisions.
struct PluckerTri {
    float m[3][3];
    float nx, ny, nz, aon;
};

__device__ __forceinline__ void plucker_edge(const float3& o, const float4& v, const float4& w,
                                             float* m) {
    const float px = __fsub_rn(v.x, o.x), py = __fsub_rn(v.y, o.y), pz = __fsub_rn(v.z, o.z);
    const float qx = __fsub_rn(w.x, o.x), qy = __fsub_rn(w.y, o.y), qz = __fsub_rn(w.z, o.z);
    m[0] = __fsub_rn(__fmul_rn(py, qz), __fmul_rn(pz, qy));
    m[1] = __fsub_rn(__fmul_rn(pz, qx), __fmul_rn(px, qz));
    m[2] = __fsub_rn(__fmul_rn(px, qy), __fmul_rn(py, qx));
}

// the triangle's (unnormalised) normal (b - a) x (c - a); independent of the origin
__device__ __forceinline__ float3 plucker_normal(const float4& a, const float4& b, const float4& c) {
    const float ux = __fsub_rn(b.x, a.x), uy = __fsub_rn(b.y, a.y), uz = __fsub_rn(b.z, a.z);
    const float vx = __fsub_rn(c.x, a.x), vy = __fsub_rn(c.y, a.y), vz = __fsub_rn(c.z, a.z);
    return make_float3(__fsub_rn(__fmul_rn(uy, vz), __fmul_rn(uz, vy)),
                       __fsub_rn(__fmul_rn(uz, vx), __fmul_rn(ux, vz)),
                       __fsub_rn(__fmul_rn(ux, vy), __fmul_rn(uy, vx)));
}

// set-up with the normal given (from plucker_normal of the same triangle)
__device__ __forceinline__ PluckerTri plucker_setup_n(const float3& o, const float4& a,
                                                      const float4& b, const float4& c,
                                                      const float3& n) {
    PluckerTri p;
    plucker_edge(o, a, b, p.m[0]);
    plucker_edge(o, b, c, p.m[1]);
    plucker_edge(o, c, a, p.m[2]);
    p.nx = n.x; p.ny = n.y; p.nz = n.z;
    p.aon = fmaf(n.z, __fsub_rn(a.z, o.z), fmaf(n.y, __fsub_rn(a.y, o.y), __fmul_rn(n.x, __fsub_rn(a.x, o.x))));
    return p;
}

__device__ __forceinline__ PluckerTri plucker_setup(const float3& o, const float4& a,
                                                    const float4& b, const float4& c) {
    return plucker_setup_n(o, a, b, c, plucker_normal(a, b, c));
}

// d . m and d . n in a fixed order, so a negated m gives an exactly negated value
__device__ __forceinline__ bool plucker_hit(const PluckerTri& p, float dx, float dy, float dz,
                                            float tmin) {
    const float s0 = fmaf(dz, p.m[0][2], fmaf(dy, p.m[0][1], __fmul_rn(dx, p.m[0][0])));
    const float s1 = fmaf(dz, p.m[1][2], fmaf(dy, p.m[1][1], __fmul_rn(dx, p.m[1][0])));
    const float s2 = fmaf(dz, p.m[2][2], fmaf(dy, p.m[2][1], __fmul_rn(dx, p.m[2][0])));
    const bool inside = (s0 >= 0.f && s1 >= 0.f && s2 >= 0.f) || (s0 <= 0.f && s1 <= 0.f && s2 <= 0.f);
    if (!inside) return false;
    const float nd = fmaf(dz, p.nz, fmaf(dy, p.ny, __fmul_rn(dx, p.nx)));
    if (nd == 0.f) return false;
    const float lim = __fmul_rn(tmin, nd);
    return nd > 0.f ? (p.aon > lim) : (p.aon < lim);
}

// the same decision as plucker_hit, evaluated without early exits, so the steps of a run
// form independent chains
__device__ __forceinline__ bool plucker_hit_all(const PluckerTri& p, float dx, float dy, float dz,
                                                float tmin) {
    const float s0 = fmaf(dz, p.m[0][2], fmaf(dy, p.m[0][1], __fmul_rn(dx, p.m[0][0])));
    const float s1 = fmaf(dz, p.m[1][2], fmaf(dy, p.m[1][1], __fmul_rn(dx, p.m[1][0])));
    const float s2 = fmaf(dz, p.m[2][2], fmaf(dy, p.m[2][1], __fmul_rn(dx, p.m[2][0])));
    const float nd = fmaf(dz, p.nz, fmaf(dy, p.ny, __fmul_rn(dx, p.nx)));
    const bool inside = fminf(s0, fminf(s1, s2)) >= 0.f || fmaxf(s0, fmaxf(s1, s2)) <= 0.f;
    const float lim = __fmul_rn(tmin, nd);
    const bool ahead = (nd > 0.f && p.aon > lim) || (nd < 0.f && p.aon < lim);
    return inside && ahead;
}

// --------------------------------------------------------------- host-side launchers
// Receivers as the kernels see them.
struct DevRecv {
    int is_grid;
    // grid
    float x0, y0, dx;
    int nx, ny;
    // points, in Morton order: origin (already offset) and t_min; perm = input index
    const float4* orig;
    const float4* nrm;      // facade normals in the same order, or null
    const int* perm;
    long long R;
};

struct DevSun {
    const StepConst* steps;
    const BlockConst* blocks;
    int S, n_blocks;
};

// outputs / state (state buffers hold gross, run, best per receiver in output order)
struct DevOut {
    int* gross;
    float* minutes;
    int* continuous;
    int* run;            // scratch: running length at the end of the last processed block
    float step_minutes;
    int accumulate_into;
    int write_final;     // 1: this launch finishes the call (write minutes)
    uint64_t* masks;     // optional [n_blocks][R]
    unsigned long long* stats;   // optional work counters (box tests, triangle tests, ...)
};

cudaError_t launch_sweep_trace(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                               const DevOut& out, cudaStream_t st);
cudaError_t launch_accrual_trace(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                 const DevOut& out, cudaStream_t st);
// traversal mode of the sweep (which = 0) and accrual (which = 1) kernels
void set_trace_mode(int which, int mode);
int get_trace_mode(int which);
// ground raster; `sun` may be the per-step partition (K = 1 blocks) for SA_SWEEP_RASTER
cudaError_t launch_raster_ground(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                 const DevOut& out, cudaStream_t st);

// Extruded convex footprints kept on the device (scenes built from footprints).
struct FootprintSet {
    int B;
    const float2* xy;      // footprint vertices, CCW per building
    const int* fp_off;     // [B + 1] offsets into xy
    const int* bands;      // [B] wall bands
    const int* vert_off;   // [B + 1] mesh vertex offsets
    const int* tri_off;    // [B + 1] mesh triangle offsets
    long long n_verts, n_tris;
};
cudaError_t extrude_footprints(const FootprintSet& fs, const float* d_heights, float* d_verts,
                               int* d_tris, int* d_tri_b, cudaStream_t st);
// d(shadow-minutes of a ground grid)/d(heights); d_S (nullable) receives S itself
cudaError_t launch_height_grad(const DevScene& sc, const FootprintSet& fs, const float* d_heights,
                               const DevRecv& rc, const DevSun& sun, float step_minutes,
                               const float* weights, float* dS_dh, double* d_S, cudaStream_t st);

// building contribution over a polygonal region (sa_analysis.cu); casting_out and
// nearest_out are host arrays of n_buildings, stats_out two host counters (cell-steps past
// 32 buildings, shadowed cell-steps whose ray met no building)
cudaError_t launch_building_contribution(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                         const std::vector<BlockConst>& runs, int n_buildings,
                                         const float* poly_xy, int n, double* casting_out,
                                         double* nearest_out, unsigned long long* stats_out,
                                         cudaStream_t st);

// direction graph (sa_graph.cu): edge of each block (blocks given by first step j0 and
// length K over dirs [S][3]), the block each edge's map is computed from (its middle
// block), and each edge's weight
void direction_graph(const float* dirs, int n_blocks, const int* j0, const int* K, double bin_deg,
                     std::vector<int>& edge, std::vector<int>& rep, std::vector<int>& weight);
// per (edge, receiver) run summary of masks [n_edges][R] into summary [n_edges][R]
cudaError_t launch_edge_summary(const unsigned long long* masks, long long R, int n_edges,
                                const int* d_edge_K, unsigned* summary, cudaStream_t st);
// gross / minutes / continuous per receiver from the summaries along each day's path; the
// walk holds every block in time order as edge | K << 20 | (first block of a day) << 27
cudaError_t launch_graph_reduce(const unsigned* summary, long long R, const int* d_walk, int n_walk,
                                float step_minutes, int* gross, float* minutes, int* continuous,
                                cudaStream_t st);

// batched scenarios (device-side descriptors; see sa_raster.cu)
struct BatchInterval {
    const StepConst* steps;
    const BlockConst* blocks;
    int n_blocks;
    const unsigned* offsets;      // [n_blocks][tiles] base bins
    const unsigned* counts;
    const int* bins;
    const int* base_counts;       // [R] gross of the base city (nullable)
    long long out_base;           // offset of this interval's outputs
};
struct BatchVariant {
    int tower_off, n_tower;       // triangles in the tower list
    int rem_off, n_rem;           // ids in the removed list
    int ix0, iy0, nx, ny;         // region in cells of the base grid
    long long out_off;            // offset within an interval's outputs
};
// Base bins of every block of one interval over all tiles (device, caller frees with
// cudaFree): offsets / counts [n_blocks][tiles], bins [total].
cudaError_t build_bins(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                       unsigned** offsets, unsigned** counts, int** bins, cudaStream_t st);
struct BatchLaunch {
    DevScene base;
    DevRecv grid;
    const BatchInterval* intervals;
    const BatchVariant* variants;
    const int4* items;
    int n_items;
    unsigned* counter;
    const int* removed;
    const float4* tower_tris;
    int* counts_out;
    int* impact_out;
    unsigned long long* stats;
    int ctas;                     // persistent CTAs
    int run;                      // raster steps per work unit
};
void set_raster_run(int run);
int get_raster_run();
// steps per light-space map of point receivers (1..16)
void set_point_run(int run);
int get_point_run();
void set_batch_tile_skip(int on);
int get_batch_tile_skip();
cudaError_t launch_batch(const BatchLaunch& bl, cudaStream_t st);

// shadow accrual map of point receivers in light space (scene_box, recv_box: lo.xyz hi.xyz)
cudaError_t launch_sam_points(const DevScene& sc, const float* scene_box, const DevRecv& rc,
                              const float* recv_box, const DevSun& sun,
                              const std::vector<BlockConst>& h_blocks,
                              const std::vector<StepConst>& h_steps, const DevOut& out,
                              cudaStream_t st);

// inverse accrual map of a ground grid (h_blocks: host copy of the block constants)
cudaError_t launch_iam(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                       const BlockConst* h_blocks, int L, const DevOut& out, cudaStream_t st);

// LBVH build (device), returns node / triangle arrays owned by the caller
struct LbvhBuild {
    float4* nodes;   // [2 * n_nodes]
    float4* tris;    // [3 * T]
    int n_nodes;
};
// Checks of an input mesh made on the device while its BVH is built: the first vertex
// with a non-finite coordinate and the first triangle with a vertex index outside
// [0, nv) or a building id outside [0, n_buildings) (-1: none), and the bounds (lo xyz,
// hi xyz) of the vertices the triangles reference (zeros without triangles).
struct MeshCheck {
    long long bad_vertex;
    long long bad_tri;
    float box[6];
};
// Builds the BVH of nt triangles (synchronises st).  With `check`, the mesh is validated
// as described above; a failed check still returns cudaSuccess with the BVH built from
// the readable part, for the caller to free.  Without it the mesh is trusted.
cudaError_t build_lbvh(const float* d_verts, long long nv, const int* d_tris, long long nt,
                       const int* d_tri_building, LbvhBuild* out, cudaStream_t st,
                       int n_buildings = 1, MeshCheck* check = nullptr);

// Morton order of point receivers: fills perm (sorted -> input index) and sorted origins
// (synchronises st).  bad_out[0] / [1]: first point with a non-finite position / normal
// (-1: none); box_out: bounds (lo xyz, hi xyz) of the offset origins.
cudaError_t sort_points(const float* d_pos, const float* d_nrm, long long n, float4* d_orig,
                        float4* d_nrm_sorted, int* d_perm, cudaStream_t st, long long* bad_out,
                        float* box_out);

// radix sort of (key, value) pairs by key (stable, 32-bit keys), in place via scratch
cudaError_t radix_sort_pairs(unsigned* keys, unsigned* vals, long long n, cudaStream_t st);

// exclusive scan of n uint32 (in place); writes the total to *d_total if non-null
cudaError_t exclusive_scan_u32(unsigned* data, long long n, unsigned* d_total, cudaStream_t st);
// the same scan with caller-provided partials (scan_partials(n) words); allocates nothing
long long scan_partials(long long n);
cudaError_t exclusive_scan_u32_with(unsigned* data, long long n, unsigned* partial,
                                    unsigned* d_total, cudaStream_t st);

// The ground accrual raster with every scratch buffer carved from `scratch` (bytes long,
// 256-byte aligned); allocates nothing.  *capacity_error is set to 1 (and cudaSuccess
// returned) when the receivers' state or a single block's bins do not fit.
cudaError_t launch_raster_ground_in(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                    const DevOut& out, cudaStream_t st, unsigned char* scratch,
                                    size_t bytes, int* capacity_error);

}  // namespace sa

namespace sa {

// Per-kernel device timing: while enabled, a CUDA event pair is recorded on the launching
// stream around each launch of the library's main kernels (not inside stream capture).
enum KernelClass { KT_RASTER = 0, KT_SAM_POINTS = 1, KT_ACCRUAL = 2, KT_SWEEP = 3, KT_IAM = 4,
                   KT_GRAPH = 5, KT_RASTER_BIN = 6, KT_CONTRIB = 7 };
void set_kernel_timing(int on);
int get_kernel_timing();
struct KernelTimer {
    int id;
    cudaStream_t st;
    void* begin;     // cudaEvent_t, or null when timing is off
    KernelTimer(int id, cudaStream_t st);
    ~KernelTimer();  // records the end event and queues the pair
    KernelTimer(const KernelTimer&) = delete;
    KernelTimer& operator=(const KernelTimer&) = delete;
};
// waits for the queued pairs, adds their durations and counts into ms[id] and n[id]
// (n_classes entries), and empties the queue
cudaError_t collect_kernel_times(double* ms, long long* n, int n_classes);

}  // namespace sa
