// sa_adjoint.cu -- derivative of the region's shadow-minutes with respect to building heights.
//
// Objective (continuous time between the sun steps): between steps j and j+1 of a day the
// sun follows the great circle d(a) = slerp(d_j, d_{j+1}, a), a in [0, 1], over one step
// length dt.  A ground receiver contributes dt * chi where the status does not change over
// the interval and dt * a* (shadow -> lit) or dt * (1 - a*) (lit -> shadow) where it flips
// at a*.  S = sum_r w_r * (those contributions).  Heights only move flip times, so
//     dS/dh_b = sum over flips f caused by building b of  w_r * dt * s_f * da*/dh_b,
// s_f = +1 for shadow -> lit and -1 for lit -> shadow.
//
// Kernels:
//   k_flip_count / k_flip_fill  walk each receiver's forward step masks (from the accrual
//                               raster) and list the intervals whose end statuses differ;
//                               intervals without a flip add dt * chi to S directly.
//   k_flip_solve                per flip, in FP64: find the buildings that shadow the
//                               receiver at the shadowed end (FP32 BVH traversal), locate
//                               each one's flip a*_b on the exact prism test, in a
//                               projective parameter of the same arc in which every prism
//                               constraint is linear: an FP32 bisection brackets the flip,
//                               the pair of constraints that close the entry interval there
//                               gives it in closed form, and FP64 statuses on both sides
//                               confirm it (otherwise an FP64 bisection finds it); then
//                               take the first (lit -> shadow) or last (shadow -> lit), and
//                               if the flip is the shadow of a roof edge e of building b
//                               crossing the receiver, differentiate the grazing condition
//                                  G(a, h) = A_e + h B_e(a) = 0,  B_e(a) = c_e x u(a),
//                               u = d_xy / d_z:  da*/dh = -B_e / (h dB_e/da).  A flip caused
//                               by a vertical edge does not depend on h.
#include <float.h>
#include <string.h>

#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxCand = 8;
constexpr int kBisect = 40;   // halvings of [0, 1]: the flip to 1e-12 of a step
constexpr int kLinEdges = 8;  // footprints up to this many edges take the linear form
constexpr int kBisectF = 22;  // FP32 halvings that bracket a flip before its closed form
constexpr double kSide = 1e-10;   // FP64 status checks this far on both sides of a root

// Visits every interval (j, j+1) inside a day of receiver r: f(j, chi0, chi1).
template <class F>
__device__ void for_intervals(const unsigned long long* masks, long long R, const BlockConst* blocks,
                              int n_blocks, long long r, F f) {
    int prev = -1;
    int prev_j = -1;
    for (int b = 0; b < n_blocks; ++b) {
        const BlockConst& bc = blocks[b];
        if (bc.new_day) prev = -1;
        const unsigned long long m = masks[(long long)bc.mask_block * R + r] >> bc.mask_bit;
        for (int k = 0; k < bc.K; ++k) {
            const int c = (int)((m >> k) & 1ull);
            if (prev >= 0) f(prev_j, prev, c);
            prev = c;
            prev_j = bc.j0 + k;
        }
    }
}

__global__ void k_flip_count(const unsigned long long* __restrict__ masks, long long R,
                             const BlockConst* __restrict__ blocks, int n_blocks,
                             const float* __restrict__ weights, double dt,
                             unsigned* __restrict__ counts, double* __restrict__ S) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (r < R) {
        unsigned n = 0;
        double steady = 0.0;
        for_intervals(masks, R, blocks, n_blocks, r, [&](int, int c0, int c1) {
            if (c0 != c1) ++n; else steady += c0;
        });
        counts[r] = n;
        s = steady * dt * (weights ? (double)weights[r] : 1.0);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(S, s);
}

__global__ void k_flip_fill(const unsigned long long* __restrict__ masks, long long R,
                            const BlockConst* __restrict__ blocks, int n_blocks,
                            const unsigned* __restrict__ offsets, int4* __restrict__ flips) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    unsigned w = offsets[r];
    for_intervals(masks, R, blocks, n_blocks, r, [&](int j, int c0, int c1) {
        if (c0 != c1) flips[w++] = make_int4((int)(r & 0x7fffffff), (int)(r >> 31), j, c0);
    });
}

struct Vec3 { double x, y, z; };

__device__ __forceinline__ Vec3 unit(const StepConst& s) {
    const double x = s.dx, y = s.dy, z = s.dz;
    const double n = sqrt(x * x + y * y + z * z);
    return Vec3{x / n, y / n, z / n};
}

struct Arc {
    Vec3 a, b;
    double theta, sin_theta;
};

__device__ __forceinline__ Vec3 arc_dir(const Arc& c, double al) {
    if (c.theta < 1e-12) {
        Vec3 d{c.a.x + al * (c.b.x - c.a.x), c.a.y + al * (c.b.y - c.a.y), c.a.z + al * (c.b.z - c.a.z)};
        const double n = sqrt(d.x * d.x + d.y * d.y + d.z * d.z);
        return Vec3{d.x / n, d.y / n, d.z / n};
    }
    const double wa = sin((1.0 - al) * c.theta) / c.sin_theta, wb = sin(al * c.theta) / c.sin_theta;
    Vec3 d{wa * c.a.x + wb * c.b.x, wa * c.a.y + wb * c.b.y, wa * c.a.z + wb * c.b.z};
    const double n = sqrt(d.x * d.x + d.y * d.y + d.z * d.z);
    return Vec3{d.x / n, d.y / n, d.z / n};
}

__device__ __forceinline__ Vec3 arc_ddir(const Arc& c, double al) {
    if (c.theta < 1e-12) return Vec3{c.b.x - c.a.x, c.b.y - c.a.y, c.b.z - c.a.z};
    const double ka = -c.theta * cos((1.0 - al) * c.theta) / c.sin_theta;
    const double kb = c.theta * cos(al * c.theta) / c.sin_theta;
    return Vec3{ka * c.a.x + kb * c.b.x, ka * c.a.y + kb * c.b.y, ka * c.a.z + kb * c.b.z};
}

// Exact prism test: does the ray from ground point (px, py) toward d cross the convex CCW
// footprint between heights 0 and h?  Returns the entry height interval and the edge that
// bounds it from below (-1: the ground).
struct Entry {
    bool inside;
    double zlo, zhi;
    int elo;
};

__device__ Entry prism(const float2* xy, int a, int v, double h, double px, double py,
                       double ux, double uy) {
    double zlo = 0.0, zhi = h;
    int elo = -1;
    for (int i = 0; i < v; ++i) {
        const float2 p0 = xy[a + i], p1 = xy[a + (i + 1 == v ? 0 : i + 1)];
        const double cx = (double)p1.x - (double)p0.x, cy = (double)p1.y - (double)p0.y;
        const double A = cx * (py - (double)p0.y) - cy * (px - (double)p0.x);
        const double Bc = cx * uy - cy * ux;     // left-of-edge constraint: A + z Bc >= 0
        if (Bc > 0.0) {
            const double z = -A / Bc;
            if (z > zlo) { zlo = z; elo = i; }
        } else if (Bc < 0.0) {
            const double z = -A / Bc;
            if (z < zhi) zhi = z;
        } else if (A < 0.0) {
            return Entry{false, 1.0, 0.0, -1};
        }
    }
    return Entry{zlo <= zhi, zlo, zhi, elo};
}

// The same decision as prism(...).inside, without divisions: each bound z = -A / B of the
// entry interval is kept as a fraction with a positive denominator and compared by cross
// multiplication.
__device__ bool prism_inside(const float2* xy, int a, int v, double h, double px, double py,
                             double ux, double uy) {
    double nlo = 0.0, dlo = 1.0;     // lower bound nlo / dlo
    double nhi = h, dhi = 1.0;       // upper bound nhi / dhi
    for (int i = 0; i < v; ++i) {
        const float2 p0 = xy[a + i], p1 = xy[a + (i + 1 == v ? 0 : i + 1)];
        const double cx = (double)p1.x - (double)p0.x, cy = (double)p1.y - (double)p0.y;
        const double A = cx * (py - (double)p0.y) - cy * (px - (double)p0.x);
        const double Bc = cx * uy - cy * ux;
        if (Bc > 0.0) {
            if (-A * dlo > nlo * Bc) { nlo = -A; dlo = Bc; }
        } else if (Bc < 0.0) {
            if (A * dhi < nhi * -Bc) { nhi = A; dhi = -Bc; }
        } else if (A < 0.0) {
            return false;
        }
    }
    return nlo * dhi <= nhi * dlo;
}

// Status of building b along the arc in the projective parameter be: the direction
// a + be (b - a) (not normalised: the slopes u = d_xy / d_z do not depend on its length)
// runs over the same great-circle arc as slerp, monotonically, so a flip found in be is
// the same physical flip; its slerp parameter follows from the angle to a.
__device__ __forceinline__ bool prism_along(const FootprintSet& fs, const float* heights, int b,
                                            double px, double py, const Arc& arc, double be) {
    const double dx = fma(be, arc.b.x - arc.a.x, arc.a.x);
    const double dy = fma(be, arc.b.y - arc.a.y, arc.a.y);
    const double dz = fma(be, arc.b.z - arc.a.z, arc.a.z);
    const double iz = 1.0 / dz;
    return prism_inside(fs.xy, fs.fp_off[b], fs.fp_off[b + 1] - fs.fp_off[b], (double)heights[b],
                        px, py, dx * iz, dy * iz);
}

// Along the arc d(be) = a + be (b - a) every edge constraint of the prism is linear in be
// once multiplied by d_z(be) > 0: the bound z = -A / B_c becomes (-A d_z) / (B_c d_z) with
// B_c d_z = c x d_xy = E0 + be E1.  Set up once per (flip, building), each bisection step
// then costs a few FP64 multiply-adds per edge and no division.
struct PrismLin {
    int v;
    double h, az, ez;
    double A[kLinEdges], E0[kLinEdges], E1[kLinEdges];
};

__device__ void prism_lin_setup(PrismLin& P, const float2* xy, int a, int v, double h, double px,
                                double py, const Arc& arc) {
    P.v = v;
    P.h = h;
    P.az = arc.a.z;
    P.ez = arc.b.z - arc.a.z;
    const double ex = arc.b.x - arc.a.x, ey = arc.b.y - arc.a.y;
    for (int i = 0; i < v; ++i) {
        const float2 p0 = xy[a + i], p1 = xy[a + (i + 1 == v ? 0 : i + 1)];
        const double cx = (double)p1.x - (double)p0.x, cy = (double)p1.y - (double)p0.y;
        P.A[i] = cx * (py - (double)p0.y) - cy * (px - (double)p0.x);
        P.E0[i] = cx * arc.a.y - cy * arc.a.x;
        P.E1[i] = cx * ey - cy * ex;
    }
}

__device__ bool prism_lin_inside(const PrismLin& P, double be) {
    const double dz = fma(be, P.ez, P.az);
    double nlo = 0.0, dlo = 1.0, nhi = P.h, dhi = 1.0;
    for (int i = 0; i < P.v; ++i) {
        const double den = fma(be, P.E1[i], P.E0[i]);
        const double num = -P.A[i] * dz;
        if (den > 0.0) {
            if (num * dlo > nlo * den) { nlo = num; dlo = den; }
        } else if (den < 0.0) {
            if (-num * dhi < nhi * -den) { nhi = -num; dhi = -den; }
        } else if (P.A[i] < 0.0) {
            return false;
        }
    }
    return nlo * dhi <= nhi * dlo;
}

// The same test with FP32 coefficients: used only to bracket the flip coarsely (the
// bracket is confirmed in FP64 below).
struct PrismLinF {
    int v;
    float h, az, ez;
    float A[kLinEdges], E0[kLinEdges], E1[kLinEdges];
};

__device__ void prism_lin_to_f(const PrismLin& P, PrismLinF& F) {
    F.v = P.v; F.h = (float)P.h; F.az = (float)P.az; F.ez = (float)P.ez;
    for (int i = 0; i < P.v; ++i) { F.A[i] = (float)P.A[i]; F.E0[i] = (float)P.E0[i]; F.E1[i] = (float)P.E1[i]; }
}

__device__ bool prism_lin_inside_f(const PrismLinF& P, float be) {
    const float dz = fmaf(be, P.ez, P.az);
    float nlo = 0.f, dlo = 1.f, nhi = P.h, dhi = 1.f;
    for (int i = 0; i < P.v; ++i) {
        const float den = fmaf(be, P.E1[i], P.E0[i]);
        const float num = -P.A[i] * dz;
        if (den > 0.f) {
            if (num * dlo > nlo * den) { nlo = num; dlo = den; }
        } else if (den < 0.f) {
            if (-num * dhi < nhi * -den) { nhi = -num; dhi = -den; }
        } else if (P.A[i] < 0.f) {
            return false;
        }
    }
    return nlo * dhi <= nhi * dlo;
}

// The constraints that bound the entry interval at be: il the lower bound (-1: the ground),
// iu the upper bound (-1: the roof height h).
__device__ void prism_lin_active(const PrismLin& P, double be, int* il, int* iu) {
    const double dz = fma(be, P.ez, P.az);
    double nlo = 0.0, dlo = 1.0, nhi = P.h, dhi = 1.0;
    *il = -1;
    *iu = -1;
    for (int i = 0; i < P.v; ++i) {
        const double den = fma(be, P.E1[i], P.E0[i]);
        const double num = -P.A[i] * dz;
        if (den > 0.0 && num * dlo > nlo * den) { nlo = num; dlo = den; *il = i; }
        if (den < 0.0 && -num * dhi < nhi * -den) { nhi = -num; dhi = -den; *iu = i; }
    }
}

// The flip where the interval closes between lower bound il and upper bound iu, in closed
// form: both bounds are ratios of functions linear in be, so their equality is linear.
//   edge il against the roof:  -A_i d_z(be) = h (E0_i + be E1_i)
//   edge il against edge iu:    A_i (E0_j + be E1_j) = A_j (E0_i + be E1_i)
__device__ bool pair_root(const PrismLin& P, int il, int iu, double* be) {
    if (il < 0) return false;
    const double Ai = P.A[il];
    if (iu < 0) {
        const double den = fma(Ai, P.ez, P.h * P.E1[il]);
        if (den == 0.0) return false;
        *be = -fma(Ai, P.az, P.h * P.E0[il]) / den;
        return true;
    }
    const double Aj = P.A[iu];
    const double den = Ai * P.E1[iu] - Aj * P.E1[il];
    if (den == 0.0) return false;
    *be = (Aj * P.E0[il] - Ai * P.E0[iu]) / den;
    return true;
}

// slerp parameter of the projective parameter be (see prism_along)
__device__ __forceinline__ double slerp_param(const Arc& arc, double be) {
    if (arc.theta < 1e-12) return be;
    const double dx = fma(be, arc.b.x - arc.a.x, arc.a.x);
    const double dy = fma(be, arc.b.y - arc.a.y, arc.a.y);
    const double dz = fma(be, arc.b.z - arc.a.z, arc.a.z);
    const double cx = arc.a.y * dz - arc.a.z * dy, cy = arc.a.z * dx - arc.a.x * dz,
                 cz = arc.a.x * dy - arc.a.y * dx;
    const double ang = atan2(sqrt(cx * cx + cy * cy + cz * cz), arc.a.x * dx + arc.a.y * dy + arc.a.z * dz);
    return fmin(1.0, fmax(0.0, ang / arc.theta));
}

// Buildings hit by the FP32 ray from o toward step s (all hits, not only the first).
__device__ int hit_buildings(const DevScene& sc, const float3& o, const StepConst& s, int* ids) {
    int n = 0;
    int i = 0;
    while (i < sc.n_nodes) {
        const float4 lo = __ldg(&sc.nodes[2 * i]);
        const float4 hi = __ldg(&sc.nodes[2 * i + 1]);
        const int esc = SA_ESC(__float_as_int(lo.w), i, sc.n_nodes, sa::CK_ADJ_ESCAPE);
        const int tri = SA_LEAF(__float_as_int(hi.w), sc.T, sa::CK_ADJ_LEAF);
        const bool in = hit_box(o, s.ix, s.iy, s.iz, lo, hi);
        if (tri >= 0) {
            if (in) {
                const float4 a = __ldg(&sc.tris[3 * tri]);
                const float4 b = __ldg(&sc.tris[3 * tri + 1]);
                const float4 c = __ldg(&sc.tris[3 * tri + 2]);
                if (hit_tri_any(s.kz, o, a, b, c, s, kGroundTmin)) {
                    const int bid = __float_as_int(a.w);
                    bool seen = false;
                    for (int q = 0; q < n; ++q) seen |= (ids[q] == bid);
                    if (!seen && n < kMaxCand) ids[n++] = bid;
                }
            }
            i = esc;
        } else {
            i = in ? i + 1 : esc;
        }
    }
    return n;
}

struct SolveArgs {
    DevScene sc;
    FootprintSet fs;
    const float* heights;
    const StepConst* steps;
    float x0, y0, dx;
    int nx;
    const float* weights;
    double dt;
    const int4* flips;
    long long n_flips;
    double* S;
    double* dSdh;
};

__global__ void k_flip_solve(SolveArgs a) {
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.n_flips) return;
    const int4 fl = a.flips[f];
    const long long r = (long long)(unsigned)fl.x | ((long long)fl.y << 31);
    const int j = fl.z, c0 = fl.w;
    const int ix = (int)(r % a.nx), iy = (int)(r / a.nx);
    float3 o;
    o.x = __fadd_rn(a.x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), a.dx));
    o.y = __fadd_rn(a.y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), a.dx));
    o.z = 0.f;
    const double px = o.x, py = o.y;
    const double w = a.weights ? (double)a.weights[r] : 1.0;
    Arc arc;
    arc.a = unit(a.steps[j]);
    arc.b = unit(a.steps[j + 1]);
    double cd = arc.a.x * arc.b.x + arc.a.y * arc.b.y + arc.a.z * arc.b.z;
    cd = fmin(cd, 1.0);
    arc.theta = acos(cd);
    arc.sin_theta = sin(arc.theta);
    // candidates: buildings hit at the shadowed end
    int ids[kMaxCand];
    const StepConst& ss = a.steps[c0 ? j : j + 1];
    const int n = hit_buildings(a.sc, o, ss, ids);
    const double al_sh = c0 ? 0.0 : 1.0, al_lit = c0 ? 1.0 : 0.0;
    double best = c0 ? -1.0 : 2.0;
    int bbest = -1;
    for (int q = 0; q < n; ++q) {
        const int b = ids[q];
        const bool s0 = c0 != 0;
        const int fa = a.fs.fp_off[b], v = a.fs.fp_off[b + 1] - fa;
        double be_star = -1.0;
        if (v <= kLinEdges) {
            PrismLin P;
            prism_lin_setup(P, a.fs.xy, fa, v, (double)a.heights[b], px, py, arc);
            if (!prism_lin_inside(P, al_sh) || prism_lin_inside(P, al_lit)) continue;
            // bracket in FP32, then the closed form of the pair of constraints that close
            // the interval, confirmed by FP64 statuses on both sides of it
            PrismLinF F;
            prism_lin_to_f(P, F);
            float flo = 0.f, fhi = 1.f;
            for (int it = 0; it < kBisectF; ++it) {
                const float mid = 0.5f * (flo + fhi);
                if (prism_lin_inside_f(F, mid) == s0) flo = mid; else fhi = mid;
            }
            int il, iu;
            prism_lin_active(P, s0 ? (double)flo : (double)fhi, &il, &iu);
            double r;
            if (pair_root(P, il, iu, &r) && r > kSide && r < 1.0 - kSide &&
                fabs(r - 0.5 * ((double)flo + (double)fhi)) < 1e-4 &&
                prism_lin_inside(P, r - kSide) == s0 && prism_lin_inside(P, r + kSide) != s0) {
                be_star = r;
            } else {
                double lo = 0.0, hi = 1.0;   // invariant: status(lo) == status at the start
                for (int it = 0; it < kBisect; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    if (prism_lin_inside(P, mid) == s0) lo = mid; else hi = mid;
                }
                be_star = 0.5 * (lo + hi);
            }
        } else {
            if (!prism_along(a.fs, a.heights, b, px, py, arc, al_sh)) continue;
            if (prism_along(a.fs, a.heights, b, px, py, arc, al_lit)) continue;
            double lo = 0.0, hi = 1.0;
            for (int it = 0; it < kBisect; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (prism_along(a.fs, a.heights, b, px, py, arc, mid) == s0) lo = mid; else hi = mid;
            }
            be_star = 0.5 * (lo + hi);
        }
        const double as = slerp_param(arc, be_star);
        if (c0 ? (as > best) : (as < best)) { best = as; bbest = b; }
    }
    if (bbest < 0) {
        // No single building explains the flip in FP64 (a step status decided within FP32
        // rounding of a boundary): the flip time is unknown, count half the interval and
        // no derivative.
        atomicAdd(a.S, 0.5 * a.dt * w);
        return;
    }
    atomicAdd(a.S, a.dt * w * (c0 ? best : 1.0 - best));
    // is the flip the shadow of a roof edge?  (entry through edge e exactly at height h)
    const int fa = a.fs.fp_off[bbest], v = a.fs.fp_off[bbest + 1] - fa;
    const double h = (double)a.heights[bbest];
    const Vec3 d = arc_dir(arc, best);
    const Vec3 dd = arc_ddir(arc, best);
    const double ux = d.x / d.z, uy = d.y / d.z;
    const double dux = (dd.x * d.z - d.x * dd.z) / (d.z * d.z);
    const double duy = (dd.y * d.z - d.y * dd.z) / (d.z * d.z);
    const Entry e = prism(a.fs.xy, fa, v, h, px, py, ux, uy);
    const double tol = 1e-6 * (h + 1.0);
    if (e.elo < 0 || fabs(e.zlo - h) > tol || e.zhi < h - tol) return;   // vertical-edge event
    const float2 p0 = a.fs.xy[fa + e.elo], p1 = a.fs.xy[fa + (e.elo + 1 == v ? 0 : e.elo + 1)];
    const double cx = (double)p1.x - (double)p0.x, cy = (double)p1.y - (double)p0.y;
    const double Bc = cx * uy - cy * ux;
    const double dB = cx * duy - cy * dux;
    if (dB == 0.0) return;
    const double dadh = -Bc / (h * dB);
    const double sf = c0 ? 1.0 : -1.0;
    atomicAdd(&a.dSdh[bbest], w * a.dt * sf * dadh);
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

}  // namespace

cudaError_t launch_height_grad(const DevScene& sc, const FootprintSet& fs, const float* d_heights,
                               const DevRecv& rc, const DevSun& sun, float step_minutes,
                               const float* weights, float* dS_dh, double* d_S, cudaStream_t st) {
    const long long R = (long long)rc.nx * rc.ny;
    cudaError_t e = cudaSuccess;
    double* dsdh = nullptr;
    double* S = nullptr;
    unsigned long long* masks = nullptr;
    unsigned* counts = nullptr;
    unsigned* d_total = nullptr;
    int4* flips = nullptr;
    int* gross = nullptr;
    const int B = fs.B;
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(sa::scratch_alloc(&dsdh, sizeof(double) * (B > 0 ? B : 1), st));
    TRY(sa::scratch_alloc(&S, sizeof(double), st));
    TRY(cudaMemsetAsync(dsdh, 0, sizeof(double) * (B > 0 ? B : 1), st));
    TRY(cudaMemsetAsync(S, 0, sizeof(double), st));
    if (R > 0 && sun.n_blocks > 0) {
        TRY(sa::scratch_alloc(&masks, sizeof(unsigned long long) * (size_t)R * sun.n_blocks, st));
        TRY(cudaMemsetAsync(masks, 0, sizeof(unsigned long long) * (size_t)R * sun.n_blocks, st));
        TRY(sa::scratch_alloc(&gross, sizeof(int) * (size_t)R, st));
        {
            DevOut out;
            memset(&out, 0, sizeof(out));
            out.gross = gross;
            out.masks = reinterpret_cast<uint64_t*>(masks);
            int* run = nullptr;
            TRY(sa::scratch_alloc(&run, sizeof(int) * (size_t)R, st));
            out.run = run;
            e = launch_raster_ground(sc, rc, sun, out, st);
            cudaFreeAsync(run, st);
            if (e != cudaSuccess) goto done;
        }
        TRY(sa::scratch_alloc(&counts, sizeof(unsigned) * (size_t)R, st));
        TRY(sa::scratch_alloc(&d_total, sizeof(unsigned), st));
        const double dt = step_minutes;
        const unsigned grid = (unsigned)((R + 255) / 256);
        k_flip_count<<<grid, 256, 0, st>>>(masks, R, sun.blocks, sun.n_blocks, weights, dt, counts, S);
        TRY(cudaGetLastError());
        TRY(exclusive_scan_u32(counts, R, d_total, st));
        unsigned total = 0;
        TRY(cudaMemcpyAsync(&total, d_total, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (total > 0) {
            TRY(sa::scratch_alloc(&flips, sizeof(int4) * (size_t)total, st));
            k_flip_fill<<<grid, 256, 0, st>>>(masks, R, sun.blocks, sun.n_blocks, counts, flips);
            SolveArgs sa;
            sa.sc = sc; sa.fs = fs; sa.heights = d_heights; sa.steps = sun.steps;
            sa.x0 = rc.x0; sa.y0 = rc.y0; sa.dx = rc.dx; sa.nx = rc.nx;
            sa.weights = weights; sa.dt = dt; sa.flips = flips; sa.n_flips = total;
            sa.S = S; sa.dSdh = dsdh;
            k_flip_solve<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(sa);
            TRY(cudaGetLastError());
        }
    }
    if (B > 0) k_to_float<<<(B + 255) / 256, 256, 0, st>>>(dsdh, dS_dh, B);
    TRY(cudaGetLastError());
    if (d_S) TRY(cudaMemcpyAsync(d_S, S, sizeof(double), cudaMemcpyDeviceToDevice, st));
done:
    if (dsdh) cudaFreeAsync(dsdh, st);
    if (S) cudaFreeAsync(S, st);
    if (masks) cudaFreeAsync(masks, st);
    if (counts) cudaFreeAsync(counts, st);
    if (d_total) cudaFreeAsync(d_total, st);
    if (flips) cudaFreeAsync(flips, st);
    if (gross) cudaFreeAsync(gross, st);
    return e;
#undef TRY
}

}  // namespace sa
