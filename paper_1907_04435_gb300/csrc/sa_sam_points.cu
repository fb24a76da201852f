// sa_sam_points.cu -- shadow accrual map for point receivers (facades), in light space.
//
// Sec. 4 renders the scene once per interval into a map on a plane orthogonal to the sun
// direction and tests every receiver against its n slices.  Here each run of <= 32
// consecutive steps of a block gets such a light-space map.  Coordinates are taken in a
// basis (e1, e2) orthogonal to the run's middle direction d_m, around a reference point.
// The map is a grid of light-space tiles:
//   - every triangle that faces the sun at some step of the run is binned into the tiles
//     its projection covers, widened by the drift of the run's rays up to the triangle's
//     top: a ray of step k from a receiver leaves the receiver's light-space point by
//     h x delta_k at height h above it (delta_k = (d_k . e1, d_k . e2) / d_k.z), and the
//     run's delta_k lie in a box that is long along the sun's motion and thin across it;
//   - every receiver goes into the single tile holding its own projection.
// A receiver and a triangle its rays can meet during the run therefore share a tile.
// One pass over the geometry per run thus serves all of the run's steps.  The test
// itself is exact: per (receiver, triangle) the Plücker edge moments are set up once,
// then each of the run's steps costs three dot products and a distance check
// (watertight with canonically ordered edges, as in the ray-traced accrual).  For a
// closed scene only sun-facing triangles are binned: any ray that meets a closed solid
// crosses one of its sun-facing faces.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sa_handles.cuh"

namespace sa {

namespace {

constexpr int kRunMax = 32;
constexpr float kLightSlack = 0.05f;    // absolute slack (m) of the light-space culls (rounding)
// threads per light-space tile (a multiple of 32) and triangles staged per chunk (<= 256)
#ifndef SA_TILE_THREADS
#define SA_TILE_THREADS 128
#endif
#ifndef SA_TILE_CHUNK
#define SA_TILE_CHUNK 128
#endif
constexpr int kTileThreads = SA_TILE_THREADS;
constexpr int kTriChunk = SA_TILE_CHUNK;
// side (m) of the light-space tiles
#ifndef SA_LIGHT_TILE
#define SA_LIGHT_TILE 32.f
#endif
// resident CTAs per SM k_sam_tile is compiled for: 9 gives 55 registers and no spills
#ifndef SA_TILE_CTAS
#define SA_TILE_CTAS 9
#endif

struct RunLight {
    float e1[3], e2[3];          // light-space basis (orthogonal to the run's middle direction)
    float c[3];                  // reference point
    float a0, b0, tile;          // tile grid origin and tile side (m)
    float zr;                    // lowest receiver height
    int nta, ntb;                // tiles along e1, e2
    int tile_base;               // first global tile index of this run
    int k0, kn;                  // steps of the run within the block
    int j0;                      // first step of the block
    int blk;                     // block within the chunk (row of the chunk's masks)
    // light-space drift per metre of height over the run's steps, as the margins it
    // implies on each side: a ray point at height h above the receiver lies within
    // [-h da_hi, h da_lo] of it along e1 and [-h db_hi, h db_lo] along e2 (all >= 0)
    float da_hi, da_lo, db_hi, db_lo;
    // every step direction of the run is d_m + alpha t + beta b + nu n (t, b, n: an FP32
    // basis around d_m), with |alpha| <= ba, |beta| <= bb, |nu| <= bn
    float dm[3], tv[3], bv[3], ba, bb, bn;
};

__device__ __forceinline__ void light_ab(const RunLight& rl, float x, float y, float z, float* a,
                                         float* b) {
    const float dx = x - rl.c[0], dy = y - rl.c[1], dz = z - rl.c[2];
    *a = rl.e1[0] * dx + rl.e1[1] * dy + rl.e1[2] * dz;
    *b = rl.e2[0] * dx + rl.e2[1] * dy + rl.e2[2] * dz;
}

__device__ __forceinline__ unsigned run_front(const float4& a, const float4& b, const float4& c,
                                              const StepConst* steps, const RunLight& rl, bool cull) {
    const float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
    const float vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
    const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    unsigned m = 0;
    for (int k = 0; k < rl.kn; ++k) {
        const StepConst& s = steps[rl.j0 + rl.k0 + k];
        const float nd = nx * s.dx + ny * s.dy + nz * s.dz;
        if (cull ? nd > 0.f : nd != 0.f) m |= 1u << k;
    }
    return m;
}

// tile range of a triangle's widened light-space box; false if outside the grid
__device__ __forceinline__ bool tri_tiles(const float4& a, const float4& b, const float4& c,
                                          const RunLight& rl, int* ta0, int* ta1, int* tb0, int* tb1) {
    float pa[3], pb[3];
    light_ab(rl, a.x, a.y, a.z, &pa[0], &pb[0]);
    light_ab(rl, b.x, b.y, b.z, &pa[1], &pb[1]);
    light_ab(rl, c.x, c.y, c.z, &pa[2], &pb[2]);
    // receivers that a ray rising at most H to the triangle's top can reach it from
    const float H = fmaxf(fmaxf(a.z, fmaxf(b.z, c.z)) - rl.zr, 0.f);
    const float amin = fminf(pa[0], fminf(pa[1], pa[2])) - fmaf(H, rl.da_hi, kLightSlack);
    const float amax = fmaxf(pa[0], fmaxf(pa[1], pa[2])) + fmaf(H, rl.da_lo, kLightSlack);
    const float bmin = fminf(pb[0], fminf(pb[1], pb[2])) - fmaf(H, rl.db_hi, kLightSlack);
    const float bmax = fmaxf(pb[0], fmaxf(pb[1], pb[2])) + fmaf(H, rl.db_lo, kLightSlack);
    const float inv = 1.f / rl.tile;
    const float fa0 = floorf((amin - rl.a0) * inv), fa1 = floorf((amax - rl.a0) * inv);
    const float fb0 = floorf((bmin - rl.b0) * inv), fb1 = floorf((bmax - rl.b0) * inv);
    if (fa1 < 0.f || fb1 < 0.f || fa0 >= (float)rl.nta || fb0 >= (float)rl.ntb) return false;
    *ta0 = (int)fmaxf(fa0, 0.f);
    *ta1 = (int)fminf(fa1, (float)(rl.nta - 1));
    *tb0 = (int)fmaxf(fb0, 0.f);
    *tb1 = (int)fminf(fb1, (float)(rl.ntb - 1));
    return true;
}

__device__ __forceinline__ int recv_tile(const float4& o, const RunLight& rl) {
    float a, b;
    light_ab(rl, o.x, o.y, o.z, &a, &b);
    const float inv = 1.f / rl.tile;
    const int ta = min(max((int)floorf((a - rl.a0) * inv), 0), rl.nta - 1);
    const int tb = min(max((int)floorf((b - rl.b0) * inv), 0), rl.ntb - 1);
    return rl.tile_base + tb * rl.nta + ta;
}

__global__ void k_lt_bin(DevScene sc, const StepConst* __restrict__ steps,
                         const RunLight* __restrict__ runs, int n_runs, bool fill,
                         unsigned* __restrict__ counts, const unsigned* __restrict__ offsets,
                         unsigned* __restrict__ cursor, int* __restrict__ bins) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (t >= sc.T || r >= n_runs) return;
    const RunLight& rl = runs[r];
    const float4 a = __ldg(&sc.tris[3 * t]), b = __ldg(&sc.tris[3 * t + 1]), c = __ldg(&sc.tris[3 * t + 2]);
    if (run_front(a, b, c, steps, rl, sc.closed != 0) == 0u) return;
    int ta0, ta1, tb0, tb1;
    if (!tri_tiles(a, b, c, rl, &ta0, &ta1, &tb0, &tb1)) return;
    for (int tb = tb0; tb <= tb1; ++tb)
        for (int ta = ta0; ta <= ta1; ++ta) {
            const int cell = rl.tile_base + tb * rl.nta + ta;
            if (fill) bins[offsets[cell] + atomicAdd(&cursor[cell], 1u)] = t;
            else atomicAdd(&counts[cell], 1u);
        }
}

// Receivers are Morton-ordered, so neighbouring lanes usually share a tile: lanes with the
// same tile are grouped (match_any) and their leader makes one atomic for the group.
__global__ void k_lr_bin(const float4* __restrict__ orig, long long R,
                         const RunLight* __restrict__ runs, int n_runs, bool fill,
                         unsigned* __restrict__ counts, const unsigned* __restrict__ offsets,
                         unsigned* __restrict__ cursor, int* __restrict__ bins) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const bool valid = s < R && r < n_runs;
    const int cell = valid ? recv_tile(orig[s], runs[r]) : -1 - lane;   // unique when invalid
    const unsigned peers = __match_any_sync(0xffffffffu, cell);
    const int leader = __ffs(peers) - 1;
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    unsigned base = 0;
    if (valid && lane == leader) {
        if (fill) base = atomicAdd(&cursor[cell], (unsigned)__popc(peers));
        else atomicAdd(&counts[cell], (unsigned)__popc(peers));
    }
    if (fill) {
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) bins[offsets[cell] + base + rank] = (int)s;
    }
}

struct TileArgs {
    DevScene sc;
    const StepConst* steps;
    const RunLight* runs;
    int n_runs;
    const int* tile_run;           // run of each global tile
    const int* order;              // tile of each CTA, most work first, empty tiles left out
    const unsigned* t_off; const unsigned* t_cnt; const int* t_bins;
    const unsigned* r_off; const unsigned* r_cnt; const int* r_bins;
    const float4* orig;
    unsigned long long* masks;     // [blocks of the chunk][R] block masks (sorted order)
    long long R;
    unsigned long long* stats;
};

// One CTA per light-space tile.  The tile's triangles are staged in shared memory with
// their light boxes, top heights and sun-facing step bits.  Each warp then takes 32 of the
// tile's receivers at a time, one per lane, and runs over the staged triangles in step:
//   - a cheap per-pair cull (the triangle is not wholly below the receiver, and the
//     receiver's light-space point lies inside the triangle's box widened by the drift a
//     ray of the run can make before it rises to the triangle's top);
//   - the pairs that survive (a few in a hundred) are appended to a per-warp queue;
//   - whenever the queue holds 32 pairs, every lane takes one and runs the exact test, so
//     the expensive set-up is never paid by idle lanes.
// Results are OR-ed into per-receiver masks in shared memory, then into the block masks.
constexpr int kQueue = 64;

// Bounds [lo, hi] on the FP32 value of d . v (in the rounding of the step tests) at every
// step d of the run, for a vector v of the triangle: d . v = d_m . v + alpha (t . v) +
// beta (b . v) + nu (n . v) exactly, n . v is within 2e-7 |v|_1 of d_m . v, and 2^-20 |v|_1
// covers the roundings of the step test's value and of these bounds (each below 8 ulp of
// |v|_1: every direction component is at most 1 in magnitude).
__device__ __forceinline__ float2 run_dot_bounds(const RunLight& rl, float vx, float vy, float vz) {
    const float c = fmaf(rl.dm[2], vz, fmaf(rl.dm[1], vy, rl.dm[0] * vx));
    const float tv = fmaf(rl.tv[2], vz, fmaf(rl.tv[1], vy, rl.tv[0] * vx));
    const float bv = fmaf(rl.bv[2], vz, fmaf(rl.bv[1], vy, rl.bv[0] * vx));
    const float l1 = fabsf(vx) + fabsf(vy) + fabsf(vz);
    const float r = fmaf(rl.ba, fabsf(tv), fmaf(rl.bb, fabsf(bv), fmaf(rl.bn, fabsf(c), 0x1p-20f * l1)));
    return make_float2(c - r, c + r);
}

// Lines of a triangle's light-space projection, as unit inward normals and offsets: a point
// x is inside iff n . x + c >= 0 for all three.  A ray of the run that meets the triangle at
// height h above the receiver passes x = r + h delta, so r can be shadowed by it only if
// n . r + c >= -h max(0, n . delta) for every line; .w holds max(0, max of n . delta over
// the run's drift box), so the cull is n . r + c >= -(rise x .w + slack).  A projection
// too thin to orient passes every point (the light box still applies).
__device__ __forceinline__ void light_edges(const float* pa, const float* pb, const RunLight& rl,
                                            float4& e0, float4& e1, float4& e2) {
    float4* e[3] = {&e0, &e1, &e2};
    const float ax = pa[1] - pa[0], ay = pb[1] - pb[0];
    const float bx = pa[2] - pa[0], by = pb[2] - pb[0];
    const float area2 = ax * by - ay * bx;
    const float l0 = sqrtf(ax * ax + ay * ay), l1 = sqrtf(bx * bx + by * by);
    const bool thin = !(fabsf(area2) > 1e-4f * l0 * l1);
    const float sg = area2 > 0.f ? 1.f : -1.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = i == 2 ? 0 : i + 1;
        const float ex = pa[j] - pa[i], ey = pb[j] - pb[i];
        const float len = sqrtf(ex * ex + ey * ey);
        if (thin || !(len > 1e-6f)) {
            *e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float nx = -sg * ey / len, ny = sg * ex / len;
        // largest n . delta over the drift box [-da_lo, da_hi] x [-db_lo, db_hi]
        const float sup = fmaxf(nx * rl.da_hi, -nx * rl.da_lo) + fmaxf(ny * rl.db_hi, -ny * rl.db_lo);
        *e[i] = make_float4(nx, ny, -(nx * pa[i] + ny * pb[i]), fmaxf(sup, 0.f) * 1.0001f);
    }
}

template <bool COUNT>
__device__ __forceinline__ void drain_pairs(const unsigned short* q, int n, int lane,
                                            const float4* s_tri, const float4* s_n,
                                            const unsigned* s_front,
                                            const float4* s_o, unsigned* s_m,
                                            const unsigned long long (*s_d2)[3], int kn,
                                            unsigned long long& n_pair,
                                            unsigned long long& n_test) {
    const bool live = lane < n;
    const unsigned e = live ? q[lane] : 0u;
    const int who = (int)(e >> 8), t = (int)(e & 0xffu);
    const float4 p = s_o[who];
    const float2 ndb = make_float2(s_tri[3 * t + 1].w, s_tri[3 * t + 2].w);
    // A receiver whose rays start at distance 0 (t_min = 0: the facade samples) with d . n
    // of one sign at every step of the run: its pair passed the plane-side cull, so the
    // distance check (a . n against 0 x d . n) holds at every step and only the inside
    // test varies.  A warp whose pairs all are so skips the distance check.
    const bool const_ahead = !live || (p.w == 0.f && (ndb.x > 0.f || ndb.y < 0.f));
    const bool all_const = __all_sync(0xffffffffu, const_ahead);
    if (!live) return;
    const float3 o = make_float3(p.x, p.y, p.z);
    const float4 a = s_tri[3 * t], b = s_tri[3 * t + 1], c = s_tri[3 * t + 2];
    const unsigned want = s_front[t];
    if (COUNT) ++n_pair;
    const float4 nv = s_n[t];
    const PluckerTri pt = plucker_setup_n(o, a, b, c, make_float3(nv.x, nv.y, nv.z));
    // every step of the run is tested without branches, two steps per packed instruction
    // (the same roundings as plucker_hit_all); steps the triangle turns away from, and the
    // repeated step of an odd run's last pair, are masked off afterwards
    unsigned long long M[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[e][c] = f2_pack(pt.m[e][c], pt.m[e][c]);
    unsigned m = 0;
    if (all_const) {
#pragma unroll
        for (int k = 0; k < kRunMax; k += 2) {
            if (k >= kn) break;
            const unsigned long long dx = s_d2[k >> 1][0], dy = s_d2[k >> 1][1], dz = s_d2[k >> 1][2];
            float sv[3][2];
#pragma unroll
            for (int e = 0; e < 3; ++e)
                f2_unpack(f2_fma(dz, M[e][2], f2_fma(dy, M[e][1], f2_mul(dx, M[e][0]))), sv[e][0], sv[e][1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool inside = min3f(sv[0][h], sv[1][h], sv[2][h]) >= 0.f ||
                                    max3f(sv[0][h], sv[1][h], sv[2][h]) <= 0.f;
                if (inside) m |= 1u << (k + h);
            }
        }
    } else {
        unsigned long long N[3];
        N[0] = f2_pack(pt.nx, pt.nx); N[1] = f2_pack(pt.ny, pt.ny); N[2] = f2_pack(pt.nz, pt.nz);
#pragma unroll
        for (int k = 0; k < kRunMax; k += 2) {
            if (k >= kn) break;
            const unsigned long long dx = s_d2[k >> 1][0], dy = s_d2[k >> 1][1], dz = s_d2[k >> 1][2];
            float sv[3][2], nd[2];
#pragma unroll
            for (int e = 0; e < 3; ++e)
                f2_unpack(f2_fma(dz, M[e][2], f2_fma(dy, M[e][1], f2_mul(dx, M[e][0]))), sv[e][0], sv[e][1]);
            f2_unpack(f2_fma(dz, N[2], f2_fma(dy, N[1], f2_mul(dx, N[0]))), nd[0], nd[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool inside = min3f(sv[0][h], sv[1][h], sv[2][h]) >= 0.f ||
                                    max3f(sv[0][h], sv[1][h], sv[2][h]) <= 0.f;
                const float lim = __fmul_rn(p.w, nd[h]);
                const bool ahead = (nd[h] > 0.f && pt.aon > lim) || (nd[h] < 0.f && pt.aon < lim);
                if (inside && ahead) m |= 1u << (k + h);
            }
        }
    }
    m &= want;
    if (COUNT) n_test += (unsigned)__popc(want);
    if (m) atomicOr(&s_m[who], m);
}

template <bool COUNT>
__global__ void __launch_bounds__(kTileThreads, SA_TILE_CTAS)
k_sam_tile(TileArgs ta) {
    constexpr int kWarps = kTileThreads / 32;
    __shared__ float4 s_tri[kTriChunk * 3];
    // staged triangles: vertices in .xyz; .w of the second and third vertex hold the
    // bounds of d . n over the run's steps (run_dot_bounds)
    __shared__ float4 s_n[kTriChunk];              // normals (origin-independent set-up), highest vertex z in .w
    __shared__ float4 s_box[kTriChunk];            // light box (amin, amax, bmin, bmax), widened by the slack
    __shared__ float4 s_edge[3][kTriChunk];        // light-space edge lines (nx, ny, c + slack, drift)
    __shared__ unsigned s_front[kTriChunk];
    __shared__ unsigned long long s_d2[kRunMax / 2][3];   // directions of steps (k, k + 1), k even
    __shared__ float4 s_o[kTileThreads];           // receiver origins (and t_min) of the pass
    __shared__ unsigned s_m[kTileThreads];         // their step bits
    __shared__ unsigned short s_q[kWarps][kQueue]; // pair queues: receiver slot << 8 | triangle
    __shared__ unsigned char s_list[kWarps][kTriChunk];  // triangles near the warp's receivers
    unsigned long long n_pair = 0, n_test = 0;
    const int tile = ta.order[blockIdx.x];
    const unsigned tcnt = ta.t_cnt[tile], rcnt = ta.r_cnt[tile];
    if (tcnt == 0 || rcnt == 0) return;
    const RunLight& rl = ta.runs[ta.tile_run[tile]];
    const int kn = rl.kn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (2 * threadIdx.x < kn) {
        const int k = 2 * threadIdx.x, k1 = min(k + 1, kn - 1);
        const StepConst& s = ta.steps[rl.j0 + rl.k0 + k];
        const StepConst& t = ta.steps[rl.j0 + rl.k0 + k1];
        s_d2[threadIdx.x][0] = f2_pack(s.dx, t.dx);
        s_d2[threadIdx.x][1] = f2_pack(s.dy, t.dy);
        s_d2[threadIdx.x][2] = f2_pack(s.dz, t.dz);
    }
    const bool cull = ta.sc.closed != 0;
    unsigned short* q = s_q[warp];
    for (unsigned base = 0; base < tcnt; base += kTriChunk) {
        const int nt = (int)min((unsigned)kTriChunk, tcnt - base);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += kTileThreads) {
            const int t = (int)SA_CHK(ta.t_bins[ta.t_off[tile] + base + i], ta.sc.T, sa::CK_POINTS_TRI);
            const float4 a = __ldg(&ta.sc.tris[3 * t]), b = __ldg(&ta.sc.tris[3 * t + 1]),
                         c = __ldg(&ta.sc.tris[3 * t + 2]);
            s_tri[3 * i] = a; s_tri[3 * i + 1] = b; s_tri[3 * i + 2] = c;
            const float3 nrm = plucker_normal(a, b, c);
            s_n[i] = make_float4(nrm.x, nrm.y, nrm.z, fmaxf(a.z, fmaxf(b.z, c.z)));
            float pa[3], pb[3];
            light_ab(rl, a.x, a.y, a.z, &pa[0], &pb[0]);
            light_ab(rl, b.x, b.y, b.z, &pa[1], &pb[1]);
            light_ab(rl, c.x, c.y, c.z, &pa[2], &pb[2]);
            // the box and the edge lines carry the culls' slack already
            s_box[i] = make_float4(fminf(pa[0], fminf(pa[1], pa[2])) - kLightSlack,
                                   fmaxf(pa[0], fmaxf(pa[1], pa[2])) + kLightSlack,
                                   fminf(pb[0], fminf(pb[1], pb[2])) - kLightSlack,
                                   fmaxf(pb[0], fmaxf(pb[1], pb[2])) + kLightSlack);
            light_edges(pa, pb, rl, s_edge[0][i], s_edge[1][i], s_edge[2][i]);
#pragma unroll
            for (int q3 = 0; q3 < 3; ++q3) s_edge[q3][i].z += kLightSlack;
            const float2 ndb = run_dot_bounds(rl, nrm.x, nrm.y, nrm.z);
            s_tri[3 * i + 1].w = ndb.x;
            s_tri[3 * i + 2].w = ndb.y;
            s_front[i] = run_front(a, b, c, ta.steps, rl, cull);
        }
        __syncthreads();
        // every warp runs the same number of passes, so the loop below stays warp-uniform
        for (unsigned r0 = (unsigned)warp * 32u; r0 < rcnt; r0 += kTileThreads) {
            const unsigned i = r0 + lane;
            const bool live = i < rcnt;
            const int s = live ? (int)SA_CHK(ta.r_bins[ta.r_off[tile] + i], ta.R, sa::CK_POINTS_RECV) : -1;
            const float4 p = live ? ta.orig[s] : make_float4(0.f, 0.f, 0.f, 0.f);
            s_o[threadIdx.x] = p;
            s_m[threadIdx.x] = 0u;
            float la = 0.f, lb = 0.f;
            light_ab(rl, p.x, p.y, p.z, &la, &lb);
            // the warp's receivers' light-space box and lowest height: triangles no ray of
            // any of them can reach are dropped for the whole warp at once
            float wa0 = live ? la : 3.4e38f, wa1 = live ? la : -3.4e38f;
            float wb0 = live ? lb : 3.4e38f, wb1 = live ? lb : -3.4e38f;
            float wz = live ? p.z : 3.4e38f;
            for (int off = 16; off > 0; off >>= 1) {
                wa0 = fminf(wa0, __shfl_xor_sync(0xffffffffu, wa0, off));
                wa1 = fmaxf(wa1, __shfl_xor_sync(0xffffffffu, wa1, off));
                wb0 = fminf(wb0, __shfl_xor_sync(0xffffffffu, wb0, off));
                wb1 = fmaxf(wb1, __shfl_xor_sync(0xffffffffu, wb1, off));
                wz = fminf(wz, __shfl_xor_sync(0xffffffffu, wz, off));
            }
            int nl = 0;
            for (int t0 = 0; t0 < nt; t0 += 32) {
                const int t = t0 + lane;           // < kTriChunk: the arrays are read in bounds
                const float rise = s_n[t].w - wz;
                const float h = fmaxf(rise, 0.f);
                const float4 bx = s_box[t];
                bool near = (t < nt) & (s_front[t] != 0u) & (rise >= -0.01f);
                near &= (fmaf(h, rl.da_hi, wa1) >= bx.x) & (fmaf(-h, rl.da_lo, wa0) <= bx.y) &
                        (fmaf(h, rl.db_hi, wb1) >= bx.z) & (fmaf(-h, rl.db_lo, wb0) <= bx.w);
#pragma unroll
                for (int q3 = 0; q3 < 3; ++q3) {
                    const float4 e = s_edge[q3][t];
                    near &= fmaf(h, e.w, fmaxf(e.x * wa0, e.x * wa1) + fmaxf(e.y * wb0, e.y * wb1) + e.z) >= 0.f;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, near);
                if (near) s_list[warp][nl + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)t;
                nl += __popc(bal);
            }
            int n = 0;
            __syncwarp();
            // a lane without a receiver rises below every triangle
            const float pz = live ? p.z : 3.4e38f;
            // j == nl drains the queue's last pairs: one call site keeps the unrolled step
            // tests in the instruction cache once
            for (int j = 0; j <= nl; ++j) {
                const int t = j < nl ? (int)s_list[warp][j] : 0;    // j == nl: nothing passes
                const float rise = j < nl ? s_n[t].w - pz : -3.4e38f;
                const float h = fmaxf(rise, 0.f);
                const float4 bx = s_box[t];
                bool pass = (rise >= -0.01f) & (fmaf(h, rl.da_hi, la) >= bx.x) & (fmaf(-h, rl.da_lo, la) <= bx.y) &
                            (fmaf(h, rl.db_hi, lb) >= bx.z) & (fmaf(-h, rl.db_lo, lb) <= bx.w);
                if (pass) {
#pragma unroll
                    for (int q3 = 0; q3 < 3; ++q3) {
                        const float4 e = s_edge[q3][t];
                        pass &= fmaf(h, e.w, fmaf(e.x, la, fmaf(e.y, lb, e.z))) >= 0.f;
                    }
                    // the receiver on the side of the triangle's plane that no ray of the run
                    // leaves toward it: the step test's own distance check (a . n against
                    // t_min d . n, same roundings) fails at every step
                    const float4 v0 = s_tri[3 * t];
                    const float4 nv = s_n[t];
                    const float aon = fmaf(nv.z, __fsub_rn(v0.z, p.z),
                                           fmaf(nv.y, __fsub_rn(v0.y, p.y), __fmul_rn(nv.x, __fsub_rn(v0.x, p.x))));
                    const float2 nd = make_float2(s_tri[3 * t + 1].w, s_tri[3 * t + 2].w);
                    if (nd.x > 0.f) pass &= aon > __fmul_rn(p.w, nd.x);
                    else if (nd.y < 0.f) pass &= aon < __fmul_rn(p.w, nd.y);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (pass) q[n + __popc(bal & ((1u << lane) - 1u))] =
                    (unsigned short)(((unsigned)threadIdx.x << 8) | (unsigned)t);
                n += __popc(bal);
                if (n >= 32 || (j == nl && n > 0)) {
                    const int cnt = min(n, 32);
                    __syncwarp();
                    drain_pairs<COUNT>(q + (n - cnt), cnt, lane, s_tri, s_n, s_front, s_o, s_m, s_d2,
                                       kn, n_pair, n_test);
                    n -= cnt;
                    __syncwarp();
                }
            }
            __syncwarp();
            const unsigned m = s_m[threadIdx.x];
            if (live && m) atomicOr(&ta.masks[(long long)rl.blk * ta.R + s], (unsigned long long)m << rl.k0);
            __syncwarp();
        }
    }
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) {
            n_pair += __shfl_down_sync(0xffffffffu, n_pair, off);
            n_test += __shfl_down_sync(0xffffffffu, n_test, off);
        }
        if (lane == 0) {
            atomicAdd(&ta.stats[0], n_pair);
            atomicAdd(&ta.stats[1], n_test);
        }
    }
}

// Launch order of the light-space tiles: descending by (triangles x receivers), bucketed at
// half powers of two; tiles with no pair go last and are not launched.  The order changes
// no result, only which CTAs start last (the cheap ones, which shortens the tail).
constexpr int kOrderBuckets = 64;

__device__ __forceinline__ int pair_bucket(unsigned tcount, unsigned rcount) {
    const unsigned long long c = (unsigned long long)tcount * rcount;
    if (c == 0ull) return kOrderBuckets - 1;
    if (c == 1ull) return kOrderBuckets - 2;
    const int l = 63 - __clzll(c);
    const int key = min(kOrderBuckets - 2, 2 * l + (int)((c >> (l - 1)) & 1ull));
    return kOrderBuckets - 2 - key;
}

__global__ void k_order_hist(const unsigned* __restrict__ tc, const unsigned* __restrict__ rc,
                             long long n, unsigned* __restrict__ hist) {
    __shared__ unsigned h[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0u;
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&h[pair_bucket(tc[i], rc[i])], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBuckets && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// exclusive scan of the histogram into the bucket cursors; n_work = tiles with a pair
__global__ void k_order_scan(unsigned* __restrict__ hist, unsigned* __restrict__ n_work) {
    if (threadIdx.x != 0) return;
    unsigned run = 0;
    for (int k = 0; k < kOrderBuckets; ++k) {
        const unsigned h = hist[k];
        hist[k] = run;
        run += h;
        if (k == kOrderBuckets - 2) *n_work = run;
    }
}

__global__ void k_order_fill(const unsigned* __restrict__ tc, const unsigned* __restrict__ rc,
                             long long n, unsigned* __restrict__ cursor, int* __restrict__ order) {
    __shared__ unsigned h[kOrderBuckets], base[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0u;
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = i < n ? pair_bucket(tc[i], rc[i]) : -1;
    unsigned rank = 0;
    if (b >= 0) rank = atomicAdd(&h[b], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBuckets && h[threadIdx.x])
        base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], h[threadIdx.x]);
    __syncthreads();
    if (b >= 0) order[base[b] + rank] = (int)i;
}

// Stitch the chunk's blocks, in order, into each receiver's gross / continuous state.
__global__ void k_points_fold(long long R, const int* __restrict__ perm,
                              const BlockConst* __restrict__ blocks, int nbc,
                              unsigned long long* __restrict__ masks, DevOut out,
                              int* __restrict__ run, int* __restrict__ best, int first, int last) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= R) return;
    const long long r = SA_CHK(perm[s], R, sa::CK_POINTS_PERM);
    RunState st{0, 0, 0};
    if (!first || out.accumulate_into) {
        st.gross = out.gross[r];
        st.best = best[r];
        st.run = first ? 0 : run[r];
    }
    for (int b = 0; b < nbc; ++b) {
        const BlockConst& bc = blocks[b];
        const unsigned long long m = masks[(long long)b * R + s];
        stitch(st, m, bc.K, bc.new_day);
        if (out.masks) out.masks[(long long)bc.mask_block * R + r] |= m;
    }
    out.gross[r] = st.gross;
    best[r] = st.best;
    run[r] = st.run;
    if (last && out.minutes) out.minutes[r] = (float)st.gross * out.step_minutes;
}

void normalize3(double* v) {
    const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
}

// The run's middle direction d_m (as stored, FP32) and an FP32 orthonormal basis around
// it: t along the run's motion, b = n x t, n = d_m / |d_m|; every step's d - d_m is solved
// in that basis (Cramer's rule in double) and the largest |coefficients|, padded, bound
// d . v - d_m . v over the run for any v (run_dot_bounds).
void run_basis(const std::vector<StepConst>& h_steps, int j, int kn, int jm, const double* e1,
               RunLight* rl) {
    const float dmf[3] = {h_steps[jm].dx, h_steps[jm].dy, h_steps[jm].dz};
    double n3[3] = {dmf[0], dmf[1], dmf[2]};
    normalize3(n3);
    const StepConst& sf = h_steps[j];
    const StepConst& sl = h_steps[j + kn - 1];
    double t3[3] = {(double)sl.dx - sf.dx, (double)sl.dy - sf.dy, (double)sl.dz - sf.dz};
    const double tn = t3[0] * n3[0] + t3[1] * n3[1] + t3[2] * n3[2];
    for (int q = 0; q < 3; ++q) t3[q] -= tn * n3[q];
    if (t3[0] * t3[0] + t3[1] * t3[1] + t3[2] * t3[2] < 1e-24)
        for (int q = 0; q < 3; ++q) t3[q] = e1[q];
    normalize3(t3);
    double b3[3] = {n3[1] * t3[2] - n3[2] * t3[1], n3[2] * t3[0] - n3[0] * t3[2], n3[0] * t3[1] - n3[1] * t3[0]};
    normalize3(b3);
    float tf[3], bf[3], nf[3];
    for (int q = 0; q < 3; ++q) {
        tf[q] = (float)t3[q];
        bf[q] = (float)b3[q];
        nf[q] = (float)n3[q];
    }
    const double M[3][3] = {{tf[0], bf[0], nf[0]}, {tf[1], bf[1], nf[1]}, {tf[2], bf[2], nf[2]}};
    auto det3 = [](const double A[3][3]) {
        return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    };
    const double D = det3(M);
    double mx[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < kn; ++k) {
        const StepConst& s = h_steps[j + k];
        const double dl[3] = {(double)s.dx - dmf[0], (double)s.dy - dmf[1], (double)s.dz - dmf[2]};
        for (int col = 0; col < 3; ++col) {
            double Mc[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) Mc[r][c] = c == col ? dl[r] : M[r][c];
            mx[col] = std::max(mx[col], fabs(det3(Mc) / D));
        }
    }
    for (int q = 0; q < 3; ++q) {
        rl->dm[q] = dmf[q];
        rl->tv[q] = tf[q];
        rl->bv[q] = bf[q];
    }
    rl->ba = (float)(mx[0] * (1.0 + 1e-6) + 1e-12);
    rl->bb = (float)(mx[1] * (1.0 + 1e-6) + 1e-12);
    rl->bn = (float)(mx[2] * (1.0 + 1e-6) + 1e-12);
}

int g_point_run = 27;

}  // namespace

void set_point_run(int run) { g_point_run = run; }
int get_point_run() { return g_point_run; }

cudaError_t launch_sam_points(const DevScene& sc, const float* scene_box, const DevRecv& rc,
                              const float* recv_box, const DevSun& sun,
                              const std::vector<BlockConst>& h_blocks,
                              const std::vector<StepConst>& h_steps, const DevOut& out,
                              cudaStream_t st) {
    const long long R = rc.R;
    if (R == 0 || h_blocks.empty()) return cudaSuccess;
    const int run_len = std::max(1, std::min(kRunMax, get_point_run()));
    const float tile = SA_LIGHT_TILE;
    // blocks per chunk: the receiver bins hold every receiver once per run (4 bytes), the
    // masks 8 bytes per receiver and block; keep both within ~1 GiB and <= 64 blocks
    const int runs_per_block = (kMaxBlock + run_len - 1) / run_len;
    const long long per_block = (long long)R * (4ll * runs_per_block + 8ll);
    const int chunk = (int)std::max(1ll, std::min(64ll, (1ll << 30) / std::max(1ll, per_block)));
    const int nbc_max = std::min(chunk, (int)h_blocks.size());
    cudaError_t e = cudaSuccess;
    unsigned long long* masks = nullptr;
    int *run = nullptr, *best = nullptr;
    e = sa::scratch_alloc(&masks, sizeof(unsigned long long) * (size_t)R * nbc_max, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&run, sizeof(int) * (size_t)R, st);
    if (e == cudaSuccess && !out.continuous) e = sa::scratch_alloc(&best, sizeof(int) * (size_t)R, st);
    if (e == cudaSuccess && out.accumulate_into && !out.continuous)
        e = cudaMemsetAsync(best, 0, sizeof(int) * (size_t)R, st);
    int* bestp = out.continuous ? out.continuous : best;
    const double c[3] = {0.5 * (recv_box[0] + recv_box[3]), 0.5 * (recv_box[1] + recv_box[4]),
                         0.5 * (recv_box[2] + recv_box[5])};
    const double zmin_r = recv_box[2];
    std::vector<RunLight> hr;
    std::vector<int> tile_run;
    const int n_blocks = (int)h_blocks.size();
    // a chunk also ends once its runs hold kMaxTiles light-space tiles
    constexpr long long kMaxTiles = 1ll << 24;
    for (int b0 = 0, nbc = 0; b0 < n_blocks && e == cudaSuccess; b0 += nbc) {
        hr.clear();
        tile_run.clear();
        int tiles = 0;
        for (nbc = 0; nbc < chunk && b0 + nbc < n_blocks && (nbc == 0 || tiles < kMaxTiles); ++nbc) {
            const int bl = nbc;
            const BlockConst& bc = h_blocks[b0 + bl];
            // the block's steps in nr runs of balanced lengths (<= run_len)
            const int nr = (bc.K + run_len - 1) / run_len;
            for (int ri = 0; ri < nr; ++ri) {
                const int k0 = ri * bc.K / nr;
                RunLight rl;
                memset(&rl, 0, sizeof(rl));
                rl.k0 = k0;
                rl.kn = (ri + 1) * bc.K / nr - k0;
                rl.j0 = bc.j0;
                rl.blk = bl;
                const int jm = bc.j0 + k0 + rl.kn / 2;
                double dm[3] = {h_steps[jm].dx, h_steps[jm].dy, h_steps[jm].dz};
                normalize3(dm);
                double e1[3] = {dm[1], -dm[0], 0.0};          // horizontal, orthogonal to dm
                if (e1[0] * e1[0] + e1[1] * e1[1] < 1e-12) { e1[0] = 1.0; e1[1] = 0.0; }
                normalize3(e1);
                double e2[3] = {dm[1] * e1[2] - dm[2] * e1[1], dm[2] * e1[0] - dm[0] * e1[2],
                                dm[0] * e1[1] - dm[1] * e1[0]};
                normalize3(e2);
                // drift per metre of height of each step's ray in light space; its box over
                // the run, padded for rounding, gives the culls' margins
                double da_lo = 0.0, da_hi = 0.0, db_lo = 0.0, db_hi = 0.0;
                for (int k = 0; k < rl.kn; ++k) {
                    const StepConst& s = h_steps[bc.j0 + k0 + k];
                    const double d[3] = {s.dx, s.dy, s.dz};
                    const double dz = std::max(d[2], 1e-6);
                    const double da = (e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2]) / dz;
                    const double db = (e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2]) / dz;
                    da_lo = std::min(da_lo, da); da_hi = std::max(da_hi, da);
                    db_lo = std::min(db_lo, db); db_hi = std::max(db_hi, db);
                }
                const double pad = 1e-6 + 1e-4 * std::max(da_hi - da_lo, db_hi - db_lo);
                rl.da_hi = (float)(da_hi * 1.0001 + pad);
                rl.da_lo = (float)(-da_lo * 1.0001 + pad);
                rl.db_hi = (float)(db_hi * 1.0001 + pad);
                rl.db_lo = (float)(-db_lo * 1.0001 + pad);
                rl.zr = (float)zmin_r - 0.01f;
                run_basis(h_steps, bc.j0 + k0, rl.kn, jm, e1, &rl);
                for (int q = 0; q < 3; ++q) { rl.e1[q] = (float)e1[q]; rl.e2[q] = (float)e2[q]; rl.c[q] = (float)c[q]; }
                // tile grid over the light-space box of the receivers
                double amin = 1e30, amax = -1e30, bmin = 1e30, bmax = -1e30;
                for (int corner = 0; corner < 8; ++corner) {
                    const double x = (corner & 1 ? recv_box[3] : recv_box[0]) - c[0];
                    const double y = (corner & 2 ? recv_box[4] : recv_box[1]) - c[1];
                    const double z = (corner & 4 ? recv_box[5] : recv_box[2]) - c[2];
                    const double a = e1[0] * x + e1[1] * y + e1[2] * z, b = e2[0] * x + e2[1] * y + e2[2] * z;
                    amin = std::min(amin, a); amax = std::max(amax, a);
                    bmin = std::min(bmin, b); bmax = std::max(bmax, b);
                }
                double ts = tile;
                while ((amax - amin) / ts * (bmax - bmin) / ts > 4.0e6) ts *= 2.0;
                rl.tile = (float)ts;
                rl.a0 = (float)(amin - 1.0);
                rl.b0 = (float)(bmin - 1.0);
                rl.nta = std::max(1, (int)std::ceil((amax - amin + 2.0) / ts));
                rl.ntb = std::max(1, (int)std::ceil((bmax - bmin + 2.0) / ts));
                rl.tile_base = tiles;
                tiles += rl.nta * rl.ntb;
                for (int q = 0; q < rl.nta * rl.ntb; ++q) tile_run.push_back((int)hr.size());
                hr.push_back(rl);
            }
        }
        const int n_runs = (int)hr.size();
        RunLight* d_runs = nullptr;
        int* d_tile_run = nullptr;
        unsigned *tc = nullptr, *toff = nullptr, *tcur = nullptr, *rcn = nullptr, *roff = nullptr,
                 *rcur = nullptr, *d_total = nullptr, *hist = nullptr;
        int *tbins = nullptr, *rbins = nullptr, *order = nullptr;
        const size_t nt = (size_t)tiles;
#define TRYB(x) do { if (e == cudaSuccess) e = (x); } while (0)
        TRYB(cudaMemsetAsync(masks, 0, sizeof(unsigned long long) * (size_t)R * nbc, st));
        TRYB(sa::scratch_alloc(&d_runs, sizeof(RunLight) * hr.size(), st));
        TRYB(sa::scratch_alloc(&d_tile_run, sizeof(int) * nt, st));
        TRYB(sa::scratch_alloc(&tc, sizeof(unsigned) * nt, st));
        TRYB(sa::scratch_alloc(&toff, sizeof(unsigned) * nt, st));
        TRYB(sa::scratch_alloc(&tcur, sizeof(unsigned) * nt, st));
        TRYB(sa::scratch_alloc(&rcn, sizeof(unsigned) * nt, st));
        TRYB(sa::scratch_alloc(&roff, sizeof(unsigned) * nt, st));
        TRYB(sa::scratch_alloc(&rcur, sizeof(unsigned) * nt, st));
        TRYB(sa::scratch_alloc(&d_total, 2 * sizeof(unsigned), st));   // bin total, tiles with work
        TRYB(sa::scratch_alloc(&hist, sizeof(unsigned) * kOrderBuckets, st));
        TRYB(sa::scratch_alloc(&order, sizeof(int) * nt, st));
        TRYB(sa::scratch_alloc(&rbins, sizeof(int) * (size_t)R * n_runs, st));
        TRYB(cudaMemcpyAsync(d_runs, hr.data(), sizeof(RunLight) * hr.size(), cudaMemcpyHostToDevice, st));
        TRYB(cudaMemcpyAsync(d_tile_run, tile_run.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st));
        TRYB(cudaMemsetAsync(tc, 0, sizeof(unsigned) * nt, st));
        TRYB(cudaMemsetAsync(tcur, 0, sizeof(unsigned) * nt, st));
        TRYB(cudaMemsetAsync(rcn, 0, sizeof(unsigned) * nt, st));
        TRYB(cudaMemsetAsync(rcur, 0, sizeof(unsigned) * nt, st));
        TRYB(cudaMemsetAsync(hist, 0, sizeof(unsigned) * kOrderBuckets, st));
        const dim3 gt((unsigned)std::max(1, (sc.T + 127) / 128), n_runs);
        const dim3 gr((unsigned)((R + 255) / 256), n_runs);
        unsigned totals[2] = {0u, 0u};
        const unsigned go = (unsigned)((nt + 255) / 256);
        if (e == cudaSuccess) {
            if (sc.T > 0) k_lt_bin<<<gt, 128, 0, st>>>(sc, sun.steps, d_runs, n_runs, false, tc, nullptr, nullptr, nullptr);
            k_lr_bin<<<gr, 256, 0, st>>>(rc.orig, R, d_runs, n_runs, false, rcn, nullptr, nullptr, nullptr);
            k_order_hist<<<go, 256, 0, st>>>(tc, rcn, (long long)nt, hist);
            k_order_scan<<<1, 32, 0, st>>>(hist, d_total + 1);
            k_order_fill<<<go, 256, 0, st>>>(tc, rcn, (long long)nt, hist, order);
            e = cudaGetLastError();
        }
        TRYB(cudaMemcpyAsync(toff, tc, sizeof(unsigned) * nt, cudaMemcpyDeviceToDevice, st));
        TRYB(cudaMemcpyAsync(roff, rcn, sizeof(unsigned) * nt, cudaMemcpyDeviceToDevice, st));
        TRYB(exclusive_scan_u32(roff, (long long)nt, nullptr, st));
        TRYB(exclusive_scan_u32(toff, (long long)nt, d_total, st));
        TRYB(cudaMemcpyAsync(totals, d_total, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        TRYB(cudaStreamSynchronize(st));
        const unsigned total = totals[0], work_tiles = totals[1];
        TRYB(sa::scratch_alloc(&tbins, sizeof(int) * ((size_t)total + 1), st));
        if (e == cudaSuccess) {
            if (sc.T > 0 && total > 0)
                k_lt_bin<<<gt, 128, 0, st>>>(sc, sun.steps, d_runs, n_runs, true, nullptr, toff, tcur, tbins);
            k_lr_bin<<<gr, 256, 0, st>>>(rc.orig, R, d_runs, n_runs, true, nullptr, roff, rcur, rbins);
            TileArgs ta;
            ta.sc = sc; ta.steps = sun.steps; ta.runs = d_runs; ta.n_runs = n_runs;
            ta.tile_run = d_tile_run;
            ta.order = order;
            ta.t_off = toff; ta.t_cnt = tc; ta.t_bins = tbins;
            ta.r_off = roff; ta.r_cnt = rcn; ta.r_bins = rbins;
            ta.orig = rc.orig; ta.masks = masks; ta.R = R; ta.stats = out.stats;
            if (work_tiles > 0) {
                KernelTimer kt(KT_SAM_POINTS, st);
                if (out.stats) k_sam_tile<true><<<work_tiles, kTileThreads, 0, st>>>(ta);
                else k_sam_tile<false><<<work_tiles, kTileThreads, 0, st>>>(ta);
            }
            k_points_fold<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(
                R, rc.perm, sun.blocks + b0, nbc, masks, out, run, bestp, b0 == 0,
                b0 + nbc == n_blocks);
            e = cudaGetLastError();
        }
        for (void* p : {(void*)d_runs, (void*)d_tile_run, (void*)tc, (void*)toff, (void*)tcur,
                        (void*)rcn, (void*)roff, (void*)rcur, (void*)d_total, (void*)tbins, (void*)rbins,
                        (void*)hist, (void*)order})
            if (p) cudaFreeAsync(p, st);
#undef TRYB
    }
    if (masks) cudaFreeAsync(masks, st);
    if (run) cudaFreeAsync(run, st);
    if (best) cudaFreeAsync(best, st);
    return e;
}

}  // namespace sa
