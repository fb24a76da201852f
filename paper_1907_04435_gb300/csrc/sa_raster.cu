// sa_raster.cu -- shadow accrual map of a ground receiver grid (Sec. 4).
//
// The paper's shadow accrual map projects every occluder point s along the block's sun
// directions onto a shadow plane and writes one depth slice per step in a single pass over
// the geometry (Sec. 4, Step 1; Theorem 1 shows the slices equal one shadow map per step).
// For receivers on the ground the shadow plane can be the ground itself: every occluder
// lies above z = 0, so a ground point is shadowed at step j exactly when it lies inside
// the projection of some triangle along d_j onto z = 0 (no depth test is needed, Step 2
// reduces to a coverage test).  The map is therefore kept in receiver space, at the
// receivers themselves, as one bit per step: no texel resampling, no aliasing, no bias.
//
// Per block of <= 64 steps:
//   k_bin_count / k_bin_fill  one pass over the triangles bins each into the 32 x 32-cell
//                             tiles its projection can reach during the block (the
//                             triangle swept along the block's slope box)
//   k_raster                  one CTA per tile keeps the tile's 1024 x 64-bit slices in
//                             registers, projects each binned triangle for every step of
//                             the block and sets bit k of each covered cell; the gross /
//                             continuous reduction is fused into the epilogue.
// With one step per block the same kernels form the per-step shadow raster baseline.
//
// Coverage is decided with edge functions evaluated from canonically ordered endpoints,
// so an edge shared by two projected triangles yields exactly negated values in the two
// and a cell centre on it is covered by at least one (watertight).
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kTile = 32;               // cells per tile side
constexpr int kRasterThreads = 256;     // 8 warps x 4 rows each
// triangles staged per batch (<= 128: a unit index t x runs + run stays below 2^13, which
// the float quotient that decodes it and the queue's 13 bits for it both need)
#ifndef SA_RASTER_BATCH
#define SA_RASTER_BATCH 64
#endif
constexpr int kTriBatch = SA_RASTER_BATCH;
// work units a warp claims at a time (<= 32: one lane each while their boxes are bounded)
#ifndef SA_RASTER_CLAIM
#define SA_RASTER_CLAIM 4
#endif
constexpr int kUnitClaim = SA_RASTER_CLAIM;
// resident CTAs per SM the raster kernels are compiled for (registers: 65536 / (256 x this));
// 6 is also what their 35.9 KB of shared memory allows
#ifndef SA_RASTER_CTAS
#define SA_RASTER_CTAS 6
#endif

struct TileGeom {
    float x0, y0, dx;
    int nx, ny, tiles_x, tiles_y;
};

__device__ __forceinline__ bool tri_above_ground(const float4& a, const float4& b, const float4& c) {
    return fmaxf(a.z, fmaxf(b.z, c.z)) > 0.f;
}

// Conservative tile range of a triangle swept over a slope box.
__device__ __forceinline__ bool swept_tiles(const float4& a, const float4& b, const float4& c,
                                            const BlockConst& bc, const TileGeom& g, int* tx0,
                                            int* tx1, int* ty0, int* ty1) {
    float xmin = 3.4e38f, xmax = -3.4e38f, ymin = 3.4e38f, ymax = -3.4e38f;
    const float4* v[3] = {&a, &b, &c};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float z = fmaxf(v[q]->z, 0.f);
        xmin = fminf(xmin, v[q]->x - z * bc.uxhi);
        xmax = fmaxf(xmax, v[q]->x - z * bc.uxlo);
        ymin = fminf(ymin, v[q]->y - z * bc.uyhi);
        ymax = fmaxf(ymax, v[q]->y - z * bc.uylo);
    }
    const float inv = 1.f / (kTile * g.dx);
    // one cell of margin on every side absorbs rounding of the projections
    const float fx0 = floorf((xmin - g.x0 - g.dx) * inv), fx1 = floorf((xmax - g.x0 + g.dx) * inv);
    const float fy0 = floorf((ymin - g.y0 - g.dx) * inv), fy1 = floorf((ymax - g.y0 + g.dx) * inv);
    if (fx1 < 0.f || fy1 < 0.f || fx0 >= (float)g.tiles_x || fy0 >= (float)g.tiles_y) return false;
    *tx0 = (int)fmaxf(fx0, 0.f);
    *tx1 = (int)fminf(fx1, (float)(g.tiles_x - 1));
    *ty0 = (int)fmaxf(fy0, 0.f);
    *ty1 = (int)fminf(fy1, (float)(g.tiles_y - 1));
    return true;
}

// For a closed scene only triangles facing the sun at some step of the block cast the
// shadow's coverage (the projection of a closed solid is covered by its sun-facing faces).
__device__ __forceinline__ bool faces_sun(const float4& a, const float4& b, const float4& c,
                                          const StepConst* steps, const BlockConst& bc) {
    const float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
    const float vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
    const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    for (int k = 0; k < bc.K; ++k) {
        const StepConst& s = steps[bc.j0 + k];
        if (nx * s.dx + ny * s.dy + nz * s.dz > 0.f) return true;
    }
    return false;
}

__global__ void k_bin_count(DevScene sc, const StepConst* __restrict__ steps,
                            const BlockConst* __restrict__ blocks, int b0,
                            TileGeom g, unsigned* __restrict__ counts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int bl = blockIdx.y;
    if (t >= sc.T) return;
    const float4 a = __ldg(&sc.tris[3 * t]), b = __ldg(&sc.tris[3 * t + 1]),
                 c = __ldg(&sc.tris[3 * t + 2]);
    if (!tri_above_ground(a, b, c)) return;
    // the tile range first: it culls the triangles whose shadow misses the grid before the
    // per-step facing test (both are conservative, so the order leaves the bins unchanged)
    int tx0, tx1, ty0, ty1;
    if (!swept_tiles(a, b, c, blocks[b0 + bl], g, &tx0, &tx1, &ty0, &ty1)) return;
    if (sc.closed && !faces_sun(a, b, c, steps, blocks[b0 + bl])) return;
    unsigned* row = counts + (size_t)bl * g.tiles_x * g.tiles_y;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&row[ty * g.tiles_x + tx], 1u);
}

__global__ void k_bin_fill(DevScene sc, const StepConst* __restrict__ steps,
                           const BlockConst* __restrict__ blocks, int b0,
                           TileGeom g, const unsigned* __restrict__ offsets,
                           unsigned* __restrict__ cursor, int* __restrict__ bins) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int bl = blockIdx.y;
    if (t >= sc.T) return;
    const float4 a = __ldg(&sc.tris[3 * t]), b = __ldg(&sc.tris[3 * t + 1]),
                 c = __ldg(&sc.tris[3 * t + 2]);
    if (!tri_above_ground(a, b, c)) return;
    int tx0, tx1, ty0, ty1;
    if (!swept_tiles(a, b, c, blocks[b0 + bl], g, &tx0, &tx1, &ty0, &ty1)) return;
    if (sc.closed && !faces_sun(a, b, c, steps, blocks[b0 + bl])) return;
    const size_t row = (size_t)bl * g.tiles_x * g.tiles_y;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const size_t cell = row + ty * g.tiles_x + tx;
            bins[offsets[cell] + atomicAdd(&cursor[cell], 1u)] = t;
        }
}

struct RasterArgs {
    DevScene sc;
    DevSun sun;
    TileGeom g;
    int b0, nbc;                     // first block and number of blocks of this chunk
    const unsigned* offsets;         // [nbc][tiles] bin offsets
    const unsigned* counts;          // [nbc][tiles] bin sizes
    const int* bins;
    DevOut out;
    int* best;                       // continuous state (== out.continuous or scratch)
    int load_state;                  // 0: start from zero, 1: from out.gross / best / run
    int final_chunk;
    int cull;                        // closed scene: only faces toward the sun
    int run;                         // steps per work unit
    long long R;
    const int* order;                // tile of each CTA (null: CTA i takes tile i)
};

constexpr int kWarpsRaster = kRasterThreads / 32;

struct BatchArgs {
    TileGeom g;
    const float4* base_tris;
    const BatchInterval* intervals;
    const BatchVariant* variants;
    const int4* items;                // (interval, variant, tile, 0)
    int n_items;
    unsigned* counter;                // work queue head, zeroed before the launch
    const int* removed;               // removed base building ids of all variants
    const float4* tower_tris;         // tower triangles of all variants (3 float4 each)
    int* counts_out;
    int* impact_out;                  // nullable
    int cull;
    int run;                          // steps per work unit
    unsigned long long* stats;        // nullable
};
// steps per work unit (run length); a process-wide option, 24 by default
int g_raster_run = 24;

// Edge function of a triangle edge (3D endpoints v -> v') projected along step k, at a
// ground point p (all xy tile-local).  With c = p - v.xy and e = v' - v,
//   E_k(p) = cross(q' - q, p - q),  q = v.xy - v.z u_k,  u_k = d_xy / d_z,
// expands to  E_k(p) = P + Qx u_k.x + Qy u_k.y  with
//   P = e.x c.y - e.y c.x,  Qx = -v.z e.y - e.z c.y,  Qy = v.z e.x + e.z c.x,
// so a cell sets (P, Qx, Qy) up once and tests a run of steps with two FMAs per edge.
// The endpoints are taken in a canonical order (the other order only flips the sign), so
// an edge shared by two triangles gives the same value in both up to an exact negation:
// a cell on it is covered by at least one (watertight).
struct EdgeRef {
    float vx, vy, vz, ex, ey, ez;   // canonical start point, and the edge vector times the
                                    // sign of the triangle's own orientation of the edge
};

// The sign is folded into the edge vector: P, Qx and Qy are then the canonical values
// times +-1, and since rounding to nearest is symmetric under negation every step's edge
// value is the canonical one times +-1 exactly, up to the sign of a zero.  The front test
// takes +0 as inside and -0 as outside; where the two triangles of an edge both get a
// zero, at least one of them gets +0 (a rounded sum of zeros is -0 only when both terms
// are -0, and the other triangle's terms are then +0), so a cell on the edge is covered.
// The back test takes both zeros as inside.
__device__ __forceinline__ EdgeRef edge_ref(const float4& a, const float4& b) {
    const bool keep = a.x < b.x || (a.x == b.x && (a.y < b.y || (a.y == b.y && a.z < b.z)));
    const float4& v = keep ? a : b;
    const float4& w = keep ? b : a;
    const float s = keep ? 1.f : -1.f;
    return EdgeRef{v.x, v.y, v.z, s * (w.x - v.x), s * (w.y - v.y), s * (w.z - v.z)};
}

// The edge's step-test terms as affine functions of the cell centre (x, y): with c = (x, y)
// - v, P = e_x c_y - e_y c_x = pa y + pb x + pc, Q_x = -(v_z e_y + e_z c_y) = -ra y + qc and
// Q_y = v_z e_x + e_z c_x = ra x + rc.  The constants are rounded once per staged triangle,
// each from the edge vector in a way that an exactly negated edge vector negates exactly,
// so the triangles sharing an edge still compute exactly negated values.
struct EdgeLin {
    float pa, pb, pc, ra, qc, rc;
};

__device__ __forceinline__ EdgeLin edge_lin(const EdgeRef& e) {
    EdgeLin l;
    l.pa = e.ex;
    l.pb = -e.ey;
    l.pc = -fmaf(l.pa, e.vy, l.pb * e.vx);
    l.ra = e.ez;
    l.qc = -fmaf(e.vz, e.ey, -(e.ez * e.vy));
    l.rc = fmaf(e.vz, e.ex, -(e.ez * e.vx));
    return l;
}

// Shared memory of one tile: staged triangles (xy tile-local), their sun-facing step
// masks, the block's directions, ground slopes and per-run slope boxes, the tile's 64-bit
// step masks and its cell centres.
struct TileSmem {
    float4 tri[kTriBatch * 3];
    unsigned long long front[kTriBatch];     // steps with n . d > 0
    unsigned long long back[kTriBatch];      // steps with n . d < 0 (open scenes only)
    int valid[kTriBatch];
    // the staged triangles' edge functions (EdgeLin, 6 floats each), 20 floats apart so
    // that a cell's test reads them as five float4
    float edges[kTriBatch * 20];
    float2 u[kMaxBlock];
    // slopes of steps (k, k + 1) packed for the paired step tests: [0][i] starts at step
    // 2i, [1][i] at step 2i + 1 (the last pair of a block repeats its last step)
    unsigned long long upx[2][kMaxBlock / 2], upy[2][kMaxBlock / 2];
    float4 d[kMaxBlock];                     // step directions
    float4 ubox[kMaxBlock];                  // per run: (min u.x, max u.x, min u.y, max u.y)
    unsigned long long mask[kTile * kTile];
    // per warp: cells waiting for their step tests, (unit << 10) | cell, drained 32 at a
    // time so that every lane tests a cell whichever unit it comes from
    unsigned queue[kRasterThreads / 32][64];
    float xl[kTile], yl[kTile];
    int next_unit;                           // next work unit of the batch to hand out
    float inv_nsub;                          // 1 / runs of the block
    unsigned char run_k0[kMaxBlock + 1];     // first step of each run, and K
};

// Tile origin and cell centres in tile-local coordinates; the centres are rounded exactly
// as the receivers' world coordinates, then shifted.
__device__ __forceinline__ void tile_setup(TileSmem& sm, const TileGeom& g, int tx, int ty,
                                           float* tox, float* toy) {
    *tox = __fadd_rn(g.x0, __fmul_rn((float)(tx * kTile), g.dx));
    *toy = __fadd_rn(g.y0, __fmul_rn((float)(ty * kTile), g.dx));
    if (threadIdx.x < kTile) {
        sm.xl[threadIdx.x] = __fadd_rn(g.x0, __fmul_rn(__fadd_rn((float)(tx * kTile + threadIdx.x), 0.5f), g.dx)) - *tox;
    } else if (threadIdx.x < 2 * kTile) {
        const int q = threadIdx.x - kTile;
        sm.yl[q] = __fadd_rn(g.y0, __fmul_rn(__fadd_rn((float)(ty * kTile + q), 0.5f), g.dx)) - *toy;
    }
    for (int c = threadIdx.x; c < kTile * kTile; c += kRasterThreads) sm.mask[c] = 0ull;
}

// The steps of one run (kn <= 32 steps from k0) that cover cell (x, y): bit k of the
// result is step k0 + k.  CULL: closed scene, only front faces count.
template <bool CULL>
__device__ __forceinline__ unsigned cell_steps(const TileSmem& sm, const EdgeLin& E0,
                                               const EdgeLin& E1, const EdgeLin& E2, float x,
                                               float y, int k0, int kn, unsigned fr, unsigned bk) {
    float P[3], QX[3], QY[3];
    const EdgeLin* ee[3] = {&E0, &E1, &E2};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const EdgeLin& e = *ee[q];
        P[q] = fmaf(e.pa, y, fmaf(e.pb, x, e.pc));
        QX[q] = fmaf(-e.ra, y, e.qc);
        QY[q] = fmaf(e.ra, x, e.rc);
    }
    // steps in pairs: E = P + Qx u_x + Qy u_y for two steps per packed instruction
    unsigned long long P2[3], QX2[3], QY2[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        P2[q] = f2_pack(P[q], P[q]);
        QX2[q] = f2_pack(QX[q], QX[q]);
        QY2[q] = f2_pack(QY[q], QY[q]);
    }
    const unsigned long long* upx = sm.upx[k0 & 1] + (k0 >> 1);
    const unsigned long long* upy = sm.upy[k0 & 1] + (k0 >> 1);
    // Fully unrolled over the longest run.  A step covers the cell from the front when no
    // edge value has its sign bit set (+0 counts as inside, -0 as outside): that bit is
    // shifted in from the sign word, so the front mask comes out in reverse step order.
    // From the back (open scenes) all three values are <= 0, zeros of either sign
    // included: two back faces sharing an edge may both get +0 there.
    unsigned hf = 0, hb = 0;
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
        if (k >= kn) break;
        const unsigned long long ux = upx[k >> 1], uy = upy[k >> 1];
        float f[3][2];
#pragma unroll
        for (int q = 0; q < 3; ++q) f2_unpack(f2_fma(QY2[q], uy, f2_fma(QX2[q], ux, P2[q])), f[q][0], f[q][1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned a = __float_as_uint(f[0][h]), b = __float_as_uint(f[1][h]), c = __float_as_uint(f[2][h]);
            hf = __funnelshift_l(~(a | b | c), hf, 1);
            if (!CULL && max3f(f[0][h], f[1][h], f[2][h]) <= 0.f) hb |= 1u << (k + h);
        }
    }
    // steps 0 .. K2 - 1 (an odd run's last pair repeats a step beyond it, which the masks
    // below drop) back in order: step k at bit k
    const int K2 = (kn + 1) & ~1;
    hf = __brev(hf) >> (32 - K2);
    return CULL ? (hf & fr) : ((hf & fr) | (hb & bk));
}

// Step tests of up to 32 queued cells, one per lane: each item names its work unit
// (triangle of the staged batch and run of the block) and its cell; the unit's run, its
// facing steps and the triangle's canonical edges are read back from shared memory.
template <bool COUNT, bool CULL>
__device__ __forceinline__ void drain_cells(TileSmem& sm, const unsigned* q, int n, int nsub,
                                            unsigned long long& n_cell,
                                            unsigned long long& n_test) {
    const int lane = threadIdx.x & 31;
    if (lane >= n) return;
    const unsigned item = q[lane];
    const int un = (int)(item >> 10), cell = (int)(item & 1023u);
    const int t = (int)(((float)un + 0.5f) * sm.inv_nsub), sub = un - t * nsub;
    const int k0 = sm.run_k0[sub], kn = sm.run_k0[sub + 1] - k0;
    const unsigned run_bits = (kn >= 32) ? 0xffffffffu : ((1u << kn) - 1u);
    const unsigned fr = (unsigned)(sm.front[t] >> k0) & run_bits;
    const unsigned bk = CULL ? 0u : ((unsigned)(sm.back[t] >> k0) & run_bits);
    const float4* ef = reinterpret_cast<const float4*>(&sm.edges[20 * t]);
    const float4 f0 = ef[0], f1 = ef[1], f2 = ef[2], f3 = ef[3], f4 = ef[4];
    const EdgeLin E0{f0.x, f0.y, f0.z, f0.w, f1.x, f1.y};
    const EdgeLin E1{f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
    const EdgeLin E2{f3.x, f3.y, f3.z, f3.w, f4.x, f4.y};
    if (COUNT) { ++n_cell; n_test += kn; }
    const unsigned hit = cell_steps<CULL>(sm, E0, E1, E2, sm.xl[cell & (kTile - 1)],
                                          sm.yl[cell >> 5], k0, kn, fr, bk);
    if (hit) atomicOr(&sm.mask[SA_CHK(cell, kTile * kTile, sa::CK_RASTER_CELL)], (unsigned long long)hit << k0);
}

// A work unit is triangle t of the staged batch and run `sub` of the block, un = t nsub +
// sub; (un + 1/2) / nsub is at least 1 / (2 nsub) from an integer, far beyond the float
// quotient's rounding (relative 2^-23) for un < 2^13.
struct UnitRun {
    int t, sub, k0;
    unsigned fr, bk;     // the run's steps the triangle faces (front; back, open scenes only)
};

template <bool CULL>
__device__ __forceinline__ UnitRun unit_run(const TileSmem& sm, int un, int nsub) {
    UnitRun u;
    u.t = (int)(((float)un + 0.5f) * sm.inv_nsub);
    u.sub = un - u.t * nsub;
    u.k0 = sm.run_k0[u.sub];
    const int kn = sm.run_k0[u.sub + 1] - u.k0;       // balanced runs
    const unsigned run_bits = (kn >= 32) ? 0xffffffffu : ((1u << kn) - 1u);
    u.fr = (unsigned)(sm.front[u.t] >> u.k0) & run_bits;
    u.bk = CULL ? 0u : ((unsigned)(sm.back[u.t] >> u.k0) & run_bits);
    return u;
}

// The cells of the tile whose centres (k + 0.5) dx fall in the swept bounding box of the
// run's projections, with 0.01 cell of slack, as columns c0..c1 and rows r0..r1 packed
// 5 bits each (c0 | c1 << 5 | r0 << 10 | r1 << 15); -1 when the unit reaches no cell.
__device__ __forceinline__ int unit_box(const TileSmem& sm, const UnitRun& u, float inv_dx) {
    if ((u.fr | u.bk) == 0u) return -1;
    const float4 a = sm.tri[3 * u.t], b = sm.tri[3 * u.t + 1], c = sm.tri[3 * u.t + 2];
    const float4 ub = sm.ubox[u.sub];
    const float uxlo = ub.x, uxhi = ub.y, uylo = ub.z, uyhi = ub.w;
    const float az = fmaxf(a.z, 0.f), bz = fmaxf(b.z, 0.f), cz = fmaxf(c.z, 0.f);
    const float xmin = fminf(a.x - az * uxhi, fminf(b.x - bz * uxhi, c.x - cz * uxhi));
    const float xmax = fmaxf(a.x - az * uxlo, fmaxf(b.x - bz * uxlo, c.x - cz * uxlo));
    const float ymin = fminf(a.y - az * uyhi, fminf(b.y - bz * uyhi, c.y - cz * uyhi));
    const float ymax = fmaxf(a.y - az * uylo, fmaxf(b.y - bz * uylo, c.y - cz * uylo));
    const float fc0 = ceilf(xmin * inv_dx - 0.51f), fc1 = floorf(xmax * inv_dx - 0.49f);
    const float fr0 = ceilf(ymin * inv_dx - 0.51f), fr1 = floorf(ymax * inv_dx - 0.49f);
    if (fc1 < 0.f || fr1 < 0.f || fc0 > (float)(kTile - 1) || fr0 > (float)(kTile - 1) ||
        fc0 > fc1 || fr0 > fr1) return -1;
    const int c0 = (int)fmaxf(fc0, 0.f), c1 = (int)fminf(fc1, (float)(kTile - 1));
    const int r0 = (int)fmaxf(fr0, 0.f), r1 = (int)fminf(fr1, (float)(kTile - 1));
    return c0 | (c1 << 5) | (r0 << 10) | (r1 << 15);
}

// Row span of a unit in tile row `row` (within its box): the cells cs .. cs + w - 1.
// Each step's projection lies inside the projection for the run's middle slope u_m
// widened by (sx, sy) = z_max |u_hi - u_lo| / 2 (a vertex at height z moves by
// z (u_m - u_k)); the x-range of the middle projection over the band [y - sy, y + sy],
// widened by sx, bounds the row's covered cells (0.05 cell and 2 mm of slack absorb
// rounding).
__device__ __forceinline__ void row_span(const TileSmem& sm, const UnitRun& u, int box, int row,
                                         float inv_dx, int* cs, int* w) {
    *cs = 0;
    *w = 0;
    const int c0 = box & 31, c1 = (box >> 5) & 31;
    const float4 a = sm.tri[3 * u.t], b = sm.tri[3 * u.t + 1], c = sm.tri[3 * u.t + 2];
    const float4 ub = sm.ubox[u.sub];
    const float uxlo = ub.x, uxhi = ub.y, uylo = ub.z, uyhi = ub.w;
    const float az = fmaxf(a.z, 0.f), bz = fmaxf(b.z, 0.f), cz = fmaxf(c.z, 0.f);
    const float umx = 0.5f * (uxlo + uxhi), umy = 0.5f * (uylo + uyhi);
    const float zm = fmaxf(az, fmaxf(bz, cz));
    const float slack = 0.05f + 2e-3f * inv_dx;                 // in cells
    const float sx = zm * (uxhi - uxlo) * 0.5f, sy = zm * (uyhi - uylo) * 0.5f;
    const float px[3] = {a.x - az * umx, b.x - bz * umx, c.x - cz * umx};
    const float py[3] = {a.y - az * umy, b.y - bz * umy, c.y - cz * umy};
    const float y = sm.yl[row];
    const float band = sy + slack / inv_dx;
    const float ya = y - band, yb = y + band;
    float lo = 3.4e38f, hi = -3.4e38f;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        if (py[v] >= ya && py[v] <= yb) { lo = fminf(lo, px[v]); hi = fmaxf(hi, px[v]); }
        const int q = v == 2 ? 0 : v + 1;
        const float dy = py[q] - py[v];
        if (dy != 0.f) {
            // the spans carry slack, so an approximate quotient suffices
            const float slope = __fdividef(px[q] - px[v], dy);
            const float e0 = fminf(py[v], py[q]), e1 = fmaxf(py[v], py[q]);
            if (ya >= e0 && ya <= e1) {
                const float x = fmaf(ya - py[v], slope, px[v]);
                lo = fminf(lo, x); hi = fmaxf(hi, x);
            }
            if (yb >= e0 && yb <= e1) {
                const float x = fmaf(yb - py[v], slope, px[v]);
                lo = fminf(lo, x); hi = fmaxf(hi, x);
            }
        }
    }
    if (lo <= hi) {
        const float f0 = fmaxf(ceilf((lo - sx) * inv_dx - 0.5f - slack), (float)c0);
        const float f1 = fminf(floorf((hi + sx) * inv_dx - 0.5f + slack), (float)c1);
        if (f0 <= f1) {
            *cs = (int)f0;
            *w = (int)f1 - *cs + 1;
        }
    }
}

// Index of the lane whose inclusive prefix sum first exceeds idx (incl non-decreasing over
// the lanes, idx < its value in lane 31).
__device__ __forceinline__ int prefix_lane(int incl, int idx) {
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, j + step - 1);
        if (v <= idx) j += step;
    }
    return j;
}

__device__ __forceinline__ int lane_prefix(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += v;
    }
    return x;
}

// Up to 32 work units un0 .. un0 + nu - 1, expanded level by level so that every lane
// has work: one lane per unit bounds its swept box; one lane per covered row finds the
// row's span; one lane per covered cell checks whether the cell is already shadowed at
// every step its unit could set (a stale read only skips less) and queues the others,
// (unit << 10) | cell, for the step tests, 32 at a time whichever unit they come from.
template <bool COUNT, bool CULL>
__device__ __forceinline__ void raster_units(TileSmem& sm, int un0, int nu, int nsub, float inv_dx,
                                             int& qn, unsigned long long& n_cell,
                                             unsigned long long& n_test,
                                             unsigned long long& n_unit,
                                             unsigned long long& n_span) {
    const int lane = threadIdx.x & 31;
    int box = -1;
    if (lane < nu) box = unit_box(sm, unit_run<CULL>(sm, un0 + lane, nsub), inv_dx);
    const int rows = box < 0 ? 0 : ((box >> 15) & 31) - ((box >> 10) & 31) + 1;
    if (COUNT) {
        const unsigned reach = __ballot_sync(0xffffffffu, rows > 0);
        if (lane == 0) n_unit += (unsigned long long)__popc(reach);
    }
    const int rincl = lane_prefix(rows);
    const int total_rows = __shfl_sync(0xffffffffu, rincl, 31);
    unsigned* q = sm.queue[threadIdx.x >> 5];
    for (int rb = 0; rb < total_rows; rb += 32) {
        // this lane's (unit, row)
        const int ridx = rb + lane;
        const int i = prefix_lane(rincl, ridx) & 31;
        const int rex = __shfl_sync(0xffffffffu, rincl - rows, i);
        const int ubox = __shfl_sync(0xffffffffu, box, i);
        const int un = un0 + i;
        int cs = 0, w = 0;
        unsigned long long can = 0ull;
        if (ridx < total_rows) {
            const UnitRun u = unit_run<CULL>(sm, un, nsub);
            const int row = ((ubox >> 10) & 31) + (ridx - rex);
            row_span(sm, u, ubox, row, inv_dx, &cs, &w);
            cs += row * kTile;                      // the row's first cell
            can = (unsigned long long)(u.fr | u.bk) << u.k0;
        }
        const int cincl = lane_prefix(w);
        const int total = __shfl_sync(0xffffffffu, cincl, 31);
        if (COUNT && lane == 0) n_span += (unsigned long long)total;
        const int cex = cincl - w;
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            const int j = prefix_lane(cincl, idx) & 31;
            const int ex = __shfl_sync(0xffffffffu, cex, j);
            const int cj = __shfl_sync(0xffffffffu, cs, j);
            const int uj = __shfl_sync(0xffffffffu, un, j);
            const unsigned long long cn = __shfl_sync(0xffffffffu, can, j);
            const int cell = cj + (idx - ex);
            const bool need = idx < total &&
                              (sm.mask[SA_CHK(cell, kTile * kTile, sa::CK_RASTER_CELL)] & cn) != cn;
            const unsigned bal = __ballot_sync(0xffffffffu, need);
            if (need) q[qn + __popc(bal & ((1u << lane) - 1u))] = ((unsigned)uj << 10) | (unsigned)cell;
            qn += __popc(bal);
            if (qn >= 32) {
                __syncwarp();
                drain_cells<COUNT, CULL>(sm, q + (qn - 32), 32, nsub, n_cell, n_test);
                qn -= 32;
                __syncwarp();
            }
        }
    }
}

// One block of steps of one tile: the n triangles given by fetch(i, vertex, &v) (false =
// skip the triangle) are staged in batches; each warp takes work units (triangle, run of
// <= 32 steps), bounds the run's swept projection, spreads its lanes over the covered
// cells (row-major, 32 at a time) and per cell tests the run's steps with the expanded
// edge functions; step bits are ORed into sm.mask.  Leaves sm.mask complete for the block.
template <bool COUNT, bool CULL, class Fetch>
__device__ void raster_block(TileSmem& sm, const Fetch& fetch, int n, const StepConst* steps,
                             int j0, int K, float tox, float toy, float inv_dx, int kSub,
                             unsigned long long& n_cell, unsigned long long& n_test,
                             unsigned long long& n_unit, unsigned long long& n_span) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nsub = (K + kSub - 1) / kSub;
    __syncthreads();
    if (threadIdx.x < K) {
        const StepConst& s = steps[j0 + threadIdx.x];
        sm.u[threadIdx.x] = make_float2(s.ux, s.uy);
        sm.d[threadIdx.x] = make_float4(s.dx, s.dy, s.dz, 0.f);
    }
    __syncthreads();
    if (threadIdx.x < K) {
        const int k = threadIdx.x, k1 = min(k + 1, K - 1);
        sm.upx[k & 1][k >> 1] = f2_pack(sm.u[k].x, sm.u[k1].x);
        sm.upy[k & 1][k >> 1] = f2_pack(sm.u[k].y, sm.u[k1].y);
    }
    if (threadIdx.x <= nsub) sm.run_k0[threadIdx.x] = (unsigned char)(threadIdx.x * K / nsub);
    if (threadIdx.x == 0) sm.inv_nsub = 1.f / (float)nsub;
    if (threadIdx.x < nsub) {
        const int k0 = threadIdx.x * K / nsub, k1 = (threadIdx.x + 1) * K / nsub;
        float4 b = make_float4(3.4e38f, -3.4e38f, 3.4e38f, -3.4e38f);
        for (int k = k0; k < k1; ++k) {
            const float2 u = sm.u[k];
            b.x = fminf(b.x, u.x); b.y = fmaxf(b.y, u.x);
            b.z = fminf(b.z, u.y); b.w = fmaxf(b.w, u.y);
        }
        sm.ubox[threadIdx.x] = b;
    }
    for (int base = 0; base < n; base += kTriBatch) {
        const int nt = min(kTriBatch, n - base);
        __syncthreads();
        for (int i = threadIdx.x; i < nt * 3; i += kRasterThreads) {
            float4 v;
            const bool ok = fetch(base + i / 3, i % 3, &v);
            v.x -= tox;
            v.y -= toy;
            sm.tri[i] = v;
            if (i % 3 == 0) sm.valid[i / 3] = ok ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) sm.next_unit = kWarpsRaster * kUnitClaim;
        // sun-facing steps of each staged triangle: a warp per triangle, a lane per step
        for (int t = warp; t < nt; t += kWarpsRaster) {
            unsigned long long fr = 0, bk = 0;
            if (sm.valid[t]) {
                const float4 a = sm.tri[3 * t], b = sm.tri[3 * t + 1], c = sm.tri[3 * t + 2];
                const float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
                const float vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
                const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;
                    float nd = 0.f;
                    if (k < K) {
                        const float4 d = sm.d[k];
                        nd = nx * d.x + ny * d.y + nz * d.z;
                    }
                    const unsigned f = __ballot_sync(0xffffffffu, nd > 0.f);
                    const unsigned g = __ballot_sync(0xffffffffu, nd < 0.f);
                    fr |= (unsigned long long)f << (32 * h);
                    bk |= (unsigned long long)g << (32 * h);
                }
                if (CULL) bk = 0ull;
            }
            if (lane == 0) {
                sm.front[t] = fr;
                sm.back[t] = bk;
            }
            if (lane < 3) {
                const float4& p = sm.tri[3 * t + lane];
                const float4& q = sm.tri[3 * t + (lane == 2 ? 0 : lane + 1)];
                const EdgeLin e = edge_lin(edge_ref(p, q));
                float* o = &sm.edges[20 * t + 6 * lane];
                o[0] = e.pa; o[1] = e.pb; o[2] = e.pc; o[3] = e.ra; o[4] = e.qc; o[5] = e.rc;
            }
        }
        __syncthreads();
        const int units = nt * nsub;
        // warps take kUnitClaim units at a time from a shared counter, so an expensive
        // group does not hold the warps that would otherwise wait for its warp at the next
        // barrier (the next group is claimed before this one is worked, hiding the
        // atomic's latency)
        int un = warp * kUnitClaim;
        int qn = 0;
        while (un < units) {
            int nx = 0;
            if (lane == 0) nx = atomicAdd(&sm.next_unit, kUnitClaim);
            raster_units<COUNT, CULL>(sm, un, min(kUnitClaim, units - un), nsub, inv_dx, qn, n_cell, n_test,
                                      n_unit, n_span);
            un = __shfl_sync(0xffffffffu, nx, 0);
        }
        // the queue's last cells, before the batch's triangles are replaced
        __syncwarp();
        drain_cells<COUNT, CULL>(sm, sm.queue[warp], qn, nsub, n_cell, n_test);
        __syncwarp();
    }
    __syncthreads();
}

__device__ __forceinline__ void flush_raster_counts(unsigned long long* stats, unsigned long long n_cell,
                                                    unsigned long long n_test,
                                                    unsigned long long n_unit,
                                                    unsigned long long n_span) {
    for (int o = 16; o > 0; o >>= 1) {
        n_cell += __shfl_down_sync(0xffffffffu, n_cell, o);
        n_test += __shfl_down_sync(0xffffffffu, n_test, o);
        n_unit += __shfl_down_sync(0xffffffffu, n_unit, o);
        n_span += __shfl_down_sync(0xffffffffu, n_span, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&stats[0], n_unit);
        atomicAdd(&stats[1], n_span);
        atomicAdd(&stats[2], n_cell);
        atomicAdd(&stats[3], n_test);
    }
}

// One CTA per 32 x 32-cell tile, every block of the chunk in order; the gross /
// continuous state of the thread's four cells stays in registers between blocks.
template <bool COUNT, bool CULL, int CTAS>
__global__ void __launch_bounds__(kRasterThreads, CTAS)
k_raster(RasterArgs ra) {
    __shared__ TileSmem sm;
    __shared__ RunState s_st[kTile * kTile];       // gross / run / best of the tile's cells
    unsigned long long n_cell = 0, n_test = 0, n_unit = 0, n_span = 0;
    const TileGeom& g = ra.g;
    const int tile = ra.order ? ra.order[blockIdx.x] : (int)blockIdx.x;
    const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = warp * 4;
    float tox, toy;
    tile_setup(sm, g, tx, ty, &tox, &toy);
    const int ix = tx * kTile + lane;
    // each thread owns the cells (row0 + q, lane), q < 4, and alone touches their state
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int iy = ty * kTile + row0 + q;
        const long long o = (long long)iy * g.nx + ix;
        RunState st{0, 0, 0};
        if (ix < g.nx && iy < g.ny && ra.load_state) {
            st.gross = ra.out.gross[o];
            st.best = ra.best[o];
            st.run = ra.out.run[o];
        }
        s_st[(row0 + q) * kTile + lane] = st;
    }
    const int n_tiles = g.tiles_x * g.tiles_y;
    const float inv_dx = 1.f / g.dx;
    for (int bl = 0; bl < ra.nbc; ++bl) {
        const BlockConst* bcp = &ra.sun.blocks[ra.b0 + bl];
        const unsigned off = ra.offsets[(size_t)bl * n_tiles + tile];
        const unsigned cnt = ra.counts[(size_t)bl * n_tiles + tile];
        const int* bins = ra.bins + off;
        const float4* tris = ra.sc.tris;
        const int T = ra.sc.T;
        auto fetch = [bins, tris, T](int i, int v, float4* out) {
            *out = __ldg(&tris[3 * SA_CHK(bins[i], T, sa::CK_RASTER_BIN) + v]);
            (void)T;
            return true;
        };
        raster_block<COUNT, CULL>(sm, fetch, (int)cnt, ra.sun.steps, bcp->j0, bcp->K, tox, toy,
                                  inv_dx, ra.run, n_cell, n_test, n_unit, n_span);
        const int K = bcp->K, new_day = bcp->new_day;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cell = (row0 + q) * kTile + lane;
            const unsigned long long m = sm.mask[cell];
            sm.mask[cell] = 0ull;
            RunState st = s_st[cell];
            stitch(st, m, K, new_day);
            s_st[cell] = st;
            const int iy = ty * kTile + row0 + q;
            if (ra.out.masks && ix < g.nx && iy < g.ny)
                ra.out.masks[(size_t)bcp->mask_block * ra.R + (long long)iy * g.nx + ix] |= m << bcp->mask_bit;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int iy = ty * kTile + row0 + q;
        if (ix >= g.nx || iy >= g.ny) continue;
        const long long o = (long long)iy * g.nx + ix;
        const RunState st = s_st[(row0 + q) * kTile + lane];
        ra.out.gross[o] = st.gross;
        ra.best[o] = st.best;
        ra.out.run[o] = st.run;
        if (ra.final_chunk && ra.out.minutes) ra.out.minutes[o] = (float)st.gross * ra.out.step_minutes;
    }
    if (COUNT) flush_raster_counts(ra.out.stats, n_cell, n_test, n_unit, n_span);
}

// --------------------------------------------------------------- batched scenarios
// A persistent launch over work items (interval, variant, tile of the variant's region).
// Each item rasters every block of its interval for one tile: the base city's binned
// triangles minus the variant's removed buildings, plus the variant's tower triangles.
// It writes the counts of the tile's cells inside the region and, where the base counts
// are given, the impact (variant minus base).
template <bool COUNT, bool CULL>
__global__ void __launch_bounds__(kRasterThreads, SA_RASTER_CTAS)
k_batch(BatchArgs ba) {
    __shared__ TileSmem sm;
    __shared__ RunState s_st[kTile * kTile];       // gross / run / best of the tile's cells
    __shared__ int s_item;
    unsigned long long n_cell = 0, n_test = 0, n_unit = 0, n_span = 0;
    const TileGeom& g = ba.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = warp * 4;
    const float inv_dx = 1.f / g.dx;
    const int n_tiles = g.tiles_x * g.tiles_y;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(ba.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= ba.n_items) break;
        const int4 it = ba.items[item];                  // interval, variant, tile, affected
        const BatchInterval& iv = ba.intervals[it.x];
        const BatchVariant& var = ba.variants[it.y];
        const int tile = it.z;
        const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
        if (!it.w) {
            // neither a removed building's nor a tower's shadow can reach this tile during
            // the interval: the variant's counts are the base counts
            for (int c = threadIdx.x; c < kTile * kTile; c += kRasterThreads) {
                const int ix = tx * kTile + (c & (kTile - 1)), iy = ty * kTile + c / kTile;
                const int lx = ix - var.ix0, ly = iy - var.iy0;
                if (ix >= g.nx || iy >= g.ny || lx < 0 || ly < 0 || lx >= var.nx || ly >= var.ny) continue;
                const long long o = iv.out_base + var.out_off + (long long)ly * var.nx + lx;
                ba.counts_out[o] = iv.base_counts[(long long)iy * g.nx + ix];
                if (ba.impact_out) ba.impact_out[o] = 0;
            }
            continue;
        }
        float tox, toy;
        tile_setup(sm, g, tx, ty, &tox, &toy);
#pragma unroll
        for (int q = 0; q < 4; ++q) s_st[(row0 + q) * kTile + lane] = RunState{0, 0, 0};
        const int* rem = ba.removed + var.rem_off;
        const int n_rem = var.n_rem;
        const float4* towers = ba.tower_tris + 3ll * var.tower_off;
        const int n_tow = var.n_tower;
        for (int bl = 0; bl < iv.n_blocks; ++bl) {
            const BlockConst& bc = iv.blocks[bl];
            const unsigned off = iv.offsets[(size_t)bl * n_tiles + tile];
            const int cnt = (int)iv.counts[(size_t)bl * n_tiles + tile];
            const int* bins = iv.bins + off;
            const float4* tris = ba.base_tris;
            auto fetch = [=](int i, int v, float4* out) {
                if (i >= cnt) {
                    *out = __ldg(&towers[3 * (i - cnt) + v]);
                    return true;
                }
                const float4 x = __ldg(&tris[3 * bins[i] + v]);
                *out = x;
                if (v != 0) return true;
                const int bid = __float_as_int(__ldg(&tris[3 * bins[i]]).w);
                for (int q = 0; q < n_rem; ++q)
                    if (rem[q] == bid) return false;
                return true;
            };
            raster_block<COUNT, CULL>(sm, fetch, cnt + n_tow, iv.steps, bc.j0, bc.K, tox, toy,
                                      inv_dx, ba.run, n_cell, n_test, n_unit, n_span);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int cell = (row0 + q) * kTile + lane;
                const unsigned long long m = sm.mask[cell];
                sm.mask[cell] = 0ull;
                RunState st = s_st[cell];
                stitch(st, m, bc.K, bc.new_day);
                s_st[cell] = st;
            }
        }
        const int ix = tx * kTile + lane;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int iy = ty * kTile + row0 + q;
            const int lx = ix - var.ix0, ly = iy - var.iy0;
            if (ix >= g.nx || iy >= g.ny || lx < 0 || ly < 0 || lx >= var.nx || ly >= var.ny) continue;
            const long long o = iv.out_base + var.out_off + (long long)ly * var.nx + lx;
            const int gross = s_st[(row0 + q) * kTile + lane].gross;
            ba.counts_out[o] = gross;
            if (ba.impact_out && iv.base_counts)
                ba.impact_out[o] = gross - iv.base_counts[(long long)iy * g.nx + ix];
        }
    }
    if (COUNT) flush_raster_counts(ba.stats, n_cell, n_test, n_unit, n_span);
}

// Launch order of the tiles: descending by the triangles binned to them over the chunk's
// blocks, bucketed at half powers of two.  The CTAs that start last are then the cheap
// ones, which shortens the launch's tail; the order does not change any result.
__global__ void k_tile_order(const unsigned* __restrict__ counts, int nbc, int n_tiles,
                             int* __restrict__ order) {
    constexpr int kBuckets = 64;
    __shared__ unsigned hist[kBuckets];
    auto bucket = [&](int t) {
        unsigned c = 0;
        for (int b = 0; b < nbc; ++b) c += counts[(size_t)b * n_tiles + t];
        if (c <= 1u) return kBuckets - 1;
        const int l = 31 - __clz(c);
        const int key = 2 * l + (int)((c >> (l - 1)) & 1u);     // 2 .. 63
        return kBuckets - 1 - key;
    };
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) atomicAdd(&hist[bucket(t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int k = 0; k < kBuckets; ++k) {
            const unsigned h = hist[k];
            hist[k] = run;
            run += h;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) order[atomicAdd(&hist[bucket(t)], 1u)] = t;
}

template <int CTAS>
void launch_k_raster_as(const RasterArgs& ra, int n_tiles, bool stats, cudaStream_t st) {
    if (ra.cull) {
        if (stats) k_raster<true, true, CTAS><<<n_tiles, kRasterThreads, 0, st>>>(ra);
        else k_raster<false, true, CTAS><<<n_tiles, kRasterThreads, 0, st>>>(ra);
    } else {
        if (stats) k_raster<true, false, CTAS><<<n_tiles, kRasterThreads, 0, st>>>(ra);
        else k_raster<false, false, CTAS><<<n_tiles, kRasterThreads, 0, st>>>(ra);
    }
}

// A launch of more tiles than 4 CTAs per SM hold takes the build for SA_RASTER_CTAS
// resident CTAs per SM (fewer registers, more warps to hide latency); a smaller one, all of
// whose tiles are resident at once anyway, takes the build for 4 (more registers, no
// spills).
void launch_k_raster(const RasterArgs& ra, int n_tiles, bool stats, cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    if (SA_RASTER_CTAS > 4 && n_tiles > 4 * sms) launch_k_raster_as<SA_RASTER_CTAS>(ra, n_tiles, stats, st);
    else launch_k_raster_as<4>(ra, n_tiles, stats, st);
}

}  // namespace

// Runs every block of `sun` through the accrual raster, in chunks of blocks whose bins
// fit a bounded scratch budget.  out.run must be scratch [R]; out.continuous may be NULL.
cudaError_t launch_raster_ground(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                 const DevOut& out, cudaStream_t st) {
    TileGeom g;
    g.x0 = rc.x0; g.y0 = rc.y0; g.dx = rc.dx; g.nx = rc.nx; g.ny = rc.ny;
    g.tiles_x = (rc.nx + kTile - 1) / kTile;
    g.tiles_y = (rc.ny + kTile - 1) / kTile;
    const int n_tiles = g.tiles_x * g.tiles_y;
    const long long R = (long long)rc.nx * rc.ny;
    if (R == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    int* best = out.continuous;
    int* best_scratch = nullptr;
    if (!best) {
        e = sa::scratch_alloc(&best_scratch, sizeof(int) * (size_t)R, st);
        if (e != cudaSuccess) return e;
        best = best_scratch;
    }
    const int chunk = 64;
    const int max_chunk_blocks = sun.n_blocks < chunk ? sun.n_blocks : chunk;
    unsigned *counts = nullptr, *offsets = nullptr, *cursor = nullptr, *d_total = nullptr;
    int *bins = nullptr, *order = nullptr;
    size_t bins_cap = 0;
    const size_t nc = (size_t)max_chunk_blocks * n_tiles;
    e = sa::scratch_alloc(&counts, sizeof(unsigned) * nc, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&offsets, sizeof(unsigned) * nc, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&cursor, sizeof(unsigned) * nc, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&d_total, sizeof(unsigned), st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&order, sizeof(int) * (size_t)n_tiles, st);
    const int tpb = 128;
    for (int b0 = 0; b0 < sun.n_blocks && e == cudaSuccess; b0 += chunk) {
        const int nbc = (sun.n_blocks - b0) < chunk ? (sun.n_blocks - b0) : chunk;
        const size_t ncc = (size_t)nbc * n_tiles;
        e = cudaMemsetAsync(counts, 0, sizeof(unsigned) * ncc, st);
        if (e != cudaSuccess) break;
        e = cudaMemsetAsync(cursor, 0, sizeof(unsigned) * ncc, st);
        if (e != cudaSuccess) break;
        unsigned total = 0;
        if (sc.T > 0) {
            dim3 grid((sc.T + tpb - 1) / tpb, nbc);
            {
                KernelTimer kt(KT_RASTER_BIN, st);
                k_bin_count<<<grid, tpb, 0, st>>>(sc, sun.steps, sun.blocks, b0, g, counts);
            }
            k_tile_order<<<1, 1024, 0, st>>>(counts, nbc, n_tiles, order);
            e = cudaMemcpyAsync(offsets, counts, sizeof(unsigned) * ncc, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) break;
            e = exclusive_scan_u32(offsets, (long long)ncc, d_total, st);
            if (e != cudaSuccess) break;
            e = cudaMemcpyAsync(&total, d_total, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) break;
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) break;
            if (total > bins_cap) {
                if (bins) cudaFreeAsync(bins, st);
                bins_cap = (size_t)total + total / 4 + 1024;
                e = sa::scratch_alloc(&bins, sizeof(int) * bins_cap, st);
                if (e != cudaSuccess) { bins = nullptr; break; }
            }
            if (total > 0) {
                KernelTimer kt(KT_RASTER_BIN, st);
                k_bin_fill<<<grid, tpb, 0, st>>>(sc, sun.steps, sun.blocks, b0, g, offsets, cursor, bins);
            }
        } else {
            e = cudaMemsetAsync(offsets, 0, sizeof(unsigned) * ncc, st);
            if (e != cudaSuccess) break;
        }
        RasterArgs ra;
        ra.sc = sc; ra.sun = sun; ra.g = g; ra.b0 = b0; ra.nbc = nbc;
        ra.offsets = offsets; ra.counts = counts; ra.bins = bins;
        ra.out = out; ra.best = best;
        ra.load_state = (b0 > 0) || out.accumulate_into;
        ra.final_chunk = (b0 + nbc >= sun.n_blocks);
        ra.R = R;
        ra.cull = sc.closed;
        ra.run = g_raster_run;
        ra.order = sc.T > 0 ? order : nullptr;
        if (b0 == 0 && out.accumulate_into) {
            // run lengths never cross calls (calls cover whole days)
            e = cudaMemsetAsync(out.run, 0, sizeof(int) * (size_t)R, st);
            if (e != cudaSuccess) break;
            if (!out.continuous) {
                e = cudaMemsetAsync(best, 0, sizeof(int) * (size_t)R, st);
                if (e != cudaSuccess) break;
            }
        }
        {
            KernelTimer kt(KT_RASTER, st);
            launch_k_raster(ra, n_tiles, out.stats != nullptr, st);
        }
        e = cudaGetLastError();
    }
    if (counts) cudaFreeAsync(counts, st);
    if (offsets) cudaFreeAsync(offsets, st);
    if (cursor) cudaFreeAsync(cursor, st);
    if (d_total) cudaFreeAsync(d_total, st);
    if (bins) cudaFreeAsync(bins, st);
    if (order) cudaFreeAsync(order, st);
    if (best_scratch) cudaFreeAsync(best_scratch, st);
    return e;
}

namespace {
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

cudaError_t launch_raster_ground_in(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                    const DevOut& out, cudaStream_t st, unsigned char* scratch,
                                    size_t bytes, int* capacity_error) {
    *capacity_error = 0;
    TileGeom g;
    g.x0 = rc.x0; g.y0 = rc.y0; g.dx = rc.dx; g.nx = rc.nx; g.ny = rc.ny;
    g.tiles_x = (rc.nx + kTile - 1) / kTile;
    g.tiles_y = (rc.ny + kTile - 1) / kTile;
    const int n_tiles = g.tiles_x * g.tiles_y;
    const long long R = (long long)rc.nx * rc.ny;
    if (R == 0) return cudaSuccess;
    const int max_chunk = 16;
    const size_t nc = (size_t)max_chunk * n_tiles;
    // carve: run [R], best [R] (when the caller passes no continuous buffer), total,
    // counts / offsets / cursor [max_chunk * tiles], scan partials, bins (the rest)
    size_t off = 0;
    int* run = reinterpret_cast<int*>(scratch + off);
    off += align256(sizeof(int) * (size_t)R);
    int* best = out.continuous;
    if (!best) {
        best = reinterpret_cast<int*>(scratch + off);
        off += align256(sizeof(int) * (size_t)R);
    }
    unsigned* d_total = reinterpret_cast<unsigned*>(scratch + off);
    off += 256;
    unsigned* counts = reinterpret_cast<unsigned*>(scratch + off);
    off += align256(sizeof(unsigned) * nc);
    unsigned* offsets = reinterpret_cast<unsigned*>(scratch + off);
    off += align256(sizeof(unsigned) * nc);
    unsigned* cursor = reinterpret_cast<unsigned*>(scratch + off);
    off += align256(sizeof(unsigned) * nc);
    unsigned* partial = reinterpret_cast<unsigned*>(scratch + off);
    off += align256(sizeof(unsigned) * (size_t)scan_partials((long long)nc));
    if (off >= bytes) { *capacity_error = 1; return cudaSuccess; }
    int* bins = reinterpret_cast<int*>(scratch + off);
    const size_t bins_cap = (bytes - off) / sizeof(int);
    DevOut o = out;
    o.run = run;
    const int tpb = 128;
    // Bins of blocks [b0, b0 + nbc): counts, their exclusive scan into offsets, and the
    // total, read back to the host.
    auto count_chunk = [&](int b0, int nbc, unsigned* total) -> cudaError_t {
        const size_t ncc = (size_t)nbc * n_tiles;
        *total = 0;
        cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned) * ncc, st);
        if (e != cudaSuccess) return e;
        if (sc.T == 0) return cudaMemsetAsync(offsets, 0, sizeof(unsigned) * ncc, st);
        dim3 grid((sc.T + tpb - 1) / tpb, nbc);
        k_bin_count<<<grid, tpb, 0, st>>>(sc, sun.steps, sun.blocks, b0, g, counts);
        e = cudaMemcpyAsync(offsets, counts, sizeof(unsigned) * ncc, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = exclusive_scan_u32_with(offsets, (long long)ncc, partial, d_total, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(total, d_total, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e;
    };
    // Sizing pass, before any output is written: cut the blocks into chunks whose bins fit
    // the scratch (halving a chunk that does not), or report that one block alone does not.
    std::vector<int2> plan;
    int b0 = 0;
    int nbc = sun.n_blocks < max_chunk ? sun.n_blocks : max_chunk;
    while (b0 < sun.n_blocks) {
        if (b0 + nbc > sun.n_blocks) nbc = sun.n_blocks - b0;
        unsigned total = 0;
        cudaError_t e = count_chunk(b0, nbc, &total);
        if (e != cudaSuccess) return e;
        if ((size_t)total > bins_cap) {
            if (nbc == 1) { *capacity_error = 1; return cudaSuccess; }
            nbc = (nbc + 1) / 2;          // retry this chunk with fewer blocks
            continue;
        }
        plan.push_back(make_int2(b0, nbc));
        b0 += nbc;
    }
    cudaError_t e = cudaSuccess;
    if (out.accumulate_into) {
        e = cudaMemsetAsync(run, 0, sizeof(int) * (size_t)R, st);
        if (e == cudaSuccess && !out.continuous) e = cudaMemsetAsync(best, 0, sizeof(int) * (size_t)R, st);
        if (e != cudaSuccess) return e;
    }
    for (const int2& c : plan) {
        unsigned total = 0;
        e = count_chunk(c.x, c.y, &total);
        if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(unsigned) * (size_t)c.y * n_tiles, st);
        if (e != cudaSuccess) return e;
        if (total > 0) {
            dim3 grid((sc.T + tpb - 1) / tpb, c.y);
            k_bin_fill<<<grid, tpb, 0, st>>>(sc, sun.steps, sun.blocks, c.x, g, offsets, cursor, bins);
        }
        RasterArgs ra;
        ra.sc = sc; ra.sun = sun; ra.g = g; ra.b0 = c.x; ra.nbc = c.y;
        ra.offsets = offsets; ra.counts = counts; ra.bins = bins;
        ra.out = o; ra.best = best;
        ra.load_state = (c.x > 0) || out.accumulate_into;
        ra.final_chunk = (c.x + c.y >= sun.n_blocks);
        ra.R = R;
        ra.cull = sc.closed;
        ra.run = g_raster_run;
        ra.order = nullptr;
        launch_k_raster(ra, n_tiles, out.stats != nullptr, st);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void set_raster_run(int run) { g_raster_run = run; }
int get_raster_run() { return g_raster_run; }

cudaError_t build_bins(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                       unsigned** offsets, unsigned** counts, int** bins, cudaStream_t st) {
    *offsets = nullptr; *counts = nullptr; *bins = nullptr;
    TileGeom g;
    g.x0 = rc.x0; g.y0 = rc.y0; g.dx = rc.dx; g.nx = rc.nx; g.ny = rc.ny;
    g.tiles_x = (rc.nx + kTile - 1) / kTile;
    g.tiles_y = (rc.ny + kTile - 1) / kTile;
    const size_t nc = (size_t)sun.n_blocks * g.tiles_x * g.tiles_y;
    if (nc == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(counts, sizeof(unsigned) * nc);
    if (e == cudaSuccess) e = cudaMalloc(offsets, sizeof(unsigned) * nc);
    unsigned* cursor = nullptr;
    unsigned* d_total = nullptr;
    if (e == cudaSuccess) e = sa::scratch_alloc(&cursor, sizeof(unsigned) * nc, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&d_total, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(*counts, 0, sizeof(unsigned) * nc, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(unsigned) * nc, st);
    unsigned total = 0;
    const int tpb = 128;
    dim3 grid((sc.T + tpb - 1) / tpb > 0 ? (sc.T + tpb - 1) / tpb : 1, sun.n_blocks);
    if (e == cudaSuccess && sc.T > 0) {
        k_bin_count<<<grid, tpb, 0, st>>>(sc, sun.steps, sun.blocks, 0, g, *counts);
        e = cudaMemcpyAsync(*offsets, *counts, sizeof(unsigned) * nc, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = exclusive_scan_u32(*offsets, (long long)nc, d_total, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_total, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    } else if (e == cudaSuccess) {
        e = cudaMemsetAsync(*offsets, 0, sizeof(unsigned) * nc, st);
    }
    if (e == cudaSuccess) e = cudaMalloc(bins, sizeof(int) * ((size_t)total + 1));
    if (e == cudaSuccess && total > 0)
        k_bin_fill<<<grid, tpb, 0, st>>>(sc, sun.steps, sun.blocks, 0, g, *offsets, cursor, *bins);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (cursor) cudaFreeAsync(cursor, st);
    if (d_total) cudaFreeAsync(d_total, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        if (*counts) cudaFree(*counts);
        if (*offsets) cudaFree(*offsets);
        if (*bins) cudaFree(*bins);
        *counts = nullptr; *offsets = nullptr; *bins = nullptr;
    }
    return e;
}

int raster_ctas_per_sm() { return SA_RASTER_CTAS; }

cudaError_t launch_batch(const BatchLaunch& bl, cudaStream_t st) {
    BatchArgs ba;
    ba.g.x0 = bl.grid.x0; ba.g.y0 = bl.grid.y0; ba.g.dx = bl.grid.dx;
    ba.g.nx = bl.grid.nx; ba.g.ny = bl.grid.ny;
    ba.g.tiles_x = (bl.grid.nx + kTile - 1) / kTile;
    ba.g.tiles_y = (bl.grid.ny + kTile - 1) / kTile;
    ba.base_tris = bl.base.tris;
    ba.intervals = bl.intervals;
    ba.variants = bl.variants;
    ba.items = bl.items;
    ba.n_items = bl.n_items;
    ba.counter = bl.counter;
    ba.removed = bl.removed;
    ba.tower_tris = bl.tower_tris;
    ba.counts_out = bl.counts_out;
    ba.impact_out = bl.impact_out;
    ba.cull = bl.base.closed;
    ba.run = bl.run;
    ba.stats = bl.stats;
    cudaError_t e = cudaMemsetAsync(bl.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (bl.n_items == 0) return cudaSuccess;
    if (ba.cull) {
        if (bl.stats) k_batch<true, true><<<bl.ctas, kRasterThreads, 0, st>>>(ba);
        else k_batch<false, true><<<bl.ctas, kRasterThreads, 0, st>>>(ba);
    } else {
        if (bl.stats) k_batch<true, false><<<bl.ctas, kRasterThreads, 0, st>>>(ba);
        else k_batch<false, false><<<bl.ctas, kRasterThreads, 0, st>>>(ba);
    }
    return cudaGetLastError();
}

}  // namespace sa
