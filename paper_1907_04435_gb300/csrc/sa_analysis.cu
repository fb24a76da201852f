// sa_analysis.cu -- analysis measures over a polygonal region of a ground grid (Sec. 7.2).
//
// Shadow area: the sum over the region's cells of shadow(p) x area(p), where shadow(p) is
// the fraction of the interval's steps the cell spends in shadow (gross counts give the
// gross fraction, continuous counts the continuous one) and area(p) = dx^2.  A cell is in
// the region when its centre is, by the even-odd rule.  The shadow score over several
// intervals is the weighted sum of their areas (weights w_t in [-1, 1]):
// sum over the region's cells of sum_t w_t x shadow_t(p) x area(p), one pass over the
// cells that reads every interval's counts of a cell together.
//
// The centres are rounded exactly as the receivers' (FP32), then tested in FP64 with
// explicit roundings, so the decision for a centre does not depend on the compiler's
// contraction of multiply-adds.
#include <math.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "sa_handles.cuh"

namespace sa {

namespace {

constexpr int kAreaThreads = 256;

// even-odd rule: count the polygon edges crossed by the ray from (x, y) toward +x
__device__ bool inside_polygon(const double2* __restrict__ poly, int n, double x, double y) {
    bool in = false;
    for (int i = 0; i < n; ++i) {
        const double2 a = poly[i], b = poly[i + 1 == n ? 0 : i + 1];
        if ((a.y > y) != (b.y > y)) {
            const double t = __ddiv_rn(__dsub_rn(y, a.y), __dsub_rn(b.y, a.y));
            const double xc = __dadd_rn(a.x, __dmul_rn(t, __dsub_rn(b.x, a.x)));
            if (x < xc) in = !in;
        }
    }
    return in;
}

__global__ void k_shadow_area(const int* __restrict__ steps, float x0, float y0, float dx, int nx,
                              long long R, const double2* __restrict__ poly, int n,
                              double inv_total, double* __restrict__ out) {
    __shared__ double s_part[kAreaThreads / 32];
    double s = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < R;
         c += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx), iy = (int)(c / nx);
        const float cx = __fadd_rn(x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), dx));
        const float cy = __fadd_rn(y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), dx));
        if (steps[c] != 0 && inside_polygon(poly, n, (double)cx, (double)cy))
            s += (double)steps[c] * inv_total;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kAreaThreads / 32; ++w) t += s_part[w];
        atomicAdd(out, t);
    }
}

// Shadow score over intervals: coef[t] = w_t / total_steps_t; counts are [n_t][R].
__global__ void k_shadow_score(const int* __restrict__ steps, long long R, int n_t,
                               const double* __restrict__ coef, float x0, float y0, float dx,
                               int nx, const double2* __restrict__ poly, int n,
                               double* __restrict__ out) {
    __shared__ double s_part[kAreaThreads / 32];
    double s = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < R;
         c += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        bool any = false;
        for (int t = 0; t < n_t; ++t) {
            const int k = __ldcs(&steps[(long long)t * R + c]);
            if (k != 0) {
                v = fma((double)k, coef[t], v);
                any = true;
            }
        }
        if (!any) continue;
        const int ix = (int)(c % nx), iy = (int)(c / nx);
        const float cx = __fadd_rn(x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), dx));
        const float cy = __fadd_rn(y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), dx));
        if (inside_polygon(poly, n, (double)cx, (double)cy)) s += v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kAreaThreads / 32; ++w) t += s_part[w];
        atomicAdd(out, t);
    }
}

// Building contribution (Sec. 7.2).  For every cell of the region and every step the
// accrual raster marks as shadowed, the buildings the ray toward the sun meets beyond
// t_min are found, and each is credited one cell-step: "casting" counts, per building,
// the cell-steps whose ray meets it (a ray meeting several buildings credits each once);
// "nearest" counts, per building, the cell-steps whose nearest hit lies on it, so that
// these partition the region's shadowed cell-steps -- except the ones the raster marks
// shadowed whose FP32 ray grazes past every triangle (shadow edges), counted apart.
//
// A first pass lists, per run of <= 32 consecutive steps of a block, the region's cells
// with a shadowed step in it.  One warp then takes 32 listed cells of one run and walks
// the depth-first node list once with the fan of the run's rays as its query (as the
// ray-traced accrual does): every triangle in the fan is tested exactly (Plucker form,
// with its distance) against the lane's shadowed steps it can reach.  Per lane and step
// the nearest hit (distance, building) is kept in shared memory, and per lane and run a
// short list of kCastList (building, steps met) pairs; a lane whose
// run meets more buildings than the list holds counts its casting again ray by ray, with
// a list of kRayList buildings per ray.  Counts are integers, credited by atomics on
// per-building totals (runs of equal nearest buildings are credited at once).
constexpr int kContribWarps = 2;
constexpr int kContribRun = 32;             // steps per fan traversal
constexpr int kCastList = 8;                // buildings per lane and run in the fan pass
constexpr int kRayList = 2 * kContribRun;   // buildings per ray in the per-ray recount

struct ContribArgs {
    DevScene sc;
    const StepConst* steps;
    const BlockConst* runs;           // runs of <= 32 steps; mask_block / mask_bit locate them
    int n_runs;
    const unsigned long long* masks;  // the raster's step masks [blocks][R]
    long long R;
    float x0, y0, dx;
    int nx;
    int bx0, by0, bnx, bny;           // the region's bounding box, in cells
    const double2* poly;
    int n;
    unsigned long long* cast_cnt;     // [B]
    unsigned long long* near_cnt;     // [B]
    unsigned long long* stats;        // [2]
    int n_b;                          // buildings (length of the counters)
    // compacted work: per run, the cells with a shadowed step in it (global cell index)
    const int* items;                 // run r's cells at item0[r] .. item0[r] + n_items[r]
    const unsigned* item0;            // [n_runs]
    const unsigned* n_items;          // [n_runs]
    const int* warp_base;             // [n_runs + 1] first warp of each run
};

// Per warp, in shared memory; Id is a 16-bit building id when the scene has fewer than
// 65,536 buildings (the smaller footprint keeps more warps resident), else 32-bit.
template <class Id>
struct ContribWarpSmem {
    float t[kContribRun][32];         // nearest hit distance per step and lane
    Id b[kContribRun][32];            // its building
    Id cb[kCastList][32];             // casting list: building
    unsigned cm[kCastList][32];       //               steps whose ray meets it
};

// what the kernel reads of a step: its direction and the direction's reciprocals
struct ContribStep {
    float dx, dy, dz, ix, iy, iz;
};

// Plucker test with the hit distance (t = ((a - o) . n) / (d . n)), the same decision as
// plucker_hit.
__device__ __forceinline__ bool plucker_hit_t(const PluckerTri& p, const ContribStep& s, float tmin,
                                              float* t) {
    if (!plucker_hit(p, s.dx, s.dy, s.dz, tmin)) return false;
    const float nd = fmaf(s.dz, p.nz, fmaf(s.dy, p.ny, __fmul_rn(s.dx, p.nx)));
    *t = p.aon / nd;
    return true;
}

// Work list of the fan traversal: per run, the region's cells with at least one shadowed
// step in it, in patch order (8 x 4 cells per patch, patches row by row), so that the 32
// cells a traversal warp takes stay close together.  Cells shadowed at no step of a run
// cost nothing there.  Two passes over the patches: counts per (run, patch), then -- after
// an exclusive scan of the counts into offsets -- the cells themselves.
__global__ void k_contrib_items(ContribArgs a, bool fill, unsigned* __restrict__ counts,
                                const unsigned* __restrict__ offsets, int* __restrict__ items) {
    const int lane = threadIdx.x & 31;
    const int tiles_x = (a.bnx + 7) >> 3;
    const long long n_patches = (long long)tiles_x * ((a.bny + 3) >> 2);
    const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp_id >= n_patches) return;                                  // whole warps
    const int ty = (int)(warp_id / tiles_x), tx = (int)(warp_id - (long long)ty * tiles_x);
    const int lx = tx * 8 + (lane & 7), ly = ty * 4 + (lane >> 3);
    const int ix = a.bx0 + lx, iy = a.by0 + ly;
    const float x = __fadd_rn(a.x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), a.dx));
    const float y = __fadd_rn(a.y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), a.dx));
    const bool in_region = lx < a.bnx && ly < a.bny && inside_polygon(a.poly, a.n, (double)x, (double)y);
    const long long cell = (long long)iy * a.nx + ix;
    for (int r = 0; r < a.n_runs; ++r) {
        const BlockConst& bc = a.runs[r];
        const unsigned run_bits = bc.K >= 32 ? 0xffffffffu : ((1u << bc.K) - 1u);
        const bool want = in_region &&
                          ((unsigned)(a.masks[(long long)bc.mask_block * a.R + cell] >> bc.mask_bit) & run_bits) != 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, want);
        const long long slot = (long long)r * n_patches + warp_id;
        if (!fill) {
            if (lane == 0) counts[slot] = (unsigned)__popc(bal);
        } else if (want) {
            items[offsets[slot] + __popc(bal & ((1u << lane) - 1u))] = (int)cell;
        }
    }
}

template <class Id>
__global__ void __launch_bounds__(32 * kContribWarps)
k_building_contribution(ContribArgs a) {
    __shared__ ContribWarpSmem<Id> s_w[kContribWarps];
    __shared__ BlockConst s_bc[kContribWarps];
    __shared__ ContribStep s_st[kContribWarps][kContribRun];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp_id = (int)(blockIdx.x * kContribWarps + wib);
    if (warp_id >= a.warp_base[a.n_runs]) return;                       // whole warps
    int r = 0;
    while (a.warp_base[r + 1] <= warp_id) ++r;
    const unsigned slot = (unsigned)(warp_id - a.warp_base[r]) * 32u + (unsigned)lane;
    const bool live = slot < a.n_items[r];
    const long long cell = live ? (long long)SA_CHK(a.items[(long long)a.item0[r] + slot], a.R, sa::CK_CONTRIB_CELL) : 0;
    const int ix = (int)(cell % a.nx), iy = (int)(cell / a.nx);
    float3 o;
    o.x = __fadd_rn(a.x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), a.dx));
    o.y = __fadd_rn(a.y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), a.dx));
    o.z = 0.f;
    ContribWarpSmem<Id>& w = s_w[wib];
    BlockConst& bc = s_bc[wib];
    ContribStep* ss = s_st[wib];
    unsigned long long n_graze = 0, n_over = 0;
    {
        for (int q = lane; q < (int)(sizeof(BlockConst) / 4); q += 32)
            reinterpret_cast<int*>(&bc)[q] = reinterpret_cast<const int*>(&a.runs[r])[q];
        __syncwarp();
        const int K = bc.K;
        if (lane < K) {
            const StepConst& sk = a.steps[bc.j0 + lane];
            ss[lane] = ContribStep{sk.dx, sk.dy, sk.dz, sk.ix, sk.iy, sk.iz};
        }
        const unsigned run_bits = K >= 32 ? 0xffffffffu : ((1u << K) - 1u);
        unsigned m = 0u;
        if (live) m = (unsigned)(a.masks[(long long)bc.mask_block * a.R + cell] >> bc.mask_bit) & run_bits;
        __syncwarp();
        for (int k = 0; k < K; ++k) w.t[k][lane] = 3.4e38f;
        int n_list = 0;
        bool ovf = false;
        unsigned found = 0u;
        const bool wedge = bc.wedge_ok != 0.f;
        const bool want = m != 0u;
        for (int i = 0; i < a.sc.n_nodes;) {
            const float4 lo = __ldg(&a.sc.nodes[2 * i]);
            const float4 hi = __ldg(&a.sc.nodes[2 * i + 1]);
            const int esc = SA_ESC(__float_as_int(lo.w), i, a.sc.n_nodes, sa::CK_CONTRIB_ESCAPE);
            const int tri = SA_LEAF(__float_as_int(hi.w), a.sc.T, sa::CK_CONTRIB_LEAF);
            const bool in = want && (wedge ? fan_box(o, bc, lo, hi) : slope_box(o, bc, lo, hi));
            if (tri >= 0) {
                unsigned cand = 0u;
                float4 ta, tb, tc;
                if (in) {
                    ta = __ldg(&a.sc.tris[3 * tri]);
                    tb = __ldg(&a.sc.tris[3 * tri + 1]);
                    tc = __ldg(&a.sc.tris[3 * tri + 2]);
                    if (plane_reachable(o, ta, tb, tc, bc)) {
                        int ka, kb;
                        candidate_steps(o, bc, bc.psi, ta, tb, tc, &ka, &kb);
                        if (ka <= kb) {
                            const unsigned hi_bits = kb >= 31 ? 0xffffffffu : ((2u << kb) - 1u);
                            cand = m & hi_bits & ~((1u << ka) - 1u);
                        }
                    }
                }
                const int wa = __reduce_min_sync(0xffffffffu, cand ? __ffs(cand) - 1 : 32);
                const int wb = __reduce_max_sync(0xffffffffu, cand ? 31 - __clz(cand) : -1);
                if (wa <= wb) {
                    unsigned hits = 0u;
                    PluckerTri pt;
                    if (cand) pt = plucker_setup(o, ta, tb, tc);
                    const int bid = cand ? (int)SA_CHK(__float_as_int(ta.w), a.n_b, sa::CK_CONTRIB_BUILDING) : 0;
                    for (int k = wa; k <= wb; ++k) {
                        float t;
                        if (((cand >> k) & 1u) && plucker_hit_t(pt, ss[k], kGroundTmin, &t)) {
                            hits |= 1u << k;
                            if (t < w.t[k][lane]) {
                                w.t[k][lane] = t;
                                w.b[k][lane] = (Id)bid;
                            }
                        }
                    }
                    if (hits) {
                        found |= hits;
                        int e = 0;
                        while (e < n_list && (int)w.cb[e][lane] != bid) ++e;
                        if (e < n_list) {
                            w.cm[e][lane] |= hits;
                        } else if (n_list < kCastList) {
                            w.cb[n_list][lane] = (Id)bid;
                            w.cm[n_list][lane] = hits;
                            ++n_list;
                        } else {
                            ovf = true;
                        }
                    }
                }
                i = esc;
            } else {
                i = __any_sync(0xffffffffu, in) ? i + 1 : esc;
            }
        }
        // nearest: runs of steps with the same nearest building are credited at once
        n_graze += (unsigned long long)__popc(m & ~found);
        unsigned rest = m & found;
        int cur = -1;
        unsigned long long cnt = 0;
        while (rest) {
            const int k = __ffs(rest) - 1;
            rest &= rest - 1u;
            const int bid = (int)w.b[k][lane];
            if (bid != cur) {
                if (cnt) atomicAdd(&a.near_cnt[cur], cnt);
                cur = bid;
                cnt = 0;
            }
            ++cnt;
        }
        if (cnt) atomicAdd(&a.near_cnt[cur], cnt);
        if (!ovf) {
            for (int e = 0; e < n_list; ++e)
                atomicAdd(&a.cast_cnt[(int)w.cb[e][lane]], (unsigned long long)__popc(w.cm[e][lane]));
        }
        // more buildings than the list holds: casting again, ray by ray (each lane alone;
        // the nearest arrays, no longer needed, hold the ray's list -- with 16-bit ids a
        // lane's list spans other lanes' columns of t, hence the warp barrier)
        __syncwarp();
        Id* ids = reinterpret_cast<Id*>(&w.t[0][0]);       // kRayList x 32 ids over t (and b)
        unsigned todo = ovf ? (m & found) : 0u;
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1u;
            const ContribStep& s = ss[k];
            int n_ids = 0;
            bool lost = false;
            for (int i = 0; i < a.sc.n_nodes;) {
                const float4 lo = __ldg(&a.sc.nodes[2 * i]);
                const float4 hi = __ldg(&a.sc.nodes[2 * i + 1]);
                const int esc = SA_ESC(__float_as_int(lo.w), i, a.sc.n_nodes, sa::CK_CONTRIB_ESCAPE);
                const int tri = SA_LEAF(__float_as_int(hi.w), a.sc.T, sa::CK_CONTRIB_LEAF);
                const bool in = hit_box(o, s.ix, s.iy, s.iz, lo, hi);
                if (tri >= 0) {
                    if (in) {
                        const float4 ta = __ldg(&a.sc.tris[3 * tri]);
                        const float4 tb = __ldg(&a.sc.tris[3 * tri + 1]);
                        const float4 tc = __ldg(&a.sc.tris[3 * tri + 2]);
                        const PluckerTri pt = plucker_setup(o, ta, tb, tc);
                        if (plucker_hit(pt, s.dx, s.dy, s.dz, kGroundTmin)) {
                            const int bid = (int)SA_CHK(__float_as_int(ta.w), a.n_b, sa::CK_CONTRIB_BUILDING);
                            int e = 0;
                            while (e < n_ids && (int)ids[e * 32 + lane] != bid) ++e;
                            if (e == n_ids) {
                                if (n_ids < kRayList) ids[(n_ids++) * 32 + lane] = (Id)bid;
                                else lost = true;
                            }
                        }
                    }
                    i = esc;
                } else {
                    i = in ? i + 1 : esc;
                }
            }
            for (int e = 0; e < n_ids; ++e) atomicAdd(&a.cast_cnt[(int)ids[e * 32 + lane]], 1ull);
            if (lost) ++n_over;
        }
    }
    for (int q = 16; q > 0; q >>= 1) {
        n_graze += __shfl_down_sync(0xffffffffu, n_graze, q);
        n_over += __shfl_down_sync(0xffffffffu, n_over, q);
    }
    if (lane == 0) {
        if (n_over) atomicAdd(&a.stats[0], n_over);
        if (n_graze) atomicAdd(&a.stats[1], n_graze);
    }
}

}  // namespace

cudaError_t launch_building_contribution(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                         const std::vector<BlockConst>& runs, int n_buildings,
                                         const float* poly_xy, int n, double* casting_out,
                                         double* nearest_out, unsigned long long* stats_out,
                                         cudaStream_t st) {
    const long long R = (long long)rc.nx * rc.ny;
    const int B = n_buildings > 0 ? n_buildings : 1;
    const size_t n_cnt = 2 * (size_t)B + 2;
    cudaError_t e = cudaSuccess;
    unsigned long long *masks = nullptr, *cnt = nullptr;
    int *gross = nullptr, *run = nullptr, *items = nullptr, *wbase = nullptr;
    unsigned *pcnt = nullptr, *poff = nullptr, *runinfo = nullptr;
    double2* dp = nullptr;
    BlockConst* druns = nullptr;
    std::vector<double2> hp((size_t)n);
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = 0; i < n; ++i) {
        hp[(size_t)i] = make_double2((double)poly_xy[2 * i], (double)poly_xy[2 * i + 1]);
        xmin = std::min(xmin, hp[(size_t)i].x); xmax = std::max(xmax, hp[(size_t)i].x);
        ymin = std::min(ymin, hp[(size_t)i].y); ymax = std::max(ymax, hp[(size_t)i].y);
    }
    // cells whose centre may lie in the polygon (one cell of margin for rounding)
    const double dx = rc.dx;
    const double fx0 = std::max(0.0, std::floor((xmin - rc.x0) / dx - 0.5) - 1.0);
    const double fx1 = std::min((double)rc.nx - 1.0, std::ceil((xmax - rc.x0) / dx - 0.5) + 1.0);
    const double fy0 = std::max(0.0, std::floor((ymin - rc.y0) / dx - 0.5) - 1.0);
    const double fy1 = std::min((double)rc.ny - 1.0, std::ceil((ymax - rc.y0) / dx - 0.5) + 1.0);
    std::vector<unsigned long long> h_cnt(n_cnt, 0ull);
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(sa::scratch_alloc(&cnt, sizeof(unsigned long long) * n_cnt, st));
    TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * n_cnt, st));
    if (R > 0 && sun.n_blocks > 0 && sc.T > 0 && !runs.empty() && fx0 <= fx1 && fy0 <= fy1) {
        TRY(sa::scratch_alloc(&dp, sizeof(double2) * (size_t)n, st));
        TRY(cudaMemcpyAsync(dp, hp.data(), sizeof(double2) * (size_t)n, cudaMemcpyHostToDevice, st));
        TRY(sa::scratch_alloc(&druns, sizeof(BlockConst) * runs.size(), st));
        TRY(cudaMemcpyAsync(druns, runs.data(), sizeof(BlockConst) * runs.size(), cudaMemcpyHostToDevice, st));
        // the accrual raster's per-block step masks mark the shadowed steps
        TRY(sa::scratch_alloc(&masks, sizeof(unsigned long long) * (size_t)R * sun.n_blocks, st));
        TRY(cudaMemsetAsync(masks, 0, sizeof(unsigned long long) * (size_t)R * sun.n_blocks, st));
        TRY(sa::scratch_alloc(&gross, sizeof(int) * (size_t)R, st));
        TRY(sa::scratch_alloc(&run, sizeof(int) * (size_t)R, st));
        {
            DevOut out;
            memset(&out, 0, sizeof(out));
            out.gross = gross;
            out.run = run;
            out.masks = reinterpret_cast<uint64_t*>(masks);
            TRY(launch_raster_ground(sc, rc, sun, out, st));
        }
        ContribArgs ca;
        ca.sc = sc; ca.steps = sun.steps; ca.runs = druns; ca.n_runs = (int)runs.size();
        ca.masks = masks; ca.R = R;
        ca.x0 = rc.x0; ca.y0 = rc.y0; ca.dx = rc.dx; ca.nx = rc.nx;
        ca.bx0 = (int)fx0; ca.by0 = (int)fy0;
        ca.bnx = (int)fx1 - (int)fx0 + 1; ca.bny = (int)fy1 - (int)fy0 + 1;
        ca.poly = dp; ca.n = n;
        ca.cast_cnt = cnt; ca.near_cnt = cnt + B; ca.stats = cnt + 2 * B; ca.n_b = B;
        // the work lists: per run, the cells with a shadowed step in it, in patch order
        const int nr = (int)runs.size();
        const long long patches = (long long)((ca.bnx + 7) / 8) * ((ca.bny + 3) / 4);
        const long long nslots = patches * nr;
        TRY(sa::scratch_alloc(&pcnt, sizeof(unsigned) * (size_t)(nslots + 1), st));
        TRY(sa::scratch_alloc(&poff, sizeof(unsigned) * (size_t)(nslots + 1), st));
        TRY(sa::scratch_alloc(&wbase, sizeof(int) * (size_t)(nr + 1), st));
        TRY(sa::scratch_alloc(&runinfo, sizeof(unsigned) * 2 * (size_t)nr, st));
        const unsigned pblocks = (unsigned)((patches + 3) / 4);
        k_contrib_items<<<pblocks, 128, 0, st>>>(ca, false, pcnt, nullptr, nullptr);
        TRY(cudaGetLastError());
        TRY(cudaMemsetAsync(pcnt + nslots, 0, sizeof(unsigned), st));
        TRY(cudaMemcpyAsync(poff, pcnt, sizeof(unsigned) * (size_t)(nslots + 1), cudaMemcpyDeviceToDevice, st));
        TRY(exclusive_scan_u32(poff, nslots + 1, nullptr, st));
        // per run: its first item and its count (run r's offsets start at slot r x patches)
        std::vector<unsigned> h_off((size_t)nr + 1);
        for (int r = 0; r <= nr; ++r)
            TRY(cudaMemcpyAsync(&h_off[(size_t)r], poff + (size_t)r * patches, sizeof(unsigned),
                                cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        const unsigned total = h_off[(size_t)nr];
        TRY(sa::scratch_alloc(&items, sizeof(int) * ((size_t)total + 1), st));
        k_contrib_items<<<pblocks, 128, 0, st>>>(ca, true, nullptr, poff, items);
        TRY(cudaGetLastError());
        std::vector<unsigned> h_run(2 * (size_t)nr);
        std::vector<int> h_base((size_t)nr + 1, 0);
        for (int r = 0; r < nr; ++r) {
            h_run[(size_t)r] = h_off[(size_t)r];
            h_run[(size_t)nr + r] = h_off[(size_t)r + 1] - h_off[(size_t)r];
            h_base[(size_t)r + 1] = h_base[(size_t)r] + (int)((h_run[(size_t)nr + r] + 31u) / 32u);
        }
        TRY(cudaMemcpyAsync(runinfo, h_run.data(), sizeof(unsigned) * 2 * (size_t)nr, cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(wbase, h_base.data(), sizeof(int) * (size_t)(nr + 1), cudaMemcpyHostToDevice, st));
        ca.items = items; ca.item0 = runinfo; ca.n_items = runinfo + nr; ca.warp_base = wbase;
        const long long warps = h_base[(size_t)nr];
        if (warps > 0) {
            KernelTimer kt(KT_CONTRIB, st);
            const unsigned ctas = (unsigned)((warps + kContribWarps - 1) / kContribWarps);
            if (B <= 65535) k_building_contribution<unsigned short><<<ctas, 32 * kContribWarps, 0, st>>>(ca);
            else k_building_contribution<int><<<ctas, 32 * kContribWarps, 0, st>>>(ca);
        }
        TRY(cudaGetLastError());
    }
    TRY(cudaMemcpyAsync(h_cnt.data(), cnt, sizeof(unsigned long long) * n_cnt, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    {
        const double wgt = sun.S > 0 ? (double)rc.dx * (double)rc.dx / (double)sun.S : 0.0;
        for (int b = 0; b < n_buildings; ++b) {
            casting_out[b] = (double)h_cnt[(size_t)b] * wgt;
            nearest_out[b] = (double)h_cnt[(size_t)B + b] * wgt;
        }
        stats_out[0] = h_cnt[2 * (size_t)B];
        stats_out[1] = h_cnt[2 * (size_t)B + 1];
    }
done:
    for (void* p : {(void*)masks, (void*)cnt, (void*)gross, (void*)run, (void*)dp, (void*)druns,
                    (void*)items, (void*)pcnt, (void*)poff, (void*)runinfo, (void*)wbase})
        if (p) cudaFreeAsync(p, st);
    return e;
#undef TRY
}

}  // namespace sa

extern "C" {

sa_status sa_shadow_area(const sa_receivers* grid, const int32_t* steps, int32_t total_steps,
                         const float* poly_xy, int32_t n, void* stream, double* area) {
    const char* who = "sa_shadow_area";
    if (!grid || !steps || !poly_xy || !area)
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_area: NULL argument");
    if (!grid->is_grid) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_area: receivers must be a ground grid");
    if (n < 3) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_area: a polygon needs 3 vertices");
    if (total_steps <= 0) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_area: total_steps <= 0");
    std::vector<double2> hp((size_t)n);
    for (int i = 0; i < n; ++i) {
        const float x = poly_xy[2 * i], y = poly_xy[2 * i + 1];
        if (!isfinite(x) || !isfinite(y))
            return sa::report_error(SA_ERR_DEGENERATE, "sa_shadow_area: non-finite polygon vertex");
        hp[(size_t)i] = make_double2((double)x, (double)y);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double2* dp = nullptr;
    double* dsum = nullptr;
    double result = 0.0;
    cudaError_t e = sa::scratch_alloc(&dp, sizeof(double2) * (size_t)n, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&dsum, sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, hp.data(), sizeof(double2) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(double), st);
    if (e == cudaSuccess && grid->R > 0) {
        const long long blocks = std::min<long long>((grid->R + sa::kAreaThreads - 1) / sa::kAreaThreads, 152ll * 16);
        sa::k_shadow_area<<<(unsigned)blocks, sa::kAreaThreads, 0, st>>>(
            steps, grid->x0, grid->y0, grid->dx, grid->nx, grid->R, dp, n,
            1.0 / (double)total_steps, dsum);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&result, dsum, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (dp) cudaFreeAsync(dp, st);
    if (dsum) cudaFreeAsync(dsum, st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "%s: %s", who, cudaGetErrorString(e));
        return sa::report_error(SA_ERR_CUDA, msg);
    }
    *area = result * (double)grid->dx * (double)grid->dx;
    return SA_OK;
}

sa_status sa_shadow_score(const sa_receivers* grid, const int32_t* steps, int32_t n_intervals,
                          const int32_t* total_steps, const float* weights, const float* poly_xy,
                          int32_t n, void* stream, double* score) {
    const char* who = "sa_shadow_score";
    if (!grid || !poly_xy || !score || !total_steps || !weights || (n_intervals > 0 && !steps))
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_score: NULL argument");
    if (!grid->is_grid) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_score: receivers must be a ground grid");
    if (n < 3) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_score: a polygon needs 3 vertices");
    if (n_intervals < 1) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_score: n_intervals < 1");
    std::vector<double> coef((size_t)n_intervals);
    for (int t = 0; t < n_intervals; ++t) {
        if (total_steps[t] <= 0) return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_score: total_steps <= 0");
        if (!(weights[t] >= -1.f && weights[t] <= 1.f))
            return sa::report_error(SA_ERR_INVALID_ARG, "sa_shadow_score: a weight outside [-1, 1]");
        coef[(size_t)t] = (double)weights[t] / (double)total_steps[t];
    }
    std::vector<double2> hp((size_t)n);
    for (int i = 0; i < n; ++i) {
        const float x = poly_xy[2 * i], y = poly_xy[2 * i + 1];
        if (!isfinite(x) || !isfinite(y))
            return sa::report_error(SA_ERR_DEGENERATE, "sa_shadow_score: non-finite polygon vertex");
        hp[(size_t)i] = make_double2((double)x, (double)y);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double2* dp = nullptr;
    double* dcoef = nullptr;
    double* dsum = nullptr;
    double result = 0.0;
    cudaError_t e = sa::scratch_alloc(&dp, sizeof(double2) * (size_t)n, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&dcoef, sizeof(double) * (size_t)n_intervals, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&dsum, sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, hp.data(), sizeof(double2) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dcoef, coef.data(), sizeof(double) * (size_t)n_intervals, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(double), st);
    if (e == cudaSuccess && grid->R > 0) {
        const long long blocks = std::min<long long>((grid->R + sa::kAreaThreads - 1) / sa::kAreaThreads, 152ll * 16);
        sa::k_shadow_score<<<(unsigned)blocks, sa::kAreaThreads, 0, st>>>(
            steps, grid->R, n_intervals, dcoef, grid->x0, grid->y0, grid->dx, grid->nx, dp, n, dsum);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&result, dsum, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (dp) cudaFreeAsync(dp, st);
    if (dcoef) cudaFreeAsync(dcoef, st);
    if (dsum) cudaFreeAsync(dsum, st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "%s: %s", who, cudaGetErrorString(e));
        return sa::report_error(SA_ERR_CUDA, msg);
    }
    *score = result * (double)grid->dx * (double)grid->dx;
    return SA_OK;
}

}  // extern "C"
