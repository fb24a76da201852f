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

// Building contribution (Sec. 7.2): for every cell of the region and every step the
// accrual raster marks as shadowed, one ray toward the sun collects the buildings it meets
// beyond t_min (all of them, through the whole BVH) and the building of the nearest hit.
// Each of them is credited dx^2 / total_steps: "casting" sums the shadow each building casts
// on the region, overlaps counted once per building; "nearest" splits the region's shadow
// area among the nearest casters, so it sums to the shadow area itself, less the cell-steps
// the raster marks shadowed whose FP32 ray grazes past every triangle (shadow edges),
// which are counted apart.
constexpr int kMaxCasters = 32;
constexpr int kContribThreads = 128;

__global__ void k_building_contribution(DevScene sc, const StepConst* __restrict__ steps,
                                        const BlockConst* __restrict__ blocks, int n_blocks,
                                        const unsigned long long* __restrict__ masks,
                                        float x0, float y0, float dx, int nx, long long R,
                                        const double2* __restrict__ poly, int n, double w,
                                        double* __restrict__ casting, double* __restrict__ nearest,
                                        unsigned long long* __restrict__ stats) {
    // Every lane of a warp stays to the end (the step loop votes across the warp); lanes
    // past the items, outside the polygon or never shadowed have no step bits.
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = item < R * n_blocks;
    const long long c = valid ? item % R : 0;
    const int bl = valid ? (int)(item / R) : 0;
    const BlockConst& bc = blocks[bl];
    unsigned long long m = 0ull;
    float3 o = make_float3(0.f, 0.f, 0.f);
    if (valid) {
        m = masks[(long long)bc.mask_block * R + c] >> bc.mask_bit;
        if (bc.K < 64) m &= (1ull << bc.K) - 1ull;
        const int ix = (int)(c % nx), iy = (int)(c / nx);
        o.x = __fadd_rn(x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), dx));
        o.y = __fadd_rn(y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), dx));
        if (m != 0ull && !inside_polygon(poly, n, (double)o.x, (double)o.y)) m = 0ull;
    }
    int ids[kMaxCasters];
    // The warp walks the steps in order, so the lanes tracing at once share a step: one
    // sun direction from neighbouring cells, a coherent traversal.
    for (int k = 0; k < 64; ++k) {
        const bool mine = (m >> k) & 1ull;
        if (!__any_sync(0xffffffffu, mine)) {
            if (!__any_sync(0xffffffffu, (m >> k) != 0ull)) break;
            continue;
        }
        if (!mine) continue;
        const StepConst& s = steps[bc.j0 + k];
        int nh = 0, best = -1;
        float best_t = 3.4e38f;
        bool lost = false;
        for (int i = 0; i < sc.n_nodes;) {
            const float4 lo = __ldg(&sc.nodes[2 * i]);
            const float4 hi = __ldg(&sc.nodes[2 * i + 1]);
            const int esc = __float_as_int(lo.w);
            const int tri = __float_as_int(hi.w);
            const bool in = hit_box(o, s.ix, s.iy, s.iz, lo, hi);
            if (tri >= 0) {
                if (in) {
                    const float4 a = __ldg(&sc.tris[3 * tri]);
                    const float4 b = __ldg(&sc.tris[3 * tri + 1]);
                    const float4 cc = __ldg(&sc.tris[3 * tri + 2]);
                    const float t = hit_dist_any(s.kz, o, a, b, cc, s, kGroundTmin);
                    if (t >= 0.f) {
                        const int bid = __float_as_int(a.w);
                        if (t < best_t) { best_t = t; best = bid; }
                        bool seen = false;
                        for (int q = 0; q < nh; ++q) seen |= (ids[q] == bid);
                        if (!seen) {
                            if (nh < kMaxCasters) ids[nh++] = bid;
                            else lost = true;
                        }
                    }
                }
                i = esc;
            } else {
                i = in ? i + 1 : esc;
            }
        }
        for (int q = 0; q < nh; ++q) atomicAdd(&casting[ids[q]], w);
        if (best >= 0) atomicAdd(&nearest[best], w);
        else atomicAdd(&stats[1], 1ull);     // marked shadowed by the raster, ray met nothing
        if (lost) atomicAdd(&stats[0], 1ull);
    }
}

}  // namespace

cudaError_t launch_building_contribution(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                         int n_buildings, const float* poly_xy, int n,
                                         double* casting_out, double* nearest_out,
                                         unsigned long long* stats_out, cudaStream_t st) {
    const long long R = (long long)rc.nx * rc.ny;
    const int B = n_buildings > 0 ? n_buildings : 1;
    cudaError_t e = cudaSuccess;
    unsigned long long *masks = nullptr, *ovf = nullptr;
    int *gross = nullptr, *run = nullptr;
    double2* dp = nullptr;
    double* acc = nullptr;
    std::vector<double2> hp((size_t)n);
    for (int i = 0; i < n; ++i) hp[(size_t)i] = make_double2((double)poly_xy[2 * i], (double)poly_xy[2 * i + 1]);
    std::vector<double> h_acc(2 * (size_t)B, 0.0);
    unsigned long long h_stats[2] = {0ull, 0ull};
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(sa::scratch_alloc(&acc, sizeof(double) * 2 * (size_t)B, st));
    TRY(sa::scratch_alloc(&ovf, 2 * sizeof(unsigned long long), st));
    TRY(sa::scratch_alloc(&dp, sizeof(double2) * (size_t)n, st));
    TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 2 * (size_t)B, st));
    TRY(cudaMemsetAsync(ovf, 0, 2 * sizeof(unsigned long long), st));
    TRY(cudaMemcpyAsync(dp, hp.data(), sizeof(double2) * (size_t)n, cudaMemcpyHostToDevice, st));
    if (R > 0 && sun.n_blocks > 0 && sc.T > 0) {
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
        const long long items = R * sun.n_blocks;
        const double w = (double)rc.dx * (double)rc.dx / (double)sun.S;
        k_building_contribution<<<(unsigned)((items + kContribThreads - 1) / kContribThreads),
                                  kContribThreads, 0, st>>>(
            sc, sun.steps, sun.blocks, sun.n_blocks, masks, rc.x0, rc.y0, rc.dx, rc.nx, R, dp, n, w,
            acc, acc + B, ovf);
        TRY(cudaGetLastError());
    }
    TRY(cudaMemcpyAsync(h_acc.data(), acc, sizeof(double) * 2 * (size_t)B, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(h_stats, ovf, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    for (int b = 0; b < n_buildings; ++b) {
        casting_out[b] = h_acc[(size_t)b];
        nearest_out[b] = h_acc[(size_t)B + b];
    }
    stats_out[0] = h_stats[0];
    stats_out[1] = h_stats[1];
done:
    for (void* p : {(void*)masks, (void*)ovf, (void*)gross, (void*)run, (void*)dp, (void*)acc})
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
