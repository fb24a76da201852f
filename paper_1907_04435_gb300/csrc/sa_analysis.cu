// sa_analysis.cu -- analysis measures over a polygonal region of a ground grid (Sec. 7.2).
//
// Shadow area: the sum over the region's cells of shadow(p) x area(p), where shadow(p) is
// the fraction of the interval's steps the cell spends in shadow (gross counts give the
// gross fraction, continuous counts the continuous one) and area(p) = dx^2.  A cell is in
// the region when its centre is, by the even-odd rule.  The shadow score over several
// intervals is the weighted sum of their areas (weights in [-1, 1]); it needs no kernel.
//
// The centres are rounded exactly as the receivers' (FP32), then tested in FP64 with
// explicit roundings, so the decision for a centre does not depend on the compiler's
// contraction of multiply-adds.
#include <math.h>
#include <stdio.h>

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

}  // namespace

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

}  // extern "C"
