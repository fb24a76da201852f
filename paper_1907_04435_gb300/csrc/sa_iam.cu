// sa_iam.cu -- inverse accrual map (Sec. 5) of a ground receiver grid.
//
// Per block of K steps:
//   k_iam_draw  every cell centre p traces toward the sun at the block's first step and
//               keeps the L nearest intersections farther than 1 m (the paper's source
//               levels and its 100 cm acne rule).  Each source s casts its shadow at step
//               k at q_k, the projection of s along d_k onto the ground; the shadow line
//               q_0 -> q_{K-1} is cut into K - 1 pieces and piece [q_k, q_{k+1}] sets bit
//               k of every grid cell it touches (closed cells), bit K-1 being set at
//               q_{K-1}.  The same is done from the block's last step with the pieces
//               running backwards (the paper's t_n -> t_1 map), which catches stretching
//               shadows and sources missed by the first map.
//   k_iam_fold  folds each cell's 64-bit vector into its gross / continuous state and
//               clears it for the next block.
// The bit vectors live in one uint64 per cell; drawing uses atomicOr, skipped when the
// bit is already set.  This is the paper's approximate method: it is compared with its
// own FP64 restatement and with the exact result (the paper's area-error bar).
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;
constexpr int kMaxLevels = 8;
constexpr float kSourceTmin = 1.0f;     // sources closer than 100 cm are ignored (Sec. 5)

// Watertight test returning the distance of the hit (see hit_tri).
template <int KZ>
__device__ __forceinline__ bool hit_tri_t(const float3& o, const float4& a, const float4& b,
                                          const float4& c, float Sx, float Sy, float Sz,
                                          float tmin, float* t_out) {
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
    const float det = U + V + W;
    if (det == 0.f) return false;
    const float T = U * (Sz * az) + V * (Sz * bz) + W * (Sz * cz);
    const float t = T / det;
    if (!(t > tmin)) return false;
    *t_out = t;
    return true;
}

// Slab test with an upper bound on the entry distance.
__device__ __forceinline__ bool hit_box_before(const float3& o, const StepConst& s, const float4& lo,
                                               const float4& hi, float tmax) {
    float tx0 = (lo.x - o.x) * s.ix, tx1 = (hi.x - o.x) * s.ix;
    float ty0 = (lo.y - o.y) * s.iy, ty1 = (hi.y - o.y) * s.iy;
    float tz0 = (lo.z - o.z) * s.iz, tz1 = (hi.z - o.z) * s.iz;
    float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    return tn <= tf * 1.0000005f && tn <= tmax;
}

// The L nearest hits (ascending) of the ray from o along step s; warp-coherent traversal.
template <int KZ>
__device__ int nearest_sources(const DevScene& sc, const float3& o, const StepConst& s,
                               bool active, int L, float* best) {
    int n = 0;
    int i = 0;
    while (i < sc.n_nodes && __any_sync(kFull, active)) {
        const float4 lo = __ldg(&sc.nodes[2 * i]);
        const float4 hi = __ldg(&sc.nodes[2 * i + 1]);
        const int esc = SA_ESC(__float_as_int(lo.w), i, sc.n_nodes, sa::CK_IAM_ESCAPE);
        const int tri = SA_LEAF(__float_as_int(hi.w), sc.T, sa::CK_IAM_LEAF);
        const float bound = n < L ? 3.4e38f : best[L - 1];
        const bool in = active && hit_box_before(o, s, lo, hi, bound);
        if (tri >= 0) {
            if (in) {
                const float4 a = __ldg(&sc.tris[3 * tri]);
                const float4 b = __ldg(&sc.tris[3 * tri + 1]);
                const float4 c = __ldg(&sc.tris[3 * tri + 2]);
                float t;
                if (hit_tri_t<KZ>(o, a, b, c, s.Sx, s.Sy, s.Sz, kSourceTmin, &t) && t < bound) {
                    int k = n < L ? n++ : L - 1;
                    while (k > 0 && best[k - 1] > t) { best[k] = best[k - 1]; --k; }
                    best[k] = t;
                }
            }
            i = esc;
        } else {
            i = __any_sync(kFull, in) ? i + 1 : esc;
        }
    }
    return n;
}

struct Grid {
    float x0, y0, dx;
    int nx, ny;
};

__device__ __forceinline__ void mark(unsigned long long* masks, long long cell, unsigned long long bit) {
    if (!(__ldcg(&masks[cell]) & bit)) atomicOr(&masks[cell], bit);
}

// Every closed grid cell touched by the segment P -> Q gets `bit`.
__device__ void draw_segment(const Grid& g, float px, float py, float qx, float qy,
                             unsigned long long* masks, unsigned long long bit) {
    const float inv = 1.f / g.dx;
    const float ymin = fminf(py, qy), ymax = fmaxf(py, qy);
    int iy0 = (int)ceilf((ymin - g.y0) * inv) - 1;
    int iy1 = (int)floorf((ymax - g.y0) * inv);
    iy0 = max(iy0, 0);
    iy1 = min(iy1, g.ny - 1);
    for (int iy = iy0; iy <= iy1; ++iy) {
        const float b0 = g.y0 + (float)iy * g.dx, b1 = b0 + g.dx;
        float xa, xb;
        if (py == qy) {
            if (py < b0 || py > b1) continue;
            xa = fminf(px, qx); xb = fmaxf(px, qx);
        } else {
            const float rdy = 1.f / (qy - py);
            const float ta = (b0 - py) * rdy, tb = (b1 - py) * rdy;
            const float lo = fmaxf(fminf(ta, tb), 0.f), hi = fminf(fmaxf(ta, tb), 1.f);
            if (lo > hi) continue;
            const float x1 = fmaf(lo, qx - px, px), x2 = fmaf(hi, qx - px, px);
            xa = fminf(x1, x2); xb = fmaxf(x1, x2);
        }
        int ix0 = (int)ceilf((xa - g.x0) * inv) - 1;
        int ix1 = (int)floorf((xb - g.x0) * inv);
        ix0 = max(ix0, 0);
        ix1 = min(ix1, g.nx - 1);
        for (int ix = ix0; ix <= ix1; ++ix) mark(masks, (long long)iy * g.nx + ix, bit);
    }
}

__global__ void __launch_bounds__(32 * kWarps)
k_iam_draw(DevScene sc, Grid g, const StepConst* __restrict__ steps, int j0, int K, int L,
           unsigned long long* __restrict__ masks) {
    const int lane = threadIdx.x & 31;
    const long long warp_id = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int tiles_x = (g.nx + 7) >> 3;
    const long long n_warps = (long long)tiles_x * ((g.ny + 3) >> 2);
    if (warp_id >= n_warps) return;
    const long long ty = warp_id / tiles_x;
    const int tx = (int)(warp_id - ty * tiles_x);
    const int ix = tx * 8 + (lane & 7);
    const long long iy = ty * 4 + (lane >> 3);
    const bool active = ix < g.nx && iy < g.ny;
    float3 o;
    o.x = __fadd_rn(g.x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), g.dx));
    o.y = __fadd_rn(g.y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), g.dx));
    o.z = 0.f;
    for (int dir = 0; dir < 2; ++dir) {
        const StepConst s = steps[dir == 0 ? j0 : j0 + K - 1];
        float best[kMaxLevels];
        int n;
        if (s.kz == 2) n = nearest_sources<2>(sc, o, s, active, L, best);
        else if (s.kz == 0) n = nearest_sources<0>(sc, o, s, active, L, best);
        else n = nearest_sources<1>(sc, o, s, active, L, best);
        for (int l = 0; l < n; ++l) {
            const float sx = fmaf(best[l], s.dx, o.x), sy = fmaf(best[l], s.dy, o.y),
                        sz = best[l] * s.dz;
            // q_k for the block's steps; the pieces run forward (dir 0) or backward (dir 1)
            if (dir == 0) {
                float px = fmaf(-sz, steps[j0].ux, sx), py = fmaf(-sz, steps[j0].uy, sy);
                for (int k = 0; k + 1 < K; ++k) {
                    const float qx = fmaf(-sz, steps[j0 + k + 1].ux, sx);
                    const float qy = fmaf(-sz, steps[j0 + k + 1].uy, sy);
                    draw_segment(g, px, py, qx, qy, masks, 1ull << k);
                    px = qx; py = qy;
                }
                draw_segment(g, px, py, px, py, masks, 1ull << (K - 1));
            } else {
                float px = fmaf(-sz, steps[j0 + K - 1].ux, sx), py = fmaf(-sz, steps[j0 + K - 1].uy, sy);
                for (int k = K - 1; k >= 1; --k) {
                    const float qx = fmaf(-sz, steps[j0 + k - 1].ux, sx);
                    const float qy = fmaf(-sz, steps[j0 + k - 1].uy, sy);
                    draw_segment(g, px, py, qx, qy, masks, 1ull << k);
                    px = qx; py = qy;
                }
                draw_segment(g, px, py, px, py, masks, 1ull);
            }
        }
    }
}

__global__ void k_iam_fold(long long R, int K, int new_day, int mask_block,
                           unsigned long long* __restrict__ masks, DevOut out, int first,
                           int last) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    RunState st{0, 0, 0};
    if (!first || out.accumulate_into) {
        st.gross = out.gross[r];
        st.best = out.continuous ? out.continuous[r] : 0;
        st.run = (first) ? 0 : out.run[r];
    }
    const unsigned long long m = masks[r];
    masks[r] = 0ull;
    stitch(st, m, K, new_day);
    out.gross[r] = st.gross;
    if (out.continuous) out.continuous[r] = st.best;
    out.run[r] = st.run;
    if (out.masks) out.masks[(long long)mask_block * R + r] |= m;
    if (last && out.minutes) out.minutes[r] = (float)st.gross * out.step_minutes;
}

}  // namespace

cudaError_t launch_iam(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                       const BlockConst* h_blocks, int L, const DevOut& out, cudaStream_t st) {
    const long long R = (long long)rc.nx * rc.ny;
    if (R == 0) return cudaSuccess;
    if (L < 1 || L > kMaxLevels) return cudaErrorInvalidValue;
    unsigned long long* masks = nullptr;
    cudaError_t e = sa::scratch_alloc(&masks, sizeof(unsigned long long) * (size_t)R, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(masks, 0, sizeof(unsigned long long) * (size_t)R, st);
    Grid g{rc.x0, rc.y0, rc.dx, rc.nx, rc.ny};
    const long long warps = (long long)((rc.nx + 7) / 8) * ((rc.ny + 3) / 4);
    const unsigned ctas = (unsigned)((warps + kWarps - 1) / kWarps);
    for (int b = 0; b < sun.n_blocks && e == cudaSuccess; ++b) {
        const BlockConst& bc = h_blocks[b];
        {
            KernelTimer kt(KT_IAM, st);
            k_iam_draw<<<ctas, 32 * kWarps, 0, st>>>(sc, g, sun.steps, bc.j0, bc.K, L, masks);
        }
        k_iam_fold<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(R, bc.K, bc.new_day, bc.mask_block,
                                                               masks, out, b == 0,
                                                               b == sun.n_blocks - 1);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(masks, st);
    return e != cudaSuccess ? e : e2;
}

}  // namespace sa
