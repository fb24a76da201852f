// sa_trace.cu -- ray-traced shadow accumulation on the linear BVH.
//
//   k_sweep    plain per-step sweep: one any-hit ray per receiver and sun step (the
//              per-minute ray-tracing baseline of Sec. 8.1).
//   k_accrual  ray-traced accrual: one traversal per receiver and block of <= 64 steps
//              whose query is the fan of the block's rays.  The shadow of an occluder
//              point sweeps a line while the sun moves (Sec. 3.2); seen from the receiver,
//              the block's rays sweep a thin wedge, and only geometry inside that wedge
//              can shadow it in the block.  Each candidate triangle is tested exactly,
//              per step, with the same watertight test as the sweep.
//
// Both kernels are warp-coherent: the 32 lanes of a warp hold neighbouring receivers (an
// 8 x 4 patch of a ground grid or 32 Morton-consecutive points) and walk the depth-first
// node list together -- a node is entered when any lane's query overlaps it -- so node
// loads are warp-uniform broadcasts and there is no divergence in the traversal itself.
// The per-receiver gross / continuous reduction is fused into the epilogue.
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 4;

struct Receiver {
    float3 o;
    float tmin;
    float3 n;        // facade normal (zero for ground receivers)
    long long out;   // output index
    bool active;
};

__device__ __forceinline__ Receiver load_receiver(const DevRecv& rc, long long warp_id, int lane) {
    Receiver r;
    if (rc.is_grid) {
        const int tiles_x = (rc.nx + 7) >> 3;
        const long long ty = warp_id / tiles_x;
        const int tx = (int)(warp_id - ty * tiles_x);
        const int ix = tx * 8 + (lane & 7);
        const long long iy = ty * 4 + (lane >> 3);
        r.active = ix < rc.nx && iy < rc.ny;
        // cell centre, rounded exactly as x0 + (ix + 0.5) * dx in FP32 without contraction
        r.o.x = __fadd_rn(rc.x0, __fmul_rn(__fadd_rn((float)ix, 0.5f), rc.dx));
        r.o.y = __fadd_rn(rc.y0, __fmul_rn(__fadd_rn((float)iy, 0.5f), rc.dx));
        r.o.z = 0.f;
        r.tmin = kGroundTmin;
        r.n = make_float3(0.f, 0.f, 0.f);
        r.out = iy * rc.nx + ix;
    } else {
        const long long s = warp_id * 32 + lane;
        r.active = s < rc.R;
        const float4 p = r.active ? rc.orig[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        r.o = make_float3(p.x, p.y, p.z);
        r.tmin = p.w;
        const float4 nn = (r.active && rc.nrm) ? rc.nrm[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        r.n = make_float3(nn.x, nn.y, nn.z);
        r.out = r.active ? rc.perm[s] : 0;
    }
    return r;
}

__device__ __forceinline__ long long warp_count(const DevRecv& rc) {
    if (rc.is_grid) return (long long)((rc.nx + 7) >> 3) * ((rc.ny + 3) >> 2);
    return (rc.R + 31) / 32;
}

__device__ __forceinline__ RunState load_state(const DevOut& out, const Receiver& r) {
    RunState s{0, 0, 0};
    if (out.accumulate_into && r.active) {
        s.gross = out.gross[r.out];
        s.best = out.continuous ? out.continuous[r.out] : 0;
    }
    return s;
}

__device__ __forceinline__ void store_state(const DevOut& out, const Receiver& r,
                                            const RunState& s) {
    if (!r.active) return;
    out.gross[r.out] = s.gross;
    if (out.continuous) out.continuous[r.out] = s.best;
    if (out.minutes) out.minutes[r.out] = (float)s.gross * out.step_minutes;
}

// Warp-coherent any-hit query of one step for the whole warp.
template <int KZ, bool COUNT>
__device__ __forceinline__ bool any_hit_packet(const DevScene& sc, const float3& o, float tmin,
                                               const StepConst& s, bool want,
                                               unsigned long long& n_box,
                                               unsigned long long& n_tri) {
    bool hit = false;
    int i = 0;
    unsigned live = __ballot_sync(kFull, want);
    while (live != 0u && i < sc.n_nodes) {
        const float4 lo = __ldg(&sc.nodes[2 * i]);
        const float4 hi = __ldg(&sc.nodes[2 * i + 1]);
        const int esc = SA_ESC(__float_as_int(lo.w), i, sc.n_nodes, sa::CK_TRACE_ESCAPE);
        const int tri = SA_LEAF(__float_as_int(hi.w), sc.T, sa::CK_TRACE_LEAF);
        const bool in = want && !hit && hit_box(o, s.ix, s.iy, s.iz, lo, hi);
        if (COUNT && want && !hit) ++n_box;
        if (tri >= 0) {
            if (in) {
                if (COUNT) ++n_tri;
                const float4 a = __ldg(&sc.tris[3 * tri]);
                const float4 b = __ldg(&sc.tris[3 * tri + 1]);
                const float4 c = __ldg(&sc.tris[3 * tri + 2]);
                hit = hit_tri<KZ>(o, a, b, c, s.Sx, s.Sy, s.Sz, tmin);
            }
            i = esc;
            live = __ballot_sync(kFull, want && !hit);
        } else {
            i = __any_sync(kFull, in) ? i + 1 : esc;
        }
    }
    return hit;
}

__device__ __forceinline__ void flush_counts(const DevOut& out, unsigned long long n_box,
                                             unsigned long long n_tri) {
    for (int o = 16; o > 0; o >>= 1) {
        n_box += __shfl_down_sync(kFull, n_box, o);
        n_tri += __shfl_down_sync(kFull, n_tri, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out.stats[0], n_box);
        atomicAdd(&out.stats[1], n_tri);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_sweep(DevScene sc, DevRecv rc, DevSun sun, DevOut out) {
    unsigned long long n_box = 0, n_tri = 0;
    const int lane = threadIdx.x & 31;
    const long long warp_id = (long long)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    if (warp_id >= warp_count(rc)) return;
    const Receiver r = load_receiver(rc, warp_id, lane);
    RunState st = load_state(out, r);
    for (int b = 0; b < sun.n_blocks; ++b) {
        const int j0 = sun.blocks[b].j0, K = sun.blocks[b].K;
        uint64_t m = 0;
        for (int k = 0; k < K; ++k) {
            const StepConst s = sun.steps[j0 + k];
            bool h;
            if (s.kz == 2) h = any_hit_packet<2, COUNT>(sc, r.o, r.tmin, s, r.active, n_box, n_tri);
            else if (s.kz == 0) h = any_hit_packet<0, COUNT>(sc, r.o, r.tmin, s, r.active, n_box, n_tri);
            else h = any_hit_packet<1, COUNT>(sc, r.o, r.tmin, s, r.active, n_box, n_tri);
            if (h) m |= 1ull << k;
        }
        stitch(st, m, K, sun.blocks[b].new_day);
        if (out.masks && r.active)
            out.masks[(long long)sun.blocks[b].mask_block * rc.R + r.out] |= m << sun.blocks[b].mask_bit;
    }
    store_state(out, r, st);
    if (COUNT) flush_counts(out, n_box, n_tri);
}

// ------------------------------------------------------------------- accrual trace
// ------------------------------------------------------------ per-lane traversal
// Watertight test with the major axis chosen at run time (component selects instead of
// the template), so lanes of a warp can test different steps at once.
__device__ __forceinline__ float pick(const float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ __forceinline__ float pick3(const float3& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ bool hit_tri_rt(const float3& o, const float4& a, const float4& b,
                                           const float4& c, const StepConst& s, float tmin) {
    const int kz = s.kz, kx = kz == 2 ? 0 : kz + 1, ky = kz == 0 ? 2 : kz - 1;
    const float oz = pick3(o, kz), ox = pick3(o, kx), oy = pick3(o, ky);
    const float az = pick(a, kz) - oz, bz = pick(b, kz) - oz, cz = pick(c, kz) - oz;
    const float ax = fmaf(-s.Sx, az, pick(a, kx) - ox), ay = fmaf(-s.Sy, az, pick(a, ky) - oy);
    const float bx = fmaf(-s.Sx, bz, pick(b, kx) - ox), by = fmaf(-s.Sy, bz, pick(b, ky) - oy);
    const float cx = fmaf(-s.Sx, cz, pick(c, kx) - ox), cy = fmaf(-s.Sy, cz, pick(c, ky) - oy);
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    const float det = U + V + W;
    if (det == 0.f) return false;
    const float T = U * (s.Sz * az) + V * (s.Sz * bz) + W * (s.Sz * cz);
    return det > 0.f ? (T > tmin * det) : (T < tmin * det);
}


template <bool COUNT>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_accrual(DevScene sc, DevRecv rc, DevSun sun, DevOut out) {
    // block and step constants are copied per warp, so warps never wait for one another
    __shared__ BlockConst s_bc[kWarpsPerCta];
    __shared__ StepConst s_st[kWarpsPerCta][kMaxBlock];
    unsigned long long n_box = 0, n_tri = 0;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long warp_id = (long long)blockIdx.x * kWarpsPerCta + wib;
    if (warp_id >= warp_count(rc)) return;
    const Receiver r = load_receiver(rc, warp_id, lane);
    RunState st = load_state(out, r);
    BlockConst& bc = s_bc[wib];
    StepConst* ss = s_st[wib];
    // occluder cache: the last triangle that shadowed this receiver is tried first in the
    // next block (shadows move slowly, so it often covers many of the block's steps)
    int ctri = -1;
    for (int b = 0; b < sun.n_blocks; ++b) {
        __syncwarp();
        for (int w = lane; w < (int)(sizeof(BlockConst) / 4); w += 32)
            reinterpret_cast<int*>(&bc)[w] = reinterpret_cast<const int*>(&sun.blocks[b])[w];
        __syncwarp();
        const int K = bc.K;
        for (int w = lane; w < K * (int)(sizeof(StepConst) / 4); w += 32)
            reinterpret_cast<int*>(ss)[w] = reinterpret_cast<const int*>(&sun.steps[bc.j0])[w];
        __syncwarp();
        const uint64_t full = (K >= 64) ? ~0ull : ((1ull << K) - 1ull);
        uint64_t m = 0;
        const bool wedge = bc.wedge_ok != 0.f;
        // lower bound of n . d over the block's direction box
        const float nd_lo = fminf(r.n.x * bc.dlo[0], r.n.x * bc.dhi[0]) +
                            fminf(r.n.y * bc.dlo[1], r.n.y * bc.dhi[1]) +
                            fminf(r.n.z * bc.dlo[2], r.n.z * bc.dhi[2]);
        const bool front = nd_lo > 1e-6f;
        if (r.active && ctri >= 0) {
            const float4 ta = __ldg(&sc.tris[3 * ctri]);
            const float4 tb = __ldg(&sc.tris[3 * ctri + 1]);
            const float4 tc = __ldg(&sc.tris[3 * ctri + 2]);
            int ka, kb;
            candidate_steps(r.o, bc, bc.psi, ta, tb, tc, &ka, &kb);
            const PluckerTri pt = plucker_setup(r.o, ta, tb, tc);
            for (int k = ka; k <= kb; ++k) {
                if (COUNT) ++n_tri;
                if (plucker_hit(pt, ss[k].dx, ss[k].dy, ss[k].dz, r.tmin)) m |= 1ull << k;
            }
        }
        int i = 0;
        unsigned live = __ballot_sync(kFull, r.active && m != full);
        while (live != 0u && i < sc.n_nodes) {
            const float4 lo = __ldg(&sc.nodes[2 * i]);
            const float4 hi = __ldg(&sc.nodes[2 * i + 1]);
            const int esc = SA_ESC(__float_as_int(lo.w), i, sc.n_nodes, sa::CK_TRACE_ESCAPE);
            const int tri = SA_LEAF(__float_as_int(hi.w), sc.T, sa::CK_TRACE_LEAF);
            const bool want = r.active && m != full;
            const bool in = want && (wedge ? fan_box(r.o, bc, lo, hi, front, r.n) : slope_box(r.o, bc, lo, hi));
            if (COUNT && want) ++n_box;
            if (tri >= 0) {
                int ka = K, kb = -1;
                float4 ta, tb, tc;
                if (in) {
                    ta = __ldg(&sc.tris[3 * tri]);
                    tb = __ldg(&sc.tris[3 * tri + 1]);
                    tc = __ldg(&sc.tris[3 * tri + 2]);
                    if (plane_reachable(r.o, ta, tb, tc, bc))
                        candidate_steps(r.o, bc, bc.psi, ta, tb, tc, &ka, &kb);
                }
                const int wa = __reduce_min_sync(kFull, ka);
                const int wb = __reduce_max_sync(kFull, kb);
                if (wa <= wb) {
                    PluckerTri pt;
                    if (ka <= kb) pt = plucker_setup(r.o, ta, tb, tc);
                    for (int k = wa; k <= wb; ++k) {
                        const bool test = k >= ka && k <= kb && !((m >> k) & 1ull);
                        if (test) {
                            if (COUNT) ++n_tri;
                            if (plucker_hit(pt, ss[k].dx, ss[k].dy, ss[k].dz, r.tmin)) {
                                m |= 1ull << k;
                                ctri = tri;
                            }
                        }
                    }
                }
                i = esc;
                live = __ballot_sync(kFull, r.active && m != full);
            } else {
                i = __any_sync(kFull, in) ? i + 1 : esc;
            }
        }
        stitch(st, m, K, bc.new_day);
        if (out.masks && r.active) out.masks[(long long)bc.mask_block * rc.R + r.out] |= m << bc.mask_bit;
    }
    store_state(out, r, st);
    if (COUNT) flush_counts(out, n_box, n_tri);
}

// Ray-traced accrual with one independent traversal per lane ("while-while": each lane
// descends internal nodes until it reaches a leaf its fan overlaps, then the lanes process
// their leaves together).  Block and step constants are copied per warp into shared
// memory, so warps of a CTA never wait for one another.
template <bool COUNT>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_accrual_lane(DevScene sc, DevRecv rc, DevSun sun, DevOut out) {
    __shared__ BlockConst s_bc[kWarpsPerCta];
    __shared__ StepConst s_st[kWarpsPerCta][kMaxBlock];
    unsigned long long n_box = 0, n_tri = 0;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long warp_id = (long long)blockIdx.x * kWarpsPerCta + wib;
    if (warp_id >= warp_count(rc)) return;
    const Receiver r = load_receiver(rc, warp_id, lane);
    RunState st = load_state(out, r);
    BlockConst& bc = s_bc[wib];
    StepConst* ss = s_st[wib];
    for (int b = 0; b < sun.n_blocks; ++b) {
        __syncwarp();
        for (int w = lane; w < (int)(sizeof(BlockConst) / 4); w += 32)
            reinterpret_cast<int*>(&bc)[w] = reinterpret_cast<const int*>(&sun.blocks[b])[w];
        __syncwarp();
        const int K = bc.K;
        for (int w = lane; w < K * (int)(sizeof(StepConst) / 4); w += 32)
            reinterpret_cast<int*>(ss)[w] = reinterpret_cast<const int*>(&sun.steps[bc.j0])[w];
        __syncwarp();
        const uint64_t full = (K >= 64) ? ~0ull : ((1ull << K) - 1ull);
        const bool wedge = bc.wedge_ok != 0.f;
        uint64_t m = 0;
        int i = r.active ? 0 : sc.n_nodes;
        while (i < sc.n_nodes && m != full) {
            int tri = -1;
            float4 lo, hi;
            while (i < sc.n_nodes) {
                lo = __ldg(&sc.nodes[2 * i]);
                hi = __ldg(&sc.nodes[2 * i + 1]);
                const int esc = SA_ESC(__float_as_int(lo.w), i, sc.n_nodes, sa::CK_TRACE_ESCAPE);
                const bool in = wedge ? fan_box(r.o, bc, lo, hi) : slope_box(r.o, bc, lo, hi);
                if (COUNT) ++n_box;
                if (!in) { i = esc; continue; }
                tri = SA_LEAF(__float_as_int(hi.w), sc.T, sa::CK_TRACE_LEAF);
                if (tri >= 0) { i = esc; break; }
                i = i + 1;
            }
            if (tri < 0) break;
            const float4 ta = __ldg(&sc.tris[3 * tri]);
            const float4 tb = __ldg(&sc.tris[3 * tri + 1]);
            const float4 tc = __ldg(&sc.tris[3 * tri + 2]);
            int ka = 0, kb = -1;
            if (plane_reachable(r.o, ta, tb, tc, bc)) candidate_steps(r.o, bc, bc.psi, ta, tb, tc, &ka, &kb);
            for (int k = ka; k <= kb; ++k) {
                if ((m >> k) & 1ull) continue;
                if (COUNT) ++n_tri;
                if (hit_tri_rt(r.o, ta, tb, tc, ss[k], r.tmin)) m |= 1ull << k;
            }
        }
        stitch(st, m, K, bc.new_day);
        if (out.masks && r.active) out.masks[(long long)bc.mask_block * rc.R + r.out] |= m << bc.mask_bit;
    }
    store_state(out, r, st);
    if (COUNT) flush_counts(out, n_box, n_tri);
}

// Per-step sweep with one independent traversal per lane.
template <bool COUNT>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_sweep_lane(DevScene sc, DevRecv rc, DevSun sun, DevOut out) {
    unsigned long long n_box = 0, n_tri = 0;
    const int lane = threadIdx.x & 31;
    const long long warp_id = (long long)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    if (warp_id >= warp_count(rc)) return;
    const Receiver r = load_receiver(rc, warp_id, lane);
    RunState st = load_state(out, r);
    for (int b = 0; b < sun.n_blocks; ++b) {
        const int j0 = sun.blocks[b].j0, K = sun.blocks[b].K;
        uint64_t m = 0;
        for (int k = 0; k < K; ++k) {
            const StepConst s = sun.steps[j0 + k];
            bool hit = false;
            int i = r.active ? 0 : sc.n_nodes;
            while (i < sc.n_nodes && !hit) {
                const float4 lo = __ldg(&sc.nodes[2 * i]);
                const float4 hi = __ldg(&sc.nodes[2 * i + 1]);
                const int esc = SA_ESC(__float_as_int(lo.w), i, sc.n_nodes, sa::CK_TRACE_ESCAPE);
                const int tri = SA_LEAF(__float_as_int(hi.w), sc.T, sa::CK_TRACE_LEAF);
                if (COUNT) ++n_box;
                if (!hit_box(r.o, s.ix, s.iy, s.iz, lo, hi)) { i = esc; continue; }
                if (tri < 0) { i = i + 1; continue; }
                if (COUNT) ++n_tri;
                hit = hit_tri_rt(r.o, __ldg(&sc.tris[3 * tri]), __ldg(&sc.tris[3 * tri + 1]),
                                 __ldg(&sc.tris[3 * tri + 2]), s, r.tmin);
                i = esc;
            }
            if (hit) m |= 1ull << k;
        }
        stitch(st, m, K, sun.blocks[b].new_day);
        if (out.masks && r.active)
            out.masks[(long long)sun.blocks[b].mask_block * rc.R + r.out] |= m << sun.blocks[b].mask_bit;
    }
    store_state(out, r, st);
    if (COUNT) flush_counts(out, n_box, n_tri);
}

long long host_warps(const DevRecv& rc) {
    if (rc.is_grid) return (long long)((rc.nx + 7) / 8) * ((rc.ny + 3) / 4);
    return (rc.R + 31) / 32;
}

}  // namespace

// Traversal mode: 1 = warp-coherent (packet), 2 = per lane, 0 = the measured default:
// per lane for the per-step sweep (single rays: lanes rarely wait on each other), packet
// for the accrual (its leaf work is a loop over steps that lanes share best in lockstep).
int g_trace_mode[2] = {0, 0};   // [0] sweep, [1] accrual

static bool use_lane(int which, const DevRecv& rc) {
    const int mode = g_trace_mode[which];
    (void)rc;
    return mode == 2 || (mode == 0 && which == 0);
}

cudaError_t launch_sweep_trace(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                               const DevOut& out, cudaStream_t st) {
    const long long warps = host_warps(rc);
    if (warps == 0) return cudaSuccess;
    const unsigned ctas = (unsigned)((warps + kWarpsPerCta - 1) / kWarpsPerCta);
    const int T = 32 * kWarpsPerCta;
    KernelTimer kt(KT_SWEEP, st);
    if (use_lane(0, rc)) {
        if (out.stats) k_sweep_lane<true><<<ctas, T, 0, st>>>(sc, rc, sun, out);
        else k_sweep_lane<false><<<ctas, T, 0, st>>>(sc, rc, sun, out);
    } else {
        if (out.stats) k_sweep<true><<<ctas, T, 0, st>>>(sc, rc, sun, out);
        else k_sweep<false><<<ctas, T, 0, st>>>(sc, rc, sun, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_accrual_trace(const DevScene& sc, const DevRecv& rc, const DevSun& sun,
                                 const DevOut& out, cudaStream_t st) {
    const long long warps = host_warps(rc);
    if (warps == 0) return cudaSuccess;
    const unsigned ctas = (unsigned)((warps + kWarpsPerCta - 1) / kWarpsPerCta);
    const int T = 32 * kWarpsPerCta;
    KernelTimer kt(KT_ACCRUAL, st);
    if (use_lane(1, rc)) {
        if (out.stats) k_accrual_lane<true><<<ctas, T, 0, st>>>(sc, rc, sun, out);
        else k_accrual_lane<false><<<ctas, T, 0, st>>>(sc, rc, sun, out);
    } else {
        if (out.stats) k_accrual<true><<<ctas, T, 0, st>>>(sc, rc, sun, out);
        else k_accrual<false><<<ctas, T, 0, st>>>(sc, rc, sun, out);
    }
    return cudaGetLastError();
}

void set_trace_mode(int which, int mode) { g_trace_mode[which] = mode; }
int get_trace_mode(int which) { return g_trace_mode[which]; }

}  // namespace sa
