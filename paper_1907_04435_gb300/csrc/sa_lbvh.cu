// sa_lbvh.cu -- linear BVH over the city triangles, built on the device.
//
// The paper indexes the city with a uniform 3D grid for its ray traversal (Sec. 8.1); this
// library uses a linear BVH instead: Morton codes of triangle centroids, a stable radix
// sort, the radix-tree topology of Karras (HPG 2012), a bottom-up box refit, and a
// depth-first node order.  In depth-first order the subtree of a node is contiguous, so
// its escape link (the node to visit when the subtree is skipped) is just its index plus
// the subtree size, and traversal needs no stack.
#include <float.h>

#include <string.h>

#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned expand_bits10(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ unsigned morton3(float x, float y, float z) {
    unsigned ix = (unsigned)fminf(fmaxf(x * 1024.f, 0.f), 1023.f);
    unsigned iy = (unsigned)fminf(fmaxf(y * 1024.f, 0.f), 1023.f);
    unsigned iz = (unsigned)fminf(fmaxf(z * 1024.f, 0.f), 1023.f);
    return (expand_bits10(ix) << 2) | (expand_bits10(iy) << 1) | expand_bits10(iz);
}

// order-preserving float <-> uint map for atomic min / max
__device__ __forceinline__ unsigned f2o(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Gather the triangles (three float4: vertex xyz, with the building id and the input
// index in .w) and reduce the centroid bounds (cw[0..5], ordered uint).  With `check`, the
// mesh is validated on the way: the first vertex with a non-finite coordinate (every
// vertex, grid-stride; cw[14..15] as u64), the first triangle with a vertex index outside
// [0, nv) or a building id outside [0, nb) (cw[12]), and the bounds of the referenced
// vertices (cw[6..11]).  An index out of range reads no memory: its corner becomes the
// origin, and the call that asked for the check fails once the results are read back.
__global__ void k_gather(const float* __restrict__ verts, long long nv, const int* __restrict__ tris,
                         const int* __restrict__ tri_b, long long nt, int nb, int check,
                         float4* __restrict__ raw, unsigned* __restrict__ cw) {
    __shared__ unsigned s_c[12];   // centroid lo xyz, hi xyz; vertex lo xyz, hi xyz
    if (threadIdx.x < 12) s_c[threadIdx.x] = (threadIdx.x % 6) < 3 ? 0xffffffffu : 0u;
    __syncthreads();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (check) {
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long v = t; v < nv; v += stride)
            if (!(isfinite(verts[3 * v]) && isfinite(verts[3 * v + 1]) && isfinite(verts[3 * v + 2])))
                atomicMin(reinterpret_cast<unsigned long long*>(cw + 14), (unsigned long long)v);
    }
    unsigned clo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, chi[3] = {0u, 0u, 0u};
    unsigned vlo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, vhi[3] = {0u, 0u, 0u};
    if (t < nt) {
        float p[3][3];
        bool ok = true;
        for (int v = 0; v < 3; ++v) {
            const int vi = tris[3 * t + v];
            const bool in = vi >= 0 && (long long)vi < nv;
            ok = ok && in;
            for (int k = 0; k < 3; ++k) p[v][k] = in ? verts[3 * (long long)vi + k] : 0.f;
        }
        const int b = tri_b ? tri_b[t] : 0;
        if (check && (!ok || b < 0 || b >= nb)) atomicMin(reinterpret_cast<int*>(cw + 12), (int)t);
        raw[3 * t + 0] = make_float4(p[0][0], p[0][1], p[0][2], __int_as_float(b));
        raw[3 * t + 1] = make_float4(p[1][0], p[1][1], p[1][2], __int_as_float((int)t));
        raw[3 * t + 2] = make_float4(p[2][0], p[2][1], p[2][2], 0.f);
        for (int k = 0; k < 3; ++k) {
            const unsigned c = f2o((p[0][k] + p[1][k] + p[2][k]) * (1.f / 3.f));
            clo[k] = c;
            chi[k] = c;
            for (int v = 0; v < 3; ++v) {
                vlo[k] = min(vlo[k], f2o(p[v][k]));
                vhi[k] = max(vhi[k], f2o(p[v][k]));
            }
        }
    }
    // warp reductions, then one shared atomic per warp and value
    for (int k = 0; k < 3; ++k) {
        clo[k] = __reduce_min_sync(0xffffffffu, clo[k]);
        chi[k] = __reduce_max_sync(0xffffffffu, chi[k]);
        vlo[k] = __reduce_min_sync(0xffffffffu, vlo[k]);
        vhi[k] = __reduce_max_sync(0xffffffffu, vhi[k]);
    }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&s_c[k], clo[k]);
            atomicMax(&s_c[3 + k], chi[k]);
            atomicMin(&s_c[6 + k], vlo[k]);
            atomicMax(&s_c[9 + k], vhi[k]);
        }
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        if ((threadIdx.x % 6) < 3) atomicMin(&cw[threadIdx.x], s_c[threadIdx.x]);
        else atomicMax(&cw[threadIdx.x], s_c[threadIdx.x]);
    }
}

__global__ void k_morton(const float4* __restrict__ raw, long long nt,
                         const unsigned* __restrict__ cbox, unsigned* __restrict__ keys,
                         unsigned* __restrict__ vals) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float lo[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = o2f(cbox[k]);
        float ext = o2f(cbox[3 + k]) - lo[k];
        inv[k] = ext > 0.f ? 1.f / ext : 0.f;
    }
    float4 a = raw[3 * t], b = raw[3 * t + 1], c = raw[3 * t + 2];
    float cx = (a.x + b.x + c.x) * (1.f / 3.f), cy = (a.y + b.y + c.y) * (1.f / 3.f),
          cz = (a.z + b.z + c.z) * (1.f / 3.f);
    keys[t] = morton3((cx - lo[0]) * inv[0], (cy - lo[1]) * inv[1], (cz - lo[2]) * inv[2]);
    vals[t] = (unsigned)t;
}

// common-prefix length of keys i and j (index tie-break for equal keys); -1 out of range
__device__ __forceinline__ int delta(const unsigned* keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned a = keys[i], b = keys[j];
    if (a == b) return 32 + __clz((unsigned)(i ^ j));
    return __clz(a ^ b);
}

// Karras 2012: internal node i covers leaves [first, last] split after `split`.
// Node ids: internal 0..n-2, leaf k = n-1+k.
__global__ void k_karras(const unsigned* __restrict__ keys, int n, int* __restrict__ left,
                         int* __restrict__ right, int* __restrict__ parent,
                         int* __restrict__ first, int* __restrict__ last, int* __restrict__ split) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int lc = (lo == gamma) ? (n - 1 + gamma) : gamma;
    int rc = (hi == gamma + 1) ? (n - 1 + gamma + 1) : gamma + 1;
    left[i] = lc;
    right[i] = rc;
    parent[lc] = i;
    parent[rc] = i;
    first[i] = lo;
    last[i] = hi;
    split[i] = gamma;
}

// Bottom-up refit: one thread per leaf; the second child to arrive at a parent merges.
__global__ void k_refit(const float4* __restrict__ tris, int n, const int* __restrict__ left,
                        const int* __restrict__ right, const int* __restrict__ parent,
                        float4* __restrict__ blo, float4* __restrict__ bhi,
                        unsigned* __restrict__ flags) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4 a = tris[3 * k], b = tris[3 * k + 1], c = tris[3 * k + 2];
    float lo[3] = {fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z))};
    float hi[3] = {fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z))};
    // pad by a few ulps so the FP32 slab test can never reject a box holding a hit
    for (int q = 0; q < 3; ++q) {
        float pad = 4e-6f * fmaxf(fabsf(lo[q]), fabsf(hi[q])) + 1e-5f;
        lo[q] -= pad;
        hi[q] += pad;
    }
    int node = n - 1 + k;
    blo[node] = make_float4(lo[0], lo[1], lo[2], 0.f);
    bhi[node] = make_float4(hi[0], hi[1], hi[2], 0.f);
    __threadfence();
    if (n == 1) return;
    int p = parent[node];
    while (true) {
        unsigned old = atomicAdd(&flags[p], 1u);
        if (old == 0) return;   // the sibling is not done yet; it will continue
        __threadfence();
        int l = left[p], r = right[p];
        float4 l0 = __ldcg(&blo[l]), l1 = __ldcg(&bhi[l]);
        float4 r0 = __ldcg(&blo[r]), r1 = __ldcg(&bhi[r]);
        blo[p] = make_float4(fminf(l0.x, r0.x), fminf(l0.y, r0.y), fminf(l0.z, r0.z), 0.f);
        bhi[p] = make_float4(fmaxf(l1.x, r1.x), fmaxf(l1.y, r1.y), fmaxf(l1.z, r1.z), 0.f);
        __threadfence();
        if (p == 0) return;
        p = parent[p];
    }
}

// Depth-first index of every node: walk to the root adding, at each step down, 1 for a
// left child and 1 + (size of the left sibling's subtree) for a right child.
__global__ void k_emit(int n, const int* __restrict__ left, const int* __restrict__ parent,
                       const int* __restrict__ first, const int* __restrict__ last,
                       const int* __restrict__ split, const float4* __restrict__ blo,
                       const float4* __restrict__ bhi, float4* __restrict__ nodes) {
    int node = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_nodes = 2 * n - 1;
    if (node >= n_nodes) return;
    int leaves = (node >= n - 1) ? 1 : (last[node] - first[node] + 1);
    int pre = 0;
    int cur = node;
    while (cur != 0 && n > 1) {
        int p = parent[cur];
        if (left[p] == cur) {
            pre += 1;
        } else {
            int left_leaves = split[p] - first[p] + 1;
            pre += 1 + (2 * left_leaves - 1);
        }
        cur = p;
    }
    int escape = pre + 2 * leaves - 1;
    int tri = (node >= n - 1) ? (node - (n - 1)) : -1;
    float4 lo = blo[node], hi = bhi[node];
    nodes[2 * pre] = make_float4(lo.x, lo.y, lo.z, __int_as_float(escape));
    nodes[2 * pre + 1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(tri));
}

__global__ void k_permute_tris(const float4* __restrict__ raw, const unsigned* __restrict__ order,
                               long long nt, float4* __restrict__ out) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    long long t = order[k];
    out[3 * k] = raw[3 * t];
    out[3 * k + 1] = raw[3 * t + 1];
    out[3 * k + 2] = raw[3 * t + 2];
}

inline int nblk(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

}  // namespace

namespace {
float o2f_host(unsigned u) {
    const unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, sizeof(f));
    return f;
}

// The mesh checks alone, for a mesh without triangles (its vertices are still checked).
cudaError_t check_vertices_only(const float* d_verts, long long nv, MeshCheck* check, cudaStream_t st) {
    unsigned* cw = nullptr;
    cudaError_t e = sa::scratch_alloc(&cw, sizeof(unsigned) * 16, st);
    unsigned h[16] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0xffffffffu, 0xffffffffu,
                      0xffffffffu, 0u, 0u, 0u, 0x7fffffffu, 0u, 0xffffffffu, 0xffffffffu};
    if (e == cudaSuccess) e = cudaMemcpyAsync(cw, h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nv > 0) {
        k_gather<<<(int)std::min<long long>(nblk(nv), 1024), kThreads, 0, st>>>(d_verts, nv, nullptr, nullptr,
                                                                               0, 1, 1, nullptr, cw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cw, sizeof(h), cudaMemcpyDeviceToHost, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (cw) cudaFreeAsync(cw, st);
    if (e == cudaSuccess) {
        unsigned long long bv;
        memcpy(&bv, h + 14, sizeof(bv));
        check->bad_vertex = bv == ~0ull ? -1 : (long long)bv;
        check->bad_tri = -1;
        for (int k = 0; k < 6; ++k) check->box[k] = 0.f;
    }
    return e;
}
}  // namespace

cudaError_t build_lbvh(const float* d_verts, long long nv, const int* d_tris, long long nt,
                       const int* d_tri_b, LbvhBuild* out, cudaStream_t st, int n_buildings,
                       MeshCheck* check) {
    out->nodes = nullptr;
    out->tris = nullptr;
    out->n_nodes = 0;
    if (nt == 0) return check ? check_vertices_only(d_verts, nv, check, st) : cudaSuccess;
    const int n = (int)nt;
    const int n_nodes = 2 * n - 1;
    cudaError_t e;
    float4 *raw = nullptr, *blo = nullptr, *bhi = nullptr;
    unsigned *cbox = nullptr, *keys = nullptr, *vals = nullptr, *flags = nullptr;
    int* ibuf = nullptr;
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto fail; } while (0)
    TRY(sa::scratch_alloc(&out->nodes, sizeof(float4) * 2 * (size_t)n_nodes, st));
    TRY(sa::scratch_alloc(&out->tris, sizeof(float4) * 3 * (size_t)n, st));
    TRY(sa::scratch_alloc(&raw, sizeof(float4) * 3 * (size_t)n, st));
    TRY(sa::scratch_alloc(&cbox, sizeof(unsigned) * 16, st));   // bounds, checks (k_gather)
    TRY(sa::scratch_alloc(&keys, sizeof(unsigned) * (size_t)n, st));
    TRY(sa::scratch_alloc(&vals, sizeof(unsigned) * (size_t)n, st));
    TRY(sa::scratch_alloc(&blo, sizeof(float4) * (size_t)n_nodes, st));
    TRY(sa::scratch_alloc(&bhi, sizeof(float4) * (size_t)n_nodes, st));
    TRY(sa::scratch_alloc(&flags, sizeof(unsigned) * (size_t)n, st));
    TRY(sa::scratch_alloc(&ibuf, sizeof(int) * 6 * (size_t)n_nodes, st));
    {
        int* left = ibuf;
        int* right = ibuf + n_nodes;
        int* parent = ibuf + 2 * n_nodes;
        int* first = ibuf + 3 * n_nodes;
        int* last = ibuf + 4 * n_nodes;
        int* split = ibuf + 5 * n_nodes;
        unsigned init[16] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0xffffffffu, 0xffffffffu,
                             0xffffffffu, 0u, 0u, 0u, 0x7fffffffu, 0u, 0xffffffffu, 0xffffffffu};
        TRY(cudaMemcpyAsync(cbox, init, sizeof(init), cudaMemcpyHostToDevice, st));
        TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)n, st));
        TRY(cudaMemsetAsync(ibuf, 0, sizeof(int) * 6 * (size_t)n_nodes, st));
        k_gather<<<nblk(n), kThreads, 0, st>>>(d_verts, nv, d_tris, d_tri_b, n, std::max(n_buildings, 1),
                                               check ? 1 : 0, raw, cbox);
        k_morton<<<nblk(n), kThreads, 0, st>>>(raw, n, cbox, keys, vals);
        TRY(cudaGetLastError());
        TRY(radix_sort_pairs(keys, vals, n, st));
        k_permute_tris<<<nblk(n), kThreads, 0, st>>>(raw, vals, n, out->tris);
        if (n > 1) k_karras<<<nblk(n - 1), kThreads, 0, st>>>(keys, n, left, right, parent, first, last, split);
        k_refit<<<nblk(n), kThreads, 0, st>>>(out->tris, n, left, right, parent, blo, bhi, flags);
        k_emit<<<nblk(n_nodes), kThreads, 0, st>>>(n, left, parent, first, last, split, blo, bhi, out->nodes);
        TRY(cudaGetLastError());
        // the checks come back with the build; the initialisation copy reads host stack
        // memory, so the call finishes before returning either way
        if (check) TRY(cudaMemcpyAsync(init, cbox, sizeof(init), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (check) {
            unsigned long long bv;
            memcpy(&bv, init + 14, sizeof(bv));
            check->bad_vertex = bv == ~0ull ? -1 : (long long)bv;
            check->bad_tri = init[12] == 0x7fffffffu ? -1 : (long long)init[12];
            // exact bounds of the referenced vertices; a zero bound is reported as +0
            for (int k = 0; k < 6; ++k) check->box[k] = o2f_host(init[6 + k]) + 0.f;
        }
    }
    out->n_nodes = n_nodes;
    cudaFreeAsync(raw, st); cudaFreeAsync(cbox, st); cudaFreeAsync(keys, st);
    cudaFreeAsync(vals, st); cudaFreeAsync(blo, st); cudaFreeAsync(bhi, st);
    cudaFreeAsync(flags, st); cudaFreeAsync(ibuf, st);
    return cudaSuccess;
fail:
    for (void* q : {(void*)raw, (void*)cbox, (void*)keys, (void*)vals, (void*)blo, (void*)bhi,
                    (void*)flags, (void*)ibuf, (void*)out->nodes, (void*)out->tris})
        if (q) cudaFreeAsync(q, st);
    cudaStreamSynchronize(st);
    out->nodes = nullptr;
    out->tris = nullptr;
    return e;
#undef TRY
}

// ----------------------------------------------------------------- point receivers
namespace {

__global__ void k_points_prep(const float* __restrict__ pos, const float* __restrict__ nrm,
                              long long n, float4* __restrict__ orig_unsorted,
                              unsigned* __restrict__ box, int* __restrict__ bad) {
    __shared__ unsigned s_lo[3], s_hi[3];
    if (threadIdx.x < 3) { s_lo[threadIdx.x] = 0xffffffffu; s_hi[threadIdx.x] = 0u; }
    __syncthreads();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float o[3];
        float tmin = kGroundTmin;
        for (int k = 0; k < 3; ++k) o[k] = pos[3 * i + k];
        if (!(isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]))) atomicMin(&bad[0], (int)i);
        if (nrm) {
            const float n0 = nrm[3 * i], n1 = nrm[3 * i + 1], n2 = nrm[3 * i + 2];
            if (!(isfinite(n0) && isfinite(n1) && isfinite(n2))) atomicMin(&bad[1], (int)i);
            for (int k = 0; k < 3; ++k) o[k] = fmaf(kFacadeOffset, nrm[3 * i + k], o[k]);
            tmin = 0.f;
        }
        orig_unsorted[i] = make_float4(o[0], o[1], o[2], tmin);
        for (int k = 0; k < 3; ++k) {
            atomicMin(&s_lo[k], f2o(o[k]));
            atomicMax(&s_hi[k], f2o(o[k]));
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&box[threadIdx.x], s_lo[threadIdx.x]);
        atomicMax(&box[3 + threadIdx.x], s_hi[threadIdx.x]);
    }
}

// Sort key of a point receiver: 30-bit Morton code of its origin; facade points are first
// grouped by the azimuth of their normal (16 sectors in the top 4 bits, Morton in the
// remaining 28), so a warp holds walls that face the same way and turn toward or away
// from the sun together.
__global__ void k_points_morton(const float4* __restrict__ o, const float* __restrict__ nrm,
                                long long n, const unsigned* __restrict__ box,
                                unsigned* __restrict__ keys, unsigned* __restrict__ vals) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float lo[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = o2f(box[k]);
        float ext = o2f(box[3 + k]) - lo[k];
        inv[k] = ext > 0.f ? 1.f / ext : 0.f;
    }
    float4 p = o[i];
    unsigned key = morton3((p.x - lo[0]) * inv[0], (p.y - lo[1]) * inv[1], (p.z - lo[2]) * inv[2]);
    if (nrm) {
        const float az = atan2f(nrm[3 * i + 1], nrm[3 * i]);          // (-pi, pi]
        unsigned sector = (unsigned)((az + 3.14159265f) * (16.f / 6.2831853f));
        sector = sector > 15u ? 15u : sector;
        key = (sector << 28) | (key >> 2);
    }
    keys[i] = key;
    vals[i] = (unsigned)i;
}

__global__ void k_points_gather(const float4* __restrict__ o, const float* __restrict__ nrm,
                                const unsigned* __restrict__ order, long long n,
                                float4* __restrict__ out, float4* __restrict__ nout,
                                int* __restrict__ perm) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    unsigned i = order[k];
    out[k] = o[i];
    perm[k] = (int)i;
    if (nout) nout[k] = make_float4(nrm[3ll * i], nrm[3ll * i + 1], nrm[3ll * i + 2], 0.f);
}

}  // namespace

cudaError_t sort_points(const float* d_pos, const float* d_nrm, long long n, float4* d_orig,
                        float4* d_nrm_sorted, int* d_perm, cudaStream_t st, long long* bad_out,
                        float* box_out) {
    bad_out[0] = bad_out[1] = -1;
    for (int k = 0; k < 6; ++k) box_out[k] = 0.f;
    if (n == 0) return cudaSuccess;
    float4* tmp = nullptr;
    unsigned *box = nullptr, *keys = nullptr, *vals = nullptr;
    cudaError_t e = sa::scratch_alloc(&tmp, sizeof(float4) * (size_t)n, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&box, sizeof(unsigned) * 8, st);   // box, bad[2]
    if (e == cudaSuccess) e = sa::scratch_alloc(&keys, sizeof(unsigned) * (size_t)n, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&vals, sizeof(unsigned) * (size_t)n, st);
    unsigned h[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0x7fffffffu, 0x7fffffffu};
    if (e == cudaSuccess) {
        e = cudaMemcpyAsync(box, h, sizeof(h), cudaMemcpyHostToDevice, st);
        k_points_prep<<<nblk(n), kThreads, 0, st>>>(d_pos, d_nrm, n, tmp, box,
                                                     reinterpret_cast<int*>(box + 6));
        k_points_morton<<<nblk(n), kThreads, 0, st>>>(tmp, d_nrm, n, box, keys, vals);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = radix_sort_pairs(keys, vals, n, st);
        k_points_gather<<<nblk(n), kThreads, 0, st>>>(tmp, d_nrm, vals, n, d_orig,
                                                       d_nrm ? d_nrm_sorted : nullptr, d_perm);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, box, sizeof(h), cudaMemcpyDeviceToHost, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
    }
    if (tmp) cudaFreeAsync(tmp, st);
    if (box) cudaFreeAsync(box, st);
    if (keys) cudaFreeAsync(keys, st);
    if (vals) cudaFreeAsync(vals, st);
    if (e == cudaSuccess) {
        for (int k = 0; k < 6; ++k) box_out[k] = o2f_host(h[k]);
        if (h[6] != 0x7fffffffu) bad_out[0] = (long long)h[6];
        if (h[7] != 0x7fffffffu) bad_out[1] = (long long)h[7];
    }
    return e;
}

}  // namespace sa
