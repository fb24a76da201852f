// sa_footprints.cu -- extruded-footprint scenes built on the device.
//
// The paper's city is a mesh of extruded building footprints (Sec. 8.2).  A building b is
// a convex counter-clockwise footprint of v vertices extruded to height h_b: walls split
// into nb horizontal bands (two triangles per band and edge), a roof fan (v - 2) and a
// bottom fan (v - 2) at z = 0.  Band heights are h * (k / nb) in FP32, so the triangles
// are exactly those of the harness's host-side extrusion.  The band counts are fixed at
// creation, so changing heights keeps the mesh topology (used by the height gradient).
#include "sa_internal.cuh"

namespace sa {

namespace {

__global__ void k_extrude(int B, const float2* __restrict__ xy, const int* __restrict__ fp_off,
                          const float* __restrict__ heights, const int* __restrict__ bands,
                          const int* __restrict__ vert_off, const int* __restrict__ tri_off,
                          float* __restrict__ verts, int* __restrict__ tris,
                          int* __restrict__ tri_b) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int a = fp_off[b], v = fp_off[b + 1] - a;
    const int nb = bands[b];
    const float h = heights[b];
    const int vb = vert_off[b];
    for (int k = 0; k <= nb; ++k) {
        const float z = (k == nb) ? h : __fmul_rn(h, __fdiv_rn((float)k, (float)nb));
        for (int i = 0; i < v; ++i) {
            const long long q = (long long)vb + (long long)k * v + i;
            verts[3 * q] = xy[a + i].x;
            verts[3 * q + 1] = xy[a + i].y;
            verts[3 * q + 2] = z;
        }
    }
    long long t = tri_off[b];
    auto ring = [&](int k, int i) { return vb + k * v + (i % v); };
    for (int k = 0; k < nb; ++k)
        for (int i = 0; i < v; ++i) {
            const int a0 = ring(k, i), b0 = ring(k, i + 1), b1 = ring(k + 1, i + 1), a1 = ring(k + 1, i);
            tris[3 * t] = a0; tris[3 * t + 1] = b0; tris[3 * t + 2] = b1; tri_b[t++] = b;
            tris[3 * t] = a0; tris[3 * t + 1] = b1; tris[3 * t + 2] = a1; tri_b[t++] = b;
        }
    for (int i = 1; i < v - 1; ++i) {
        tris[3 * t] = ring(nb, 0); tris[3 * t + 1] = ring(nb, i); tris[3 * t + 2] = ring(nb, i + 1);
        tri_b[t++] = b;
    }
    for (int i = 1; i < v - 1; ++i) {
        tris[3 * t] = ring(0, 0); tris[3 * t + 1] = ring(0, i + 1); tris[3 * t + 2] = ring(0, i);
        tri_b[t++] = b;
    }
}

}  // namespace

cudaError_t extrude_footprints(const FootprintSet& fs, const float* d_heights, float* d_verts,
                               int* d_tris, int* d_tri_b, cudaStream_t st) {
    if (fs.B == 0) return cudaSuccess;
    k_extrude<<<(fs.B + 127) / 128, 128, 0, st>>>(fs.B, fs.xy, fs.fp_off, d_heights, fs.bands,
                                                   fs.vert_off, fs.tri_off, d_verts, d_tris, d_tri_b);
    return cudaGetLastError();
}

}  // namespace sa
