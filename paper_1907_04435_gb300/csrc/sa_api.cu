// sa_api.cu -- C ABI of libshadowaccrual: handles, validation, sun-table partitioning and
// dispatch of the accumulation methods.  See include/shadowaccrual.h for the contract.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sa_handles.cuh"

namespace {

thread_local char g_err[512] = "";

sa_status fail(sa_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

sa_status cuda_fail(cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(SA_ERR_OOM, "%s: out of device memory", where);
    return fail(SA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void make_step(const float* d, sa::StepConst* s) {
    s->dx = d[0]; s->dy = d[1]; s->dz = d[2];
    s->ux = (float)((double)d[0] / (double)d[2]);
    s->uy = (float)((double)d[1] / (double)d[2]);
    float inv[3];
    for (int k = 0; k < 3; ++k) {
        double v = d[k];
        if (fabs(v) < 1e-20) v = v < 0 ? -1e-20 : 1e-20;
        inv[k] = (float)(1.0 / v);
    }
    s->ix = inv[0]; s->iy = inv[1]; s->iz = inv[2];
    int kz = 2;
    if (fabsf(d[0]) > fabsf(d[kz])) kz = 0;
    if (fabsf(d[1]) > fabsf(d[kz])) kz = 1;
    const int kx = (kz + 1) % 3, ky = (kz + 2) % 3;
    s->kz = kz;
    s->Sx = (float)((double)d[kx] / (double)d[kz]);
    s->Sy = (float)((double)d[ky] / (double)d[kz]);
    s->Sz = (float)(1.0 / (double)d[kz]);
    s->pad0 = s->pad1 = s->pad2 = s->pad3 = 0;
}

void cross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
double dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void normalize(double* a) {
    double n = sqrt(dot(a, a));
    for (int k = 0; k < 3; ++k) a[k] /= n;
}

// Block constants for steps [j0, j0 + K): slope box, and the wedge bounding the fan of
// the block's rays (plane through the first and last directions, in-plane angles psi).
sa::BlockConst make_block(const float* dirs, const std::vector<sa::StepConst>& steps, int j0,
                          int K, int new_day, bool with_wedge) {
    sa::BlockConst b;
    memset(&b, 0, sizeof(b));
    b.j0 = j0; b.K = K; b.new_day = new_day; b.monotone = 0;
    b.mask_block = 0; b.mask_bit = 0;
    b.uxlo = b.uylo = 3.4e38f; b.uxhi = b.uyhi = -3.4e38f;
    for (int q = 0; q < 3; ++q) { b.dlo[q] = 3.4e38f; b.dhi[q] = -3.4e38f; }
    for (int k = 0; k < K; ++k)
        for (int q = 0; q < 3; ++q) {
            b.dlo[q] = std::min(b.dlo[q], dirs[3 * (j0 + k) + q]);
            b.dhi[q] = std::max(b.dhi[q], dirs[3 * (j0 + k) + q]);
        }
    for (int k = 0; k < K; ++k) {
        b.uxlo = std::min(b.uxlo, steps[j0 + k].ux); b.uxhi = std::max(b.uxhi, steps[j0 + k].ux);
        b.uylo = std::min(b.uylo, steps[j0 + k].uy); b.uyhi = std::max(b.uyhi, steps[j0 + k].uy);
    }
    b.wedge_ok = 0.f;
    if (!with_wedge || K < 2) return b;
    double a[3], c[3], n[3];
    for (int q = 0; q < 3; ++q) { a[q] = dirs[3 * j0 + q]; c[q] = dirs[3 * (j0 + K - 1) + q]; }
    normalize(a); normalize(c);
    cross(a, c, n);
    const double nn = sqrt(dot(n, n));
    if (nn < 1e-7) return b;
    for (int q = 0; q < 3; ++q) n[q] /= nn;
    double e1[3] = {a[0] + c[0], a[1] + c[1], a[2] + c[2]};
    const double pn = dot(e1, n);
    for (int q = 0; q < 3; ++q) e1[q] -= pn * n[q];
    normalize(e1);
    double e2[3];
    cross(n, e1, e2);
    double soff = 0.0, pmin = 1e9, pmax = -1e9;
    int mono = 1;
    double prev = -1e9;
    for (int k = 0; k < K; ++k) {
        double d[3];
        for (int q = 0; q < 3; ++q) d[q] = dirs[3 * (j0 + k) + q];
        normalize(d);
        soff = std::max(soff, fabs(dot(n, d)));
        const double psi = atan2(dot(e2, d), dot(e1, d));
        b.psi[k] = (float)psi;
        pmin = std::min(pmin, psi);
        pmax = std::max(pmax, psi);
        if (psi < prev) mono = 0;
        prev = psi;
    }
    if (pmax - pmin > 3.0) return b;   // not a thin fan: keep the slope box
    const double eps = 1e-5;
    b.monotone = mono;
    b.psi_eps = 2e-5f;
    b.s_off = (float)(soff + 1e-6);
    b.nx = (float)n[0]; b.ny = (float)n[1]; b.nz = (float)n[2];
    b.e1x = (float)e1[0]; b.e1y = (float)e1[1]; b.e1z = (float)e1[2];
    b.e2x = (float)e2[0]; b.e2y = (float)e2[1]; b.e2z = (float)e2[2];
    const double lo = pmin - eps, hi = pmax + eps;
    for (int q = 0; q < 3; ++q) {
        (&b.g1x)[q] = (float)(-sin(lo) * e1[q] + cos(lo) * e2[q]);
        (&b.g2x)[q] = (float)(sin(hi) * e1[q] - cos(hi) * e2[q]);
    }
    b.wedge_ok = 1.f;
    return b;
}

sa::DevScene dev_scene(const sa_scene* s) {
    sa::DevScene d;
    d.nodes = s->bvh.nodes;
    d.tris = s->bvh.tris;
    d.n_nodes = s->bvh.n_nodes;
    d.T = (int)s->T;
    d.closed = s->closed;
    return d;
}

sa::DevRecv dev_recv(const sa_receivers* r) {
    sa::DevRecv d;
    d.is_grid = r->is_grid;
    d.x0 = r->x0; d.y0 = r->y0; d.dx = r->dx; d.nx = r->nx; d.ny = r->ny;
    d.orig = r->d_orig;
    d.nrm = r->d_nrm;
    d.perm = r->d_perm;
    d.R = r->R;
    return d;
}

template <class T>
cudaError_t upload(const void* src, size_t n, int device_ptrs, T** dst, cudaStream_t st) {
    *dst = nullptr;
    if (n == 0) return cudaSuccess;
    cudaError_t e = sa::scratch_alloc(dst, sizeof(T) * n, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dst, src, sizeof(T) * n,
                           device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
}

// host copy of a caller buffer (host or device) for validation
template <class T>
sa_status host_copy(const T* src, size_t n, int device_ptrs, std::vector<T>* out) {
    out->resize(n);
    if (n == 0) return SA_OK;
    if (!device_ptrs) {
        memcpy(out->data(), src, sizeof(T) * n);
        return SA_OK;
    }
    cudaError_t e = cudaMemcpy(out->data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading caller buffer");
    return SA_OK;
}

}  // namespace

namespace sa {
sa_status report_error(sa_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace sa

extern "C" {

const char* sa_last_error(void) { return g_err; }

int32_t sa_version(void) { return (1 << 16) | 0; }

// ------------------------------------------------------------------------------ scene
sa_status sa_scene_from_mesh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                             const int32_t* tri_building, int32_t n_buildings,
                             int32_t device_ptrs, void* stream, sa_scene** out) {
    if (!out) return fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: out is NULL");
    *out = nullptr;
    if (nv < 0 || nt < 0) return fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: negative size");
    if (nt > (1ll << 30)) return fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: too many triangles");
    if ((nv > 0 && !verts) || (nt > 0 && !tris))
        return fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: NULL buffer");
    if (n_buildings < 0) return fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: n_buildings < 0");
    // The mesh is validated on the device while its BVH is built (non-finite vertices,
    // vertex indices and building ids out of range), and the bounds of the referenced
    // vertices come back with the checks.
    cudaStream_t st = as_stream(stream);
    sa_scene* sc = new (std::nothrow) sa_scene();
    if (!sc) return fail(SA_ERR_OOM, "sa_scene_from_mesh: host allocation");
    sc->T = nt;
    sc->n_buildings = n_buildings;
    // inputs to the device: device buffers are used in place, host buffers go through
    // stream-ordered staging (pinned host memory copies asynchronously)
    const float* dv = verts;
    const int *dt = tris, *db = tri_building;
    float* sv = nullptr;
    int *stt = nullptr, *sb = nullptr;
    cudaError_t e = cudaSuccess;
    if (!device_ptrs) {
        if (nv > 0) {
            e = sa::scratch_alloc(&sv, sizeof(float) * 3 * (size_t)nv, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sv, verts, sizeof(float) * 3 * (size_t)nv, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess && nt > 0) {
            e = sa::scratch_alloc(&stt, sizeof(int) * 3 * (size_t)nt, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(stt, tris, sizeof(int) * 3 * (size_t)nt, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess && nt > 0 && tri_building) {
            e = sa::scratch_alloc(&sb, sizeof(int) * (size_t)nt, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sb, tri_building, sizeof(int) * (size_t)nt, cudaMemcpyHostToDevice, st);
        }
        dv = sv;
        dt = stt;
        db = tri_building ? sb : nullptr;
    }
    sa::MeshCheck chk{};
    if (e == cudaSuccess) e = sa::build_lbvh(dv, nv, dt, nt, db, &sc->bvh, st, std::max(n_buildings, 1), &chk);
    // the failing triangle's indices, for the message (read before the staging is freed)
    int32_t bad[4] = {0, 0, 0, 0};
    if (e == cudaSuccess && chk.bad_vertex < 0 && chk.bad_tri >= 0) {
        const int32_t* src = device_ptrs ? dt : tris;
        const int32_t* srcb = device_ptrs ? db : tri_building;
        if (device_ptrs) {
            e = cudaMemcpy(bad, src + 3 * chk.bad_tri, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && srcb) e = cudaMemcpy(bad + 3, srcb + chk.bad_tri, sizeof(int32_t), cudaMemcpyDeviceToHost);
        } else {
            memcpy(bad, src + 3 * chk.bad_tri, sizeof(int32_t) * 3);
            if (srcb) bad[3] = srcb[chk.bad_tri];
        }
    }
    if (sv) cudaFreeAsync(sv, st);
    if (stt) cudaFreeAsync(stt, st);
    if (sb) cudaFreeAsync(sb, st);
    sa_status verdict = SA_OK;
    if (e != cudaSuccess) {
        verdict = cuda_fail(e, "sa_scene_from_mesh");
    } else if (chk.bad_vertex >= 0) {
        verdict = fail(SA_ERR_DEGENERATE, "sa_scene_from_mesh: non-finite vertex %lld", chk.bad_vertex);
    } else if (chk.bad_tri >= 0) {
        int q = 0;
        while (q < 3 && bad[q] >= 0 && bad[q] < nv) ++q;
        if (q < 3)
            verdict = fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: triangle %lld indexes vertex %d", chk.bad_tri, bad[q]);
        else
            verdict = fail(SA_ERR_INVALID_ARG, "sa_scene_from_mesh: building id %d of triangle %lld", bad[3], chk.bad_tri);
    }
    if (verdict != SA_OK) {
        if (sc->bvh.nodes) cudaFreeAsync(sc->bvh.nodes, st);
        if (sc->bvh.tris) cudaFreeAsync(sc->bvh.tris, st);
        delete sc;
        return verdict;
    }
    sc->min_z = chk.box[2];
    for (int q = 0; q < 6; ++q) sc->box[q] = chk.box[q];
    *out = sc;
    return SA_OK;
}

void sa_scene_destroy(sa_scene* scene) {
    if (!scene) return;
    cudaDeviceSynchronize();
    if (scene->bvh.nodes) cudaFree(scene->bvh.nodes);
    if (scene->bvh.tris) cudaFree(scene->bvh.tris);
    if (scene->d_fp_mem) cudaFree(scene->d_fp_mem);
    if (scene->d_heights) cudaFree(scene->d_heights);
    delete scene;
}

// Extrude the footprint set with the scene's current device heights and rebuild the BVH.
static cudaError_t rebuild_from_footprints(sa_scene* sc, cudaStream_t st) {
    const sa::FootprintSet& fs = sc->fs;
    float* dv = nullptr;
    int *dt = nullptr, *db = nullptr;
    cudaError_t e = cudaSuccess;
    if (fs.n_tris > 0) {
        e = sa::scratch_alloc(&dv, sizeof(float) * 3 * (size_t)fs.n_verts, st);
        if (e == cudaSuccess) e = sa::scratch_alloc(&dt, sizeof(int) * 3 * (size_t)fs.n_tris, st);
        if (e == cudaSuccess) e = sa::scratch_alloc(&db, sizeof(int) * (size_t)fs.n_tris, st);
        if (e == cudaSuccess) e = sa::extrude_footprints(fs, sc->d_heights, dv, dt, db, st);
    }
    sa::LbvhBuild nb{};
    if (e == cudaSuccess) e = sa::build_lbvh(dv, fs.n_verts, dt, fs.n_tris, db, &nb, st);
    if (dv) cudaFreeAsync(dv, st);
    if (dt) cudaFreeAsync(dt, st);
    if (db) cudaFreeAsync(db, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (sc->bvh.nodes) cudaFree(sc->bvh.nodes);
    if (sc->bvh.tris) cudaFree(sc->bvh.tris);
    sc->bvh = nb;
    sc->T = fs.n_tris;
    return cudaSuccess;
}

static sa_status check_heights(const std::vector<float>& h, const char* who) {
    for (size_t b = 0; b < h.size(); ++b)
        if (!isfinite(h[b]) || !(h[b] > 0.f))
            return fail(SA_ERR_INVALID_ARG, "%s: height of building %zu must be finite and > 0", who, b);
    return SA_OK;
}

sa_status sa_scene_from_footprints(const float* xy, const int32_t* poly_off, int32_t n_buildings,
                                   const float* heights, float band_height, int32_t device_ptrs,
                                   void* stream, sa_scene** out) {
    const char* who = "sa_scene_from_footprints";
    if (!out) return fail(SA_ERR_INVALID_ARG, "%s: out is NULL", who);
    *out = nullptr;
    if (n_buildings < 0 || (n_buildings > 0 && (!xy || !poly_off || !heights)))
        return fail(SA_ERR_INVALID_ARG, "%s: bad sizes or NULL pointers", who);
    if (!isfinite(band_height) || band_height < 0.f) return fail(SA_ERR_INVALID_ARG, "%s: band_height", who);
    std::vector<int32_t> off;
    sa_status s = host_copy(poly_off, (size_t)n_buildings + 1, device_ptrs, &off);
    if (s != SA_OK) return s;
    if (off[0] != 0) return fail(SA_ERR_INVALID_ARG, "%s: poly_off[0] must be 0", who);
    for (int b = 0; b < n_buildings; ++b)
        if (off[b + 1] - off[b] < 3)
            return fail(SA_ERR_INVALID_ARG, "%s: building %d has fewer than 3 vertices", who, b);
    const int nv = off[n_buildings];
    std::vector<float> hxy, hh;
    s = host_copy(xy, (size_t)nv * 2, device_ptrs, &hxy);
    if (s == SA_OK) s = host_copy(heights, (size_t)n_buildings, device_ptrs, &hh);
    if (s != SA_OK) return s;
    s = check_heights(hh, who);
    if (s != SA_OK) return s;
    for (size_t i = 0; i < hxy.size(); ++i)
        if (!isfinite(hxy[i])) return fail(SA_ERR_DEGENERATE, "%s: non-finite footprint vertex", who);
    // convex, counter-clockwise footprints
    for (int b = 0; b < n_buildings; ++b) {
        const int a = off[b], v = off[b + 1] - a;
        double area = 0.0;
        for (int i = 0; i < v; ++i) {
            const int i1 = a + (i + 1) % v, i2 = a + (i + 2) % v;
            const double e1x = (double)hxy[2 * i1] - hxy[2 * (a + i)], e1y = (double)hxy[2 * i1 + 1] - hxy[2 * (a + i) + 1];
            const double e2x = (double)hxy[2 * i2] - hxy[2 * i1], e2y = (double)hxy[2 * i2 + 1] - hxy[2 * i1 + 1];
            if (e1x * e2y - e1y * e2x < 0.0)
                return fail(SA_ERR_INVALID_ARG, "%s: footprint %d is not convex and counter-clockwise", who, b);
            area += (double)hxy[2 * (a + i)] * hxy[2 * i1 + 1] - (double)hxy[2 * i1] * hxy[2 * (a + i) + 1];
        }
        if (!(area > 0.0)) return fail(SA_ERR_INVALID_ARG, "%s: footprint %d has no positive area", who, b);
    }
    std::vector<int32_t> bands(n_buildings), voff(n_buildings + 1, 0), toff(n_buildings + 1, 0);
    for (int b = 0; b < n_buildings; ++b) {
        const int v = off[b + 1] - off[b];
        int nb = 1;
        if (band_height > 0.f) nb = std::max(1, (int)ceil((double)hh[b] / (double)band_height));
        bands[b] = nb;
        voff[b + 1] = voff[b] + (nb + 1) * v;
        toff[b + 1] = toff[b] + 2 * v * nb + 2 * (v - 2);
    }
    sa_scene* sc = new (std::nothrow) sa_scene();
    if (!sc) return fail(SA_ERR_OOM, "%s: host allocation", who);
    sc->n_buildings = n_buildings;
    sc->min_z = 0.f;
    sc->has_footprints = 1;
    for (int q = 0; q < 3; ++q) { sc->box[q] = INFINITY; sc->box[3 + q] = -INFINITY; }
    for (int i = 0; i < nv; ++i)
        for (int q = 0; q < 2; ++q) {
            sc->box[q] = std::min(sc->box[q], hxy[2 * i + q]);
            sc->box[3 + q] = std::max(sc->box[3 + q], hxy[2 * i + q]);
        }
    sc->box[2] = 0.f;
    sc->box[5] = 0.f;
    for (int b = 0; b < n_buildings; ++b) sc->box[5] = std::max(sc->box[5], hh[b]);
    if (n_buildings == 0) for (int q = 0; q < 6; ++q) sc->box[q] = 0.f;
    sc->closed = 1;
    cudaStream_t st = as_stream(stream);
    // one device block: xy (float2) | fp_off | bands | vert_off | tri_off
    const size_t b_xy = sizeof(float) * 2 * (size_t)std::max(nv, 1);
    const size_t b_i = sizeof(int) * (size_t)(n_buildings + 1);
    cudaError_t e = sa::scratch_alloc_bytes(&sc->d_fp_mem, b_xy + 4 * b_i, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&sc->d_heights, sizeof(float) * (size_t)std::max(n_buildings, 1), st);
    if (e == cudaSuccess) {
        char* base = static_cast<char*>(sc->d_fp_mem);
        float2* dxy = reinterpret_cast<float2*>(base);
        int* doff = reinterpret_cast<int*>(base + b_xy);
        int* dband = doff + (n_buildings + 1);
        int* dvoff = dband + (n_buildings + 1);
        int* dtoff = dvoff + (n_buildings + 1);
        if (nv > 0) e = cudaMemcpyAsync(dxy, hxy.data(), sizeof(float) * 2 * nv, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(doff, off.data(), b_i, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && n_buildings > 0)
            e = cudaMemcpyAsync(dband, bands.data(), sizeof(int) * n_buildings, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dvoff, voff.data(), b_i, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dtoff, toff.data(), b_i, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && n_buildings > 0)
            e = cudaMemcpyAsync(sc->d_heights, hh.data(), sizeof(float) * n_buildings, cudaMemcpyHostToDevice, st);
        sc->fs.B = n_buildings;
        sc->fs.xy = dxy;
        sc->fs.fp_off = doff;
        sc->fs.bands = dband;
        sc->fs.vert_off = dvoff;
        sc->fs.tri_off = dtoff;
        sc->fs.n_verts = voff[n_buildings];
        sc->fs.n_tris = toff[n_buildings];
    }
    if (e == cudaSuccess) e = rebuild_from_footprints(sc, st);
    if (e != cudaSuccess) {
        sa_scene_destroy(sc);
        return cuda_fail(e, who);
    }
    *out = sc;
    return SA_OK;
}

sa_status sa_scene_set_heights(sa_scene* scene, const float* heights, int32_t device_ptrs,
                               void* stream) {
    const char* who = "sa_scene_set_heights";
    if (!scene || !heights) return fail(SA_ERR_INVALID_ARG, "%s: NULL argument", who);
    if (!scene->has_footprints) return fail(SA_ERR_UNSUPPORTED, "%s: scene was not built from footprints", who);
    std::vector<float> hh;
    sa_status s = host_copy(heights, (size_t)scene->n_buildings, device_ptrs, &hh);
    if (s != SA_OK) return s;
    s = check_heights(hh, who);
    if (s != SA_OK) return s;
    scene->box[5] = 0.f;
    for (float h : hh) scene->box[5] = std::max(scene->box[5], h);
    cudaStream_t st = as_stream(stream);
    cudaError_t e = scene->n_buildings > 0
        ? cudaMemcpyAsync(scene->d_heights, hh.data(), sizeof(float) * scene->n_buildings, cudaMemcpyHostToDevice, st)
        : cudaSuccess;
    if (e == cudaSuccess) e = rebuild_from_footprints(scene, st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return SA_OK;
}

sa_status sa_set_option(int32_t key, int32_t value) {
    switch (key) {
        case SA_OPT_SWEEP_TRAVERSAL:
        case SA_OPT_ACCRUAL_TRAVERSAL:
            if (value < 0 || value > 2) return fail(SA_ERR_INVALID_ARG, "sa_set_option: traversal mode %d", value);
            sa::set_trace_mode(key == SA_OPT_SWEEP_TRAVERSAL ? 0 : 1, value);
            return SA_OK;
        case SA_OPT_RASTER_RUN:
            if (value < 1 || value > 32) return fail(SA_ERR_INVALID_ARG, "sa_set_option: raster run %d", value);
            sa::set_raster_run(value);
            return SA_OK;
        case SA_OPT_POINT_RUN:
            if (value < 1 || value > 32) return fail(SA_ERR_INVALID_ARG, "sa_set_option: point run %d", value);
            sa::set_point_run(value);
            return SA_OK;
        case SA_OPT_KERNEL_TIMING:
            if (value < 0 || value > 1) return fail(SA_ERR_INVALID_ARG, "sa_set_option: kernel timing %d", value);
            sa::set_kernel_timing(value);
            return SA_OK;
        case SA_OPT_BATCH_TILE_SKIP:
            if (value < 0 || value > 1) return fail(SA_ERR_INVALID_ARG, "sa_set_option: batch tile skip %d", value);
            sa::set_batch_tile_skip(value);
            return SA_OK;
        default:
            return fail(SA_ERR_INVALID_ARG, "sa_set_option: unknown key %d", key);
    }
}

int32_t sa_get_option(int32_t key) {
    if (key == SA_OPT_SWEEP_TRAVERSAL) return sa::get_trace_mode(0);
    if (key == SA_OPT_ACCRUAL_TRAVERSAL) return sa::get_trace_mode(1);
    if (key == SA_OPT_RASTER_RUN) return sa::get_raster_run();
    if (key == SA_OPT_KERNEL_TIMING) return sa::get_kernel_timing();
    if (key == SA_OPT_POINT_RUN) return sa::get_point_run();
    if (key == SA_OPT_BATCH_TILE_SKIP) return sa::get_batch_tile_skip();
    return -1;
}

sa_status sa_kernel_times(double* ms, int64_t* launches, int32_t n) {
    if (n < 0) return fail(SA_ERR_INVALID_ARG, "sa_kernel_times: n = %d", n);
    std::vector<long long> cnt((size_t)n, 0);
    cudaError_t e = sa::collect_kernel_times(ms, cnt.data(), n);
    if (launches)
        for (int i = 0; i < n; ++i) launches[i] += (int64_t)cnt[i];
    if (e != cudaSuccess) return cuda_fail(e, "sa_kernel_times");
    return SA_OK;
}

sa_status sa_scene_declare_closed(sa_scene* scene, int32_t closed) {
    if (!scene) return fail(SA_ERR_INVALID_ARG, "sa_scene_declare_closed: NULL scene");
    scene->closed = closed ? 1 : 0;
    return SA_OK;
}

sa_status sa_scene_info(const sa_scene* scene, int64_t* n_tris, int64_t* n_nodes,
                        int32_t* n_buildings, float* min_z) {
    if (!scene) return fail(SA_ERR_INVALID_ARG, "sa_scene_info: NULL scene");
    if (n_tris) *n_tris = scene->T;
    if (n_nodes) *n_nodes = scene->bvh.n_nodes;
    if (n_buildings) *n_buildings = scene->n_buildings;
    if (min_z) *min_z = scene->min_z;
    return SA_OK;
}

// -------------------------------------------------------------------------------- sun
}  // extern "C"

namespace {

// Checks of a sun table shared by sa_sun_create and sa_sun_interpolate; *block_len 0
// becomes 60.
sa_status check_sun_table(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                          int32_t* block_len, const char* who) {
    if (S < 0 || D < 0 || (S > 0 && !dirs) || !day_start)
        return fail(SA_ERR_INVALID_ARG, "%s: bad sizes or NULL pointers", who);
    if (*block_len == 0) *block_len = 60;
    if (*block_len < 1 || *block_len > sa::kMaxBlock)
        return fail(SA_ERR_INVALID_ARG, "%s: block_len %d outside 1..64", who, *block_len);
    if (day_start[0] != 0 || day_start[D] != S)
        return fail(SA_ERR_INVALID_ARG, "%s: day_start must run from 0 to S", who);
    for (int k = 0; k < D; ++k)
        if (day_start[k + 1] < day_start[k])
            return fail(SA_ERR_INVALID_ARG, "%s: day_start decreases at day %d", who, k);
    for (int j = 0; j < S; ++j) {
        const float* d = dirs + 3 * j;
        if (!isfinite(d[0]) || !isfinite(d[1]) || !isfinite(d[2]))
            return fail(SA_ERR_INVALID_ARG, "%s: non-finite direction at step %d", who, j);
        const double n = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
        if (fabs(n - 1.0) > 1e-5)
            return fail(SA_ERR_INVALID_ARG, "%s: |d| = %.8f at step %d", who, n, j);
        if (!(d[2] > 0.f))
            return fail(SA_ERR_SUN_BELOW_HORIZON, "%s: d_z <= 0 at step %d", who, j);
    }
    return SA_OK;
}

// Calls fn(first step, steps, block of the day) for every block: each day of n steps is
// cut into ceil(n / block_len) consecutive blocks whose sizes differ by at most one, the
// longer ones first.
template <class Fn>
void for_each_block(const int32_t* day_start, int32_t D, int32_t block_len, Fn fn) {
    for (int k = 0; k < D; ++k) {
        const int a = day_start[k], n = day_start[k + 1] - a;
        if (n == 0) continue;
        const int nb = (n + block_len - 1) / block_len;
        const int base = n / nb, rem = n % nb;
        int j = a;
        for (int q = 0; q < nb; ++q) {
            const int K = base + (q < rem ? 1 : 0);
            fn(j, K, q);
            j += K;
        }
    }
}

}  // namespace

extern "C" {

sa_status sa_sun_create(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                        int32_t block_len, void* stream, sa_sun** out) {
    if (!out) return fail(SA_ERR_INVALID_ARG, "sa_sun_create: out is NULL");
    *out = nullptr;
    const sa_status chk = check_sun_table(dirs, S, day_start, D, &block_len, "sa_sun_create");
    if (chk != SA_OK) return chk;
    sa_sun* sun = new (std::nothrow) sa_sun();
    if (!sun) return fail(SA_ERR_OOM, "sa_sun_create: host allocation");
    sun->S = S;
    sun->D = D;
    sun->h_steps.resize(S);
    for (int j = 0; j < S; ++j) make_step(dirs + 3 * j, &sun->h_steps[j]);
    for_each_block(day_start, D, block_len, [&](int j, int K, int q) {
        const int mb = (int)sun->h_blocks.size();
        sun->h_blocks.push_back(make_block(dirs, sun->h_steps, j, K, q == 0, true));
        sun->h_blocks.back().mask_block = mb;
        for (int i = 0; i < K; ++i) {
            sun->h_step_blocks.push_back(make_block(dirs, sun->h_steps, j + i, 1, q == 0 && i == 0, false));
            sun->h_step_blocks.back().mask_block = mb;
            sun->h_step_blocks.back().mask_bit = i;
        }
    });
    cudaStream_t st = as_stream(stream);
    cudaError_t e = upload(sun->h_steps.data(), sun->h_steps.size(), 0, &sun->d_steps, st);
    if (e == cudaSuccess) e = upload(sun->h_blocks.data(), sun->h_blocks.size(), 0, &sun->d_blocks, st);
    if (e == cudaSuccess)
        e = upload(sun->h_step_blocks.data(), sun->h_step_blocks.size(), 0, &sun->d_step_blocks, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        sa_sun_destroy(sun);
        return cuda_fail(e, "sa_sun_create");
    }
    *out = sun;
    return SA_OK;
}

sa_status sa_sun_interpolate(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                             int32_t block_len, float* dirs_out) {
    const sa_status chk = check_sun_table(dirs, S, day_start, D, &block_len, "sa_sun_interpolate");
    if (chk != SA_OK) return chk;
    if (S > 0 && !dirs_out) return fail(SA_ERR_INVALID_ARG, "sa_sun_interpolate: dirs_out is NULL");
    // a copy, so that dirs_out may alias dirs
    std::vector<double> d((size_t)S * 3);
    for (size_t i = 0; i < d.size(); ++i) d[i] = (double)dirs[i];
    for (size_t i = 0; i < d.size(); ++i) dirs_out[i] = (float)d[i];
    for_each_block(day_start, D, block_len, [&](int a, int n, int) {
        if (n <= 2) return;
        double d1[3], dn[3];
        const double l1 = sqrt(d[3 * a] * d[3 * a] + d[3 * a + 1] * d[3 * a + 1] + d[3 * a + 2] * d[3 * a + 2]);
        const size_t e = 3 * (size_t)(a + n - 1);
        const double ln = sqrt(d[e] * d[e] + d[e + 1] * d[e + 1] + d[e + 2] * d[e + 2]);
        for (int c = 0; c < 3; ++c) {
            d1[c] = d[3 * (size_t)a + c] / l1;
            dn[c] = d[e + c] / ln;
        }
        const double cx = d1[1] * dn[2] - d1[2] * dn[1], cy = d1[2] * dn[0] - d1[0] * dn[2],
                     cz = d1[0] * dn[1] - d1[1] * dn[0];
        const double theta = atan2(sqrt(cx * cx + cy * cy + cz * cz), d1[0] * dn[0] + d1[1] * dn[1] + d1[2] * dn[2]);
        for (int i = 1; i < n - 1; ++i) {
            double w1 = 1.0, wn = 0.0;
            if (theta >= 1e-12) {
                const double tau = (double)i / (double)(n - 1);
                w1 = sin((1.0 - tau) * theta) / sin(theta);
                wn = sin(tau * theta) / sin(theta);
            }
            for (int c = 0; c < 3; ++c) dirs_out[3 * (size_t)(a + i) + c] = (float)(w1 * d1[c] + wn * dn[c]);
        }
    });
    return SA_OK;
}

sa_status sa_direction_graph(const float* dirs, int32_t S, const int32_t* day_start, int32_t D,
                             int32_t block_len, float bin_deg, int32_t* n_blocks, int32_t* n_edges,
                             int32_t* edge_of_block, int32_t* map_block, int32_t* weight) {
    const char* who = "sa_direction_graph";
    if (!n_blocks || !n_edges) return fail(SA_ERR_INVALID_ARG, "%s: NULL count", who);
    if (!(bin_deg > 0.f && bin_deg <= 90.f)) return fail(SA_ERR_INVALID_ARG, "%s: bin_deg outside (0, 90]", who);
    const sa_status chk = check_sun_table(dirs, S, day_start, D, &block_len, who);
    if (chk != SA_OK) return chk;
    std::vector<int> j0, K, edge, rep, wt;
    for_each_block(day_start, D, block_len, [&](int j, int k, int) {
        j0.push_back(j);
        K.push_back(k);
    });
    sa::direction_graph(dirs, (int)j0.size(), j0.data(), K.data(), (double)bin_deg, edge, rep, wt);
    *n_blocks = (int32_t)j0.size();
    *n_edges = (int32_t)rep.size();
    for (size_t b = 0; edge_of_block && b < edge.size(); ++b) edge_of_block[b] = edge[b];
    for (size_t e = 0; map_block && e < rep.size(); ++e) map_block[e] = rep[e];
    for (size_t e = 0; weight && e < wt.size(); ++e) weight[e] = wt[e];
    return SA_OK;
}

sa_status sa_block_partition(const int32_t* day_start, int32_t D, int32_t block_len,
                             int32_t* n_blocks, int32_t* j0, int32_t* K) {
    const char* who = "sa_block_partition";
    if (!day_start || !n_blocks || D < 0) return fail(SA_ERR_INVALID_ARG, "%s: NULL argument or D < 0", who);
    if (block_len == 0) block_len = 60;
    if (block_len < 1 || block_len > sa::kMaxBlock)
        return fail(SA_ERR_INVALID_ARG, "%s: block_len %d outside 1..64", who, block_len);
    if (day_start[0] != 0) return fail(SA_ERR_INVALID_ARG, "%s: day_start must start at 0", who);
    for (int k = 0; k < D; ++k)
        if (day_start[k + 1] < day_start[k])
            return fail(SA_ERR_INVALID_ARG, "%s: day_start decreases at day %d", who, k);
    int32_t nb = 0;
    for_each_block(day_start, D, block_len, [&](int j, int k, int) {
        if (j0) j0[nb] = j;
        if (K) K[nb] = k;
        ++nb;
    });
    *n_blocks = nb;
    return SA_OK;
}

void sa_sun_destroy(sa_sun* sun) {
    if (!sun) return;
    cudaDeviceSynchronize();
    if (sun->d_steps) cudaFree(sun->d_steps);
    if (sun->d_blocks) cudaFree(sun->d_blocks);
    if (sun->d_step_blocks) cudaFree(sun->d_step_blocks);
    delete sun;
}

sa_status sa_sun_info(const sa_sun* sun, int32_t* S, int32_t* D, int32_t* n_blocks) {
    if (!sun) return fail(SA_ERR_INVALID_ARG, "sa_sun_info: NULL sun");
    if (S) *S = sun->S;
    if (D) *D = sun->D;
    if (n_blocks) *n_blocks = (int32_t)sun->h_blocks.size();
    return SA_OK;
}

// -------------------------------------------------------------------------- receivers
sa_status sa_receivers_grid(float x0, float y0, float dx, int32_t nx, int32_t ny,
                            sa_receivers** out) {
    if (!out) return fail(SA_ERR_INVALID_ARG, "sa_receivers_grid: out is NULL");
    *out = nullptr;
    if (!(dx > 0.f) || !isfinite(dx) || !isfinite(x0) || !isfinite(y0))
        return fail(SA_ERR_INVALID_ARG, "sa_receivers_grid: bad origin or spacing");
    if (nx < 0 || ny < 0 || nx > (1 << 24) || ny > (1 << 24))
        return fail(SA_ERR_INVALID_ARG, "sa_receivers_grid: bad grid size");
    sa_receivers* r = new (std::nothrow) sa_receivers();
    if (!r) return fail(SA_ERR_OOM, "sa_receivers_grid: host allocation");
    r->is_grid = 1;
    r->x0 = x0; r->y0 = y0; r->dx = dx; r->nx = nx; r->ny = ny;
    r->R = (long long)nx * ny;
    *out = r;
    return SA_OK;
}

sa_status sa_receivers_points(const float* pos, const float* normal, int64_t n,
                              int32_t device_ptrs, void* stream, sa_receivers** out) {
    if (!out) return fail(SA_ERR_INVALID_ARG, "sa_receivers_points: out is NULL");
    *out = nullptr;
    if (n < 0 || n > (1ll << 31) - 1) return fail(SA_ERR_INVALID_ARG, "sa_receivers_points: bad count");
    if (n > 0 && !pos) return fail(SA_ERR_INVALID_ARG, "sa_receivers_points: NULL positions");
    sa_receivers* r = new (std::nothrow) sa_receivers();
    if (!r) return fail(SA_ERR_OOM, "sa_receivers_points: host allocation");
    r->is_grid = 0;
    r->R = n;
    cudaStream_t st = as_stream(stream);
    // host inputs are copied to stream-ordered staging; device inputs are read in place.
    // Validation (finite values) and the bounds run on the device, in the sort's pass.
    const float *dp = pos, *dn = normal;
    float *sp = nullptr, *sn = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t bytes = sizeof(float) * 3 * (size_t)n;
    if (n > 0 && !device_ptrs) {
        e = sa::scratch_alloc(&sp, bytes, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sp, pos, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && normal) e = sa::scratch_alloc(&sn, bytes, st);
        if (e == cudaSuccess && normal) e = cudaMemcpyAsync(sn, normal, bytes, cudaMemcpyHostToDevice, st);
        dp = sp;
        dn = normal ? sn : nullptr;
    }
    if (e == cudaSuccess && n > 0) e = sa::scratch_alloc(&r->d_orig, sizeof(float4) * (size_t)n, st);
    if (e == cudaSuccess && n > 0) e = sa::scratch_alloc(&r->d_perm, sizeof(int) * (size_t)n, st);
    if (e == cudaSuccess && n > 0 && normal) e = sa::scratch_alloc(&r->d_nrm, sizeof(float4) * (size_t)n, st);
    long long bad[2] = {-1, -1};
    if (e == cudaSuccess)
        e = sa::sort_points(dp, dn, n, r->d_orig, r->d_nrm, r->d_perm, st, bad, r->box);
    if (sp) cudaFreeAsync(sp, st);
    if (sn) cudaFreeAsync(sn, st);
    if (e != cudaSuccess) {
        sa_receivers_destroy(r);
        return cuda_fail(e, "sa_receivers_points");
    }
    if (bad[0] >= 0 || bad[1] >= 0) {
        sa_receivers_destroy(r);
        return bad[0] >= 0
            ? fail(SA_ERR_DEGENERATE, "sa_receivers_points: non-finite position %lld", bad[0])
            : fail(SA_ERR_DEGENERATE, "sa_receivers_points: non-finite normal %lld", bad[1]);
    }
    *out = r;
    return SA_OK;
}

void sa_receivers_destroy(sa_receivers* recv) {
    if (!recv) return;
    cudaDeviceSynchronize();
    if (recv->d_orig) cudaFree(recv->d_orig);
    if (recv->d_perm) cudaFree(recv->d_perm);
    if (recv->d_nrm) cudaFree(recv->d_nrm);
    delete recv;
}

int64_t sa_receivers_count(const sa_receivers* recv) { return recv ? recv->R : -1; }

// ------------------------------------------------------------------------- accumulate
static sa_status run_method(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                            sa_method method, int32_t iam_levels, sa::DevOut out,
                            cudaStream_t st, const char* who) {
    if (!scene || !recv || !sun) return fail(SA_ERR_INVALID_ARG, "%s: NULL handle", who);
    if (iam_levels < 0 || iam_levels > 8) return fail(SA_ERR_INVALID_ARG, "%s: iam_levels", who);
    const bool raster = method == SA_SWEEP_RASTER || (method == SA_ACCRUAL_SAM && recv->is_grid);
    if ((method == SA_SWEEP_RASTER || method == SA_IAM) && !recv->is_grid)
        return fail(SA_ERR_UNSUPPORTED, "%s: method %d needs a ground grid", who, (int)method);
    if (raster && scene->min_z < 0.f)
        return fail(SA_ERR_UNSUPPORTED, "%s: raster methods need geometry at z >= 0", who);
    if (method < SA_SWEEP_TRACE || method > SA_IAM)
        return fail(SA_ERR_INVALID_ARG, "%s: unknown method %d", who, (int)method);
    sa::DevScene dsc = dev_scene(scene);
    sa::DevRecv drc = dev_recv(recv);
    sa::DevSun dsun;
    dsun.steps = sun->d_steps;
    dsun.S = sun->S;
    if (method == SA_SWEEP_RASTER) {
        dsun.blocks = sun->d_step_blocks;
        dsun.n_blocks = (int)sun->h_step_blocks.size();
    } else {
        dsun.blocks = sun->d_blocks;
        dsun.n_blocks = (int)sun->h_blocks.size();
    }
    const long long R = recv->R;
    if (R == 0) return SA_OK;
    cudaError_t e = cudaSuccess;
    if (dsun.n_blocks == 0) {
        // no steps: counts are zero (or unchanged when accumulating)
        if (!out.accumulate_into) {
            e = cudaMemsetAsync(out.gross, 0, sizeof(int) * (size_t)R, st);
            if (e == cudaSuccess && out.continuous) e = cudaMemsetAsync(out.continuous, 0, sizeof(int) * (size_t)R, st);
            if (e == cudaSuccess && out.minutes) e = cudaMemsetAsync(out.minutes, 0, sizeof(float) * (size_t)R, st);
        }
        return e == cudaSuccess ? SA_OK : cuda_fail(e, who);
    }
    int* run = nullptr;
    if (method == SA_IAM) {
        e = sa::scratch_alloc(&run, sizeof(int) * (size_t)R, st);
        if (e != cudaSuccess) return cuda_fail(e, who);
        out.run = run;
        e = sa::launch_iam(dsc, drc, dsun, sun->h_blocks.data(), iam_levels ? iam_levels : 3, out, st);
    } else if (raster) {
        e = sa::scratch_alloc(&run, sizeof(int) * (size_t)R, st);
        if (e != cudaSuccess) return cuda_fail(e, who);
        out.run = run;
        e = sa::launch_raster_ground(dsc, drc, dsun, out, st);
    } else if (method == SA_SWEEP_TRACE) {
        e = sa::launch_sweep_trace(dsc, drc, dsun, out, st);
    } else if (method == SA_ACCRUAL_SAM) {
        e = sa::launch_sam_points(dsc, scene->box, drc, recv->box, dsun, sun->h_blocks, sun->h_steps,
                                  out, st);
    } else {
        e = sa::launch_accrual_trace(dsc, drc, dsun, out, st);
    }
    if (run) cudaFreeAsync(run, st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return sa::check_after_call(st, who);
}

sa_status sa_accumulate(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                        float step_minutes, sa_method method, int32_t iam_levels,
                        int32_t flags, int32_t* gross_steps, float* gross_minutes,
                        int32_t* continuous_steps, void* stream) {
    if (!gross_steps && recv && recv->R > 0)
        return fail(SA_ERR_INVALID_ARG, "sa_accumulate: gross_steps is NULL");
    if (!isfinite(step_minutes) || step_minutes < 0.f)
        return fail(SA_ERR_INVALID_ARG, "sa_accumulate: bad step_minutes");
    if (flags & ~SA_ACCUMULATE_INTO) return fail(SA_ERR_INVALID_ARG, "sa_accumulate: unknown flags");
    sa::DevOut out;
    memset(&out, 0, sizeof(out));
    out.gross = gross_steps;
    out.minutes = gross_minutes;
    out.continuous = continuous_steps;
    out.step_minutes = step_minutes;
    out.accumulate_into = (flags & SA_ACCUMULATE_INTO) ? 1 : 0;
    out.write_final = 1;
    return run_method(scene, recv, sun, method, iam_levels, out, as_stream(stream), "sa_accumulate");
}

sa_status sa_shadow_masks(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                          sa_method method, int32_t iam_levels, uint64_t* masks, void* stream) {
    if (!masks && recv && recv->R > 0) return fail(SA_ERR_INVALID_ARG, "sa_shadow_masks: NULL masks");
    if (!recv) return fail(SA_ERR_INVALID_ARG, "sa_shadow_masks: NULL receivers");
    cudaStream_t st = as_stream(stream);
    int* gross = nullptr;
    if (recv->R > 0) {
        cudaError_t e = sa::scratch_alloc(&gross, sizeof(int) * (size_t)recv->R, st);
        if (e != cudaSuccess) return cuda_fail(e, "sa_shadow_masks");
    }
    if (recv->R > 0 && sun) {
        cudaError_t e = cudaMemsetAsync(masks, 0, sizeof(uint64_t) * (size_t)recv->R * sun->h_blocks.size(), st);
        if (e != cudaSuccess) { cudaFreeAsync(gross, st); return cuda_fail(e, "sa_shadow_masks"); }
    }
    sa::DevOut out;
    memset(&out, 0, sizeof(out));
    out.gross = gross;
    out.masks = reinterpret_cast<uint64_t*>(masks);
    out.write_final = 1;
    sa_status s = run_method(scene, recv, sun, method, iam_levels, out, st, "sa_shadow_masks");
    if (gross) cudaFreeAsync(gross, st);
    return s;
}

sa_status sa_accumulate_graph(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                              sa_method method, int32_t iam_levels, float bin_deg, float step_minutes,
                              int32_t* gross_steps, float* gross_minutes, int32_t* continuous_steps,
                              int32_t* n_edges, void* stream) {
    const char* who = "sa_accumulate_graph";
    if (!scene || !recv || !sun) return fail(SA_ERR_INVALID_ARG, "%s: NULL handle", who);
    if (!(bin_deg > 0.f && bin_deg <= 90.f)) return fail(SA_ERR_INVALID_ARG, "%s: bin_deg outside (0, 90]", who);
    if (!isfinite(step_minutes) || step_minutes < 0.f) return fail(SA_ERR_INVALID_ARG, "%s: step_minutes", who);
    if (recv->R > 0 && !gross_steps) return fail(SA_ERR_INVALID_ARG, "%s: gross_steps is NULL", who);
    cudaStream_t st = as_stream(stream);
    // the graph over the sun table's own blocks
    const int nb = (int)sun->h_blocks.size();
    std::vector<float> dirs((size_t)sun->S * 3);
    for (int j = 0; j < sun->S; ++j) {
        dirs[3 * (size_t)j] = sun->h_steps[j].dx;
        dirs[3 * (size_t)j + 1] = sun->h_steps[j].dy;
        dirs[3 * (size_t)j + 2] = sun->h_steps[j].dz;
    }
    std::vector<int> j0(nb), K(nb), path, rep, wt;
    for (int b = 0; b < nb; ++b) {
        j0[b] = sun->h_blocks[b].j0;
        K[b] = sun->h_blocks[b].K;
    }
    sa::direction_graph(dirs.data(), nb, j0.data(), K.data(), (double)bin_deg, path, rep, wt);
    const int E = (int)rep.size();
    if (n_edges) *n_edges = E;
    if (E >= (1 << 20)) return fail(SA_ERR_INVALID_ARG, "%s: %d edges (at most 2^20 - 1)", who, E);
    // every block in time order: its edge, its steps and whether it starts a day
    std::vector<int> walk((size_t)nb);
    for (int b = 0; b < nb; ++b)
        walk[(size_t)b] = path[(size_t)b] | (K[(size_t)b] << 20) | ((sun->h_blocks[b].new_day ? 1 : 0) << 27);
    const long long R = recv->R;
    if (R == 0) return SA_OK;
    cudaError_t e = cudaSuccess;
    if (nb == 0) {
        e = cudaMemsetAsync(gross_steps, 0, sizeof(int) * (size_t)R, st);
        if (e == cudaSuccess && continuous_steps) e = cudaMemsetAsync(continuous_steps, 0, sizeof(int) * (size_t)R, st);
        if (e == cudaSuccess && gross_minutes) e = cudaMemsetAsync(gross_minutes, 0, sizeof(float) * (size_t)R, st);
        return e == cudaSuccess ? SA_OK : cuda_fail(e, who);
    }
    std::vector<int> edge_K((size_t)E);
    for (int q = 0; q < E; ++q) edge_K[(size_t)q] = K[(size_t)rep[(size_t)q]];
    unsigned* summary = nullptr;
    unsigned long long* masks = nullptr;
    int *d_walk = nullptr, *d_K = nullptr, *scratch = nullptr;
    // one chunk of edges' masks at a time, at most 4 GiB (the scratch pool keeps 4 GiB
    // across synchronisations; larger chunks are mapped again on every call), in multiples
    // of the raster's own 64-block chunks where it holds that many
    const long long per_edge = 8ll * R;
    long long fit = std::max(1ll, (4ll << 30) / per_edge);
    if (fit >= 64) fit -= fit % 64;
    const int chunk = (int)std::min((long long)E, fit);
    sa_status status = SA_OK;
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(sa::scratch_alloc(&summary, sizeof(unsigned) * (size_t)E * (size_t)R, st));
    TRY(sa::scratch_alloc(&masks, sizeof(unsigned long long) * (size_t)chunk * (size_t)R, st));
    TRY(sa::scratch_alloc(&scratch, sizeof(int) * (size_t)R, st));
    TRY(sa::scratch_alloc(&d_walk, sizeof(int) * (size_t)nb, st));
    TRY(sa::scratch_alloc(&d_K, sizeof(int) * (size_t)E, st));
    TRY(cudaMemcpyAsync(d_walk, walk.data(), sizeof(int) * (size_t)nb, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(d_K, edge_K.data(), sizeof(int) * (size_t)E, cudaMemcpyHostToDevice, st));
    for (int e0 = 0; e0 < E; e0 += chunk) {
        const int e1 = std::min(E, e0 + chunk);
        // a sun table holding the chunk's map blocks, one per edge, each its own day; it
        // borrows the steps of `sun`
        sa_sun gs;
        gs.S = sun->S;
        gs.D = e1 - e0;
        gs.h_steps = sun->h_steps;
        for (int q = e0; q < e1; ++q) {
            sa::BlockConst bc = sun->h_blocks[(size_t)rep[(size_t)q]];
            bc.mask_block = q - e0;
            bc.mask_bit = 0;
            bc.new_day = 1;
            gs.h_blocks.push_back(bc);
            for (int i = 0; i < bc.K; ++i) {
                sa::BlockConst sb = sun->h_step_blocks[(size_t)bc.j0 + i];
                sb.mask_block = q - e0;
                sb.mask_bit = i;
                sb.new_day = i == 0;
                gs.h_step_blocks.push_back(sb);
            }
        }
        gs.d_steps = sun->d_steps;
        e = upload(gs.h_blocks.data(), gs.h_blocks.size(), 0, &gs.d_blocks, st);
        if (e == cudaSuccess) e = upload(gs.h_step_blocks.data(), gs.h_step_blocks.size(), 0, &gs.d_step_blocks, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(masks, 0, sizeof(unsigned long long) * (size_t)(e1 - e0) * (size_t)R, st);
        if (e == cudaSuccess) {
            sa::DevOut out;
            memset(&out, 0, sizeof(out));
            out.gross = scratch;
            out.masks = reinterpret_cast<uint64_t*>(masks);
            out.write_final = 1;
            status = run_method(scene, recv, &gs, method, iam_levels, out, st, who);
        }
        if (e == cudaSuccess && status == SA_OK)
            e = sa::launch_edge_summary(masks, R, e1 - e0, d_K + e0, summary + (size_t)e0 * (size_t)R, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (gs.d_blocks) cudaFree(gs.d_blocks);
        if (gs.d_step_blocks) cudaFree(gs.d_step_blocks);
        gs.d_steps = nullptr;
        if (e != cudaSuccess || status != SA_OK) goto done;
    }
    TRY(sa::launch_graph_reduce(summary, R, d_walk, nb, step_minutes, gross_steps, gross_minutes,
                                continuous_steps, st));
done:
    for (void* p : {(void*)summary, (void*)masks, (void*)scratch, (void*)d_walk, (void*)d_K})
        if (p) cudaFreeAsync(p, st);
#undef TRY
    if (status != SA_OK) return status;
    if (e != cudaSuccess) return cuda_fail(e, who);
    return sa::check_after_call(st, who);
}

sa_status sa_height_grad(const sa_scene* scene, const sa_receivers* grid, const sa_sun* sun,
                         float step_minutes, const float* weights, float* dS_dh, double* S_out,
                         void* stream) {
    const char* who = "sa_height_grad";
    if (!scene || !grid || !sun) return fail(SA_ERR_INVALID_ARG, "%s: NULL handle", who);
    if (!scene->has_footprints) return fail(SA_ERR_UNSUPPORTED, "%s: scene was not built from footprints", who);
    if (!grid->is_grid) return fail(SA_ERR_UNSUPPORTED, "%s: receivers must be a ground grid", who);
    if (scene->n_buildings > 0 && !dS_dh) return fail(SA_ERR_INVALID_ARG, "%s: dS_dh is NULL", who);
    if (!isfinite(step_minutes) || step_minutes < 0.f) return fail(SA_ERR_INVALID_ARG, "%s: step_minutes", who);
    sa::DevSun dsun;
    dsun.steps = sun->d_steps;
    dsun.blocks = sun->d_blocks;
    dsun.S = sun->S;
    dsun.n_blocks = (int)sun->h_blocks.size();
    cudaError_t e = sa::launch_height_grad(dev_scene(scene), scene->fs, scene->d_heights, dev_recv(grid), dsun,
                                           step_minutes, weights, dS_dh, S_out, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return sa::check_after_call(as_stream(stream), who);
}

sa_status sa_building_contribution(const sa_scene* scene, const sa_receivers* grid,
                                   const sa_sun* sun, const float* poly_xy, int32_t n,
                                   void* stream, double* casting, double* nearest,
                                   int64_t* stats) {
    const char* who = "sa_building_contribution";
    if (!scene || !grid || !sun || !poly_xy) return fail(SA_ERR_INVALID_ARG, "%s: NULL argument", who);
    if (scene->n_buildings > 0 && (!casting || !nearest))
        return fail(SA_ERR_INVALID_ARG, "%s: NULL output", who);
    if (!grid->is_grid) return fail(SA_ERR_INVALID_ARG, "%s: receivers must be a ground grid", who);
    if (n < 3) return fail(SA_ERR_INVALID_ARG, "%s: a polygon needs 3 vertices", who);
    for (int i = 0; i < 2 * n; ++i)
        if (!isfinite(poly_xy[i])) return fail(SA_ERR_DEGENERATE, "%s: non-finite polygon vertex", who);
    if (scene->T > 0 && scene->min_z < 0.f)
        return fail(SA_ERR_UNSUPPORTED, "%s: scene geometry below z = 0", who);
    const double mask_bytes = 8.0 * (double)grid->R * (double)sun->h_blocks.size();
    if (mask_bytes > 4.0 * 1024.0 * 1024.0 * 1024.0)
        return fail(SA_ERR_INVALID_ARG, "%s: step masks of %.0f bytes exceed 4 GiB; split the interval", who,
                    mask_bytes);
    sa::DevSun dsun;
    dsun.steps = sun->d_steps;
    dsun.blocks = sun->d_blocks;
    dsun.S = sun->S;
    dsun.n_blocks = (int)sun->h_blocks.size();
    // runs of <= 32 steps of each block, each with its own fan, pointing into the block's mask
    std::vector<float> dirs(3 * (size_t)sun->S);
    for (int j = 0; j < sun->S; ++j) {
        dirs[3 * (size_t)j] = sun->h_steps[j].dx;
        dirs[3 * (size_t)j + 1] = sun->h_steps[j].dy;
        dirs[3 * (size_t)j + 2] = sun->h_steps[j].dz;
    }
    std::vector<sa::BlockConst> runs;
    for (const sa::BlockConst& b : sun->h_blocks) {
        const int nsub = (b.K + 31) / 32;
        for (int q = 0; q < nsub; ++q) {
            const int k0 = q * b.K / nsub, k1 = (q + 1) * b.K / nsub;
            sa::BlockConst r = make_block(dirs.data(), sun->h_steps, b.j0 + k0, k1 - k0, 0, true);
            r.mask_block = b.mask_block;
            r.mask_bit = b.mask_bit + k0;
            runs.push_back(r);
        }
    }
    unsigned long long h[2] = {0ull, 0ull};
    cudaError_t e = sa::launch_building_contribution(dev_scene(scene), dev_recv(grid), dsun, runs,
                                                     scene->n_buildings, poly_xy, n, casting, nearest, h,
                                                     as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    const sa_status chk = sa::check_after_call(as_stream(stream), who);
    if (chk != SA_OK) return chk;
    if (stats) {
        stats[0] = (int64_t)h[0];
        stats[1] = (int64_t)h[1];
    }
    if (h[0] > 0)
        return fail(SA_ERR_UNSUPPORTED, "%s: %llu cell-steps met more than 64 buildings along one ray; "
                    "their casting credit is incomplete", who, h[0]);
    return SA_OK;
}

sa_status sa_work_counters(const sa_scene* scene, const sa_receivers* recv, const sa_sun* sun,
                           sa_method method, uint64_t* counters, void* stream) {
    if (!counters) return fail(SA_ERR_INVALID_ARG, "sa_work_counters: NULL counters");
    if (!recv) return fail(SA_ERR_INVALID_ARG, "sa_work_counters: NULL receivers");
    cudaStream_t st = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(uint64_t) * 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "sa_work_counters");
    int* gross = nullptr;
    if (recv->R > 0) {
        e = sa::scratch_alloc(&gross, sizeof(int) * (size_t)recv->R, st);
        if (e != cudaSuccess) return cuda_fail(e, "sa_work_counters");
    }
    sa::DevOut out;
    memset(&out, 0, sizeof(out));
    out.gross = gross;
    out.write_final = 1;
    out.stats = reinterpret_cast<unsigned long long*>(counters);
    sa_status s = run_method(scene, recv, sun, method, 0, out, st, "sa_work_counters");
    if (gross) cudaFreeAsync(gross, st);
    return s;
}

}  // extern "C"
