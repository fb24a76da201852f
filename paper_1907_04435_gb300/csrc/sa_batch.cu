// sa_batch.cu -- batched development scenarios (impact of new towers, Sec. 7.1 / Sec. 9).
//
// The impact of a new building is the difference of the accumulation with and without it
// (Sec. 7.1).  A batch holds one base city, V variants (towers added, overlapped base
// buildings removed), a square receiver region per variant and several sun intervals.  At
// creation it bins the base city's triangles once per block of every interval (the bins
// do not depend on the variant), computes the base counts over the whole grid, and lists
// the work items (interval, variant, tile of the region).  sa_batch_run then executes a
// CUDA graph holding one persistent launch that drains the work queue: each item rasters
// its tile with the base bins minus the removed buildings plus the variant's towers.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sa_handles.cuh"

struct sa_batch {
    const sa_scene* base = nullptr;
    sa::DevRecv grid{};
    int V = 0, I = 0;
    long long cells_per_interval = 0;
    std::vector<long long> var_off;                 // per variant, within an interval
    std::vector<sa::BatchInterval> h_iv;
    std::vector<void*> owned;                       // device buffers to free
    sa::BatchInterval* d_iv = nullptr;
    sa::BatchVariant* d_var = nullptr;
    int4* d_items = nullptr;
    int n_items = 0;
    int n_affected = 0;
    unsigned* d_counter = nullptr;
    int* d_removed = nullptr;
    float4* d_towers = nullptr;
    int ctas = 0;
    int run = 8;
    int sms = 0;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* g_counts = nullptr;
    int* g_impact = nullptr;
};

namespace sa {
namespace {
// 1: tiles no changed building can shadow keep the base counts (default); 0: every tile
// of a region is rastered (to measure what the skipping saves)
int g_tile_skip = 1;
}  // namespace
void set_batch_tile_skip(int on) { g_tile_skip = on; }
int get_batch_tile_skip() { return g_tile_skip; }
int raster_ctas_per_sm();   // sa_raster.cu: the CTAs per SM its kernels are compiled for
}  // namespace sa

namespace {

inline int __float_as_int_host(float f) {
    int i;
    memcpy(&i, &f, sizeof(i));
    return i;
}

sa::BatchLaunch launch_of(const sa_batch* b, int* counts, int* impact, int n_items, int ctas,
                          int run, unsigned long long* stats) {
    sa::BatchLaunch bl;
    bl.base.nodes = b->base->bvh.nodes;
    bl.base.tris = b->base->bvh.tris;
    bl.base.n_nodes = b->base->bvh.n_nodes;
    bl.base.T = (int)b->base->T;
    bl.base.closed = b->base->closed;
    bl.grid = b->grid;
    bl.intervals = b->d_iv;
    bl.variants = b->d_var;
    bl.items = b->d_items;
    bl.n_items = n_items;
    bl.counter = b->d_counter;
    bl.removed = b->d_removed;
    bl.tower_tris = b->d_towers;
    bl.counts_out = counts;
    bl.impact_out = impact;
    bl.stats = stats;
    bl.ctas = ctas;
    bl.run = run;
    return bl;
}

void drop_graph(sa_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

template <class T>
cudaError_t dev_copy(sa_batch* b, const T* src, size_t n, T** dst) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc(dst, sizeof(T) * std::max<size_t>(n, 1));
    if (e != cudaSuccess) return e;
    b->owned.push_back(*dst);
    if (n == 0) return cudaSuccess;
    return cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

void sa_batch_destroy(sa_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->capture) cudaStreamDestroy(b->capture);
    for (void* p : b->owned) cudaFree(p);
    delete b;
}

sa_status sa_batch_create(const sa_scene* base, const sa_receivers* grid, const sa_variants* v,
                          const sa_sun* const* intervals, int32_t n_intervals,
                          int32_t with_impact, void* stream, sa_batch** out) {
    if (!out) return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: out is NULL");
    *out = nullptr;
    if (!base || !grid || !v || (n_intervals > 0 && !intervals) || n_intervals < 0)
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: NULL argument or bad count");
    if (!grid->is_grid) return sa::report_error(SA_ERR_UNSUPPORTED, "sa_batch_create: receivers must be a ground grid");
    if (base->min_z < 0.f) return sa::report_error(SA_ERR_UNSUPPORTED, "sa_batch_create: base geometry below z = 0");
    const int V = v->n_variants;
    if (V < 0 || (V > 0 && (!v->tower_off || !v->removed_off || !v->regions)))
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: bad variant description");
    for (int i = 0; i < n_intervals; ++i)
        if (!intervals[i]) return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: NULL interval");
    const int n_tow = V > 0 ? v->tower_off[V] : 0, n_rem = V > 0 ? v->removed_off[V] : 0;
    if (V > 0 && (v->tower_off[0] != 0 || v->removed_off[0] != 0 || n_tow < 0 || n_rem < 0 ||
                  (n_tow > 0 && !v->tower_tris) || (n_rem > 0 && !v->removed_ids)))
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: bad offsets");
    std::vector<sa::BatchVariant> hv(V);
    const int tiles_x = (grid->nx + 31) / 32, tiles_y = (grid->ny + 31) / 32;
    long long cells = 0;
    for (int k = 0; k < V; ++k) {
        const int* r = v->regions + 4 * k;
        if (v->tower_off[k + 1] < v->tower_off[k] || v->removed_off[k + 1] < v->removed_off[k])
            return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: offsets decrease");
        if (r[0] < 0 || r[1] < 0 || r[2] < 0 || r[3] < 0 || r[0] + r[2] > grid->nx || r[1] + r[3] > grid->ny)
            return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: region outside the grid");
        hv[k].tower_off = v->tower_off[k];
        hv[k].n_tower = v->tower_off[k + 1] - v->tower_off[k];
        hv[k].rem_off = v->removed_off[k];
        hv[k].n_rem = v->removed_off[k + 1] - v->removed_off[k];
        hv[k].ix0 = r[0]; hv[k].iy0 = r[1]; hv[k].nx = r[2]; hv[k].ny = r[3];
        hv[k].out_off = cells;
        cells += (long long)r[2] * r[3];
    }
    std::vector<float4> towers((size_t)n_tow * 3);
    for (int t = 0; t < n_tow; ++t)
        for (int q = 0; q < 3; ++q) {
            const float* f = v->tower_tris + 9 * (size_t)t + 3 * q;
            if (!isfinite(f[0]) || !isfinite(f[1]) || !isfinite(f[2]) || f[2] < 0.f)
                return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_create: tower vertex non-finite or below z = 0");
            towers[3 * (size_t)t + q] = make_float4(f[0], f[1], f[2], 0.f);
        }
    sa_batch* b = new (std::nothrow) sa_batch();
    if (!b) return sa::report_error(SA_ERR_OOM, "sa_batch_create: host allocation");
    b->base = base;
    b->grid.is_grid = 1;
    b->grid.x0 = grid->x0; b->grid.y0 = grid->y0; b->grid.dx = grid->dx;
    b->grid.nx = grid->nx; b->grid.ny = grid->ny;
    b->grid.orig = nullptr; b->grid.nrm = nullptr; b->grid.perm = nullptr;
    b->grid.R = grid->R;
    b->V = V;
    b->I = n_intervals;
    b->cells_per_interval = cells;
    for (int k = 0; k < V; ++k) b->var_off.push_back(hv[k].out_off);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->ctas = 4 * b->sms;
    b->run = sa::get_raster_run();
    if (e == cudaSuccess) e = dev_copy(b, hv.data(), hv.size(), &b->d_var);
    if (e == cudaSuccess) e = dev_copy(b, towers.data(), towers.size(), &b->d_towers);
    if (e == cudaSuccess) e = dev_copy(b, v->removed_ids, (size_t)n_rem, &b->d_removed);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned));
    if (e == cudaSuccess) b->owned.push_back(b->d_counter);
    // per interval: base bins and base counts
    sa::DevScene dsc;
    dsc.nodes = base->bvh.nodes; dsc.tris = base->bvh.tris; dsc.n_nodes = base->bvh.n_nodes;
    dsc.T = (int)base->T; dsc.closed = base->closed;
    for (int i = 0; i < n_intervals && e == cudaSuccess; ++i) {
        const sa_sun* sun = intervals[i];
        sa::DevSun ds;
        ds.steps = sun->d_steps; ds.blocks = sun->d_blocks; ds.S = sun->S;
        ds.n_blocks = (int)sun->h_blocks.size();
        sa::BatchInterval bi{};
        bi.steps = sun->d_steps;
        bi.blocks = sun->d_blocks;
        bi.n_blocks = ds.n_blocks;
        bi.out_base = (long long)i * cells;
        unsigned *off = nullptr, *cnt = nullptr;
        int* bins = nullptr;
        e = sa::build_bins(dsc, b->grid, ds, &off, &cnt, &bins, st);
        if (off) b->owned.push_back(off);
        if (cnt) b->owned.push_back(cnt);
        if (bins) b->owned.push_back(bins);
        bi.offsets = off; bi.counts = cnt; bi.bins = bins;
        bi.base_counts = nullptr;
        if (e == cudaSuccess && grid->R > 0) {
            int *bc = nullptr, *run = nullptr;
            e = cudaMalloc(&bc, sizeof(int) * (size_t)grid->R);
            if (e == cudaSuccess) b->owned.push_back(bc);
            if (e == cudaSuccess) e = sa::scratch_alloc(&run, sizeof(int) * (size_t)grid->R, st);
            if (e == cudaSuccess) {
                sa::DevOut o;
                memset(&o, 0, sizeof(o));
                o.gross = bc;
                o.run = run;
                e = sa::launch_raster_ground(dsc, b->grid, ds, o, st);
                cudaFreeAsync(run, st);
            }
            bi.base_counts = bc;
        }
        b->h_iv.push_back(bi);
    }
    if (e == cudaSuccess) e = dev_copy(b, b->h_iv.data(), b->h_iv.size(), &b->d_iv);
    // Boxes of what each variant changes: its removed base buildings and its towers.
    std::vector<std::vector<float>> changed(V);     // per variant: lo.xyz hi.xyz ...
    if (e == cudaSuccess && V > 0) {
        std::vector<float4> bt((size_t)base->T * 3);
        if (base->T > 0)
            e = cudaMemcpy(bt.data(), base->bvh.tris, sizeof(float4) * bt.size(), cudaMemcpyDeviceToHost);
        std::vector<float> bbox((size_t)std::max(base->n_buildings, 1) * 6);
        for (size_t q = 0; q < bbox.size(); q += 6) {
            bbox[q] = bbox[q + 1] = bbox[q + 2] = 3.4e38f;
            bbox[q + 3] = bbox[q + 4] = bbox[q + 5] = -3.4e38f;
        }
        for (long long t = 0; t < base->T; ++t) {
            const int bid = __float_as_int_host(bt[3 * t].w);
            if (bid < 0 || bid >= base->n_buildings) continue;
            float* bb = &bbox[6 * (size_t)bid];
            for (int q = 0; q < 3; ++q) {
                const float4& p = bt[3 * t + q];
                bb[0] = std::min(bb[0], p.x); bb[1] = std::min(bb[1], p.y); bb[2] = std::min(bb[2], p.z);
                bb[3] = std::max(bb[3], p.x); bb[4] = std::max(bb[4], p.y); bb[5] = std::max(bb[5], p.z);
            }
        }
        for (int k = 0; k < V; ++k) {
            for (int q = v->removed_off[k]; q < v->removed_off[k + 1]; ++q) {
                const int bid = v->removed_ids[q];
                if (bid < 0 || bid >= base->n_buildings) continue;
                changed[k].insert(changed[k].end(), &bbox[6 * (size_t)bid], &bbox[6 * (size_t)bid] + 6);
            }
            for (int t = v->tower_off[k]; t < v->tower_off[k + 1]; ++t) {
                float b6[6] = {3.4e38f, 3.4e38f, 3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
                for (int q = 0; q < 3; ++q)
                    for (int c = 0; c < 3; ++c) {
                        const float x = v->tower_tris[9 * (size_t)t + 3 * q + c];
                        b6[c] = std::min(b6[c], x);
                        b6[3 + c] = std::max(b6[3 + c], x);
                    }
                changed[k].insert(changed[k].end(), b6, b6 + 6);
            }
        }
    }
    // Work items: every tile of every variant's region, for every interval.  A tile is
    // marked affected if the shadow of a changed box, swept over the interval's slope
    // range, can reach it (one cell of margin); other tiles keep the base counts.
    std::vector<int4> items;
    std::vector<unsigned char> hit((size_t)tiles_x * tiles_y);
    for (int i = 0; i < n_intervals; ++i) {
        float uxlo = 3.4e38f, uxhi = -3.4e38f, uylo = 3.4e38f, uyhi = -3.4e38f;
        for (const sa::StepConst& sc : intervals[i]->h_steps) {
            uxlo = std::min(uxlo, sc.ux); uxhi = std::max(uxhi, sc.ux);
            uylo = std::min(uylo, sc.uy); uyhi = std::max(uyhi, sc.uy);
        }
        for (int k = 0; k < V; ++k) {
            const sa::BatchVariant& var = hv[k];
            if (var.nx == 0 || var.ny == 0) continue;
            std::fill(hit.begin(), hit.end(), 0);
            const std::vector<float>& ch = changed[k];
            for (size_t q = 0; q < ch.size(); q += 6) {
                const float zh = std::max(ch[q + 5], 0.f);
                const double x0 = ch[q] - zh * std::max(uxhi, 0.f), x1 = ch[q + 3] - zh * std::min(uxlo, 0.f);
                const double y0 = ch[q + 1] - zh * std::max(uyhi, 0.f), y1 = ch[q + 4] - zh * std::min(uylo, 0.f);
                const double cell = grid->dx;
                const int tx0 = (int)std::max(0.0, std::floor((x0 - grid->x0 - cell) / (32.0 * cell)));
                const int tx1 = (int)std::min((double)tiles_x - 1, std::floor((x1 - grid->x0 + cell) / (32.0 * cell)));
                const int ty0 = (int)std::max(0.0, std::floor((y0 - grid->y0 - cell) / (32.0 * cell)));
                const int ty1 = (int)std::min((double)tiles_y - 1, std::floor((y1 - grid->y0 + cell) / (32.0 * cell)));
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int tx = tx0; tx <= tx1; ++tx) hit[(size_t)ty * tiles_x + tx] = 1;
            }
            if (!sa::get_batch_tile_skip()) std::fill(hit.begin(), hit.end(), 1);
            const int tx0 = var.ix0 / 32, tx1 = (var.ix0 + var.nx - 1) / 32;
            const int ty0 = var.iy0 / 32, ty1 = (var.iy0 + var.ny - 1) / 32;
            for (int ty = ty0; ty <= std::min(ty1, tiles_y - 1); ++ty)
                for (int tx = tx0; tx <= std::min(tx1, tiles_x - 1); ++tx)
                    items.push_back(make_int4(i, k, ty * tiles_x + tx, hit[(size_t)ty * tiles_x + tx]));
        }
    }
    // affected items first, so the persistent CTAs take the heavy work early
    std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
    b->n_affected = 0;
    for (const int4& it : items) b->n_affected += it.w;
    b->n_items = (int)items.size();
    if (e == cudaSuccess) e = dev_copy(b, items.data(), items.size(), &b->d_items);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        sa_batch_destroy(b);
        return sa::report_error(e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = b;
    return SA_OK;
}

int64_t sa_batch_output_count(const sa_batch* b) {
    return b ? (int64_t)b->I * b->cells_per_interval : -1;
}

int64_t sa_batch_output_offset(const sa_batch* b, int32_t interval, int32_t variant) {
    if (!b || interval < 0 || interval >= b->I || variant < 0 || variant >= b->V) return -1;
    return (int64_t)interval * b->cells_per_interval + b->var_off[variant];
}

int32_t sa_batch_work_items(const sa_batch* b) { return b ? b->n_items : -1; }
int32_t sa_batch_affected_items(const sa_batch* b) { return b ? b->n_affected : -1; }

sa_status sa_batch_run(sa_batch* b, int32_t* counts, int32_t* impact, void* stream) {
    if (!b) return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_run: NULL batch");
    if (!counts && b->n_items > 0) return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_run: NULL counts");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!b->exec || b->g_counts != counts || b->g_impact != impact) {
        drop_graph(b);
        e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = sa::launch_batch(launch_of(b, counts, impact, b->n_items, b->ctas, b->run, nullptr),
                                              b->capture);
            e = cudaStreamEndCapture(b->capture, &b->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
        }
        b->g_counts = counts;
        b->g_impact = impact;
    }
    e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
    return sa::check_after_call(st, "sa_batch_run");
}

// Launch shape: 2, 3 or 4 persistent CTAs per SM and 8, 16 or 24 steps per raster run,
// each timed on the first eighth of the work queue; the fastest is kept for sa_batch_run.
sa_status sa_batch_tune(sa_batch* b, int32_t* best_ctas, int32_t* best_run, void* stream) {
    if (!b) return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_tune: NULL batch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = std::max(1, b->n_items / 8);
    int* scratch = nullptr;
    cudaError_t e = sa::scratch_alloc(&scratch, sizeof(int) * (size_t)std::max<long long>(1, b->I * b->cells_per_interval), st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 3.4e38f;
    int bc = b->ctas, br = b->run;
    const int runs[3] = {8, 16, 24};
    for (int c = 2; c <= sa::raster_ctas_per_sm() && e == cudaSuccess; ++c)
        for (int r : runs) {
            const sa::BatchLaunch bl = launch_of(b, scratch, nullptr, n, c * b->sms, r, nullptr);
            e = sa::launch_batch(bl, st);                                   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = sa::launch_batch(bl, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best) { best = ms; bc = c * b->sms; br = r; }
            if (e != cudaSuccess) break;
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (scratch) cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
    if (bc != b->ctas || br != b->run) drop_graph(b);
    b->ctas = bc;
    b->run = br;
    if (best_ctas) *best_ctas = bc;
    if (best_run) *best_run = br;
    return SA_OK;
}

// Work counters of one batch run (ground-raster counters [2], [3]; see sa_work_counters).
sa_status sa_batch_work_counters(sa_batch* b, uint64_t* counters, void* stream) {
    if (!b || !counters) return sa::report_error(SA_ERR_INVALID_ARG, "sa_batch_work_counters: NULL argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int* scratch = nullptr;
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(uint64_t) * 4, st);
    if (e == cudaSuccess)
        e = sa::scratch_alloc(&scratch, sizeof(int) * (size_t)std::max<long long>(1, b->I * b->cells_per_interval), st);
    if (e == cudaSuccess)
        e = sa::launch_batch(launch_of(b, scratch, nullptr, b->n_items, b->ctas, b->run,
                                       reinterpret_cast<unsigned long long*>(counters)), st);
    if (scratch) cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
    return SA_OK;
}

}  // extern "C"
