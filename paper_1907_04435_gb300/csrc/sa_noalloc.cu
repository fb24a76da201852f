// sa_noalloc.cu -- sa_accumulate_grid_noalloc: the ground-grid accrual raster with its
// scratch memory in a fixed device array instead of the stream-ordered allocator.
//
// Some callers cannot allocate device memory while they run: a host application that
// reserved the device's memory for itself before loading this library, or a loop that
// must not pay the allocator's synchronisation and latency.  This entry point takes all
// of its scratch (per-receiver run state, tile bin counters, scan partials and the bins)
// from one file-scope __device__ array of SA_NOALLOC_SCRATCH_BYTES, which every GPU that
// loads the library keeps for the life of the process.  The paper has no counterpart.
#include <string.h>

#include "sa_handles.cuh"

namespace {

// Host code must not use this symbol as a device address; it obtains the address with
// cudaGetSymbolAddress (see scratch_of_current_device).
static __device__ __align__(256) unsigned char g_grid_scratch[SA_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current device's context.  It is looked up
// on every call (a cheap driver query beside the call's own synchronisations), so an
// address never outlives the context it was taken in.
sa_status scratch_of_current_device(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_grid_scratch);
    if (e != cudaSuccess || !p)
        return sa::report_error(SA_ERR_CUDA, "sa_accumulate_grid_noalloc: cudaGetSymbolAddress of the scratch array failed");
    *out = static_cast<unsigned char*>(p);
    return SA_OK;
}

}  // namespace

extern "C" sa_status sa_accumulate_grid_noalloc(const sa_scene* scene, const sa_receivers* grid,
                                                const sa_sun* sun, float step_minutes,
                                                int32_t flags, int32_t* gross_steps,
                                                float* gross_minutes, int32_t* continuous_steps,
                                                void* stream) {
    if (!scene || !grid || !sun)
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_accumulate_grid_noalloc: NULL handle");
    if (!grid->is_grid)
        return sa::report_error(SA_ERR_UNSUPPORTED, "sa_accumulate_grid_noalloc: receivers must be a ground grid");
    if (grid->R > (long long)SA_NOALLOC_MAX_CELLS)
        return sa::report_error(SA_ERR_INVALID_ARG,
                                "sa_accumulate_grid_noalloc: grid has more than SA_NOALLOC_MAX_CELLS "
                                "(4194304) cells; split it or use sa_accumulate");
    if (scene->min_z < 0.f)
        return sa::report_error(SA_ERR_UNSUPPORTED, "sa_accumulate_grid_noalloc: geometry below z = 0");
    if (flags & ~SA_ACCUMULATE_INTO)
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_accumulate_grid_noalloc: unknown flags");
    if (!(step_minutes >= 0.f) || step_minutes > 3.4e38f)
        return sa::report_error(SA_ERR_INVALID_ARG, "sa_accumulate_grid_noalloc: bad step_minutes");
    if (grid->R == 0) return SA_OK;
    if (!gross_steps) return sa::report_error(SA_ERR_INVALID_ARG, "sa_accumulate_grid_noalloc: gross_steps is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (sun->h_blocks.empty()) {
        // no steps: counts are zero, or unchanged when accumulating (as sa_accumulate)
        cudaError_t e = cudaSuccess;
        if (!(flags & SA_ACCUMULATE_INTO)) {
            const size_t n = (size_t)grid->R;
            e = cudaMemsetAsync(gross_steps, 0, sizeof(int32_t) * n, st);
            if (e == cudaSuccess && continuous_steps) e = cudaMemsetAsync(continuous_steps, 0, sizeof(int32_t) * n, st);
            if (e == cudaSuccess && gross_minutes) e = cudaMemsetAsync(gross_minutes, 0, sizeof(float) * n, st);
        }
        return e == cudaSuccess ? SA_OK : sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
    }
    unsigned char* scratch = nullptr;
    sa_status s = scratch_of_current_device(&scratch);
    if (s != SA_OK) return s;

    sa::DevScene dsc;
    dsc.nodes = scene->bvh.nodes;
    dsc.tris = scene->bvh.tris;
    dsc.n_nodes = scene->bvh.n_nodes;
    dsc.T = (int)scene->T;
    dsc.closed = scene->closed;
    sa::DevRecv drc;
    drc.is_grid = 1;
    drc.x0 = grid->x0; drc.y0 = grid->y0; drc.dx = grid->dx; drc.nx = grid->nx; drc.ny = grid->ny;
    drc.orig = nullptr; drc.nrm = nullptr; drc.perm = nullptr; drc.R = grid->R;
    sa::DevSun dsun;
    dsun.steps = sun->d_steps;
    dsun.blocks = sun->d_blocks;
    dsun.S = sun->S;
    dsun.n_blocks = (int)sun->h_blocks.size();
    sa::DevOut out;
    memset(&out, 0, sizeof(out));
    out.gross = gross_steps;
    out.minutes = gross_minutes;
    out.continuous = continuous_steps;
    out.step_minutes = step_minutes;
    out.accumulate_into = (flags & SA_ACCUMULATE_INTO) ? 1 : 0;
    out.write_final = 1;
    int capacity_error = 0;
    cudaError_t e = sa::launch_raster_ground_in(dsc, drc, dsun, out, st, scratch,
                                                SA_NOALLOC_SCRATCH_BYTES, &capacity_error);
    if (e != cudaSuccess) return sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
    if (capacity_error)
        return sa::report_error(SA_ERR_INVALID_ARG,
                                "sa_accumulate_grid_noalloc: one block's triangle-tile bins do not fit the "
                                "fixed scratch (no output was written); use a shorter block_len, a smaller "
                                "grid or sa_accumulate");
    return sa::check_after_call(st, "sa_accumulate_grid_noalloc");
}
