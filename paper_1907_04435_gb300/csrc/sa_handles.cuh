// sa_handles.cuh -- definitions of the opaque handles of the C ABI (internal).
#pragma once

#include <vector>

#include "sa_internal.cuh"

struct sa_scene {
    sa::LbvhBuild bvh;
    long long T;
    int n_buildings;
    float min_z;
    float box[6] = {0, 0, 0, 0, 0, 0};  // bounds of all vertices: lo.xyz, hi.xyz
    int closed = 0;                    // buildings declared closed, outward-oriented solids
    // scenes built from footprints keep them (height changes, height gradient)
    int has_footprints = 0;
    sa::FootprintSet fs{};
    float* d_heights = nullptr;
    void* d_fp_mem = nullptr;          // one allocation behind the FootprintSet arrays
};

struct sa_sun {
    int S, D;
    std::vector<sa::StepConst> h_steps;
    std::vector<sa::BlockConst> h_blocks;        // requested block length
    std::vector<sa::BlockConst> h_step_blocks;   // one step per block
    sa::StepConst* d_steps = nullptr;
    sa::BlockConst* d_blocks = nullptr;
    sa::BlockConst* d_step_blocks = nullptr;
};

struct sa_receivers {
    int is_grid;
    float x0, y0, dx;
    int nx, ny;
    long long R;
    float4* d_orig = nullptr;
    float4* d_nrm = nullptr;           // facade normals (sorted), null for ground points
    int* d_perm = nullptr;
    float box[6] = {0, 0, 0, 0, 0, 0};  // bounds of the ray origins (points)
};

namespace sa {
// Records `msg` as the calling thread's last error and returns `s`.
sa_status report_error(sa_status s, const char* msg);
// In the bounds-checked build: synchronise `st` and turn a recorded out-of-range index into
// SA_ERR_INTERNAL (naming `who`, the site, the index and its bound); SA_OK otherwise.
sa_status check_after_call(cudaStream_t st, const char* who);
}  // namespace sa
