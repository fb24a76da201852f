// sa_graph.cu -- direction bins and the direction graph for long periods (Sec. 6).
//
// Over many days the sun retraces nearly the same hourly arcs, so an interval is reduced to
// the pair (bin of its first direction, bin of its last direction), the bins being quads of
// the hemisphere bounded by `bin_deg` in elevation and in azimuth.  Intervals with the same
// pair (and the same number of steps) are one edge of the direction graph; one shadow map
// is computed per edge and reused for every interval the edge stands for.  The paper does
// not say which interval's sun the map uses; here it is the edge's middle interval in
// time order, so that the map's sun lies inside the spread of the suns it stands for (the
// first interval biases a season's shadow toward the season's start).
//
//   direction_graph   host: edge of every block, the block each edge's map is computed
//                     from, weights.
//   k_edge_summary    per (edge, receiver): popcount, leading run (prefix), trailing run
//                     (suffix) and longest run of the edge's step mask, packed in 32 bits.
//   k_graph_reduce    per receiver: gross = sum over the blocks of all days of the edge's
//                     popcount (Eq. 1: each edge's count times its weight), and the longest
//                     continuous run, stitched along each day's path of edges in time order
//                     from the prefix / longest / suffix runs (Sec. 6, continuous shadows).
#include <math.h>

#include <map>
#include <tuple>
#include <vector>

#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kGraphThreads = 256;

__device__ __forceinline__ unsigned longest_run(unsigned long long x) {
    unsigned n = 0;
    while (x) {        // each pass shortens every run of ones by one
        x &= x >> 1;
        ++n;
    }
    return n;
}

__global__ void k_edge_summary(const unsigned long long* __restrict__ masks, long long R, int n_edges,
                               const int* __restrict__ edge_K, unsigned* __restrict__ summary) {
    const long long items = R * n_edges;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(it / R);
        const int K = __ldg(&edge_K[e]);
        const unsigned long long low = K >= 64 ? ~0ull : ((1ull << K) - 1ull);
        const unsigned long long m = masks[it] & low;
        const unsigned pop = (unsigned)__popcll(m);
        unsigned pre, suf, best;
        if (pop == (unsigned)K) {
            pre = suf = best = (unsigned)K;
        } else {
            pre = (unsigned)(__ffsll((long long)~m) - 1);            // ones below the first zero
            suf = (unsigned)__clzll((long long)~(m << (64 - K)));   // ones above the last zero
            best = longest_run(m);
        }
        summary[it] = pop | (pre << 8) | (suf << 16) | (best << 24);
    }
}

__global__ void k_graph_reduce(const unsigned* __restrict__ summary, long long R,
                               const int* __restrict__ path, const int* __restrict__ day_block,
                               int D, const int* __restrict__ edge_K, float step_minutes,
                               int* __restrict__ gross, float* __restrict__ minutes,
                               int* __restrict__ continuous) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (long long)gridDim.x * blockDim.x) {
        int g = 0, best_all = 0;
        for (int d = 0; d < D; ++d) {
            int run = 0, best = 0;
            const int b1 = __ldg(&day_block[d + 1]);
            for (int b = __ldg(&day_block[d]); b < b1; ++b) {
                const int e = __ldg(&path[b]);
                const unsigned s = summary[(long long)e * R + r];
                const int pop = (int)(s & 255u);
                if (pop == __ldg(&edge_K[e])) {
                    run += pop;
                } else {
                    best = max(best, max(run + (int)((s >> 8) & 255u), (int)(s >> 24)));
                    run = (int)((s >> 16) & 255u);
                }
                g += pop;
            }
            best_all = max(best_all, max(best, run));
        }
        gross[r] = g;
        if (minutes) minutes[r] = (float)g * step_minutes;
        if (continuous) continuous[r] = best_all;
    }
}

int grid_for(long long items) {
    const long long b = (items + kGraphThreads - 1) / kGraphThreads;
    return (int)(b < 152ll * 16 ? (b > 0 ? b : 1) : 152ll * 16);
}

}  // namespace

void direction_graph(const float* dirs, int n_blocks, const int* j0, const int* K, double bin_deg,
                     std::vector<int>& edge, std::vector<int>& rep, std::vector<int>& weight) {
    const double to_deg = 180.0 / M_PI;
    auto bins = [&](int j, long long* eb, long long* ab) {
        const double x = dirs[3 * (size_t)j], y = dirs[3 * (size_t)j + 1], z = dirs[3 * (size_t)j + 2];
        const double n = sqrt(x * x + y * y + z * z);
        const double el = asin(fmin(fmax(z / n, -1.0), 1.0)) * to_deg;
        const double az = atan2(x, y) * to_deg;
        *eb = (long long)floor(el / bin_deg);
        *ab = (long long)floor(az / bin_deg);
    };
    std::map<std::tuple<long long, long long, long long, long long, int>, int> ids;
    edge.assign((size_t)n_blocks, 0);
    rep.clear();
    weight.clear();
    for (int b = 0; b < n_blocks; ++b) {
        long long e1, a1, e2, a2;
        bins(j0[b], &e1, &a1);
        bins(j0[b] + K[b] - 1, &e2, &a2);
        const auto key = std::make_tuple(e1, a1, e2, a2, K[b]);
        auto it = ids.find(key);
        if (it == ids.end()) {
            it = ids.emplace(key, (int)rep.size()).first;
            rep.push_back(b);
            weight.push_back(0);
        }
        edge[(size_t)b] = it->second;
        weight[(size_t)it->second] += 1;
    }
    // each edge's map comes from its middle block: member (m - 1) / 2 of its m blocks
    std::vector<int> seen(rep.size(), 0);
    for (int b = 0; b < n_blocks; ++b) {
        const int q = edge[(size_t)b];
        if (seen[(size_t)q]++ == (weight[(size_t)q] - 1) / 2) rep[(size_t)q] = b;
    }
}

cudaError_t launch_edge_summary(const unsigned long long* masks, long long R, int n_edges,
                                const int* d_edge_K, unsigned* summary, cudaStream_t st) {
    if (R <= 0 || n_edges <= 0) return cudaSuccess;
    k_edge_summary<<<grid_for(R * n_edges), kGraphThreads, 0, st>>>(masks, R, n_edges, d_edge_K, summary);
    return cudaGetLastError();
}

cudaError_t launch_graph_reduce(const unsigned* summary, long long R, const int* d_path,
                                const int* d_day_block, int D, const int* d_edge_K, float step_minutes,
                                int* gross, float* minutes, int* continuous, cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    k_graph_reduce<<<grid_for(R), kGraphThreads, 0, st>>>(summary, R, d_path, d_day_block, D, d_edge_K,
                                                          step_minutes, gross, minutes, continuous);
    return cudaGetLastError();
}

}  // namespace sa
