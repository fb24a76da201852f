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
//                     The days' paths are one walk of packed codes staged in shared memory.
#include <math.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kGraphThreads = 256;
constexpr int kGather = 8;        // summaries a thread loads ahead in the walk
constexpr int kWalkTile = 2048;   // walk codes staged in shared memory at a time

// Longest run of ones in x, which is not all ones.  With A_k the bits i at which a run of
// at least k ones starts (A_1 = x, A_{a+b} = A_a & (A_b >> a)), the longest run is the
// largest n with A_n != 0; it is found bit by bit from 32 down, since it is below 64.
__device__ __forceinline__ unsigned longest_run(unsigned long long x) {
    const unsigned long long a1 = x, a2 = a1 & (a1 >> 1), a4 = a2 & (a2 >> 2), a8 = a4 & (a4 >> 4),
                             a16 = a8 & (a8 >> 8), a32 = a16 & (a16 >> 16);
    unsigned long long cur = ~0ull;   // A_0
    unsigned n = 0;
    unsigned long long c;
    c = cur & (a32 >> n); if (c) { cur = c; n += 32; }
    c = cur & (a16 >> n); if (c) { cur = c; n += 16; }
    c = cur & (a8 >> n);  if (c) { cur = c; n += 8; }
    c = cur & (a4 >> n);  if (c) { cur = c; n += 4; }
    c = cur & (a2 >> n);  if (c) { cur = c; n += 2; }
    c = cur & (a1 >> n);  if (c) { n += 1; }
    return n;
}

// grid: x over receivers, y over edges (strided)
__global__ void k_edge_summary(const unsigned long long* __restrict__ masks, long long R, int n_edges,
                               const int* __restrict__ edge_K, unsigned* __restrict__ summary) {
    for (int e = blockIdx.y; e < n_edges; e += gridDim.y) {
        const int K = __ldg(&edge_K[e]);
        const unsigned long long low = K >= 64 ? ~0ull : ((1ull << K) - 1ull);
        const unsigned long long* __restrict__ me = masks + (long long)e * R;
        unsigned* __restrict__ se = summary + (long long)e * R;
        for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R;
             r += (long long)gridDim.x * blockDim.x) {
            const unsigned long long m = me[r] & low;
            if (m == 0ull) {            // lit at every step: the most common case
                se[r] = 0u;
                continue;
            }
            const unsigned pop = (unsigned)__popcll(m);
            unsigned pre, suf, best;
            if (pop == (unsigned)K) {
                pre = suf = best = (unsigned)K;
            } else {
                pre = (unsigned)(__ffsll((long long)~m) - 1);            // ones below the first zero
                suf = (unsigned)__clzll((long long)~(m << (64 - K)));   // ones above the last zero
                best = longest_run(m);
            }
            se[r] = pop | (pre << 8) | (suf << 16) | (best << 24);
        }
    }
}

// The walk: every block of every day in time order, packed as edge | K << 20 | new_day << 27.
// Each CTA stages kWalkTile codes of it in shared memory; each thread walks them for its
// receiver, loading kGather summaries ahead of their use.
__global__ void __launch_bounds__(kGraphThreads) k_graph_reduce(
    const unsigned* __restrict__ summary, long long R, const int* __restrict__ walk, int n_walk,
    float step_minutes, int* __restrict__ gross, float* __restrict__ minutes, int* __restrict__ continuous) {
    __shared__ int s_walk[kWalkTile];
    for (long long base = (long long)blockIdx.x * blockDim.x; base < R; base += (long long)gridDim.x * blockDim.x) {
        const long long r = base + threadIdx.x;
        const bool valid = r < R;
        int g = 0, best_all = 0, run = 0, best = 0;
        for (int p0 = 0; p0 < n_walk; p0 += kWalkTile) {
            const int n = min(kWalkTile, n_walk - p0);
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) s_walk[i] = __ldg(&walk[p0 + i]);
            __syncthreads();
            if (!valid) continue;
            for (int i = 0; i < n; i += kGather) {
                unsigned sm[kGather];
                int code[kGather];
#pragma unroll
                for (int q = 0; q < kGather; ++q) {
                    code[q] = i + q < n ? s_walk[i + q] : -1;
                    sm[q] = code[q] >= 0 ? summary[(long long)(code[q] & 0xFFFFF) * R + r] : 0u;
                }
#pragma unroll
                for (int q = 0; q < kGather; ++q) {
                    if (code[q] < 0) break;
                    if (code[q] & (1 << 27)) {          // a new day: close the previous one
                        best_all = max(best_all, max(best, run));
                        run = best = 0;
                    }
                    const int K = (code[q] >> 20) & 127;
                    const int pop = (int)(sm[q] & 255u);
                    if (pop == K) {
                        run += pop;
                    } else {
                        best = max(best, max(run + (int)((sm[q] >> 8) & 255u), (int)(sm[q] >> 24)));
                        run = (int)((sm[q] >> 16) & 255u);
                    }
                    g += pop;
                }
            }
        }
        if (valid) {
            best_all = max(best_all, max(best, run));
            gross[r] = g;
            if (minutes) minutes[r] = (float)g * step_minutes;
            if (continuous) continuous[r] = best_all;
        }
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
    const long long bx = (R + kGraphThreads - 1) / kGraphThreads;
    dim3 grid((unsigned)std::min(bx, 152ll * 8), (unsigned)std::min(n_edges, 65535));
    KernelTimer kt(KT_GRAPH, st);
    k_edge_summary<<<grid, kGraphThreads, 0, st>>>(masks, R, n_edges, d_edge_K, summary);
    return cudaGetLastError();
}

cudaError_t launch_graph_reduce(const unsigned* summary, long long R, const int* d_walk, int n_walk,
                                float step_minutes, int* gross, float* minutes, int* continuous,
                                cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    KernelTimer kt(KT_GRAPH, st);
    k_graph_reduce<<<grid_for(R), kGraphThreads, 0, st>>>(summary, R, d_walk, n_walk, step_minutes, gross,
                                                          minutes, continuous);
    return cudaGetLastError();
}

}  // namespace sa
