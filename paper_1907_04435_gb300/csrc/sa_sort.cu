// sa_sort.cu -- device-wide exclusive scan and a stable LSD radix sort of (key, value)
// pairs, used for Morton ordering of triangles (BVH build) and of point receivers, and for
// the tile bins of the accrual raster.
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048 values per CTA

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
__device__ unsigned block_excl_scan(unsigned v, unsigned* total) {
    __shared__ unsigned warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    unsigned incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned s = lane < nwarps ? warp_sums[lane] : 0u;
        unsigned si = warp_incl_scan(s);
        if (lane < nwarps) warp_sums[lane] = si - s;
        if (lane == nwarps - 1) warp_sums[31] = si;
    }
    __syncthreads();
    unsigned res = incl - v + warp_sums[warp];
    if (total) *total = warp_sums[31];
    __syncthreads();
    return res;
}

__global__ void k_scan_reduce(const unsigned* __restrict__ in, long long n,
                              unsigned* __restrict__ partial) {
    const long long base = (long long)blockIdx.x * kScanTile;
    unsigned s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    unsigned total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// single CTA: exclusive scan of the partials in place (any count), total to *d_total
__global__ void k_scan_partials(unsigned* partial, int np, unsigned* d_total) {
    unsigned carry = 0;
    for (int base = 0; base < np; base += kScanThreads) {
        int i = base + threadIdx.x;
        unsigned v = i < np ? partial[i] : 0u;
        unsigned tot;
        unsigned ex = block_excl_scan(v, &tot);
        if (i < np) partial[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void k_scan_apply(unsigned* __restrict__ data, long long n,
                             const unsigned* __restrict__ partial) {
    __shared__ unsigned tile[kScanTile];
    const long long base = (long long)blockIdx.x * kScanTile;
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < n ? data[i] : 0u;
    }
    __syncthreads();
    // each thread scans kScanItems consecutive values
    unsigned loc[kScanItems];
    unsigned s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = s;
        s += tile[threadIdx.x * kScanItems + k];
    }
    unsigned tot;
    unsigned ex = block_excl_scan(s, &tot) + partial[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = loc[k] + ex;
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        if (i < n) data[i] = tile[k * kScanThreads + threadIdx.x];
    }
}

// ------------------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;                              // keys per thread per tile
constexpr int kSortTile = kSortThreads * kSortRounds;       // 2048 keys per CTA
constexpr int kRadix = 256;

__global__ void k_radix_hist(const unsigned* __restrict__ keys, long long n, int shift,
                             unsigned* __restrict__ hist, int n_tiles) {
    __shared__ unsigned h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortRounds; ++k) {
        long long i = base + (long long)k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Stable scatter: keys of a tile are ranked round by round (256 consecutive keys per
// round, in thread order); within a round, warps rank equal digits with match_any and
// warps are ordered by a per-digit prefix over the 8 warps.
__global__ void k_radix_scatter(const unsigned* __restrict__ keys_in,
                                const unsigned* __restrict__ vals_in, long long n, int shift,
                                const unsigned* __restrict__ offsets, int n_tiles,
                                unsigned* __restrict__ keys_out, unsigned* __restrict__ vals_out) {
    __shared__ unsigned base_off[kRadix];
    __shared__ unsigned warp_cnt[kSortThreads / 32][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base_off[threadIdx.x] = offsets[(long long)threadIdx.x * n_tiles + blockIdx.x];
    const long long tile = (long long)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        for (int w = 0; w < kSortThreads / 32; ++w) warp_cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const long long i = tile + (long long)r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        unsigned key = valid ? keys_in[i] : 0u, val = valid ? vals_in[i] : 0u;
        unsigned digit = valid ? (key >> shift) & 0xff : 0x100u + lane;   // unique per lane
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        unsigned rank_in_warp = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) warp_cnt[warp][digit] = __popc(peers);
        __syncthreads();
        // thread t owns digit t: exclusive prefix over warps, then advance base
        {
            unsigned s = 0;
            for (int w = 0; w < kSortThreads / 32; ++w) {
                unsigned c = warp_cnt[w][threadIdx.x];
                warp_cnt[w][threadIdx.x] = s;
                s += c;
            }
            __syncthreads();
            if (valid) {
                unsigned pos = base_off[digit] + warp_cnt[warp][digit] + rank_in_warp;
                keys_out[pos] = key;
                vals_out[pos] = val;
            }
            __syncthreads();
            base_off[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t exclusive_scan_u32(unsigned* data, long long n, unsigned* d_total, cudaStream_t st) {
    if (n <= 0) {
        if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(unsigned), st);
        return cudaSuccess;
    }
    const int np = (int)((n + kScanTile - 1) / kScanTile);
    unsigned* partial = nullptr;
    cudaError_t e = sa::scratch_alloc(&partial, sizeof(unsigned) * np, st);
    if (e != cudaSuccess) return e;
    k_scan_reduce<<<np, kScanThreads, 0, st>>>(data, n, partial);
    k_scan_partials<<<1, kScanThreads, 0, st>>>(partial, np, d_total);
    k_scan_apply<<<np, kScanThreads, 0, st>>>(data, n, partial);
    e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(partial, st);
    return e != cudaSuccess ? e : e2;
}

long long scan_partials(long long n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t exclusive_scan_u32_with(unsigned* data, long long n, unsigned* partial,
                                    unsigned* d_total, cudaStream_t st) {
    if (n <= 0) {
        if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(unsigned), st);
        return cudaSuccess;
    }
    const int np = (int)scan_partials(n);
    k_scan_reduce<<<np, kScanThreads, 0, st>>>(data, n, partial);
    k_scan_partials<<<1, kScanThreads, 0, st>>>(partial, np, d_total);
    k_scan_apply<<<np, kScanThreads, 0, st>>>(data, n, partial);
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(unsigned* keys, unsigned* vals, long long n, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int n_tiles = (int)((n + kSortTile - 1) / kSortTile);
    unsigned *k2 = nullptr, *v2 = nullptr, *hist = nullptr;
    cudaError_t e = sa::scratch_alloc(&k2, sizeof(unsigned) * n, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&v2, sizeof(unsigned) * n, st);
    if (e == cudaSuccess) e = sa::scratch_alloc(&hist, sizeof(unsigned) * kRadix * (size_t)n_tiles, st);
    if (e != cudaSuccess) {
        if (k2) cudaFreeAsync(k2, st);
        if (v2) cudaFreeAsync(v2, st);
        return e;
    }
    unsigned *ka = keys, *va = vals, *kb = k2, *vb = v2;
    for (int shift = 0; shift < 32 && e == cudaSuccess; shift += 8) {
        k_radix_hist<<<n_tiles, kSortThreads, 0, st>>>(ka, n, shift, hist, n_tiles);
        e = exclusive_scan_u32(hist, (long long)kRadix * n_tiles, nullptr, st);
        if (e != cudaSuccess) break;
        k_radix_scatter<<<n_tiles, kSortThreads, 0, st>>>(ka, va, n, shift, hist, n_tiles, kb, vb);
        e = cudaGetLastError();
        unsigned* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    // four passes: the result is back in the caller's buffers
    cudaFreeAsync(k2, st);
    cudaFreeAsync(v2, st);
    cudaFreeAsync(hist, st);
    return e;
}

}  // namespace sa
