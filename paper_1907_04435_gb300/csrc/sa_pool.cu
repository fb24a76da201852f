// sa_pool.cu -- the library's stream-ordered memory pool.
//
// Scratch (bins, masks, sort buffers) is allocated and freed on the caller's stream within
// each call, and the handles' own arrays (BVH, sun tables, sorted receivers) come from the
// same pool, freed when the handle is destroyed.  The default pool would return memory to
// the device at every synchronisation, so a repeated call would map it again each time;
// this pool keeps up to kKeep bytes reserved instead, and a handle built again (a scene
// rebuilt every step) takes memory already mapped instead of paying cudaMalloc's latency.
#include <atomic>
#include <mutex>
#include <vector>

#include "sa_handles.cuh"

namespace sa {

namespace {
constexpr unsigned long long kKeep = 4ull << 30;
std::mutex g_pool_mu;
std::vector<cudaMemPool_t> g_pools;   // by device ordinal; null until first use
std::atomic<unsigned long long> g_n_allocs{0}, g_alloc_bytes{0};

cudaError_t pool_of_current_device(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = kKeep;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t scratch_alloc_bytes(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_of_current_device(&pool);
    if (e != cudaSuccess) return e;
    g_n_allocs.fetch_add(1, std::memory_order_relaxed);
    g_alloc_bytes.fetch_add(bytes, std::memory_order_relaxed);
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

}  // namespace sa

extern "C" sa_status sa_scratch_stats(uint64_t* stats) {
    if (!stats) return sa::report_error(SA_ERR_INVALID_ARG, "sa_scratch_stats: stats is NULL");
    stats[0] = sa::g_n_allocs.load(std::memory_order_relaxed);
    stats[1] = sa::g_alloc_bytes.load(std::memory_order_relaxed);
    stats[2] = 0;
    stats[3] = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SA_OK;
    }
    std::lock_guard<std::mutex> lk(sa::g_pool_mu);
    if (dev < (int)sa::g_pools.size() && sa::g_pools[dev]) {
        unsigned long long v = 0;
        if (cudaMemPoolGetAttribute(sa::g_pools[dev], cudaMemPoolAttrReservedMemCurrent, &v) == cudaSuccess)
            stats[2] = v;
        if (cudaMemPoolGetAttribute(sa::g_pools[dev], cudaMemPoolAttrUsedMemHigh, &v) == cudaSuccess)
            stats[3] = v;
    }
    return SA_OK;
}
