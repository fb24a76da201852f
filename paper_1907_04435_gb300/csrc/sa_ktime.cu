// sa_ktime.cu -- per-kernel device timing.
//
// Events are recorded on the stream that launches the kernel, so the measured interval is
// that launch alone (plus the event records themselves, a few microseconds).  Pairs are
// queued and resolved only when the caller collects them, so timing adds no host
// synchronisation to the timed calls.
#include <mutex>
#include <vector>

#include "sa_internal.cuh"

namespace sa {

namespace {
struct Pending {
    int id;
    cudaEvent_t a, b;
};
std::mutex g_mu;
int g_on = 0;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;

cudaEvent_t take_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

void set_kernel_timing(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on ? 1 : 0;
}

int get_kernel_timing() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

KernelTimer::KernelTimer(int id_, cudaStream_t st_) : id(id_), st(st_), begin(nullptr) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cudaEvent_t e = take_event();
    if (!e) return;
    if (cudaEventRecord(e, st) != cudaSuccess) {
        g_free.push_back(e);
        return;
    }
    begin = (void*)e;
}

KernelTimer::~KernelTimer() {
    if (!begin) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t a = (cudaEvent_t)begin;
    cudaEvent_t b = take_event();
    if (!b || cudaEventRecord(b, st) != cudaSuccess) {
        g_free.push_back(a);
        if (b) g_free.push_back(b);
        return;
    }
    g_pending.push_back({id, a, b});
}

cudaError_t collect_kernel_times(double* ms, long long* n, int n_classes) {
    std::vector<Pending> todo;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        todo.swap(g_pending);
    }
    cudaError_t first = cudaSuccess;
    for (const Pending& p : todo) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
        if (e == cudaSuccess) {
            if (p.id >= 0 && p.id < n_classes) {
                if (ms) ms[p.id] += (double)t;
                if (n) n[p.id] += 1;
            }
        } else if (first == cudaSuccess) {
            first = e;
        }
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending& p : todo) {
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    return first;
}

}  // namespace sa

static_assert(sa::KT_RASTER == SA_KERNEL_RASTER && sa::KT_SAM_POINTS == SA_KERNEL_SAM_POINTS &&
                  sa::KT_ACCRUAL == SA_KERNEL_ACCRUAL && sa::KT_SWEEP == SA_KERNEL_SWEEP &&
                  sa::KT_IAM == SA_KERNEL_IAM && sa::KT_GRAPH == SA_KERNEL_GRAPH &&
                  sa::KT_RASTER_BIN == SA_KERNEL_RASTER_BIN && sa::KT_CONTRIB == SA_KERNEL_CONTRIB &&
                  SA_KERNEL_CLASSES == 8,
              "kernel classes of the C ABI and the library agree");
