// sa_check.cu -- the bounds-checked build's registry of per-file violation words, and the
// calls that report them (sa_checked_build, sa_check_status).
#include <stdio.h>

#include <mutex>
#include <vector>

#include "sa_handles.cuh"

namespace sa {

namespace {
std::mutex& reader_mu() {
    static std::mutex m;
    return m;
}
std::vector<CheckReader>& readers() {
    static std::vector<CheckReader> v;
    return v;
}
}  // namespace

int register_check_reader(CheckReader r) {
    std::lock_guard<std::mutex> lk(reader_mu());
    readers().push_back(r);
    return (int)readers().size();
}

cudaError_t read_check_words(unsigned long long* w) {
    w[0] = w[1] = w[2] = 0ull;
    std::lock_guard<std::mutex> lk(reader_mu());
    for (CheckReader r : readers()) {
        unsigned long long x[3] = {0ull, 0ull, 0ull};
        const cudaError_t e = r(x, 1);
        if (e != cudaSuccess) return e;
        if (x[0] && !w[0]) { w[0] = x[0]; w[1] = x[1]; w[2] = x[2]; }
    }
    return cudaSuccess;
}

const char* check_site_name(int site) {
    static const char* names[CK_SITES] = {
        "none", "ray traversal: leaf triangle", "ray traversal: escape link",
        "ground raster: binned triangle", "ground raster: tile cell", "binning: bin slot",
        "light-space map: binned triangle", "light-space map: binned receiver",
        "light-space map: receiver permutation", "light-space map: receiver mask",
        "building contribution: leaf triangle", "building contribution: escape link",
        "building contribution: building id", "building contribution: listed cell",
        "inverse map: leaf triangle",
        "inverse map: escape link", "height adjoint: leaf triangle", "height adjoint: escape link"};
    return site >= 0 && site < CK_SITES ? names[site] : "unknown";
}

sa_status check_after_call(cudaStream_t st, const char* who) {
#ifdef SA_CHECKED
    cudaError_t e = cudaStreamSynchronize(st);
    unsigned long long w[3] = {0ull, 0ull, 0ull};
    if (e == cudaSuccess) e = read_check_words(w);
    char msg[256];
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "%s: %s", who, cudaGetErrorString(e));
        return report_error(SA_ERR_CUDA, msg);
    }
    if (w[0]) {
        snprintf(msg, sizeof(msg), "%s: index %lld outside its bound %lld at %s (bounds-checked build)",
                 who, (long long)w[1], (long long)w[2], check_site_name((int)w[0]));
        return report_error(SA_ERR_INTERNAL, msg);
    }
#else
    (void)st;
    (void)who;
#endif
    return SA_OK;
}

}  // namespace sa

extern "C" {

int32_t sa_checked_build(void) {
#ifdef SA_CHECKED
    return 1;
#else
    return 0;
#endif
}

sa_status sa_check_status(int32_t* site, int64_t* index, int64_t* bound) {
    if (site) *site = 0;
    if (index) *index = 0;
    if (bound) *bound = 0;
#ifdef SA_CHECKED
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long w[3] = {0ull, 0ull, 0ull};
    if (e == cudaSuccess) e = sa::read_check_words(w);
    if (e != cudaSuccess) return sa::report_error(SA_ERR_CUDA, cudaGetErrorString(e));
    if (w[0]) {
        if (site) *site = (int32_t)w[0];
        if (index) *index = (int64_t)w[1];
        if (bound) *bound = (int64_t)w[2];
        char msg[256];
        snprintf(msg, sizeof(msg), "sa_check_status: index %lld outside its bound %lld at %s",
                 (long long)w[1], (long long)w[2], sa::check_site_name((int)w[0]));
        return sa::report_error(SA_ERR_INTERNAL, msg);
    }
#endif
    return SA_OK;
}

}  // extern "C"
