// Device buffers of released workspaces, kept for reuse (per device).
//
// A plan's numeric workspace is a dozen buffers of up to a few hundred MB
// (panel-sized scratch, digit planes, exact sums).  Creating and destroying
// plans of one pattern again and again (the end-to-end path re-plans from
// host arrays every call) would pay a cudaMalloc and a synchronizing
// cudaFree for each of them every time.  Released buffers go into a cache
// keyed by their device and exact size instead, up to kCacheCap bytes; the owner
// synchronizes the device once before releasing, so that no kernel can still
// be using a cached buffer when it is handed out again.  A failed cudaMalloc
// empties the cache and retries; selinv_release_cached_memory empties it on
// request.
#include <cuda_runtime.h>

#include <cstddef>
#include <map>
#include <mutex>
#include <utility>

#include "selinv.h"
#include "plan.h"

namespace selinv {

namespace {
constexpr size_t kCacheCap = size_t(8) << 30;   // bytes kept at most
std::mutex g_mu;
std::multimap<std::pair<int, size_t>, void *> g_cache;   // (device, bytes) -> buffer
size_t g_cached = 0;

// frees every cached buffer on its own device (the current device is kept)
void trim_locked() {
    if (g_cache.empty()) return;   // nothing to free: no device call
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    for (auto &e : g_cache) {
        cudaSetDevice(e.first.first);
        cudaFree(e.second);
    }
    if (have) cudaSetDevice(cur);
    g_cache.clear();
    g_cached = 0;
}

int current_device() {
    int d = 0;
    return cudaGetDevice(&d) == cudaSuccess ? d : 0;
}

// the device a buffer was allocated on
int device_of(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) == cudaSuccess) return a.device;
    cudaGetLastError();
    return current_device();
}
}  // namespace

cudaError_t dev_alloc(void **ptr, size_t bytes) {
    const int dev = current_device();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(std::make_pair(dev, bytes));
        if (it != g_cache.end()) {
            *ptr = it->second;
            g_cache.erase(it);
            g_cached -= bytes;
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();   // the failed allocation is not sticky
        {
            std::lock_guard<std::mutex> lk(g_mu);
            trim_locked();
        }
        e = cudaMalloc(ptr, bytes);
    }
    if (e != cudaSuccess) *ptr = nullptr;
    return e;
}

void dev_release(void *ptr, size_t bytes) {
    if (!ptr) return;
    const int dev = device_of(ptr);
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_cached + bytes <= kCacheCap) {
        g_cache.emplace(std::make_pair(dev, bytes), ptr);
        g_cached += bytes;
    } else {
        cudaFree(ptr);
    }
}

}  // namespace selinv

extern "C" int selinv_release_cached_memory(void) {
    std::lock_guard<std::mutex> lk(selinv::g_mu);
    selinv::trim_locked();
    return SELINV_OK;
}
