// Device buffers of released workspaces, kept for reuse.
//
// A plan's numeric workspace is a dozen buffers of up to a few hundred MB
// (panel-sized scratch, digit planes, exact sums).  Creating and destroying
// plans of one pattern again and again (the end-to-end path re-plans from
// host arrays every call) would pay a cudaMalloc and a synchronizing
// cudaFree for each of them every time.  Released buffers go into a cache
// keyed by their exact size instead, up to kCacheCap bytes; the owner
// synchronizes the device once before releasing, so that no kernel can still
// be using a cached buffer when it is handed out again.  A failed cudaMalloc
// empties the cache and retries; selinv_release_cached_memory empties it on
// request.
#include <cuda_runtime.h>

#include <cstddef>
#include <map>
#include <mutex>

#include "selinv.h"
#include "plan.h"

namespace selinv {

namespace {
constexpr size_t kCacheCap = size_t(8) << 30;   // bytes kept at most
std::mutex g_mu;
std::multimap<size_t, void *> g_cache;
size_t g_cached = 0;

void trim_locked() {
    for (auto &e : g_cache) cudaFree(e.second);
    g_cache.clear();
    g_cached = 0;
}
}  // namespace

cudaError_t dev_alloc(void **ptr, size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(bytes);
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
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_cached + bytes <= kCacheCap) {
        g_cache.emplace(bytes, ptr);
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
