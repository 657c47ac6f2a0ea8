// Allocation-free variant of the diagonal-block kernel k_linv:
// Dinv = L_KK^{-T} D_K^{-1} L_KK^{-1} for one unit-lower diagonal block.
//
// Some callers cannot allocate device memory: code in a latency-critical
// loop (cudaMalloc and cudaFree synchronize the whole device and take an
// unbounded amount of time), code whose device memory is entirely owned by
// another allocator (a framework's caching allocator or a fixed arena sized
// up front), and code running where allocation is not permitted at all
// (inside a host callback).  For them this entry point keeps its scratch --
// the s x s block L_KK^{-1} -- in a file-scope static device array of fixed
// size instead of plan- or caller-allocated memory; the caller still passes
// the input block, D and the output.
#include <cuda_runtime.h>

#include <mutex>

#include "selinv.h"

namespace {

constexpr int kMaxS = SELINV_NOALLOC_MAX_S;
constexpr int kMaxDevices = 64;

// L_KK^{-1} of the current call, column-major s x s.  Every GPU that loads
// the library holds this array (kMaxS^2 doubles = 128 KB) until the process
// exits.  All calls share it.
static __device__ __align__(256) double g_linv_scratch[kMaxS * kMaxS];

// Device address of g_linv_scratch per device ordinal, looked up once per
// device (in host code the symbol is only a host-side stand-in).  The
// address belongs to the device's primary context: after cudaDeviceReset
// the module is loaded again and the cached address is stale, so a process
// that resets a device must not call this entry point on it afterwards.
std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};

int scratch_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SELINV_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_linv_scratch) != cudaSuccess || !p) return SELINV_ERR_CUDA;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return SELINV_OK;
}

// One CTA: columns of L_KK^{-1} by forward substitution (thread per column),
// then Dinv(i, j) = sum_{k >= max(i,j)} Linv(k, i) Linv(k, j) / D_k.  Every
// entry of the scratch block that is read is written first in this call, so
// nothing needs clearing between calls.
__global__ void __launch_bounds__(128) k_dinv_noalloc(int s, const double *__restrict__ L, int64_t ld,
                                                      const double *__restrict__ D,
                                                      double *__restrict__ Dinv, int64_t ldo,
                                                      double *__restrict__ Li) {
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        double *x = Li + (int64_t)j * s;
        for (int i = 0; i < j; i++) x[i] = 0.0;
        x[j] = 1.0;
        for (int i = j + 1; i < s; i++) {
            double acc = 0.0;
            for (int k = j; k < i; k++) acc = fma(L[(int64_t)k * ld + i], x[k], acc);
            x[i] = -acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int i = e % s, j = e / s;
        double acc = 0.0;
        for (int k = (i > j ? i : j); k < s; k++)
            acc = fma(Li[(int64_t)i * s + k] / D[k], Li[(int64_t)j * s + k], acc);
        Dinv[(int64_t)j * ldo + i] = acc;
    }
}

}  // namespace

extern "C" int selinv_dinv_noalloc(int32_t s, const double *Lkk, int64_t ld, const double *D,
                                   double *Dinv, int64_t ldo, void *cuda_stream) {
    if (s < 0 || s > kMaxS) return SELINV_ERR_INVALID_ARG;  // beyond the static scratch
    if (s == 0) return SELINV_OK;
    if (!Lkk || !D || !Dinv || ld < s || ldo < s) return SELINV_ERR_INVALID_ARG;
    double *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    k_dinv_noalloc<<<1, 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(s, Lkk, ld, D, Dinv, ldo, scratch);
    return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}
