// Internal types shared by the host plan code and the sm_103a kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "selinv.h"

namespace selinv {

// Programmatic dependent launch: in the captured level loops every
// kernel-to-kernel edge is a programmatic one, so the next grid is scheduled
// as the previous one drains instead of after a full serialization; each
// kernel waits here, before it reads anything, until its predecessors have
// completed and their memory operations are visible.  A grid launched
// without such an edge passes at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


// complex128 as two doubles.  Transposes are plain for complex symmetric
// problems (A = A^T); a Hermitian problem (ProbDesc::herm) conjugates every
// transposed factor (cjif below).
struct __align__(16) zd {
    double x, y;
};

__host__ __device__ inline zd make_zd(double a, double b) { zd r; r.x = a; r.y = b; return r; }

template <typename T> struct Sc;
template <> struct Sc<double> {
    static __host__ __device__ inline double zero() { return 0.0; }
    static __host__ __device__ inline double one() { return 1.0; }
    static constexpr int kWords = 1;  // doubles per element
};
template <> struct Sc<zd> {
    static __host__ __device__ inline zd zero() { return make_zd(0.0, 0.0); }
    static __host__ __device__ inline zd one() { return make_zd(1.0, 0.0); }
    static constexpr int kWords = 2;
};

// acc += a * b
__host__ __device__ inline void madd(double &acc, double a, double b) { acc = fma(a, b, acc); }
__host__ __device__ inline void madd(zd &acc, zd a, zd b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc -= a * b
__host__ __device__ inline void msub(double &acc, double a, double b) { acc = fma(-a, b, acc); }
__host__ __device__ inline void msub(zd &acc, zd a, zd b) {
    acc.x = fma(-a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(-a.x, b.y, fma(-a.y, b.x, acc.y));
}
__host__ __device__ inline double add(double a, double b) { return a + b; }
__host__ __device__ inline zd add(zd a, zd b) { return make_zd(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double sub(double a, double b) { return a - b; }
__host__ __device__ inline zd sub(zd a, zd b) { return make_zd(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double mul(double a, double b) { return a * b; }
__host__ __device__ inline zd mul(zd a, zd b) {
    return make_zd(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double neg(double a) { return -a; }
__host__ __device__ inline zd neg(zd a) { return make_zd(-a.x, -a.y); }
__host__ __device__ inline double half(double a) { return 0.5 * a; }
__host__ __device__ inline zd half(zd a) { return make_zd(0.5 * a.x, 0.5 * a.y); }
__host__ __device__ inline double scal(double a, double s) { return a * s; }
__host__ __device__ inline zd scal(zd a, double s) { return make_zd(a.x * s, a.y * s); }
// 1 / a (complex: by the textbook formula conj(a) / |a|^2 with scaling)
__host__ __device__ inline double recip(double a) { return 1.0 / a; }
__host__ __device__ inline zd recip(zd a) {
    double m = fabs(a.x) > fabs(a.y) ? fabs(a.x) : fabs(a.y);
    double s = m > 0 ? 1.0 / m : 0.0;
    double ax = a.x * s, ay = a.y * s;
    double d = ax * ax + ay * ay;
    return make_zd(ax * s / d, -ay * s / d);
}
// conjugate (identity for real values); cjif: only when h is set
__host__ __device__ inline double cj(double a) { return a; }
__host__ __device__ inline zd cj(zd a) { return make_zd(a.x, -a.y); }
template <typename T> __host__ __device__ inline T cjif(T a, bool h) { return h ? cj(a) : a; }
__host__ __device__ inline bool is_zero(double a) { return a == 0.0; }
__host__ __device__ inline bool is_zero(zd a) { return a.x == 0.0 && a.y == 0.0; }
__host__ __device__ inline bool finite_val(double a) { return isfinite(a); }
__host__ __device__ inline bool finite_val(zd a) { return isfinite(a.x) && isfinite(a.y); }

// Device view of one problem (one plan + one set of numeric buffers).
struct ProbDesc {
    // plan (device arrays)
    const int32_t *super_ptr;   // [ns+1]
    const int64_t *rowptr;      // [ns+1]
    const int32_t *rows;        // row lists
    const int64_t *panel_off;   // [ns+1]
    const int64_t *colbase;     // [n] panel address of column j in its owner's panel
    const int64_t *relbase;     // [rowptr[ns]] per C position: rel_ptr(segment) - seg_start
    const int32_t *relidx;      // relative row indices
    const int64_t *linv_off;    // [ns+1] offsets of L_KK^{-1} blocks (s*s each)
    const int64_t *part_off;    // [ns] offset of K's split partials inside its level
    const int32_t *sparent;     // [ns]
    const int64_t *seg_ptr;     // [ns+1] owner segments of each C (push schedule)
    const int32_t *seg_start;   // first C position of each segment
    // numeric buffers
    const void *L;              // panels
    const void *D;              // [n]
    void *Z;                    // panels (output A^{-1}; the gather source)
    void *Yout;                 // panels: where the tcgen05 gather-GEMM writes -A^{-1}(C,C) B (= Z by default)
    void *LD;                   // panels: Dinv_K in the diagonal block, Lhat below
    void *Linv;                 // sum s^2
    void *partial;              // split-k partials of A^{-1}_KK
    int *counter;               // [ns] tiles done per supernode
    int *done;                  // [ns] completion flags (persistent schedule)
    int *status;                // latched error code
    uint16_t *lhs;              // fp16 digit planes of Lhat, [plane][column][q] (mma.sync kernels)
    const int64_t *lhs_off;     // [ns+1] offsets into lhs (elements)
    uint16_t *lhsu;             // the same digits in the tcgen05 operand layout: per 16-row step
                                // and plane (the 7 planes of a step one after the other) a block
                                // of roundup(s, 64) columns x 16 q, K-major 8 x 8 core matrices
                                // (column groups 256 bytes apart); zero padding
    const int64_t *lhsu_off;    // [ns+1] offsets into lhsu (elements)
    int *colexp;                // [n] biased exponent of each column of Lhat
    int *colexpY;               // [n] biased exponent of each column of A^{-1}_{C,K} (atomic max)
    long long *dacc;            // [2 * sum s^2] exact int64 sums of the diagonal-block products
    int *colexpZ;               // [n] biased exponent of each whole column of the A^{-1} panels
    uint16_t *linvd;            // bf16 digit planes of L_KK^{-1} (tensor-core Lhat)
    const int64_t *linvd_off;   // [ns+1]
    int *linvexp;               // [n] column exponents of L_KK^{-1}
    long long *yacc;            // [2 * nnz] exact int64 sums of split contractions, zero between calls
    int *tcount;                // [sum ntiles] arrivals per (K, row tile), zero between calls
    const int64_t *tile_base;   // [ns+1] prefix sums of the row tiles of each supernode
    int32_t ns, n;
    int64_t nnz;                // panel entries (every gather address lies in [0, nnz))
    int32_t check_gather;       // 1: bounds-check gather addresses (debug_checks bit 2)
    int32_t dtype;              // element type: SELINV_F64 or SELINV_C128
    int32_t prod_op;            // product mode of the transposed tcgen05 kernel (out = LD):
                                // 0: out = acc, 1: out -= acc, 2: out = Yout - acc
    int32_t symmetrize;
    int32_t herm;               // complex Hermitian (SELINV_C128H): conjugate transposes
    // nonsymmetric values (LU form): U transposed in the panel layout, the
    // upper part of A^{-1} transposed, Uhat^T, and (U_KK^T)^{-1} blocks
    int32_t lu;
    const void *Ut;
    void *Zu;
    void *LDu;
    void *Vt;
};

// One unit of work of a tiled kernel: rows [tile*TM, tile*TM+TM) of C(K).
struct Item {
    int32_t prob;
    int32_t K;
    int32_t tile;
    int32_t ntiles;
};

constexpr int kTM = 64;   // rows of C per work item
constexpr int kDiagCols = 32;   // columns j per work item of the tensor-core diagonal block
// slab slot of a split-k tcgen05 item (int64 words): (hi, lo) of a 128 x 64 tile, then 128 row exponents
constexpr long long kTcSlotWords = 2 * 128 * 64 + 64;

#ifdef __CUDACC__
// Optional bounds check of gather addresses (debug_checks bit 2): an address
// outside the panel array latches SELINV_ERR_BAD_INDEX and is not read.
struct GatherCheck {
    int64_t nnz = 0;
    int *status = nullptr;
    int on = 0;
    __device__ __forceinline__ bool ok(int64_t addr) const {
        if (!on || (addr >= 0 && addr < nnz)) return true;
        atomicCAS(status, 0, SELINV_ERR_BAD_INDEX);
        return false;
    }
};
__device__ __forceinline__ GatherCheck gather_check(const ProbDesc &P) {
    GatherCheck g;
    g.nnz = P.nnz;
    g.status = P.status;
    g.on = P.check_gather;
    return g;
}

// atomicMax on a shared slot that every active lane of the warp targets: one
// atomic per warp instead of one per lane (the lanes would serialize on it)
__device__ __forceinline__ void warp_uniform_atomic_max(int *slot, int v) {
    const unsigned mask = __activemask();
    const int m = __reduce_max_sync(mask, v);
    if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicMax(slot, m);
}
#endif

// Size class of a supernode's width s: the column tile TN of its kernels.
inline int bucket_of(int s) {
    if (s <= 8) return 0;
    if (s <= 16) return 1;
    if (s <= 32) return 2;
    if (s <= 64) return 3;
    return 4;
}
constexpr int kNumBuckets = 5;
constexpr int kBucketTN[kNumBuckets] = {8, 16, 32, 64, 128};

}  // namespace selinv
