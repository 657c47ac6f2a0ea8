// Complex symmetric selected inversion on the tensor cores: the operands of
// the real digit contractions for A = A^T with complex values (Sec. II-C:
// plain transposes), and the finisher of the complex diagonal block.
//
// A complex product sum_q X(q, j) Y(q, i) is one real contraction over the
// 2c-long index k' = 2q + part:
//   rows j     of the left operand: (Re X(q, j), -Im X(q, j)) at k' = 2q, 2q + 1
//   rows s + j of the left operand: (Im X(q, j),  Re X(q, j))
//   right operand:                  (Re Y(q, i),  Im Y(q, i))
// so that row j gives Re(X^T Y)(j, i) and row s + j gives Im(X^T Y)(j, i).
// With X = Lhat this left operand serves both A^{-1}_{C,K} = -A^{-1}_{C,C}
// Lhat (k_selinv_tcw, the right operand being the gathered A^{-1}_{C,C}, which
// is symmetric) and the diagonal product Lhat^T A^{-1}_{C,K} (k_diag_tc).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "fixedpoint.cuh"
#include "launch.h"
#include "diag_fin.cuh"
#include "tile_gemm.cuh"

namespace selinv {


// ---------------------------------------------------------------------------
// k_lhat_digits_z: the left operand above for X = Lhat (complex), as fp16
// digit planes in the tcgen05 operand layout: per 16-step of k' and plane
// (the 7 planes of a step one after the other) a block of roundup(2s, 64)
// rows x 16, K-major 8 x 8 core matrices.  One exponent per column j of
// Lhat over both parts (shared by rows j and s + j).  One warp per column;
// work = (problem, (K << 8) | block of 8 columns).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_lhat_digits_z(const ProbDesc *__restrict__ descs,
                                                       const int2 *__restrict__ work, int nwork) {
    grid_dep_wait();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const ProbDesc &P = descs[work[w].x];
    const int K = work[w].y >> 8;
    const int jb = work[w].y & 0xFF;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int j = jb * 8 + warp;
    if (j >= s) return;
    const double2 *Lh = static_cast<const double2 *>(P.LD) + P.panel_off[K] + (int64_t)j * ld + s;
    int E = 0;
    for (int q = lane; q < c; q += 32) {
        const double2 v = Lh[q];
        E = max(E, max(bexp(v.x), bexp(v.y)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) P.colexp[fc + j] = E;
    const int64_t s64 = (2 * s + 63) / 64 * 64;
    const int k16 = (2 * c + 15) / 16 * 16;
    uint16_t *pu = P.lhsu + P.lhsu_off[K];
    for (int kp = lane; kp < k16; kp += 32) {
        const int q = kp >> 1, part = kp & 1;
        double re = 0.0, im = 0.0;
        if (q < c) {
            const double2 v = Lh[q];
            re = part ? -v.y : v.x;   // row j:     (Re, -Im)
            im = part ? v.x : v.y;    // row s + j: (Im,  Re)
        }
        int dr[kDig], di[kDig];
        digits7(re, E, dr);
        digits7(im, E, di);
        const int64_t base = (int64_t)(kp / 16) * kDig * s64 * 16 + ((kp % 16) / 8) * 64 + kp % 8;
        const int r1 = j, r2 = s + j;
        const int64_t o1 = base + (r1 / 8) * 128 + (r1 % 8) * 8, o2 = base + (r2 / 8) * 128 + (r2 % 8) * 8;
#pragma unroll
        for (int i = 0; i < kDig; i++) {
            pu[i * s64 * 16 + o1] = f16_of_int(dr[i]);
            pu[i * s64 * 16 + o2] = f16_of_int(di[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// k_diag_fin_z: A^{-1}_KK = Dinv_K - Lhat^T A^{-1}_{C,K} (complex) from the
// exact sums of k_diag_tc, symmetrized with the plain transpose (Sec. II-C);
// Hermitian: Dinv_K - Lhat^H A^{-1}_{C,K}, symmetrized as (X + X^H) / 2
// (diag_fin_pair).  One CTA per (K, 2 columns).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_diag_fin_z(const ProbDesc *__restrict__ descs,
                                                    const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    diag_fin_pair<true>(descs[it.prob], it.K, 2 * it.tile, 1);
}

cudaError_t launch_lhat_digits_z(const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    k_lhat_digits_z<<<nwork, 256, 0, st>>>(d, work, nwork);
    return cudaGetLastError();
}

cudaError_t launch_diag_fin_z(const ProbDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_diag_fin_z<<<n, 256, 0, st>>>(d, items, n);
    return cudaGetLastError();
}

}  // namespace selinv
