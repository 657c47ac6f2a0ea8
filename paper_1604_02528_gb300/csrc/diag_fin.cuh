// The diagonal block of a supernode from the exact sums of its tensor-core
// products (Alg. 1: A^{-1}_KK = Dinv_K - Lhat^T A^{-1}_{C,K}, symmetrized as
// in Sec. II-C), for the finisher kernels k_diag_fin (real) and k_diag_fin_z
// (complex).
//
// The sums (hi, lo) per entry (four words for complex values: Re hi, Re lo,
// Im hi, Im lo) hold (Lhat^T Y)(i, j), Y = A^{-1}_{C,K}, on the grid of
// Lhat's column exponent i and Y's column exponent j; bshift is 1 for the
// tcgen05 digit grids and 0 for the mma.sync ones.  Entry (i, j) and its
// mirror come from the same sums in the same order, so the block is exactly
// symmetric.
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "fixedpoint.cuh"
#include "tile_gemm.cuh"

namespace selinv {

// Rows i = i0, i0 + 32, ... (i < i1) of column j of A^{-1}_KK: one warp,
// lanes over the rows; returns the largest exponent of the warp's entries
// (the same in every lane).
template <bool CPLX>
__device__ __forceinline__ int diag_fin_rows(const ProbDesc &P, int K, int j, int bshift, int i0, int i1) {
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    int mj = 0;
    if constexpr (!CPLX) {
        const double *LDk = static_cast<const double *>(P.LD) + P.panel_off[K];
        double *Zk = static_cast<double *>(P.Z) + P.panel_off[K];
        const long long *acc64 = P.dacc + 2 * P.linv_off[K];
        auto prod = [&](int a, int b) -> double {   // (Lhat^T Y)(a, b)
            const long long *q = acc64 + 2 * ((int64_t)b * s + a);
            const long long hi = q[0], lo = q[1];
            const int ey = P.colexpY[fc + b];
            if (ey == 0 || (hi == 0 && lo == 0)) return 0.0;
            const int sc = (P.colexp[fc + a] - 1022) + (ey - 1022) - 14 + bshift;
            return fixed_to_double(hi, lo, sc);
        };
        for (int i = i0; i < i1 && i < s; i += 32) {
            double x = LDk[(int64_t)j * ld + i] - prod(i, j);
            if (P.symmetrize) x = 0.5 * (x + (LDk[(int64_t)i * ld + j] - prod(j, i)));
            Zk[(int64_t)j * ld + i] = x;
            mj = max(mj, bexp(x));
        }
    } else {
        // Hermitian: the sums are those of Lhat^T conj(Y), conjugated here,
        // and the block is symmetrized as (X + X^H) / 2
        const double2 *LDk = static_cast<const double2 *>(P.LD) + P.panel_off[K];
        double2 *Zk = static_cast<double2 *>(P.Z) + P.panel_off[K];
        const long long *acc64 = P.dacc + 4 * P.linv_off[K];
        const bool herm = P.herm;
        auto prod = [&](int a, int b) -> double2 {
            const long long *q = acc64 + 4 * ((int64_t)b * s + a);
            const int ey = P.colexpY[fc + b];
            if (ey == 0) return make_double2(0.0, 0.0);
            const int sc = (P.colexp[fc + a] - 1022) + (ey - 1022) - 14 + bshift;
            const double im = fixed_to_double(q[2], q[3], sc);
            return make_double2(fixed_to_double(q[0], q[1], sc), herm ? -im : im);
        };
        for (int i = i0; i < i1 && i < s; i += 32) {
            const double2 d1 = LDk[(int64_t)j * ld + i], p1 = prod(i, j);
            double2 x = make_double2(d1.x - p1.x, d1.y - p1.y);
            if (P.symmetrize) {
                const double2 d2 = LDk[(int64_t)i * ld + j], p2 = prod(j, i);
                const double2 y = make_double2(d2.x - p2.x, herm ? -(d2.y - p2.y) : d2.y - p2.y);
                x = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
            }
            Zk[(int64_t)j * ld + i] = x;
            mj = max(mj, max(bexp(x.x), bexp(x.y)));
        }
    }
    return __reduce_max_sync(0xffffffffu, mj);
}

// The finisher's CTA (256 threads) for two columns j0, j0 + 1 of K: four
// warps per column, a quarter of its rows each (short chains of dependent
// loads and conversions: the finisher is latency-bound); the column's
// exponent (whole column of K's panel: the block and the rows below) is
// reduced through shared memory.
template <bool CPLX>
__device__ __forceinline__ void diag_fin_pair(const ProbDesc &P, int K, int j0, int bshift) {
    __shared__ int wmax[8];
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int j = j0 + warp / 4, q = warp % 4;
    const int rows = (s + 3) / 4;   // rows per warp, a multiple of 32 or the rest
    const int r0 = ((rows + 31) / 32) * 32 * q;
    int mj = 0;
    if (j < s) mj = diag_fin_rows<CPLX>(P, K, j, bshift, r0 + lane, r0 + ((rows + 31) / 32) * 32);
    if (lane == 0) wmax[warp] = mj;
    __syncthreads();
    if (threadIdx.x < 2 && j0 + (int)threadIdx.x < s) {
        const int t = threadIdx.x;
        const int m = max(max(wmax[4 * t], wmax[4 * t + 1]), max(wmax[4 * t + 2], wmax[4 * t + 3]));
        P.colexpZ[fc + j0 + t] = max(m, P.colexpY[fc + j0 + t]);
    }
}

}  // namespace selinv
