// Register-tiled update of one target tile by one owner segment:
//   out(p, q) -= sum_k X(p, k) Y(q, k),  p in [pa, pa + np), q in [st, st + nq), p >= q
// where the rows p of a descendant's C land in the target tile and the
// columns q are the segment's run of C owned by the target supernode.  Used
// by the factorization's Schur update (X = L_CK D_K, Y = L_CK) and by the
// selected-inversion adjoint's reverse gather (X = [Ybar, Lhat], Y = [Lhat,
// Ybar]).  The whole CTA (256 threads) works on B x B output blocks (B = 64,
// or 32 for more CTAs on narrow levels), k staged kSegK at a time in shared
// memory; every output has one owner, the order of the k sum is fixed:
// deterministic.
#pragma once

#include "common.cuh"

namespace selinv {

constexpr int kSegK = 16;
constexpr int kSegB = 64;

template <typename T, int B = kSegB> struct SegSmem {
    T Xs[kSegK][B + 1];
    T Ys[kSegK][B + 1];
};

// x(pl, k) = X(pa + pl, k), y(ql, k) = Y(st + ql, k); out(pl, ql, v) applies
// the update v to the target entry of (pa + pl, st + ql).  The caller
// guarantees np <= B.
template <typename T, class FX, class FY, class FO, int B = kSegB>
__device__ void seg_update(int pa, int np, int st, int nq, int kdim, const FX &x, const FY &y, const FO &out,
                           SegSmem<T, B> &sm) {
    constexpr int R = B / 16;   // outputs per thread along each side
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int q0 = 0; q0 < nq; q0 += B) {
        const int nqc = nq - q0 < B ? nq - q0 : B;
        // columns q of this chunk above every row p of the tile contribute nothing
        if (st + q0 > pa + np - 1) break;
        T acc[R][R];
#pragma unroll
        for (int i = 0; i < R; i++)
#pragma unroll
            for (int j = 0; j < R; j++) acc[i][j] = Sc<T>::zero();
        for (int k0 = 0; k0 < kdim; k0 += kSegK) {
            __syncthreads();
            for (int e = threadIdx.x; e < kSegK * B; e += 256) {
                const int r = e % B, kk = e / B, k = k0 + kk;
                sm.Xs[kk][r] = (r < np && k < kdim) ? x(r, k) : Sc<T>::zero();
                sm.Ys[kk][r] = (r < nqc && k < kdim) ? y(q0 + r, k) : Sc<T>::zero();
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kSegK; kk++) {
                T a[R], b[R];
#pragma unroll
                for (int i = 0; i < R; i++) a[i] = sm.Xs[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < R; j++) b[j] = sm.Ys[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < R; i++)
#pragma unroll
                    for (int j = 0; j < R; j++) madd(acc[i][j], a[i], b[j]);
            }
        }
#pragma unroll
        for (int i = 0; i < R; i++)
#pragma unroll
            for (int j = 0; j < R; j++) {
                const int pl = ty + 16 * i, ql = q0 + tx + 16 * j;
                if (pl < np && ql < nq && pa + pl >= st + ql) out(pl, ql, acc[i][j]);
            }
    }
}

}  // namespace selinv
