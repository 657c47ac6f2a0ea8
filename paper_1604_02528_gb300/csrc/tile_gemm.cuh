// Shared tile machinery of the FP64 / complex128 kernels: a register-tiled
// GEMM core over shared-memory stages filled by loader functors, and the
// loaders (column-major blocks, panel rows, the indexed gather of a
// symmetric block of A^{-1} -- or of any panel-layout array -- on C x C).
#pragma once

#include "common.cuh"

namespace selinv {

constexpr int kThreads = 256;
constexpr int kTK = 16;

// biased exponent of |x| (0 for zero / subnormal); complex: of the larger part
__device__ __forceinline__ int bexp(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
__device__ __forceinline__ int bexp(zd x) { return max(bexp(x.x), bexp(x.y)); }

// loads that bypass L1 (data written by other CTAs of the same launch)
__device__ inline double ldcg(const double *p) { return __ldcg(p); }
__device__ inline zd ldcg(const zd *p) {
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return make_zd(v.x, v.y);
}

// ---------------------------------------------------------------------------
// register-tiled GEMM core: acc[MI][NJ] += A(TM x kdim) * B(kdim x TN),
// A and B staged tile by tile (TK) in shared memory by loader functors.
// Thread (tx, ty) owns rows ty + TY*i and columns tx + TX*j.
// ---------------------------------------------------------------------------
template <int TN> struct Shape {
    static constexpr int TX = TN < 16 ? TN : 16;
    static constexpr int TY = kThreads / TX;
    static constexpr int MI = kTM / TY;
    static constexpr int NJ = TN / TX;
};

template <typename T, int TN, class LA, class LB>
__device__ inline void tile_gemm(int kdim, const LA &la, const LB &lb,
                                 T (&acc)[Shape<TN>::MI][Shape<TN>::NJ], T *As, T *Bs) {
    using S = Shape<TN>;
    const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
    for (int k0 = 0; k0 < kdim; k0 += kTK) {
        __syncthreads();
        la(k0, As);
        lb(k0, Bs);
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kTK; kk++) {
            T a[S::MI], b[S::NJ];
#pragma unroll
            for (int i = 0; i < S::MI; i++) a[i] = As[kk * kTM + ty + S::TY * i];
#pragma unroll
            for (int j = 0; j < S::NJ; j++) b[j] = Bs[kk * TN + tx + S::TX * j];
#pragma unroll
            for (int i = 0; i < S::MI; i++)
#pragma unroll
                for (int j = 0; j < S::NJ; j++) madd(acc[i][j], a[i], b[j]);
        }
    }
}

// B loader: a column-major block X (ld ldx) restricted to kdim rows, s columns
template <typename T, int TN> struct LoadColMajor {
    const T *X;
    int64_t ldx;
    int kdim, s;
    __device__ void operator()(int k0, T *Bs) const {
        for (int e = threadIdx.x; e < kTK * TN; e += kThreads) {
            const int kk = e % kTK, j = e / kTK;
            const int k = k0 + kk;
            Bs[kk * TN + j] = (k < kdim && j < s) ? X[(int64_t)j * ldx + k] : Sc<T>::zero();
        }
    }
};

// ---------------------------------------------------------------------------
// Gather of entry (p, q) of a symmetric C x C block stored lower in the
// ancestors' panels: at (max(p,q), min(p,q)); with b = min, a = max it sits
// in the panel of the owner of column C[b], column address colbase[b], row
// relidx[relbase[b] + a].  kDoubleDiag doubles the diagonal (reverse-mode
// use, where the symmetric cotangent counts the diagonal twice).
// ---------------------------------------------------------------------------
template <typename T, int TN, bool kDoubleDiag = false> struct LoadGather {
    const T *Z;
    const int64_t *pcb;   // per C position: panel address of column C[q] (+ plan base)
    const int64_t *prb;   // per C position: base into relidx
    const int32_t *relidx;
    const int64_t *tile_cb;  // shared: pcb of the tile's rows
    const int64_t *tile_rb;  // shared: prb of the tile's rows
    int p0, c;
    bool herm = false;    // Hermitian: an entry above the diagonal is the stored one's conjugate
    const T *Zup = nullptr;   // LU form: the entries above the diagonal come from this panel set
    GatherCheck chk{};        // optional bounds check of the addresses
    __device__ void operator()(int k0, T *As) const {
        for (int e = threadIdx.x; e < kTK * kTM; e += kThreads) {
            const int pl = e % kTM, kk = e / kTM;
            const int p = p0 + pl, q = k0 + kk;
            T v = Sc<T>::zero();
            if (p < c && q < c) {
                int64_t addr;
                if (p >= q) addr = pcb[q] + relidx[prb[q] + p];
                else addr = tile_cb[pl] + relidx[tile_rb[pl] + q];
                if (chk.ok(addr)) v = ldcg((p < q && Zup ? Zup : Z) + addr);  // L2: written by other CTAs of a persistent launch
                if (p < q) v = cjif(v, herm);
                if (kDoubleDiag && p == q) v = add(v, v);
            }
            As[kk * kTM + pl] = v;
        }
    }
};

// ---------------------------------------------------------------------------
// After a tile has written its split partial of the diagonal block: the last
// tile of K to arrive (counter) reduces all partials in tile order
// (deterministic) into A^{-1}_KK = Dinv_K - sum_t Ptile, symmetrized, and
// flags K done when a completion array is present.
// ---------------------------------------------------------------------------
// Zuk (LU form): receives the transpose of the block as well
template <typename T>
__device__ void diag_finish(const ProbDesc &P, int K, int s, int64_t ld, int ntiles, const T *LDk, T *Zk,
                            T *Zuk = nullptr) {
    __shared__ int s_last;
    // the last tile of K to finish reduces the partials in tile order
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int prev = atomicAdd(&P.counter[K], 1);
        s_last = (prev == ntiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const T *part0 = static_cast<const T *>(P.partial) + P.part_off[K];
    const int64_t ss = (int64_t)s * s;
    __shared__ int cz[128];   // exponent of each whole column of K's panel
    for (int j = threadIdx.x; j < s; j += kThreads)
        cz[j] = __ldcg(P.colexpY + P.super_ptr[K] + j);   // atomics of this launch
    __syncthreads();
    // a warp per column j, lanes over the rows i >= j: column j's exponent is
    // reduced in the warp, row i's (column i of the mirror) has one lane
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int j = warp; j < s; j += kThreads / 32) {
        int mj = 0;
        for (int i = j + lane; i < s; i += 32) {
            T xij = LDk[(int64_t)j * ld + i], xji = LDk[(int64_t)i * ld + j];
            for (int t = 0; t < ntiles; t++) {
                xij = sub(xij, ldcg(part0 + t * ss + (int64_t)j * s + i));
                xji = sub(xji, ldcg(part0 + t * ss + (int64_t)i * s + j));
            }
            if (P.symmetrize && !Zuk) {   // (X + X^T)/2, or (X + X^H)/2 (the diagonal becomes real)
                const T v = half(add(xij, cjif(xji, P.herm != 0)));
                xij = v;
                xji = cjif(v, P.herm != 0);
            }
            Zk[(int64_t)j * ld + i] = xij;
            Zk[(int64_t)i * ld + j] = xji;
            if (Zuk) {
                Zuk[(int64_t)j * ld + i] = xji;
                Zuk[(int64_t)i * ld + j] = xij;
            }
            mj = max(mj, bexp(xij));
            atomicMax(&cz[i], bexp(xji));
        }
        mj = __reduce_max_sync(0xffffffffu, mj);
        if (lane == 0) atomicMax(&cz[j], mj);
    }
    __syncthreads();
    // exponent of every whole column of K's panel (rows below: atomic max taken
    // when they were written), for the row bounds of the descendants' gathers
    for (int j = threadIdx.x; j < s; j += kThreads) {
        P.colexpZ[P.super_ptr[K] + j] = cz[j];
        P.colexpY[P.super_ptr[K] + j] = 0;
    }
    if (threadIdx.x == 0) P.counter[K] = 0;
    if (P.done) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(&P.done[K], 1);
    }
}

}  // namespace selinv
