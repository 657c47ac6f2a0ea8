// sm_103a kernels of the selected-inversion traversal (Alg. 1 of the paper):
//   k_linv    L_KK^{-1} and Dinv_K = L_KK^{-T} D_K^{-1} L_KK^{-1}       (Alg. 1 loop 1)
//             (L_KK^{-H} for a Hermitian problem, Sec. II-C; likewise Lhat^H below)
//   k_lhat    Lhat_{C,K} = L_{C,K} L_KK^{-1}, tiled over rows of C       (Alg. 1 loop 1)
//   k_selinv  A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat_{C,K} with the gather of
//             A^{-1}_{C,C} from the ancestors' panels fused into the GEMM,
//             then the split contribution Lhat^T A^{-1}_{C,K} of every row
//             tile, reduced in a fixed order by the last tile of K into
//             A^{-1}_KK = Dinv_K - Lhat^T A^{-1}_{C,K}, symmetrized (Sec. II-C).
// Every kernel works on a list of work items that may mix supernodes of
// several problems (batched pole shifts / matrices) at one tree level.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "launch.h"
#include "tile_gemm.cuh"

namespace selinv {


__device__ inline void latch_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// k_linv: one CTA per supernode.  X = L_KK^{-1} by row-oriented forward
// substitution on all columns at once: row k of X is final after step k-1,
// and step k updates every X(i, j), i > k, j <= k, in parallel.  X stays in
// shared memory when it fits (odd stride: row and column walks hit distinct
// banks), else in the global scratch.  When there is room, the columns of
// L_KK arrive in shared memory 32 at a time, the next block copied
// (cp.async) while the current one is used, so that no step waits on a
// global load: the s - 1 dependent steps are then bound by the FP64 pipe.
// Then the symmetric Dinv(i, j) = sum_{k >= max(i, j)} X(k, i) X(k, j) / D_k,
// lower half computed and mirrored.
// ---------------------------------------------------------------------------
constexpr int kLinvThreads = 256;
constexpr size_t kLinvSmemMax = (128 * 129 + 128 + 64 * 128) * sizeof(double);

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *g) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// LU form of the normalisation (Alg. 1 first loop with U kept separately):
// X = L_KK^{-1} and V = (U_KK^T)^{-1} (U_KK^T is the lower diagonal block of
// Ut, non-unit diagonal) by row-oriented forward substitution, row k of V
// scaled by 1 / U_kk when it is final; Dinv = U_KK^{-1} L_KK^{-1}, entry
// (i, j) = sum_{k >= max(i, j)} V(k, i) X(k, j), the full (nonsymmetric) block.
template <typename T>
__device__ void linv_lu(const ProbDesc &P, int K, int s, int64_t ld, const T *L, T *X, T *LD) {
    const T *U = static_cast<const T *>(P.Ut) + P.panel_off[K];   // U_KK^T(i, k) = U[k*ld + i]
    T *V = static_cast<T *>(P.Vt) + P.linv_off[K];
    for (int e = threadIdx.x; e < s * s; e += kLinvThreads) {
        const int i = e % s, j = e / s;
        X[e] = i == j ? Sc<T>::one() : Sc<T>::zero();
        V[e] = i == j ? Sc<T>::one() : Sc<T>::zero();
    }
    for (int k = 0; k < s; k++) {
        __syncthreads();
        const T ukk = U[(int64_t)k * ld + k];
        if (threadIdx.x == 0 && (is_zero(ukk) || !finite_val(ukk))) latch_status(P.status, SELINV_ERR_ZERO_PIVOT);
        const T r = recip(ukk);
        for (int j = threadIdx.x; j <= k; j += kLinvThreads) V[j * s + k] = mul(V[j * s + k], r);
        __syncthreads();
        const int m = s - 1 - k;
        for (int e = threadIdx.x; e < m * (k + 1); e += kLinvThreads) {
            const int i = k + 1 + e % m, j = e / m;
            msub(X[j * s + i], L[(int64_t)k * ld + i], X[j * s + k]);
            msub(V[j * s + i], U[(int64_t)k * ld + i], V[j * s + k]);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += kLinvThreads) {
        const int i = e % s, j = e / s;
        T acc = Sc<T>::zero();
        for (int k = i > j ? i : j; k < s; k++) madd(acc, V[i * s + k], X[j * s + k]);
        LD[(int64_t)j * ld + i] = acc;
    }
}

// with_dinv = 0: only L_KK^{-1} (k_dinv forms Dinv_K afterwards, spread over tiles)
template <typename T>
__global__ void __launch_bounds__(kLinvThreads) k_linv(const ProbDesc *__restrict__ descs,
                                                       const int2 *__restrict__ work, int nwork,
                                                       size_t smem_cap, int with_dinv) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const ProbDesc &P = descs[work[w].x];
    const int K = work[w].y;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const T *L = static_cast<const T *>(P.L) + P.panel_off[K];
    const T *D = static_cast<const T *>(P.D) + fc;
    T *Li = static_cast<T *>(P.Linv) + P.linv_off[K];
    T *LD = static_cast<T *>(P.LD) + P.panel_off[K];
    if (P.lu) {   // nonsymmetric values: L_KK^{-1}, (U_KK^T)^{-1} and U_KK^{-1} L_KK^{-1} in global memory
        linv_lu<T>(P, K, s, ld, L, Li, LD);
        return;
    }
    const int sp = s | 1;
    const bool in_smem = sizeof(T) * ((size_t)s * sp + s) <= smem_cap;
    const int lx = in_smem ? sp : s;                              // X(i, j) = X[j*lx + i]
    T *X = in_smem ? reinterpret_cast<T *>(smem_raw) : Li;
    T *rD = in_smem ? X + (size_t)s * sp : nullptr;
    for (int e = threadIdx.x; e < s * s; e += kLinvThreads) {
        const int i = e % s, j = e / s;
        X[j * lx + i] = i == j ? Sc<T>::one() : Sc<T>::zero();
    }
    for (int j = threadIdx.x; j < s; j += kLinvThreads) {
        if (is_zero(D[j]) || !finite_val(D[j])) latch_status(P.status, SELINV_ERR_ZERO_PIVOT);
        if (in_smem) rD[j] = recip(D[j]);
    }
    // two blocks of 32 columns of L_KK in shared memory, [column][row]
    const bool stage = in_smem && sizeof(T) * ((size_t)s * sp + s + 64 * (size_t)s) <= smem_cap;
    T *Lb = stage ? rD + s : nullptr;
    const int nb = (s + 31) / 32;
    auto fetch = [&](int b) {   // columns 32 b .. 32 b + 31 (rows below the diagonal) into buffer b & 1
        T *dst = Lb + (size_t)(b & 1) * 32 * s;
        for (int e = threadIdx.x; e < 32 * s; e += kLinvThreads) {
            const int kk = e / s, i = e % s, k = 32 * b + kk;
            if (k < s && i > k) cp_async_elem(dst + e, L + (int64_t)k * ld + i);
        }
        cp_async_commit();
    };
    if (stage) fetch(0);
    __syncthreads();
    for (int k = 0; k + 1 < s; k++) {
        const T *Lk = L + (int64_t)k * ld;       // L(i, k) = Lk[i]
        if (stage) {
            if (k % 32 == 0) {
                // the next block goes out now (its buffer was last read before
                // the previous step's barrier); then this block must be in
                if (k / 32 + 1 < nb) {
                    fetch(k / 32 + 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
            }
            Lk = Lb + (size_t)((k / 32) & 1) * 32 * s + (size_t)(k % 32) * s;
        }
        const int m = s - 1 - k;                 // rows i = k+1 .. s-1
        for (int e = threadIdx.x; e < m * (k + 1); e += kLinvThreads) {
            const int i = k + 1 + e % m, j = e / m;
            msub(X[j * lx + i], Lk[i], X[j * lx + k]);
        }
        __syncthreads();
    }
    if (in_smem)
        for (int e = threadIdx.x; e < s * s; e += kLinvThreads) Li[e] = X[(e / s) * lx + e % s];
    if (!with_dinv) return;
    const bool h = P.herm != 0;
    for (int e = threadIdx.x; e < s * s; e += kLinvThreads) {
        const int i = e % s, j = e / s;
        if (i < j) continue;
        T acc = Sc<T>::zero();
        for (int k = i; k < s; k++)
            madd(acc, mul(cjif(X[i * lx + k], h), in_smem ? rD[k] : recip(D[k])), X[j * lx + k]);
        LD[(int64_t)j * ld + i] = acc;
        LD[(int64_t)i * ld + j] = cjif(acc, h);
    }
}

// ---------------------------------------------------------------------------
// k_dinv: Dinv_K = X^T D_K^{-1} X (X^H for a Hermitian problem), X = L_KK^{-1}
// from k_linv, for the wide supernodes: one 32 x 32 tile (i0 >= j0) of the
// lower triangle per CTA, mirrored; k runs from i0 (X is lower triangular).
// work (problem, K << 8 | tile), tiles row-major over the lower triangle.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_dinv(const ProbDesc *__restrict__ descs, const int2 *__restrict__ work,
                                              int nwork) {
    grid_dep_wait();
    __shared__ T As[32][33], Bs[32][33];
    __shared__ T rD[128];
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const ProbDesc &P = descs[work[w].x];
    const int K = work[w].y >> 8, t = work[w].y & 0xFF;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    int ti = 0, r = t;
    while (r > ti) { r -= ti + 1; ti++; }            // tile t -> (ti, tj), tj <= ti
    const int i0 = ti * 32, j0 = r * 32;
    const T *X = static_cast<const T *>(P.Linv) + P.linv_off[K];   // X(k, j) = X[j*s + k]
    const T *D = static_cast<const T *>(P.D) + fc;
    T *LD = static_cast<T *>(P.LD) + P.panel_off[K];
    const bool h = P.herm != 0;
    for (int k = threadIdx.x; k < s; k += 256) rD[k] = recip(D[k]);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[2][2] = {{Sc<T>::zero(), Sc<T>::zero()}, {Sc<T>::zero(), Sc<T>::zero()}};
    for (int k0 = i0; k0 < s; k0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int q = e % 32, rr = e / 32, k = k0 + q;   // k fastest: contiguous in X's columns
            As[q][rr] = (k < s && i0 + rr < s) ? mul(cjif(X[(int64_t)(i0 + rr) * s + k], h), rD[k]) : Sc<T>::zero();
            Bs[q][rr] = (k < s && j0 + rr < s) ? X[(int64_t)(j0 + rr) * s + k] : Sc<T>::zero();
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 32; q++) {
            const T a0 = As[q][ty], a1 = As[q][ty + 16], b0 = Bs[q][tx], b1 = Bs[q][tx + 16];
            madd(acc[0][0], a0, b0);
            madd(acc[0][1], a0, b1);
            madd(acc[1][0], a1, b0);
            madd(acc[1][1], a1, b1);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            if (i >= s || j >= s || i < j) continue;
            LD[(int64_t)j * ld + i] = acc[u][v];
            LD[(int64_t)i * ld + j] = cjif(acc[u][v], h);
        }
}

// ---------------------------------------------------------------------------
// k_lhat: Lhat(p, :) = L(s + p, :) L_KK^{-1} for the TM rows of one item.
// ---------------------------------------------------------------------------
template <typename T, int TN> struct LoadPanelRows {  // A = L rows s+p0.., k = column of K
    const T *L;
    int64_t ld;
    int s, p0, c;
    __device__ void operator()(int k0, T *As) const {
        for (int e = threadIdx.x; e < kTK * kTM; e += kThreads) {
            const int p = e % kTM, kk = e / kTM;
            const int k = k0 + kk, pr = p0 + p;
            As[kk * kTM + p] = (k < s && pr < c) ? L[(int64_t)k * ld + s + pr] : Sc<T>::zero();
        }
    }
};

template <typename T, int TN> __host__ __device__ constexpr int smem_a_elems() { return kTK * (kTM > TN ? kTM : TN); }
template <typename T, int TN> __host__ __device__ constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(smem_a_elems<T, TN>() + kTK * TN);
}

template <typename T, int TN>
__global__ void __launch_bounds__(kThreads) k_lhat(const ProbDesc *__restrict__ descs,
                                                   const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    using S = Shape<TN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Bs = As + smem_a_elems<T, TN>();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int s = P.super_ptr[K + 1] - P.super_ptr[K];
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    // LU form: a second pass forms Uhat^T = U(K,C)^T (U_KK^T)^{-1}
    for (int side = 0; side < (P.lu ? 2 : 1); side++) {
        const T *L = static_cast<const T *>(side ? P.Ut : P.L) + P.panel_off[K];
        const T *Li = static_cast<const T *>(side ? P.Vt : P.Linv) + P.linv_off[K];
        T *LD = static_cast<T *>(side ? P.LDu : P.LD) + P.panel_off[K];
        T acc[S::MI][S::NJ];
#pragma unroll
        for (int i = 0; i < S::MI; i++)
#pragma unroll
            for (int j = 0; j < S::NJ; j++) acc[i][j] = Sc<T>::zero();
        LoadPanelRows<T, TN> la{L, ld, s, p0, c};
        LoadColMajor<T, TN> lb{Li, (int64_t)s, s, s};
        tile_gemm<T, TN>(s, la, lb, acc, As, Bs);
        const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
#pragma unroll
        for (int i = 0; i < S::MI; i++)
#pragma unroll
            for (int j = 0; j < S::NJ; j++) {
                const int p = p0 + ty + S::TY * i, col = tx + S::TX * j;
                if (p < c && col < s) LD[(int64_t)col * ld + s + p] = acc[i][j];
            }
    }
}

// Split contribution of one row tile to the diagonal block,
// Ptile(i, j) = sum_{p in tile} Lhat(p, i) Y(p, j), written to the partial
// buffer; the last tile of K to arrive reduces the partials in tile order
// (deterministic) into A^{-1}_KK = Dinv_K - sum_t Ptile, symmetrized.
template <typename T, int TN>
__device__ void diag_block(const ProbDesc &P, const Item &it, int K, int s, int64_t ld, int c, int p0,
                           int pm, const T *LDk, T *Zk, T *As, T *Bs) {
    __syncthreads();  // this CTA's rows of A^{-1}_{C,K} are visible to the CTA
    // split contribution of this tile: Ptile(i, j) = sum_{p in tile} Lhat(p, i) Y(p, j)
    // (LU form: Uhat^T(p, i) in place of Lhat(p, i), A^{-1}_KK = U_KK^{-1} L_KK^{-1} - Uhat A^{-1}_{C,K})
    T *part = static_cast<T *>(P.partial) + P.part_off[K] + (int64_t)it.tile * s * s;
    const T *Ak = P.lu ? static_cast<const T *>(P.LDu) + P.panel_off[K] : LDk;
    constexpr int OPT = 8;
    for (int ob = 0; ob < s * s; ob += kThreads * OPT) {
        T pacc[OPT];
#pragma unroll
        for (int o = 0; o < OPT; o++) pacc[o] = Sc<T>::zero();
        for (int pc = 0; pc < pm; pc += kTK) {
            __syncthreads();
            for (int e = threadIdx.x; e < kTK * TN; e += kThreads) {
                const int kk = e % kTK, j = e / kTK;
                const int p = p0 + pc + kk;
                const bool ok = (pc + kk < pm) && j < s;
                As[kk * TN + j] = ok ? cjif(Ak[(int64_t)j * ld + s + p], P.herm != 0) : Sc<T>::zero();   // Lhat (conj.)
                Bs[kk * TN + j] = ok ? Zk[(int64_t)j * ld + s + p] : Sc<T>::zero();        // Y
            }
            __syncthreads();
#pragma unroll
            for (int o = 0; o < OPT; o++) {
                const int e = ob + threadIdx.x + kThreads * o;
                if (e < s * s) {
                    const int i = e % s, j = e / s;
#pragma unroll 4
                    for (int kk = 0; kk < kTK; kk++) madd(pacc[o], As[kk * TN + i], Bs[kk * TN + j]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < OPT; o++) {
            const int e = ob + threadIdx.x + kThreads * o;
            if (e < s * s) part[e] = pacc[o];
        }
    }
    diag_finish<T>(P, K, s, ld, it.ntiles, LDk, Zk, P.lu ? static_cast<T *>(P.Zu) + P.panel_off[K] : nullptr);
}

// ---------------------------------------------------------------------------
// k_selinv: one row tile of C(K).
// Gather: entry (p, q) of A^{-1}_{C,C} is stored, by symmetry, at
// (max(p,q), min(p,q)); with b = min, a = max it sits in the panel of the
// owner of column C[b] at row relidx[prb[b] + a], column address pcb[b].
// ---------------------------------------------------------------------------
template <typename T, int TN>
__device__ void selinv_item(const ProbDesc &P, const Item &it, unsigned char *smem_raw) {
    using S = Shape<TN>;
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Bs = As + smem_a_elems<T, TN>();
    __shared__ int64_t tile_cb[kTM], tile_rb[kTM];
    const int K = it.K;
    const int s = P.super_ptr[K + 1] - P.super_ptr[K];
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;  // rows in this tile (may be <= 0 when c == 0)
    const int64_t pos0 = P.rowptr[K] + s;         // position of C[0] in the row lists
    const T *Zc = static_cast<const T *>(P.Z);
    T *Zk = static_cast<T *>(P.Z) + P.panel_off[K];
    const T *LDk = static_cast<const T *>(P.LD) + P.panel_off[K];

    for (int e = threadIdx.x; e < kTM; e += kThreads) {
        const int p = p0 + e;
        tile_cb[e] = p < c ? P.colbase[pos0 + p] : 0;
        tile_rb[e] = p < c ? P.relbase[pos0 + p] : 0;
    }
    T acc[S::MI][S::NJ];
#pragma unroll
    for (int i = 0; i < S::MI; i++)
#pragma unroll
        for (int j = 0; j < S::NJ; j++) acc[i][j] = Sc<T>::zero();
    if (pm > 0) {
        // LU form: entries above the diagonal from the transposed upper panels
        LoadGather<T, TN> la{Zc, P.colbase + pos0, P.relbase + pos0, P.relidx, tile_cb, tile_rb, p0, c,
                             P.herm != 0, P.lu ? static_cast<const T *>(P.Zu) : nullptr, gather_check(P)};
        LoadColMajor<T, TN> lb{LDk + s, ld, c, s};  // Lhat(q, j) = LD[j*ld + s + q]
        tile_gemm<T, TN>(c, la, lb, acc, As, Bs);
    }
    // write A^{-1}_{C,K} = -acc
    const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
    __shared__ int ymax[TN];
    for (int e = threadIdx.x; e < TN; e += kThreads) ymax[e] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::MI; i++)
#pragma unroll
        for (int j = 0; j < S::NJ; j++) {
            const int p = p0 + ty + S::TY * i, col = tx + S::TX * j;
            if (p < c && col < s) {
                Zk[(int64_t)col * ld + s + p] = neg(acc[i][j]);
                atomicMax(&ymax[col], bexp(acc[i][j]));
            }
        }
    __syncthreads();
    for (int e = threadIdx.x; e < s; e += kThreads)
        if (ymax[e] > 0) atomicMax(&P.colexpY[P.super_ptr[K] + e], ymax[e]);
    if (P.lu && pm > 0) {
        // LU form: A^{-1}(K,C)^T = -A^{-1}(C,C)^T Uhat^T; entry (p, q) of the
        // transposed gather is A^{-1}(C[q], C[p]): the same addresses with the
        // two panel sets exchanged
        T *Zu = static_cast<T *>(P.Zu);
        const T *LDu = static_cast<const T *>(P.LDu) + P.panel_off[K];
#pragma unroll
        for (int i = 0; i < S::MI; i++)
#pragma unroll
            for (int j = 0; j < S::NJ; j++) acc[i][j] = Sc<T>::zero();
        LoadGather<T, TN> lu{Zu, P.colbase + pos0, P.relbase + pos0, P.relidx, tile_cb, tile_rb, p0, c, false, Zc,
                             gather_check(P)};
        LoadColMajor<T, TN> lb{LDu + s, ld, c, s};
        tile_gemm<T, TN>(c, lu, lb, acc, As, Bs);
        T *Zuk = Zu + P.panel_off[K];
#pragma unroll
        for (int i = 0; i < S::MI; i++)
#pragma unroll
            for (int j = 0; j < S::NJ; j++) {
                const int p = p0 + ty + S::TY * i, col = tx + S::TX * j;
                if (p < c && col < s) Zuk[(int64_t)col * ld + s + p] = neg(acc[i][j]);
            }
    }
    diag_block<T, TN>(P, it, K, s, ld, c, p0, pm, LDk, Zk, As, Bs);
}

template <typename T, int TN>
__global__ void __launch_bounds__(kThreads) k_selinv(const ProbDesc *__restrict__ descs,
                                                     const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    selinv_item<T, TN>(descs[it.prob], it, smem_raw);
}

// ---------------------------------------------------------------------------
// Push schedule: the left-looking form of Alg. 2.  A^{-1} starts at zero and
// the levels run root first.  When K's level comes, every ancestor of K has
// pushed its updates into K's rows C, so A^{-1}_{C,K} is complete, and
// k_push_diag forms the diagonal block from it (the Ptile sums of k_selinv).
// k_push then sends K's contributions to every descendant I' whose C' meets
// K's columns, in one owner segment [q0, q1) of C': with the entries (p, q) of
// A^{-1}_{C',C'} whose smaller index lies in the segment (all of them stored
// in K's panel),
//   inner product: rows p in [q0, q1), q in [q0, c')   (A^{-1}_{K,I'} of Alg. 2)
//   outer product: rows p in [q1, c'), q in [q0, q1)   (A^{-1}_{I,I'}, I in C(K))
//   A^{-1}(C'[p], I') -= sum_q A^{-1}(C'[p], C'[q]) Lhat(C'[q], I').
// Over the owners of C' these regions cover every (p, q) once.  Two
// supernodes of one level are never both ancestors of one I', so the writes
// of one launch never meet, and their sources (panels of the level being
// pushed) are not written by it.
// ---------------------------------------------------------------------------
template <typename T, int TN>
__global__ void __launch_bounds__(kThreads) k_push_diag(const ProbDesc *__restrict__ descs,
                                                        const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int s = P.super_ptr[K + 1] - P.super_ptr[K];
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Bs = As + smem_a_elems<T, TN>();
    diag_block<T, TN>(P, it, K, s, ld, c, p0, pm, static_cast<const T *>(P.LD) + P.panel_off[K],
                      static_cast<T *>(P.Z) + P.panel_off[K], As, Bs);
}

// A(pl, k) = A^{-1}(C[p0 + pl], C[q0 + k]); min of the two positions in the
// segment, so the entry sits in the segment owner's panel (conjugated above
// the diagonal for a Hermitian problem)
template <typename T> struct LoadPush {
    const T *Z;
    const int64_t *pcb, *prb;   // per C position of I': column address / relidx base
    const int32_t *relidx;
    int p0, pm, q0, kd;
    bool herm;
    GatherCheck chk;
    __device__ void operator()(int k0, T *As) const {
        for (int e = threadIdx.x; e < kTK * kTM; e += kThreads) {
            const int pl = e % kTM, kk = e / kTM;
            T v = Sc<T>::zero();
            if (pl < pm && k0 + kk < kd) {
                const int p = p0 + pl, q = q0 + k0 + kk;
                const int m = p < q ? p : q, M = p < q ? q : p;
                const int64_t addr = pcb[m] + relidx[prb[m] + M];
                if (chk.ok(addr)) v = Z[addr];
                if (p < q) v = cjif(v, herm);
            }
            As[kk * kTM + pl] = v;
        }
    }
};

// item: K = I', tile = row tile of the region, ntiles = (segment of I' << 1) | inner
template <typename T, int TN>
__global__ void __launch_bounds__(kThreads) k_push(const ProbDesc *__restrict__ descs,
                                                   const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    using S = Shape<TN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Bs = As + smem_a_elems<T, TN>();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int I = it.K;
    const int s = P.super_ptr[I + 1] - P.super_ptr[I];
    const int64_t ld = P.rowptr[I + 1] - P.rowptr[I];
    const int c = (int)(ld - s);
    const int64_t e = P.seg_ptr[I] + (it.ntiles >> 1);
    const bool inner = (it.ntiles & 1) != 0;
    const int q0 = P.seg_start[e];
    const int q1 = e + 1 < P.seg_ptr[I + 1] ? P.seg_start[e + 1] : c;
    const int rb = inner ? q0 : q1, re = inner ? q1 : c;
    const int p0 = rb + it.tile * kTM;
    const int pm = re - p0 < kTM ? re - p0 : kTM;
    if (pm <= 0) return;
    const int kd = (inner ? c : q1) - q0;
    const int64_t pos0 = P.rowptr[I] + s;
    const int64_t off = P.panel_off[I];
    T *Z = static_cast<T *>(P.Z);
    const T *LDi = static_cast<const T *>(P.LD) + off;
    T acc[S::MI][S::NJ];
#pragma unroll
    for (int i = 0; i < S::MI; i++)
#pragma unroll
        for (int j = 0; j < S::NJ; j++) acc[i][j] = Sc<T>::zero();
    LoadPush<T> la{Z, P.colbase + pos0, P.relbase + pos0, P.relidx, p0, pm, q0, kd, P.herm != 0, gather_check(P)};
    LoadColMajor<T, TN> lb{LDi + s + q0, ld, kd, s};   // Lhat(q0 + k, j)
    tile_gemm<T, TN>(kd, la, lb, acc, As, Bs);
    const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
    T *Zi = Z + off;
#pragma unroll
    for (int i = 0; i < S::MI; i++)
#pragma unroll
        for (int j = 0; j < S::NJ; j++) {
            const int pl = ty + S::TY * i, col = tx + S::TX * j;
            if (pl < pm && col < s) {
                T *dst = Zi + (int64_t)col * ld + s + p0 + pl;
                *dst = sub(*dst, acc[i][j]);
            }
        }
}

// ---------------------------------------------------------------------------
// k_selinv_tiny: the whole of Alg. 1's second loop for a supernode with s <= 8
// columns and c <= 64 rows below them, one warp per supernode (eight per CTA):
// the deep levels of a nested-dissection tree hold thousands of these, for
// which a CTA per row tile is mostly synchronisation.  Lane l owns rows l and
// l + 32 of A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat (the gather as in k_selinv,
// 16 columns of C at a time with all their loads in flight -- the kernel is
// bound by the latency of the gathers' dependent loads --, Lhat rows
// broadcast); each entry of the s x s diagonal
// block Dinv - Lhat^T A^{-1}_{C,K} is a warp sum over the lanes' own rows,
// symmetrized through shared memory.  Writes the whole-column exponents for
// the row bounds of later tensor-core gathers.
// ---------------------------------------------------------------------------
constexpr int kTinyS = 8, kTinyC = 64;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ zd warp_sum(zd v) { return make_zd(warp_sum(v.x), warp_sum(v.y)); }

// The supernode's work with its width S known at compile time, and nr = 1
// or 2 row groups of 32 (c <= 32 or c <= 64): no product term is spent on
// columns past s or rows past c (the kernel is bound by the FP64 pipe).
template <typename T, int S>
__device__ __forceinline__ void tiny_one(const ProbDesc &P, const int K, const int lane, T *Xw) {
    const int fc = P.super_ptr[K];
    const int s = S;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int nr = c > 32 ? 2 : 1;
    const int64_t pos0 = P.rowptr[K] + s;
    const bool h = P.herm != 0;
    const T *Zc = static_cast<const T *>(P.Z);
    T *Zk = static_cast<T *>(P.Z) + P.panel_off[K];
    const T *LDk = static_cast<const T *>(P.LD) + P.panel_off[K];
    const int64_t *pcb = P.colbase + pos0, *prb = P.relbase + pos0;
    T acc[2][S];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int j = 0; j < S; j++) acc[r][j] = Sc<T>::zero();
    // the column data of C, lane l holding positions l and l + 32 (the lanes'
    // own rows p use theirs for the entries above the diagonal); then QB
    // columns q at a time: all their relative rows in flight together, then
    // all their values
    const GatherCheck chk = gather_check(P);
    int64_t cbq[2] = {0, 0}, rbq[2] = {0, 0};
#pragma unroll
    for (int r = 0; r < 2; r++)
        if (lane + 32 * r < c) {
            cbq[r] = pcb[lane + 32 * r];
            rbq[r] = prb[lane + 32 * r];
        }
    constexpr int QB = sizeof(T) == sizeof(double) ? 16 : 4;
    for (int q0 = 0; q0 < c; q0 += QB) {
        int32_t rel[2][QB];
#pragma unroll
        for (int u = 0; u < QB; u++) {
            const int q = q0 + u;   // the same in every lane
            const int64_t rq = __shfl_sync(0xffffffffu, q < 32 ? rbq[0] : rbq[1], q & 31);
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const int p = lane + 32 * r;
                // entry (p, q) of A^{-1}_{C,C}: stored at (max, min)
                rel[r][u] = (p < c && q < c) ? P.relidx[p >= q ? rq + p : rbq[r] + q] : 0;
            }
        }
        T v[2][QB];
#pragma unroll
        for (int u = 0; u < QB; u++) {
            const int q = q0 + u;
            const int64_t cq = __shfl_sync(0xffffffffu, q < 32 ? cbq[0] : cbq[1], q & 31);
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const int p = lane + 32 * r;
                v[r][u] = Sc<T>::zero();
                if (p >= c || q >= c) continue;
                const int64_t addr = (p >= q ? cq : cbq[r]) + rel[r][u];
                if (chk.ok(addr)) v[r][u] = Zc[addr];
                if (p < q) v[r][u] = cjif(v[r][u], h);
            }
        }
#pragma unroll
        for (int u = 0; u < QB; u++) {
            const int q = q0 + u;
            if (q >= c) break;
            T lh[S];
#pragma unroll
            for (int j = 0; j < S; j++) lh[j] = LDk[(int64_t)j * ld + s + q];
#pragma unroll
            for (int r = 0; r < 2; r++) {
                if (r >= nr) break;
#pragma unroll
                for (int j = 0; j < S; j++) madd(acc[r][j], v[r][u], lh[j]);
            }
        }
    }
    // A^{-1}_{C,K} = -acc, written; the lanes' own Lhat rows for the diagonal block
    T own[2][S];
    int ye[S];
#pragma unroll
    for (int j = 0; j < S; j++) {
        int e = 0;
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int p = lane + 32 * r;
            const bool ok = p < c;
            acc[r][j] = ok ? neg(acc[r][j]) : Sc<T>::zero();
            own[r][j] = ok ? cjif(LDk[(int64_t)j * ld + s + p], h) : Sc<T>::zero();
            if (ok) {
                Zk[(int64_t)j * ld + s + p] = acc[r][j];
                e = max(e, bexp(acc[r][j]));
            }
        }
        ye[j] = __reduce_max_sync(0xffffffffu, e);
    }
    // X(i, j) = Dinv(i, j) - sum_p Lhat(p, i) A^{-1}_{C,K}(p, j)  (Lhat conjugated: Hermitian)
#pragma unroll
    for (int i = 0; i < S; i++)
#pragma unroll
        for (int j = 0; j < S; j++) {
            T part = Sc<T>::zero();
#pragma unroll
            for (int r = 0; r < 2; r++) {
                if (r >= nr) break;
                madd(part, own[r][i], acc[r][j]);
            }
            part = warp_sum(part);
            if (lane == 0) Xw[j * kTinyS + i] = sub(LDk[(int64_t)j * ld + i], part);
        }
    __syncwarp();
    int ze = 0;
    for (int e = lane; e < s * s; e += 32) {
        const int i = e % s, j = e / s;
        T x = Xw[j * kTinyS + i];
        if (P.symmetrize) x = half(add(x, cjif(Xw[i * kTinyS + j], h)));
        Zk[(int64_t)j * ld + i] = x;
        ze = max(ze, bexp(x));
    }
    // one bound for the whole block and the rows below each column (a column's
    // own maximum would do; a larger bound keeps the gathers exact as well)
    ze = __reduce_max_sync(0xffffffffu, ze);
    if (lane < s) {
        int y = 0;
#pragma unroll
        for (int j = 0; j < S; j++)
            if (j == lane) y = ye[j];
        P.colexpZ[fc + lane] = max(ze, y);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_selinv_tiny(const ProbDesc *__restrict__ descs,
                                                     const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    __shared__ T Xs[8][kTinyS * kTinyS];   // per warp: the unsymmetrized diagonal block
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = blockIdx.x * 8 + warp;
    if (w >= nitems) return;               // the whole warp
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    switch (P.super_ptr[K + 1] - P.super_ptr[K]) {
    case 1: tiny_one<T, 1>(P, K, lane, Xs[warp]); break;
    case 2: tiny_one<T, 2>(P, K, lane, Xs[warp]); break;
    case 3: tiny_one<T, 3>(P, K, lane, Xs[warp]); break;
    case 4: tiny_one<T, 4>(P, K, lane, Xs[warp]); break;
    case 5: tiny_one<T, 5>(P, K, lane, Xs[warp]); break;
    case 6: tiny_one<T, 6>(P, K, lane, Xs[warp]); break;
    case 7: tiny_one<T, 7>(P, K, lane, Xs[warp]); break;
    default: tiny_one<T, 8>(P, K, lane, Xs[warp]); break;
    }
}

cudaError_t launch_selinv_tiny(int dtype, const ProbDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (dtype == SELINV_C128) k_selinv_tiny<zd><<<(n + 7) / 8, 256, 0, st>>>(d, items, n);
    else k_selinv_tiny<double><<<(n + 7) / 8, 256, 0, st>>>(d, items, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_selinv_persist: the whole traversal in one launch.  Work items are listed
// root level first; each CTA claims the next item from a global ticket and,
// before working on supernode K, waits for the completion flag of K's parent
// (set by the last tile of the parent after its diagonal block is written;
// done-ness is transitive up the tree).  An item only waits on items with
// smaller tickets, which running CTAs have already claimed, so the schedule
// cannot deadlock.  Every wait is capped at spin_limit polls; a wait that runs
// out latches SELINV_ERR_TIMEOUT in the status word and the item proceeds (its
// output is then invalid), so the kernel always terminates.  With
// wait_on_unset the waits target a flag that nothing sets (a test of the
// timeout path).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_selinv_persist(const ProbDesc *__restrict__ descs,
                                                             const Item *__restrict__ items,
                                                             const int8_t *__restrict__ buckets, int nitems,
                                                             int *ticket, long long spin_limit,
                                                             int wait_on_unset) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
        __syncthreads();
        const int task = s_task;
        if (task >= nitems) return;
        const Item it = items[task];
        const ProbDesc &P = descs[it.prob];
        const int par = P.sparent[it.K];
        if (par >= 0 && threadIdx.x == 0) {
            const volatile int *flag = P.done + (wait_on_unset ? P.ns : par);
            long long polls = 0;
            while (*flag == 0) {
                if (++polls > spin_limit) {
                    latch_status(P.status, SELINV_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(256);
            }
            __threadfence();
        }
        __syncthreads();
        switch (buckets[task]) {
        case 0: selinv_item<T, 8>(P, it, smem_raw); break;
        case 1: selinv_item<T, 16>(P, it, smem_raw); break;
        case 2: selinv_item<T, 32>(P, it, smem_raw); break;
        case 3: selinv_item<T, 64>(P, it, smem_raw); break;
        default: selinv_item<T, 128>(P, it, smem_raw); break;
        }
    }
}

// debug check of the inputs: latches SELINV_ERR_NONFINITE when any of the n
// doubles is a NaN or an infinity (complex data: both parts)
__global__ void __launch_bounds__(256) k_check_finite(const double *__restrict__ x, int64_t n, int *status) {
    grid_dep_wait();
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[e]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) latch_status(status, SELINV_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_check_finite(const void *x, int64_t n, int *status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_check_finite<<<grid, 256, 0, st>>>(static_cast<const double *>(x), n, status);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_linv_t(const ProbDesc *d, const int2 *work, int nwork, int large, int with_dinv,
                                 cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    // small blocks (s <= 32) need at most 33 KB (X and a staged block of L);
    // large ones get room for s = 128 (real)
    const size_t cap = large ? kLinvSmemMax : (32 * 33 + 32 + 64 * 32) * sizeof(T);
    k_linv<T><<<nwork, kLinvThreads, cap, st>>>(d, work, nwork, cap, with_dinv);
    return cudaGetLastError();
}

cudaError_t launch_linv(int dtype, const ProbDesc *d, const int2 *work, int nwork, int large, cudaStream_t st,
                        int with_dinv) {
    return dtype == SELINV_C128 ? launch_linv_t<zd>(d, work, nwork, large, with_dinv, st)
                                : launch_linv_t<double>(d, work, nwork, large, with_dinv, st);
}

cudaError_t launch_dinv(int dtype, const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    if (dtype == SELINV_C128) k_dinv<zd><<<nwork, 256, 0, st>>>(d, work, nwork);
    else k_dinv<double><<<nwork, 256, 0, st>>>(d, work, nwork);
    return cudaGetLastError();
}

template <typename T, int TN>
static cudaError_t launch_items_t(int kernel, const ProbDesc *d, const Item *items, int n,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    constexpr size_t smem = smem_bytes<T, TN>();
    if (kernel == 0) k_lhat<T, TN><<<n, kThreads, smem, st>>>(d, items, n);
    else if (kernel == 1) k_selinv<T, TN><<<n, kThreads, smem, st>>>(d, items, n);
    else if (kernel == 2) k_push_diag<T, TN><<<n, kThreads, smem, st>>>(d, items, n);
    else k_push<T, TN><<<n, kThreads, smem, st>>>(d, items, n);
    return cudaGetLastError();
}

template <typename T, int TN>
static cudaError_t configure_t() {
    constexpr int smem = (int)smem_bytes<T, TN>();
    cudaError_t e = cudaFuncSetAttribute(k_lhat<T, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_selinv<T, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_push_diag<T, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_push<T, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <typename T>
static cudaError_t configure_dt() {
    cudaError_t e = configure_t<T, 8>();
    if (e == cudaSuccess) e = configure_t<T, 16>();
    if (e == cudaSuccess) e = configure_t<T, 32>();
    if (e == cudaSuccess) e = configure_t<T, 64>();
    if (e == cudaSuccess) e = configure_t<T, 128>();
    return e;
}

template <typename T> constexpr size_t persist_smem() { return smem_bytes<T, 128>(); }

cudaError_t launch_selinv_persist(int dtype, const ProbDesc *d, const Item *items, const int8_t *buckets,
                                  int n, int *ticket, long long spin_limit, int wait_on_unset,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (dtype == SELINV_C128) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_selinv_persist<zd>, kThreads, persist_smem<zd>());
        const int grid = std::max(1, std::min(n, nsm * std::max(per_sm, 1)));
        k_selinv_persist<zd><<<grid, kThreads, persist_smem<zd>(), st>>>(d, items, buckets, n, ticket, spin_limit, wait_on_unset);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_selinv_persist<double>, kThreads, persist_smem<double>());
        const int grid = std::max(1, std::min(n, nsm * std::max(per_sm, 1)));
        k_selinv_persist<double><<<grid, kThreads, persist_smem<double>(), st>>>(d, items, buckets, n, ticket, spin_limit, wait_on_unset);
    }
    return cudaGetLastError();
}

// opt every kernel in to its dynamic shared memory (outside any graph capture)
cudaError_t configure_selinv_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_linv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinvSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_linv<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinvSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_selinv_persist<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persist_smem<double>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_selinv_persist<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persist_smem<zd>());
    if (e == cudaSuccess) e = configure_dt<double>();
    if (e == cudaSuccess) e = configure_dt<zd>();
    return e;
}

template <typename T>
static cudaError_t launch_items_dt(int kernel, int bucket, const ProbDesc *d, const Item *items,
                                   int n, cudaStream_t st) {
    switch (bucket) {
    case 0: return launch_items_t<T, 8>(kernel, d, items, n, st);
    case 1: return launch_items_t<T, 16>(kernel, d, items, n, st);
    case 2: return launch_items_t<T, 32>(kernel, d, items, n, st);
    case 3: return launch_items_t<T, 64>(kernel, d, items, n, st);
    default: return launch_items_t<T, 128>(kernel, d, items, n, st);
    }
}

cudaError_t launch_lhat(int dtype, int bucket, const ProbDesc *d, const Item *items, int n,
                        cudaStream_t st) {
    return dtype == SELINV_C128 ? launch_items_dt<zd>(0, bucket, d, items, n, st)
                                : launch_items_dt<double>(0, bucket, d, items, n, st);
}

cudaError_t launch_selinv(int dtype, int bucket, const ProbDesc *d, const Item *items, int n,
                          cudaStream_t st) {
    return dtype == SELINV_C128 ? launch_items_dt<zd>(1, bucket, d, items, n, st)
                                : launch_items_dt<double>(1, bucket, d, items, n, st);
}

// push schedule: kind 0 = diagonal blocks, 1 = the pushes (bucket of the target's width)
cudaError_t launch_push(int dtype, int kind, int bucket, const ProbDesc *d, const Item *items, int n,
                        cudaStream_t st) {
    return dtype == SELINV_C128 ? launch_items_dt<zd>(2 + kind, bucket, d, items, n, st)
                                : launch_items_dt<double>(2 + kind, bucket, d, items, n, st);
}


}  // namespace selinv
