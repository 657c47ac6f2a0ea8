// FP64-exact contraction A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat_{C,K} on the fp16
// tensor cores (mma.sync m16n8k16, fp32 accumulate).
//
// GB300's FP64 pipe delivers ~1.26 TFLOP/s, while its 16-bit tensor path is
// hundreds of times faster.  Each FP64 operand is cut, without rounding
// error, into 7 balanced base-256 digits in [-128, 128] on a fixed-point
// grid shared by its row (A: the gathered A^{-1}_{C,C}, exponent = row
// maximum) or its column (B: Lhat, exponent = column maximum).  Every digit
// is exact in fp16 and every digit product (<= 2^14) is exact in fp32.
// Products of digit pairs (i, j) with i + j = g share the scale 2^{-8g}, so
// they are summed into one fp32 accumulator per g; with at most 7 pairs per
// g and 128 k-values between flushes the sums stay below 2^24 and are
// therefore exact.  Every 128 k-values the 7 accumulators are folded exactly
// into two int64 words per output element; the FP64 result is formed once
// at the end.  Pairs with i + j > 6 are dropped: the result carries
// 2^-53-level error relative to (row max) x (column max), like a DGEMM with
// a max-norm bound.  FP64 accumulation is kept throughout (the int64 sums
// are exact), as the tree recursion propagates error.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"
#include "launch.h"
#include "tile_gemm.cuh"
#include "fixedpoint.cuh"
#include "diag_fin.cuh"

namespace selinv {

constexpr int kOzK = 16;         // k per mma step
constexpr int kFlushSteps = 8;   // 128 k per exact fp32 chunk
constexpr int kApad = 24;        // smem row stride (fp16) of a 16-wide k slab: conflict-free
constexpr int kOzThreads = 256;

// ---------------------------------------------------------------------------
// k_lhat_digits: digit planes of Lhat_{C,K} (per column j: exponent over all
// q) in the tcgen05 operand layout and, unless the work item says that only
// that one is read, in the mma.sync layout plane[j][q] (q contiguous, padded
// to c16 with zeros).  One CTA per 8 columns: a warp per column finds its
// exponent, then each thread cuts 8 consecutive q of one column, whose digits
// of a plane are one 16-byte store in both layouts.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_lhat_digits(const ProbDesc *__restrict__ descs,
                                                     const int2 *__restrict__ work, int nwork) {
    grid_dep_wait();
    __shared__ int colE[8];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const ProbDesc &P = descs[work[w].x];
    const int K = work[w].y >> 8;           // (K << 8) | only_u << 7 | column block of 8
    const int jb = work[w].y & 0x7F;
    const bool both = !(work[w].y & 0x80);   // also the mma.sync layout
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int c16 = (c + 15) & ~15;
    const int j0 = jb * 8, nj = s - j0 < 8 ? s - j0 : 8;
    const double *LDk = static_cast<const double *>(P.LD) + P.panel_off[K] + s;   // Lhat(q, j) = LDk[j*ld + q]
    if (warp < nj) {
        const double *Lh = LDk + (int64_t)(j0 + warp) * ld;
        int E = 0;
        for (int q = lane; q < c; q += 32) E = max(E, bexp(Lh[q]));
#pragma unroll
        for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
        if (lane == 0) {
            colE[warp] = E;
            P.colexp[fc + j0 + warp] = E;
        }
    }
    __syncthreads();
    uint16_t *pl = P.lhs + P.lhs_off[K];
    const int64_t plane = (int64_t)s * c16;
    // tcgen05 layout: block (step, plane) of s64 x 16 (the 7 planes of a step
    // one after the other), column group j/8 at 128 elements, k group
    // (q % 16) / 8 at 64, row j % 8 at 8, q % 8
    uint16_t *pu = P.lhsu + P.lhsu_off[K];
    const int64_t s64 = (s + 63) / 64 * 64;
    for (int e = threadIdx.x; e < 8 * (c16 / 8); e += 256) {
        const int jl = e % 8, q0 = (e / 8) * 8, j = j0 + jl;
        if (jl >= nj) continue;
        const double *Lh = LDk + (int64_t)j * ld;
        uint32_t h[kDig][4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            int d0[kDig], d1[kDig];
            digits7(q0 + t < c ? Lh[q0 + t] : 0.0, colE[jl], d0);
            digits7(q0 + t + 1 < c ? Lh[q0 + t + 1] : 0.0, colE[jl], d1);
#pragma unroll
            for (int i = 0; i < kDig; i++) h[i][t / 2] = f16_of_int(d0[i]) | (f16_of_int(d1[i]) << 16);
        }
        const int64_t ub = (int64_t)(q0 / 16) * kDig * s64 * 16 + (j / 8) * 128 + ((q0 % 16) / 8) * 64 + (j % 8) * 8;
#pragma unroll
        for (int i = 0; i < kDig; i++) {
            const uint4 v = make_uint4(h[i][0], h[i][1], h[i][2], h[i][3]);
            *reinterpret_cast<uint4 *>(pu + i * s64 * 16 + ub) = v;
            if (both) *reinterpret_cast<uint4 *>(pl + i * plane + (int64_t)j * c16 + q0) = v;
        }
    }
}

__device__ __forceinline__ void mma_f16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// ---------------------------------------------------------------------------
// Entry (p, q) of A^{-1}_{C,C} gathered from the ancestors' panels: stored at
// (max, min) by symmetry; (p, q) are positions in C(K), pl = p - p0.
// ---------------------------------------------------------------------------
struct Gather {
    const double *Z;
    const int64_t *pcb, *prb;        // per C position of K
    const int32_t *relidx;
    const int64_t *tile_cb, *tile_rb; // the tile's rows (shared memory)
    int p0, c;
    GatherCheck chk;
    __device__ __forceinline__ double operator()(int pl, int q) const {
        const int p = p0 + pl;
        if (p >= c || q >= c) return 0.0;
        const int64_t addr = p >= q ? pcb[q] + relidx[prb[q] + p] : tile_cb[pl] + relidx[tile_rb[pl] + q];
        return chk.ok(addr) ? Z[addr] : 0.0;
    }
};

// ---------------------------------------------------------------------------
// k_selinv_oz<TN>: one (K, row tile of 64, column tile of TN, k-range) item.
// Items carry tile = (row_tile * ncol + col_tile) * nsplit + k_split and
// ntiles = nsplit.  8 warps: warp w owns m-tile (w % 4) and n-tiles
// (w / 4) + 2 t, t < TN/16.  The k loop is double buffered: the gather for
// step + 1 is issued before the tensor-core work of step.  With nsplit > 1
// the k-ranges of one row tile add their exact int64 sums into a global
// buffer (integer atomics: order independent) and the last one to arrive
// writes A^{-1}_{C,K} for the whole row tile.
// ---------------------------------------------------------------------------
template <int TN> struct OzShape {
    static constexpr int NT = TN / 16;   // n-tiles (of 8) per warp
};

template <int TN>
__global__ void __launch_bounds__(kOzThreads, 1) k_selinv_oz(const ProbDesc *__restrict__ descs,
                                                             const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    constexpr int NT = OzShape<TN>::NT;
    constexpr int ABUF = kDig * kTM * kApad, BBUF = kDig * TN * kApad;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // layout: A digits [2][7][64][kApad] fp16 | B digits [2][7][TN][kApad] fp16 |
    //         acc hi/lo [64][TN] int64 x 2 | row exponents [64] int
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Bs = As + 2 * ABUF;
    long long *Hi = reinterpret_cast<long long *>(Bs + 2 * BBUF);
    long long *Lo = Hi + kTM * TN;
    int *rowE = reinterpret_cast<int *>(Lo + kTM * TN);
    __shared__ int64_t tile_cb[kTM], tile_rb[kTM];
    __shared__ int s_last;

    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int c16 = (c + 15) & ~15;
    const int ncol = (s + TN - 1) / TN;
    const int nsplit = it.ntiles;
    const int ksp = it.tile % nsplit;
    const int ct = (it.tile / nsplit) % ncol;
    const int tile = it.tile / nsplit / ncol;
    const int p0 = tile * kTM, n0 = ct * TN;
    const int64_t pos0 = P.rowptr[K] + s;
    const int nsteps = c16 / kOzK;
    const int chunk = ((nsteps + nsplit - 1) / nsplit + kFlushSteps - 1) / kFlushSteps * kFlushSteps;
    const int st0 = ksp * chunk;
    const int st1 = st0 + chunk < nsteps ? st0 + chunk : nsteps;

    // Row exponents of the gathered block, bounded without gathering: entry
    // (p, q) sits in the ancestor panel column C[min(p, q)], so row p is bounded
    // by the largest whole-column exponent over C[0..p].
    __shared__ int s_pre;
    if (threadIdx.x == 0) s_pre = 0;
    __syncthreads();
    {
        int e = 0;
        for (int q = threadIdx.x; q < p0 && q < c; q += kOzThreads) e = max(e, P.colexpZ[P.rows[pos0 + q]]);
        if (e) atomicMax(&s_pre, e);
    }
    for (int e = threadIdx.x; e < kTM; e += kOzThreads) {
        const int p = p0 + e;
        tile_cb[e] = p < c ? P.colbase[pos0 + p] : 0;
        tile_rb[e] = p < c ? P.relbase[pos0 + p] : 0;
        rowE[e] = p < c ? P.colexpZ[P.rows[pos0 + p]] : 0;
    }
    for (int e = threadIdx.x; e < kTM * TN; e += kOzThreads) { Hi[e] = 0; Lo[e] = 0; }
    __syncthreads();
    if (threadIdx.x < 32) {                   // prefix max over the tile's 64 rows
        int lo = max(rowE[threadIdx.x], s_pre), hi = rowE[threadIdx.x + 32];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, lo, o);
            if ((int)threadIdx.x >= o) lo = max(lo, v);
        }
        const int carry = __shfl_sync(0xffffffffu, lo, 31);
        hi = max(hi, carry);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, hi, o);
            if ((int)threadIdx.x >= o) hi = max(hi, v);
        }
        rowE[threadIdx.x] = lo;
        rowE[threadIdx.x + 32] = hi;
    }
    __syncthreads();
    const Gather g{static_cast<const double *>(P.Z), P.colbase + pos0, P.relbase + pos0, P.relidx,
                   tile_cb, tile_rb, p0, c, gather_check(P)};

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int mt = warp % 4;                  // m-tile: rows mt*16 .. +15
    const int grp = lane / 4, qd = lane % 4;
    // this thread's gather slots: row gl, k offsets gk, gk+1, gk+8, gk+9
    const int gl = threadIdx.x % kTM, gk = (threadIdx.x / kTM) * 2;
    float acc[NT][kDig][4];
#pragma unroll
    for (int t = 0; t < NT; t++)
#pragma unroll
        for (int gg = 0; gg < kDig; gg++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[t][gg][r] = 0.f;

    const uint16_t *Bg = P.lhs + P.lhs_off[K];
    const int64_t bplane = (int64_t)s * c16;
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if (st0 < st1) {
        const int k0 = st0 * kOzK;
        v0 = g(gl, k0 + gk); v1 = g(gl, k0 + gk + 1); v2 = g(gl, k0 + gk + 8); v3 = g(gl, k0 + gk + 9);
    }
    for (int step = st0; step < st1; step++) {
        const int k0 = step * kOzK;
        const int buf = (step - st0) & 1;
        uint16_t *Ab = As + buf * ABUF;
        uint16_t *Bb = Bs + buf * BBUF;
        // B digits: plane i, column n0 + j, q = k0 .. k0 + 15 (two 16-byte halves)
        for (int e = threadIdx.x; e < kDig * TN * 2; e += kOzThreads) {
            const int half = e & 1, j = (e >> 1) % TN, i = (e >> 1) / TN;
            uint16_t *dst = Bb + (i * TN + j) * kApad + half * 8;
            if (n0 + j < s) cp_async16(dst, Bg + i * bplane + (int64_t)(n0 + j) * c16 + k0 + half * 8);
            else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        }
        // A digits of this step from the values gathered during the previous step
        {
            int d0[kDig], d1[kDig];
            const int E = rowE[gl];
            digits7(v0, E, d0);
            digits7(v1, E, d1);
#pragma unroll
            for (int i = 0; i < kDig; i++)
                *reinterpret_cast<uint32_t *>(Ab + (i * kTM + gl) * kApad + gk) =
                    f16_of_int(d0[i]) | (f16_of_int(d1[i]) << 16);
            digits7(v2, E, d0);
            digits7(v3, E, d1);
#pragma unroll
            for (int i = 0; i < kDig; i++)
                *reinterpret_cast<uint32_t *>(Ab + (i * kTM + gl) * kApad + gk + 8) =
                    f16_of_int(d0[i]) | (f16_of_int(d1[i]) << 16);
        }
        // gather of the next step, in flight during this step's tensor-core work
        if (step + 1 < st1) {
            const int k1 = k0 + kOzK;
            v0 = g(gl, k1 + gk); v1 = g(gl, k1 + gk + 1); v2 = g(gl, k1 + gk + 8); v3 = g(gl, k1 + gk + 9);
        }
        cp_async_wait_all();
        __syncthreads();
        // 28 digit pairs (i + j <= 6) per n-tile; consecutive mma target
        // different accumulators (group i + j varies fastest, then the n-tile)
        uint32_t b[NT][kDig][2];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const int nt = (warp / 4) + 2 * t;  // n-tile index (8 columns)
#pragma unroll
            for (int j = 0; j < kDig; j++) {
                const uint16_t *bb = Bb + (j * TN + nt * 8 + grp) * kApad;
                b[t][j][0] = *reinterpret_cast<const uint32_t *>(bb + qd * 2);
                b[t][j][1] = *reinterpret_cast<const uint32_t *>(bb + qd * 2 + 8);
            }
        }
#pragma unroll
        for (int i = 0; i < kDig; i++) {
            const uint16_t *base = Ab + (i * kTM + mt * 16) * kApad;
            const uint32_t a0 = *reinterpret_cast<const uint32_t *>(base + grp * kApad + qd * 2);
            const uint32_t a1 = *reinterpret_cast<const uint32_t *>(base + (grp + 8) * kApad + qd * 2);
            const uint32_t a2 = *reinterpret_cast<const uint32_t *>(base + grp * kApad + qd * 2 + 8);
            const uint32_t a3 = *reinterpret_cast<const uint32_t *>(base + (grp + 8) * kApad + qd * 2 + 8);
#pragma unroll
            for (int t = 0; t < NT; t++)
#pragma unroll
                for (int j = 0; i + j < kDig; j++)
                    mma_f16(acc[t][i + j], a0, a1, a2, a3, b[t][j][0], b[t][j][1]);
        }
        // fold the exact fp32 group sums into the int64 accumulators (each
        // element has one owning thread: no synchronization needed)
        if ((step - st0 + 1) % kFlushSteps == 0 || step + 1 == st1) {
#pragma unroll
            for (int t = 0; t < NT; t++) {
                const int nt = (warp / 4) + 2 * t;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int row = mt * 16 + grp + (r >= 2 ? 8 : 0);
                    const int col = nt * 8 + qd * 2 + (r & 1);
                    long long gq[kDig];
#pragma unroll
                    for (int q = 0; q < kDig; q++) { gq[q] = (long long)__float2int_rn(acc[t][q][r]); acc[t][q][r] = 0.f; }
                    Hi[row * TN + col] += (gq[0] << 16) + (gq[1] << 8) + gq[2];
                    Lo[row * TN + col] += (gq[3] << 24) + (gq[4] << 16) + (gq[5] << 8) + gq[6];
                }
            }
        }
    }
    __shared__ int ymax[128];
    for (int e = threadIdx.x; e < 128; e += kOzThreads) ymax[e] = 0;
    __syncthreads();
    double *Zk = static_cast<double *>(P.Z) + P.panel_off[K];
    // Y = -(A^{-1}_{C,C} Lhat) in FP64: scale 2^(e_p + f_j - 14) (e = E - 1022)
    auto emit = [&](int row, int j, long long hi, long long lo) {
        const int sc = (rowE[row] - 1022) + (P.colexp[fc + j] - 1022) - 14;
        const double y = fixed_to_double(hi, lo, sc);
        Zk[(int64_t)j * ld + s + p0 + row] = -y;
        warp_uniform_atomic_max(&ymax[j], bexp(y));   // the lanes of a warp share column j
    };
    if (nsplit == 1) {
        for (int e = threadIdx.x; e < kTM * TN; e += kOzThreads) {
            const int row = e % kTM, col = e / kTM;
            if (p0 + row < c && n0 + col < s) emit(row, n0 + col, Hi[row * TN + col], Lo[row * TN + col]);
        }
    } else {
        long long *Yacc = P.yacc + 2 * P.panel_off[K];    // (hi, lo) per element of K's panel
        for (int e = threadIdx.x; e < kTM * TN; e += kOzThreads) {
            const int row = e % kTM, col = e / kTM;
            if (p0 + row >= c || n0 + col >= s) continue;
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(Yacc + 2 * ((int64_t)(n0 + col) * ld + s + p0 + row));
            if (Hi[row * TN + col]) atomicAdd(dst, (unsigned long long)Hi[row * TN + col]);
            if (Lo[row * TN + col]) atomicAdd(dst + 1, (unsigned long long)Lo[row * TN + col]);
        }
        __threadfence();
        __syncthreads();
        int *ctr = P.tcount + P.tile_base[K] + tile;
        if (threadIdx.x == 0) s_last = (atomicAdd(ctr, 1) == ncol * nsplit - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        for (int e = threadIdx.x; e < kTM * s; e += kOzThreads) {
            const int row = e % kTM, j = e / kTM;
            if (p0 + row >= c) continue;
            unsigned long long *q = reinterpret_cast<unsigned long long *>(Yacc + 2 * ((int64_t)j * ld + s + p0 + row));
            const long long hi = (long long)__ldcg(q), lo = (long long)__ldcg(q + 1);
            q[0] = 0ull;
            q[1] = 0ull;
            emit(row, j, hi, lo);
        }
        if (threadIdx.x == 0) *ctr = 0;
    }
    __syncthreads();
    // column exponents of A^{-1}_{C,K} over all row tiles (used by the diagonal block)
    for (int j = threadIdx.x; j < s; j += kOzThreads)
        if (ymax[j] > 0) atomicMax(&P.colexpY[fc + j], ymax[j]);
}

// ---------------------------------------------------------------------------
// k_linv_digits: fp16 digit planes of L_KK^{-1} for the tensor-core Lhat
// product: per column j, exponent over k; layout plane[j][k], k padded to s16
// (k_lhat_oz), or, when the work item says so, the tcgen05 operand layout of
// the transposed product (rows j, k in 16-steps).  One warp per column.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_linv_digits(const ProbDesc *__restrict__ descs,
                                                     const int2 *__restrict__ work, int nwork) {
    grid_dep_wait();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const ProbDesc &P = descs[work[w].x];
    const int K = work[w].y >> 8;
    const int jb = work[w].y & 0x7F;
    const bool tcl = work[w].y & 0x80;      // the tcgen05 operand layout
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int s16 = (s + 15) & ~15;
    const int j = jb * 8 + warp;
    if (j >= s) return;
    const double *X = static_cast<const double *>(P.Linv) + P.linv_off[K] + (int64_t)j * s;  // X(k, j)
    int E = 0;
    for (int k = lane; k < s; k += 32) E = max(E, bexp(X[k]));
#pragma unroll
    for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) P.linvexp[fc + j] = E;
    uint16_t *pl = P.linvd + P.linvd_off[K];
    const int64_t plane = (int64_t)s * s16;
    for (int k = lane; k < s16; k += 32) {
        int d[kDig];
        if (k < s) digits7(X[k], E, d);
        else {
#pragma unroll
            for (int i = 0; i < kDig; i++) d[i] = 0;
        }
        if (tcl) {
            // rows j, k in 16-steps: per step the 7 planes of s64 x 16 one
            // after the other, K-major 8 x 8 core matrices
            const int64_t s64 = (s + 63) / 64 * 64;
            const int64_t ub = (int64_t)(k / 16) * kDig * s64 * 16 + (j / 8) * 128 + ((k % 16) / 8) * 64 + (j % 8) * 8 + k % 8;
#pragma unroll
            for (int i = 0; i < kDig; i++) pl[i * s64 * 16 + ub] = (uint16_t)f16_of_int(d[i]);
        } else {
#pragma unroll
            for (int i = 0; i < kDig; i++) pl[i * plane + (int64_t)j * s16 + k] = (uint16_t)f16_of_int(d[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// k_lhat_oz<TN>: Lhat(p, j) = sum_k L(s + p, k) L_KK^{-1}(k, j) for one 64-row
// tile and one column tile, on the fp16 tensor cores.  A = rows of L_{C,K}
// (row exponent over its s entries), B = the digit planes of L_KK^{-1}.
// k = s <= 128: a single exact fp32 chunk.
// ---------------------------------------------------------------------------
template <int TN>
__global__ void __launch_bounds__(kOzThreads, TN <= 32 ? 2 : 1) k_lhat_oz(const ProbDesc *__restrict__ descs,
                                                           const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    constexpr int NT = TN / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);     // [7][64][kApad]
    uint16_t *Bs = As + kDig * kTM * kApad;                    // [7][TN][kApad]
    __shared__ int rowE[kTM];
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int s16 = (s + 15) & ~15;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int ncol = (s + TN - 1) / TN;
    const int tile = it.tile / ncol, ct = it.tile % ncol;
    const int p0 = tile * kTM, n0 = ct * TN;
    const double *Lc = static_cast<const double *>(P.L) + P.panel_off[K] + s;   // L_C(p, k) = Lc[k*ld + p]
    for (int e = threadIdx.x; e < kTM; e += kOzThreads) rowE[e] = 0;
    __syncthreads();
    {
        const int pl = threadIdx.x % kTM, part = threadIdx.x / kTM;
        int E = 0;
        if (p0 + pl < c)
            for (int k = part; k < s; k += kOzThreads / kTM) E = max(E, bexp(Lc[(int64_t)k * ld + p0 + pl]));
        atomicMax(&rowE[pl], E);
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int mt = warp % 4, grp = lane / 4, qd = lane % 4;
    float acc[NT][kDig][4];
#pragma unroll
    for (int t = 0; t < NT; t++)
#pragma unroll
        for (int g = 0; g < kDig; g++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[t][g][r] = 0.f;
    const uint16_t *Bg = P.linvd + P.linvd_off[K];
    const int64_t bplane = (int64_t)s * s16;
    for (int k0 = 0; k0 < s16; k0 += kOzK) {
        __syncthreads();
        for (int e = threadIdx.x; e < kDig * TN * 2; e += kOzThreads) {
            const int half = e & 1, j = (e >> 1) % TN, i = (e >> 1) / TN;
            uint16_t *dst = Bs + (i * TN + j) * kApad + half * 8;
            if (n0 + j < s) cp_async16(dst, Bg + i * bplane + (int64_t)(n0 + j) * s16 + k0 + half * 8);
            else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        }
        for (int e = threadIdx.x; e < kTM * (kOzK / 2); e += kOzThreads) {
            const int pl = e % kTM, kk = (e / kTM) * 2;
            const int p = p0 + pl, k = k0 + kk;
            const double x0 = (p < c && k < s) ? Lc[(int64_t)k * ld + p] : 0.0;
            const double x1 = (p < c && k + 1 < s) ? Lc[(int64_t)(k + 1) * ld + p] : 0.0;
            int d0[kDig], d1[kDig];
            digits7(x0, rowE[pl], d0);
            digits7(x1, rowE[pl], d1);
#pragma unroll
            for (int i = 0; i < kDig; i++)
                *reinterpret_cast<uint32_t *>(As + (i * kTM + pl) * kApad + kk) =
                    f16_of_int(d0[i]) | (f16_of_int(d1[i]) << 16);
        }
        cp_async_wait_all();
        __syncthreads();
        uint32_t b[NT][kDig][2];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const int nt = (warp / 4) + 2 * t;
#pragma unroll
            for (int j = 0; j < kDig; j++) {
                const uint16_t *bb = Bs + (j * TN + nt * 8 + grp) * kApad;
                b[t][j][0] = *reinterpret_cast<const uint32_t *>(bb + qd * 2);
                b[t][j][1] = *reinterpret_cast<const uint32_t *>(bb + qd * 2 + 8);
            }
        }
#pragma unroll
        for (int i = 0; i < kDig; i++) {
            const uint16_t *base = As + (i * kTM + mt * 16) * kApad;
            const uint32_t a0 = *reinterpret_cast<const uint32_t *>(base + grp * kApad + qd * 2);
            const uint32_t a1 = *reinterpret_cast<const uint32_t *>(base + (grp + 8) * kApad + qd * 2);
            const uint32_t a2 = *reinterpret_cast<const uint32_t *>(base + grp * kApad + qd * 2 + 8);
            const uint32_t a3 = *reinterpret_cast<const uint32_t *>(base + (grp + 8) * kApad + qd * 2 + 8);
#pragma unroll
            for (int t = 0; t < NT; t++)
#pragma unroll
                for (int j = 0; i + j < kDig; j++)
                    mma_f16(acc[t][i + j], a0, a1, a2, a3, b[t][j][0], b[t][j][1]);
        }
    }
    double *LD = static_cast<double *>(P.LD) + P.panel_off[K] + s;
#pragma unroll
    for (int t = 0; t < NT; t++) {
        const int nt = (warp / 4) + 2 * t;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int row = mt * 16 + grp + (r >= 2 ? 8 : 0);
            const int j = n0 + nt * 8 + qd * 2 + (r & 1);
            if (p0 + row >= c || j >= s) continue;
            long long gq[kDig];
#pragma unroll
            for (int q = 0; q < kDig; q++) gq[q] = (long long)__float2int_rn(acc[t][q][r]);
            const long long hi = (gq[0] << 16) + (gq[1] << 8) + gq[2];
            const long long lo = (gq[3] << 24) + (gq[4] << 16) + (gq[5] << 8) + gq[6];
            const int sc = (rowE[row] - 1022) + (P.linvexp[fc + j] - 1022) - 14;
            LD[(int64_t)j * ld + p0 + row] = fixed_to_double(hi, lo, sc);
        }
    }
}

// ---------------------------------------------------------------------------
// k_diag_oz: contribution of one 64-row tile to the diagonal block,
// sum_{p in tile} Lhat(p, i) Y(p, j), Y = A^{-1}_{C,K} (already written), on
// the fp16 tensor cores with the same exact digit scheme:
//   A = Lhat^T restricted to the tile (rows i, k = p): the Lhat digit planes,
//       exponent = column exponent of Lhat over all of C;
//   B = Y restricted to the tile: digits on Y's column exponent over all of C
//       (atomic max taken when Y was written).
// k = 64 needs no flush (7 * 64 * 2^14 < 2^24).  Since every tile works on the
// same grid, the tiles' integer sums are added exactly (int64 atomics, order
// independent); k_diag_fin then forms A^{-1}_KK = Dinv - Lhat^T Y in FP64.
// 8 warps: warp w owns m-tile w (16 rows i) and the 4 n-tiles of a 32-column
// pass over j.
// ---------------------------------------------------------------------------
constexpr int kDK = 64;          // k extent (rows of the tile)
constexpr int kDpad = kDK + 8;   // smem row stride (fp16), conflict-free fragment loads
constexpr int kDJ = kDiagCols;   // columns j per item

__global__ void __launch_bounds__(kOzThreads, 1) k_diag_oz(const ProbDesc *__restrict__ descs,
                                                           const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);          // [7][128][kDpad]
    uint16_t *Bs = As + kDig * 128 * kDpad;                         // [7][kDJ][kDpad]
    int *colE = reinterpret_cast<int *>(Bs + kDig * kDJ * kDpad);   // [128]
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int c16 = (c + 15) & ~15;
    const int npass = (s + kDJ - 1) / kDJ;         // items (row tile, column pass)
    const int pass = it.tile % npass;
    const int p0 = (it.tile / npass) * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;
    const int s16 = (s + 15) & ~15;
    double *Zk = static_cast<double *>(P.Z) + P.panel_off[K];
    const double *LDk = static_cast<const double *>(P.LD) + P.panel_off[K];
    const double *Y = Zk + s;                                       // Y(p, j) = Y[j*ld + p]
    const uint16_t *Ag = P.lhs + P.lhs_off[K];
    const int64_t aplane = (int64_t)s * c16;
    const int64_t ss = (int64_t)s * s;
    long long *acc64 = P.dacc + 2 * P.linv_off[K];            // [s*s] x (hi, lo)

    if (pm > 0) {
        // A digits: rows i < s16, k = p0 .. p0 + 63 (zero past c16 and for i >= s)
        const int kvalid = c16 - p0 < kDK ? c16 - p0 : kDK;     // multiple of 16
        for (int e = threadIdx.x; e < kDig * s16 * (kDK / 8); e += kOzThreads) {
            const int ch = e % (kDK / 8), i = (e / (kDK / 8)) % s16, pl = e / (kDK / 8) / s16;
            uint16_t *dst = As + (pl * 128 + i) * kDpad + ch * 8;
            if (i < s && ch * 8 < kvalid) cp_async16(dst, Ag + pl * aplane + (int64_t)i * c16 + p0 + ch * 8);
            else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        }
        // column exponents of Y over all of C (shared by every tile: exact sums)
        for (int j = threadIdx.x; j < 128; j += kOzThreads) colE[j] = j < s ? P.colexpY[fc + j] : 0;
        cp_async_wait_all();
        __syncthreads();
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int grp = lane / 4, qd = lane % 4;
    const int mt = warp;                       // rows i = mt*16 .. mt*16+15
    for (int jb = pass * kDJ; jb < s && jb < (pass + 1) * kDJ; jb += kDJ) {
        if (pm > 0) {
            __syncthreads();                   // previous pass done with Bs
            // B digits: columns jb .. jb+31, k = tile rows (two adjacent p per word)
            for (int e = threadIdx.x; e < kDJ * (kDK / 2); e += kOzThreads) {
                const int jl = e % kDJ, kk = (e / kDJ) * 2;
                const int j = jb + jl;
                int d0[kDig], d1[kDig];
                const double y0 = (j < s && kk < pm) ? Y[(int64_t)j * ld + p0 + kk] : 0.0;
                const double y1 = (j < s && kk + 1 < pm) ? Y[(int64_t)j * ld + p0 + kk + 1] : 0.0;
                const int E = j < s ? colE[j] : 0;
                digits7(y0, E, d0);
                digits7(y1, E, d1);
#pragma unroll
                for (int i = 0; i < kDig; i++)
                    *reinterpret_cast<uint32_t *>(Bs + (i * kDJ + jl) * kDpad + kk) =
                        f16_of_int(d0[i]) | (f16_of_int(d1[i]) << 16);
            }
            __syncthreads();
        }
        float acc[4][kDig][4];
#pragma unroll
        for (int t = 0; t < 4; t++)
#pragma unroll
            for (int g = 0; g < kDig; g++)
#pragma unroll
                for (int r = 0; r < 4; r++) acc[t][g][r] = 0.f;
        if (pm > 0 && mt * 16 < s) {
#pragma unroll 1
            for (int ks = 0; ks < kDK / kOzK; ks++) {
                uint32_t a[kDig][4];
#pragma unroll
                for (int i = 0; i < kDig; i++) {
                    const uint16_t *base = As + (i * 128 + mt * 16) * kDpad + ks * 16;
                    a[i][0] = *reinterpret_cast<const uint32_t *>(base + grp * kDpad + qd * 2);
                    a[i][1] = *reinterpret_cast<const uint32_t *>(base + (grp + 8) * kDpad + qd * 2);
                    a[i][2] = *reinterpret_cast<const uint32_t *>(base + grp * kDpad + qd * 2 + 8);
                    a[i][3] = *reinterpret_cast<const uint32_t *>(base + (grp + 8) * kDpad + qd * 2 + 8);
                }
#pragma unroll
                for (int t = 0; t < 4; t++) {
#pragma unroll
                    for (int j = 0; j < kDig; j++) {
                        const uint16_t *bb = Bs + (j * kDJ + t * 8 + grp) * kDpad + ks * 16;
                        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(bb + qd * 2);
                        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(bb + qd * 2 + 8);
#pragma unroll
                        for (int i = 0; i + j < kDig; i++)
                            mma_f16(acc[t][i + j], a[i][0], a[i][1], a[i][2], a[i][3], b0, b1);
                    }
                }
            }
        }
        // exact group sums of this tile -> int64, added exactly to the sums of
        // all tiles of K (integer addition: the order does not matter)
        if (pm > 0 && mt * 16 < s) {
#pragma unroll
            for (int t = 0; t < 4; t++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = mt * 16 + grp + (r >= 2 ? 8 : 0);
                    const int j = jb + t * 8 + qd * 2 + (r & 1);
                    if (i >= s || j >= s) continue;
                    long long g[kDig];
#pragma unroll
                    for (int q = 0; q < kDig; q++) g[q] = (long long)__float2int_rn(acc[t][q][r]);
                    const long long hi = (g[0] << 16) + (g[1] << 8) + g[2];
                    const long long lo = (g[3] << 24) + (g[4] << 16) + (g[5] << 8) + g[6];
                    unsigned long long *dst = reinterpret_cast<unsigned long long *>(acc64 + 2 * ((int64_t)j * s + i));
                    if (hi) atomicAdd(dst, (unsigned long long)hi);
                    if (lo) atomicAdd(dst + 1, (unsigned long long)lo);
                }
        }
    }
}

// ---------------------------------------------------------------------------
// k_diag_fin: A^{-1}_KK = Dinv_K - Lhat^T Y from the exact sums of k_diag_oz
// (bshift 0) or k_diag_tc (bshift 1), symmetrized: one CTA per (K, 2 columns)
// (diag_fin_pair).  items: (K, column pair, bshift).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_diag_fin(const ProbDesc *__restrict__ descs,
                                                  const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const Item it = items[w];
    diag_fin_pair<false>(descs[it.prob], it.K, 2 * it.tile, it.ntiles);
}

constexpr size_t diag_oz_smem() {
    return sizeof(uint16_t) * (size_t)kDig * (128 + kDJ) * kDpad + sizeof(int) * 128;
}

cudaError_t launch_diag_oz(const ProbDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_diag_oz<<<n, kOzThreads, diag_oz_smem(), st>>>(d, items, n);
    return cudaGetLastError();
}

cudaError_t launch_diag_fin(const ProbDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_diag_fin<<<n, 256, 0, st>>>(d, items, n);
    return cudaGetLastError();
}

template <int TN> constexpr size_t oz_smem_bytes() {
    return sizeof(uint16_t) * 2 * (size_t)kDig * (kTM + TN) * kApad + 2 * sizeof(long long) * kTM * TN +
           sizeof(int) * kTM;
}

template <int TN> constexpr size_t lhat_oz_smem() {
    return sizeof(uint16_t) * (size_t)kDig * (kTM + TN) * kApad;
}

cudaError_t configure_ozaki_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_selinv_oz<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes<16>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selinv_oz<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes<32>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selinv_oz<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes<64>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diag_oz_smem());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lhat_oz<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lhat_oz_smem<16>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lhat_oz<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lhat_oz_smem<32>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lhat_oz<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lhat_oz_smem<64>());
    return e;
}

cudaError_t launch_linv_digits(const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    k_linv_digits<<<nwork, 256, 0, st>>>(d, work, nwork);
    return cudaGetLastError();
}

cudaError_t launch_lhat_oz(int tn, const ProbDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (tn == 16) k_lhat_oz<16><<<n, kOzThreads, lhat_oz_smem<16>(), st>>>(d, items, n);
    else if (tn == 32) k_lhat_oz<32><<<n, kOzThreads, lhat_oz_smem<32>(), st>>>(d, items, n);
    else k_lhat_oz<64><<<n, kOzThreads, lhat_oz_smem<64>(), st>>>(d, items, n);
    return cudaGetLastError();
}

cudaError_t launch_lhat_digits(const ProbDesc *d, const int2 *work, int nwork, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    k_lhat_digits<<<nwork, 256, 0, st>>>(d, work, nwork);
    return cudaGetLastError();
}

// TN = 16, 32 or 64 (a column tile); items carry tile = row_tile * ncol + col_tile
cudaError_t launch_selinv_oz(int tn, const ProbDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (tn == 16) k_selinv_oz<16><<<n, kOzThreads, oz_smem_bytes<16>(), st>>>(d, items, n);
    else if (tn == 32) k_selinv_oz<32><<<n, kOzThreads, oz_smem_bytes<32>(), st>>>(d, items, n);
    else k_selinv_oz<64><<<n, kOzThreads, oz_smem_bytes<64>(), st>>>(d, items, n);
    return cudaGetLastError();
}

}  // namespace selinv
