// Digit slicing and digit-pair products shared by the tcgen05 kernels: an
// FP64 value is cut into 7 balanced base-256 digits on a fixed-point grid
// (2^(E - 1076) for the grid exponent E), each digit held exactly in fp16;
// the products of digit pairs with the same i + j are summed into one exact
// fp32 accumulator in tensor memory.
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "umma.cuh"

namespace selinv {

constexpr int kTcM = 128;          // tensor-memory lanes (M of every MMA)
constexpr int kTcDig = 7;          // digits per FP64 operand
constexpr int kTcFlush = 8;        // k16 steps per exact fp32 chunk (128 k)
static_assert(kTcFlush == 8, "the planner sizes k-ranges in whole chunks of 8 steps");
// Bounded mbarrier waits inside one CTA get at least this many polls
// (about a second), whatever the caller's bound on waits between CTAs.
constexpr long long kMbarMinPolls = 1ll << 22;

// x = M * 2^(E - 1076) with |M| < 2^54 (E >= the biased exponent of x),
// truncated toward zero; integer operations only.
__device__ __forceinline__ long long fixed54(double x, int E) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    const long long mant = ex ? ((b & 0xFFFFFFFFFFFFFll) | (1ll << 52)) : 0ll;
    const int sh = E - ex - 1;
    const long long M = sh < 0 ? (mant << 1) : (sh < 63 ? (mant >> sh) : 0ll);
    return b < 0 ? -M : M;
}

// With u = M + 0x80808080808080 (M as above), byte t of u minus 128 is the
// balanced base-256 digit of weight 256^t, in [-128, 127].  The digits of
// byte t of two values as an fp16 pair (w0's in the low half): the bytes are
// placed in the mantissas of 1024 + byte (fp16 bits 0x6400 | byte) and 1152
// is subtracted -- exact, three instructions per pair.
template <int T>
__device__ __forceinline__ uint32_t digit_pair(uint32_t w0, uint32_t w1) {
    const uint32_t b = __byte_perm(w0, w1, (T & 3) | (((T & 3) + 4) << 8) | (((T & 3) + 4) << 16)) & 0x00FF00FFu;
    const uint32_t h = b | 0x64006400u;
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(h), "r"(0xE480E480u));   // + (-1152, -1152)
    return r;
}

// The digit products of one k16 step, A digit planes i (128 rows) against B
// digit planes j (TN rows each), summed into group i + j at tensor-memory
// columns (i + j) TN.  The 7 B planes lie one after the other with the
// row-group stride of the operand layout, so planes j0 .. j0 + m - 1 form one
// operand of m TN rows: one MMA of N = m TN (at most 256) at columns
// (i + j0) TN computes A_i B_j0 .. A_i B_{j0+m-1} into groups i + j0 ..
// i + j0 + m - 1.  Per step 10 MMAs for TN = 64, 7 for TN <= 32 (against 28
// of N = TN).  A group starts from zero at the first step of a chunk, with
// the products of A plane 0.
template <int TN, int A_PLANE, int B_PLANE>
__device__ __forceinline__ void digit_products(uint32_t tmem, uint64_t ad0, uint64_t bd0, bool first) {
    constexpr int kPer = 256 / TN;   // B planes per MMA (N <= 256)
#pragma unroll
    for (int i = 0; i < kTcDig; i++) {
        const uint64_t ad = ad0 + (uint64_t)(i * A_PLANE * 2 / 16);
#pragma unroll
        for (int j0 = 0; j0 < kTcDig - i; j0 += kPer) {
            const int m = kTcDig - i - j0 < kPer ? kTcDig - i - j0 : kPer;
            const uint64_t bd = bd0 + (uint64_t)(j0 * B_PLANE * 2 / 16);
            umma::mma_f16kind(tmem + (uint32_t)((i + j0) * TN), ad, bd, umma::idesc_f16_f32(kTcM, m * TN),
                              (first && i == 0) ? 0u : 1u);
        }
    }
}

// Digit plane PL (weight 256^(6 - PL)) of the 4 values whose biased fixed-
// point words are (lo[u], hi[u]): half a 16-byte core-matrix row of fp16.
template <int PL>
__device__ __forceinline__ void store_plane4(uint16_t *dst, const uint32_t (&lo)[4], const uint32_t (&hi)[4]) {
    constexpr int T = 6 - PL;
    const uint32_t(&w)[4] = T >= 4 ? hi : lo;
    uint2 q;
    q.x = digit_pair<T>(w[0], w[1]);
    q.y = digit_pair<T>(w[2], w[3]);
    *reinterpret_cast<uint2 *>(dst) = q;
}

// Address of entry (p, q) of A^{-1}_{C,C} in the ancestors' panels (stored at
// (max, min) by symmetry), in three dependent parts so that a producer can
// keep each load a whole step ahead of its use: the column data of q (panel
// address of column C[q] in its owner and the start of its relative rows),
// then the base and the relative row (a load), then the value; base -1
// outside C x C.  pl = p - p0; the tile's own rows come from shared memory.
// parts() also reports whether (p, q) lies above the diagonal (stored as its
// mirror: a Hermitian matrix stores the conjugate there).
struct TcGather {
    const int64_t *pcb, *prb;
    const int32_t *relidx;
    const int64_t *tile_cb, *tile_rb;
    int p0, c;
    GatherCheck chk;   // optional bounds check of the addresses (applied by the loads)
    __device__ __forceinline__ void cols(int q, int64_t &cb, int64_t &rb) const {
        if (q < c) {
            cb = pcb[q];
            rb = prb[q];
        } else {
            cb = -1;
            rb = 0;
        }
    }
    __device__ __forceinline__ void parts(int pl, int q, int64_t cb, int64_t rb, int64_t &base, int32_t &rel,
                                          bool &upper) const {
        const int p = p0 + pl;
        upper = p < q;
        if (p >= c || q >= c) {
            base = -1;
            rel = 0;
        } else if (p >= q) {
            base = cb;
            rel = relidx[rb + p];
        } else {
            base = tile_cb[pl];
            rel = relidx[tile_rb[pl] + q];
        }
    }
};

}  // namespace selinv
