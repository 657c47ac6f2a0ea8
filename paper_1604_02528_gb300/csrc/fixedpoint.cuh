// Exact fixed-point helpers shared by the tensor-core kernels.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace selinv {

constexpr int kDig = 7;          // digits per FP64 operand of the tensor-core products

// fp16 bit pattern of a small integer v (|v| <= 128): exact via an fp32
// round trip through the magic constant 1.5 * 2^23, then an exact narrowing.
__device__ __forceinline__ uint32_t f16_of_int(int v) {
    const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
    return (uint32_t)__half_as_ushort(__float2half_rn(f));
}

// 7 balanced base-256 digits (most significant first) of x on the grid of
// biased exponent E (E >= exponent of x): x ~= sum_i d_i 2^(E-1022-7-8i).
__device__ __forceinline__ void digits7(double x, int E, int d[kDig]) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = ex ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
    const int sh = E - ex - 2;                       // M = mant * 2^(2 - (E - ex)) < 2^55
    unsigned long long M = sh < 0 ? (mant << (-sh)) : (sh < 64 ? (mant >> sh) : 0ull);
#pragma unroll
    for (int i = kDig - 1; i >= 1; i--) {
        int v = (int)(M & 0xFFull);
        M >>= 8;
        if (v >= 128) { v -= 256; M += 1; }
        d[i] = v;
    }
    d[0] = (int)M;                                   // <= 128
    if (b < 0) {
#pragma unroll
        for (int i = 0; i < kDig; i++) d[i] = -d[i];
    }
}


// (hi * 2^32 + lo) * 2^(sc - 48) as a double, rounded once to nearest even,
// with integer operations only (the FP64 pipe is GB300's scarcest unit).
__device__ __forceinline__ double fixed_to_double(long long hi, long long lo, int sc) {
    const __int128 n = ((__int128)hi << 32) + (__int128)lo;
    if (n == 0) return 0.0;
    const unsigned long long sgn = n < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned __int128 m = n < 0 ? (unsigned __int128)(-n) : (unsigned __int128)n;
    const unsigned long long mh = (unsigned long long)(m >> 64), ml = (unsigned long long)m;
    const int nb = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);   // bit length
    unsigned long long q;
    int e2 = sc - 48;                                   // value = q * 2^e2 below
    if (nb <= 53) {
        q = ml << (53 - nb);
        e2 -= 53 - nb;
    } else {
        const int r = nb - 53;
        q = (unsigned long long)(m >> r);
        const unsigned __int128 rem = m & ((((unsigned __int128)1) << r) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (r - 1);
        if (rem > half || (rem == half && (q & 1ull))) q++;
        e2 += r;
        if (q >> 53) { q >>= 1; e2++; }
    }
    const int be = e2 + 52 + 1023;                      // q in [2^52, 2^53)
    if (be <= 0 || be >= 2047) {                        // outside the normal range
        const double v = ldexp((double)q, e2);
        return sgn ? -v : v;
    }
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (q & 0xFFFFFFFFFFFFFull)));
}

}  // namespace selinv
