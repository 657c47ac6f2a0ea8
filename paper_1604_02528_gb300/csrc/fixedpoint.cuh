// Exact fixed-point helpers shared by the tensor-core kernels.
#pragma once

#include <stdint.h>

namespace selinv {

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
