// Exact sums of absolute values of float64 numbers, in integer arithmetic.
//
// The Gershgorin radius of a row, r_i = sum_{j != i} |h_ij| (Sec. "Chebyshev expansions": the
// bounds that map the spectrum of H into [-1, 1]), is accumulated in a 128-bit fixed-point
// integer instead of float64 additions: the float64 pipe of this GPU retires about two lane
// operations per clock and SM, so one float64 add per entry of H bounded the kernel, while
// integer operations run at many times that rate. The fixed point follows the largest
// exponent seen: acc = (hi:lo) 2^(e - 1133), so that a number with the biased exponent e and
// the 53-bit significand m (subnormals: e = 1, no implicit bit) enters as m << 58 (bits 58 to
// 110), 17 bits of headroom hold up to 2^16 such terms, and a number 2^s smaller enters as
// m << (58 - s), or m >> (s - 58) when s > 58 (bits below 2^(e - 1133) are dropped: at most
// n 2^-110 of the sum). A larger exponent rescales the accumulator first. Two accumulators
// merge by aligning the smaller scale to the larger. The result is rounded to float64 once
// (round to nearest, ties to even), so it is the correctly rounded sum up to those dropped
// bits, whatever the order of the terms: every reduction tree gives the same bits.
// Host-compilable, so that a host test can compare it with a correctly rounded float64 sum.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define FO_XS __host__ __device__
#else
#define FO_XS
#endif

namespace fo {

struct XAcc {
    uint64_t lo, hi;   // the sum in units of 2^(e - 1133)
    int e;             // largest biased exponent seen (0: nothing added yet)
};

FO_XS inline int xs_clz64(uint64_t a) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}

// acc >>= s (s >= 0), dropping the bits shifted out
FO_XS inline void xacc_shr(XAcc& a, int s) {
    if (s <= 0) return;
    if (s >= 128) {
        a.lo = a.hi = 0;
    } else if (s >= 64) {
        a.lo = a.hi >> (s - 64);
        a.hi = 0;
    } else {
        a.lo = (a.lo >> s) | (a.hi << (64 - s));
        a.hi >>= s;
    }
}

// acc += |x| for the finite float64 x with bit pattern `bits`
FO_XS inline void xacc_add_abs(XAcc& a, uint64_t bits) {
    const uint64_t u = bits & 0x7fffffffffffffffull;
    if (u == 0) return;
    int e = (int)(u >> 52);
    uint64_t m = u & 0x000fffffffffffffull;
    if (e == 0) e = 1;
    else m |= 1ull << 52;
    if (e > a.e) {   // a new largest exponent: rescale what was summed so far
        xacc_shr(a, e - a.e);
        a.e = e;
    }
    const int sh = a.e - e;
    uint64_t tlo, thi;
    if (sh <= 58) {
        const int s = 58 - sh;
        tlo = m << s;
        thi = s ? m >> (64 - s) : 0;
    } else if (sh < 58 + 53) {
        tlo = m >> (sh - 58);
        thi = 0;
    } else {
        return;
    }
    a.lo += tlo;
    a.hi += thi + (a.lo < tlo ? 1u : 0u);
}

// a += b (both accumulators of the same kind of sum)
FO_XS inline void xacc_merge(XAcc& a, XAcc b) {
    if (b.e > a.e) {
        const XAcc t = a;
        a = b;
        b = t;
    }
    xacc_shr(b, a.e - b.e);
    a.lo += b.lo;
    a.hi += b.hi + (a.lo < b.lo ? 1u : 0u);
}

// The accumulated sum rounded to float64 (to nearest, ties to even; +inf past the largest
// finite value).
FO_XS inline double xacc_to_double(const XAcc& a) {
    if ((a.lo | a.hi) == 0) return 0.0;
    const int p = a.hi ? 127 - xs_clz64(a.hi) : 63 - xs_clz64(a.lo);   // leading bit
    int E = p + a.e - 110;   // biased exponent when the result is normal
    int sh = p - 52;         // right shift that leaves 53 significant bits
    if (E <= 0) {            // subnormal: fewer bits
        sh += 1 - E;
        E = 0;
    }
    uint64_t m;
    bool up = false;
    if (sh <= 0) {
        m = a.lo << (-sh);   // p <= 52: the sum is in lo and fits
    } else {
        uint64_t guard, sticky;
        if (sh < 64) {
            m = (a.lo >> sh) | (a.hi << (64 - sh));
            guard = (a.lo >> (sh - 1)) & 1u;
            sticky = a.lo & ((1ull << (sh - 1)) - 1);
        } else if (sh == 64) {
            m = a.hi;
            guard = a.lo >> 63;
            sticky = a.lo << 1;
        } else if (sh < 128) {
            const int s2 = sh - 64;
            m = a.hi >> s2;
            guard = (a.hi >> (s2 - 1)) & 1u;
            sticky = (a.hi & ((1ull << (s2 - 1)) - 1)) | a.lo;
        } else {
            m = 0;
            guard = sh == 128 ? a.hi >> 63 : 0;
            sticky = sh == 128 ? ((a.hi << 1) | a.lo) : (a.hi | a.lo);
        }
        up = guard && (sticky != 0 || (m & 1u));
    }
    m += up ? 1u : 0u;
    // a carry out of the significand moves into the exponent field by itself
    uint64_t bits = E == 0 ? m : ((uint64_t)(E - 1) << 52) + m;
    if (bits >= 0x7ff0000000000000ull) bits = 0x7ff0000000000000ull;
    double d;
    memcpy(&d, &bits, 8);
    return d;
}

}  // namespace fo
