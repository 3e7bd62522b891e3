// float32 <-> float64 conversions, and the float32 of a float64 product, with integer
// operations only.
//
// The conversion instructions run on the float64 pipe, which on this GPU retires about two
// lane operations per clock and SM; the epilogues that write the float64 density matrix
// widen every entry, and the scaling multiplies every entry of H and rounds it to float32, so
// they build the bit patterns with integer operations instead. Widening
// (IEEE 754 binary32 -> binary64 is exact: the exponent is rebiased by 1023 - 127, the 23
// fraction bits move to the top of the 52; a subnormal float32 becomes a normal float64).
// NaN keeps its payload and quiet bit. Host-compilable, so that a host test can compare them
// with the C++ conversions (every float32 bit pattern; random and rounding-boundary float64
// patterns) and the product with an fma-based reference.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define FO_HD __host__ __device__
#else
#define FO_HD
#endif

namespace fo {

FO_HD inline int fo_clz32(uint32_t a) {
#if defined(__CUDA_ARCH__)
    return __clz((int)a);
#else
    return a ? __builtin_clz(a) : 32;
#endif
}

FO_HD inline double widen_f32(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    const uint32_t a = b & 0x7fffffffu;
    uint64_t r;
    if (a - 0x00800000u < 0x7f000000u) {
        // normal: exponent field and fraction move up 29 bits, exponent rebiased
        r = ((uint64_t)a << 29) + ((uint64_t)(1023 - 127) << 52);
    } else if (a >= 0x7f800000u) {
        // infinity, NaN
        r = 0x7ff0000000000000ull | ((uint64_t)(a & 0x007fffffu) << 29);
    } else if (a == 0) {
        r = 0;
    } else {
        // subnormal a * 2^-149: the leading bit at position p gives 2^(p - 149)
        const int p = 31 - fo_clz32(a);
        r = ((uint64_t)(p - 149 + 1023) << 52) | (((uint64_t)a << (52 - p)) & 0x000fffffffffffffull);
    }
    r |= (uint64_t)(b & 0x80000000u) << 32;
    double d;
    memcpy(&d, &r, 8);
    return d;
}

// float64 -> float32, round to nearest, ties to even (IEEE 754 convertFormat), with integer
// operations only: 29 fraction bits are dropped from a normal result, more from a subnormal
// one; a carry out of the fraction moves into the exponent (and from the largest finite value
// to infinity). NaN stays NaN (quiet).
FO_HD inline float narrow_f64(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff);
    const uint64_t frac = b & 0x000fffffffffffffull;
    uint32_t r;
    if (e == 0x7ff) {
        r = 0x7f800000u | (frac ? 0x00400000u | (uint32_t)(frac >> 29) : 0u);
    } else if (e >= 1023 - 126) {   // normal float32 range or above
        const int fe = e - 1023 + 127;
        if (fe >= 0xff) {
            r = 0x7f800000u;
        } else {
            r = ((uint32_t)fe << 23) | (uint32_t)(frac >> 29);
            const uint64_t rem = frac & 0x1fffffffull;
            if (rem > 0x10000000ull || (rem == 0x10000000ull && (r & 1u))) ++r;
        }
    } else if (e == 0) {
        r = 0;   // float64 subnormals are far below half the smallest float32 subnormal
    } else {
        // subnormal float32 result: (2^52 + frac) * 2^(e - 1075) in units of 2^-149
        const uint64_t m = frac | (1ull << 52);
        const int sh = 926 - e;   // bits dropped, >= 30
        if (sh > 53) {
            r = 0;
        } else {
            r = (uint32_t)(m >> sh);
            const uint64_t rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
            if (rem > half || (rem == half && (r & 1u))) ++r;
        }
    }
    r |= sign;
    float f;
    memcpy(&f, &r, 4);
    return f;
}

// float32 of the exact product a * b of two finite float64 numbers (round to nearest, ties to
// even; one rounding, where RN32(RN64(a b)) rounds twice), with integer operations only: the
// 53-bit significands multiply into a 106-bit integer, whose leading 24 bits with the guard
// and sticky bits below give the float32 significand; a subnormal float32 result keeps
// fewer bits, an overflow gives infinity. The scaling of H multiplies every upper entry by
// 2 / (e_b - e_a) and stores it as float32: a float64 multiply per entry ran on the narrow
// float64 pipe.
FO_HD inline uint64_t fo_mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
FO_HD inline int fo_clz64(uint64_t a) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}
FO_HD inline float mul_rn_f32(double a, double b) {
    uint64_t ua, ub;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    const uint32_t sign = (uint32_t)((ua ^ ub) >> 32) & 0x80000000u;
    int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
    uint64_t ma = ua & 0x000fffffffffffffull, mb = ub & 0x000fffffffffffffull;
    uint32_t r = 0;
    if ((ea | ma) != 0 && (eb | mb) != 0) {
        if (ea == 0) ea = 1;
        else ma |= 1ull << 52;
        if (eb == 0) eb = 1;
        else mb |= 1ull << 52;
        const uint64_t lo = ma * mb, hi = fo_mulhi64(ma, mb);   // the product, < 2^106
        const int p = hi ? 127 - fo_clz64(hi) : 63 - fo_clz64(lo);
        // product = (hi:lo) 2^(ea + eb - 2150); float32 biased exponent when normal:
        int E = p + ea + eb - 2150 + 127;
        int sh = p - 23;   // right shift that leaves 24 significant bits
        if (E <= 0) {      // subnormal: fewer bits
            sh += 1 - E;
            E = 0;
        }
        uint64_t m = 0, guard = 0, sticky = 0;
        if (sh <= 0) {
            m = lo << (-sh);
        } else if (sh < 64) {
            m = (lo >> sh) | (hi << (64 - sh));
            guard = (lo >> (sh - 1)) & 1u;
            sticky = lo & ((1ull << (sh - 1)) - 1);
        } else if (sh == 64) {
            m = hi;
            guard = lo >> 63;
            sticky = lo << 1;
        } else if (sh < 128) {
            const int s2 = sh - 64;
            m = hi >> s2;
            guard = (hi >> (s2 - 1)) & 1u;
            sticky = (hi & ((1ull << (s2 - 1)) - 1)) | lo;
        }   // sh >= 128: below half the smallest subnormal (the product is < 2^106)
        if (guard && (sticky != 0 || (m & 1u))) ++m;
        // a carry out of the significand moves into the exponent field by itself
        const uint64_t bits = E == 0 ? m : ((uint64_t)(E - 1) << 23) + m;
        r = bits >= 0x7f800000ull ? 0x7f800000u : (uint32_t)bits;
    }
    r |= sign;
    float f;
    memcpy(&f, &r, 4);
    return f;
}

}  // namespace fo
