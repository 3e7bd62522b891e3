"""The library's integer float32 <-> float64 conversions (csrc/fpbits.h: widening in the
product epilogues that write the float64 density matrix, narrowing in the scaling of H)
against the C++ conversions: widening on every one of the 2^32 float32 bit patterns,
narrowing (round to nearest, ties to even) on random float64 patterns and on patterns at and
next to every rounding boundary (ties, the normal/subnormal and overflow thresholds); the same
bits for every number, NaN for every NaN. And the integer float32 product of two float64
numbers (the scaling's off-diagonal entries) against a reference from the FPU: the float64
product, its exact error by fma, and the float32 rounding decided by that error at ties."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2306_12616_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include "fpbits.h"
int main() {
    unsigned long long bad = 0, nans = 0;
    for (unsigned long long u = 0; u <= 0xffffffffull; ++u) {
        const unsigned int b = (unsigned int)u;
        float f;
        std::memcpy(&f, &b, 4);
        const double w = fo::widen_f32(f);
        if (std::isnan(f)) {
            ++nans;
            if (!std::isnan(w)) ++bad;
            continue;
        }
        const double ref = (double)f;
        unsigned long long x, y;
        std::memcpy(&x, &w, 8);
        std::memcpy(&y, &ref, 8);
        if (x != y) {
            if (bad < 5) std::printf("mismatch %08x\n", b);
            ++bad;
        }
    }
    std::printf("%llu %llu\n", bad, nans);
    return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_widen_f32_every_bit_pattern(tmp_path):
    src = tmp_path / "widen.cpp"
    exe = tmp_path / "widen"
    src.write_text(PROGRAM)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    bad, nans = (int(x) for x in out.stdout.split()[-2:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert nans == 2 * (2 ** 23 - 1)


NARROW = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include "fpbits.h"
static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next() {   // splitmix64
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static unsigned long long checked = 0, bad = 0;
static void check(uint64_t u) {
    double x;
    std::memcpy(&x, &u, 8);
    const float a = fo::narrow_f64(x), ref = (float)x;
    ++checked;
    if (std::isnan(x)) { if (!std::isnan(a)) ++bad; return; }
    uint32_t p, q;
    std::memcpy(&p, &a, 4);
    std::memcpy(&q, &ref, 4);
    if (p != q) { if (bad < 5) std::printf("mismatch %016llx\n", (unsigned long long)u); ++bad; }
}
int main() {
    for (int i = 0; i < 50000000; ++i) check(next());
    // every float32 value f: the float64 at f, at the midpoint to the next float32 up, and
    // one float64 ulp on either side of the midpoint (both signs, subnormals included)
    for (uint64_t b = 0; b < 0x7f800000ull; b += 1 + (next() & 63)) {
        uint32_t fb = (uint32_t)b;
        float f;
        std::memcpy(&f, &fb, 4);
        double d = (double)f;
        uint64_t u;
        std::memcpy(&u, &d, 8);
        uint32_t gb = fb + 1;
        float g;
        std::memcpy(&g, &gb, 4);
        const double mid = 0.5 * ((double)f + (double)g);
        uint64_t m;
        std::memcpy(&m, &mid, 8);
        for (uint64_t s : {0ull, 0x8000000000000000ull}) {
            check(u | s); check(m | s); check((m + 1) | s); check((m - 1) | s);
        }
    }
    // below the smallest float32 subnormal, exponent by exponent
    for (uint64_t e = 0; e < 0x7ff; ++e)
        for (int i = 0; i < 64; ++i) check((e << 52) | (next() & 0x000fffffffffffffull));
    std::printf("%llu %llu\n", checked, bad);
    return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_narrow_f64_random_and_boundaries(tmp_path):
    src = tmp_path / "narrow.cpp"
    exe = tmp_path / "narrow"
    src.write_text(NARROW)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    checked, bad = (int(x) for x in out.stdout.split()[-2:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert checked > 100_000_000


MUL = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include "fpbits.h"
static uint64_t state = 0x2306126161234567ull;
static uint64_t next() {   // splitmix64
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static double unit() { return (double)(next() >> 11) * 0x1.0p-53; }
// float32 of the exact a * b from the FPU: p = RN64(a b) and its exact error e = fma(a, b, -p);
// RN32(a b) = RN32(p) unless p is a float32 midpoint, where the sign of e decides
static float ref_mul(double a, double b) {
    const double p = a * b;
    const double e = std::fma(a, b, -p);
    float f = (float)p;
    if (!std::isfinite(f) || e == 0.0) return f;
    const float g = (double)f < p ? std::nextafterf(f, INFINITY) : std::nextafterf(f, -INFINITY);
    if (!std::isfinite(g)) return f;
    const double mid = 0.5 * ((double)f + (double)g);
    if (p != mid) return f;
    const float lo = f < g ? f : g, hi = f < g ? g : f;
    return e > 0.0 ? hi : lo;
}
static unsigned long long checked = 0, bad = 0;
static void check(double a, double b) {
    const float x = fo::mul_rn_f32(a, b), y = ref_mul(a, b);
    uint32_t p, q;
    std::memcpy(&p, &x, 4);
    std::memcpy(&q, &y, 4);
    ++checked;
    if (p != q) {
        if (bad < 5) std::printf("mismatch %a * %a: %a vs %a\n", a, b, (double)x, (double)y);
        ++bad;
    }
}
int main() {
    for (int i = 0; i < 20000000; ++i) {   // H-like entries times scale factors
        const double a = (unit() * 2 - 1) * std::ldexp(1.0, (int)(next() % 40) - 20);
        const double b = std::ldexp(1.0 + unit(), -(int)(next() % 12));
        check(a, b);
    }
    for (int i = 0; i < 20000000; ++i) {   // random finite bit patterns
        uint64_t u = next(), v = next();
        double a, b;
        std::memcpy(&a, &u, 8);
        std::memcpy(&b, &v, 8);
        if (!std::isfinite(a) || !std::isfinite(b)) continue;
        check(a, b);
    }
    for (int i = 0; i < 20000000; ++i) {   // products around the float32 range limits
        const int ea = (int)(next() % 400) - 200, eb = -150 - ea + (int)(next() % 30) + (i & 1 ? 0 : 276);
        check(std::ldexp(1.0 + unit(), ea), std::ldexp(1.0 + unit(), eb));
    }
    for (int i = 0; i < 4000000; ++i) {    // products of short significands: exact ties
        const double a = (double)(next() % (1u << 13)) * std::ldexp(1.0, (int)(next() % 60) - 30);
        const double b = (double)(next() % (1u << 13)) * std::ldexp(1.0, (int)(next() % 60) - 30);
        check(a, -b);
    }
    check(0.0, 3.0); check(-0.0, 3.0); check(1e-320, 1e-10); check(3.4e38, 2.0);
    std::printf("%llu %llu\n", checked, bad);
    return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_mul_rn_f32_against_fma_reference(tmp_path):
    src = tmp_path / "mul.cpp"
    exe = tmp_path / "mul"
    src.write_text(MUL)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    checked, bad = (int(x) for x in out.stdout.split()[-2:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert checked > 60_000_000
