"""The exact float64 sums of the Gershgorin row radii (csrc/exactsum.h: 128-bit fixed point
that follows the largest exponent, rounded to float64 once) against Python's math.fsum, which
returns the correctly rounded sum: rows of random values over narrow and very wide exponent
ranges, with zeros, subnormals and values near the largest float64, summed in order, in a
shuffled order and as 32 lane-strided partial sums merged by a butterfly (the kernels' warp
reduction): the same bits as fsum every time."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2306_12616_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include "exactsum.h"
using namespace fo;
static uint64_t bits_of(double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; }
int main(int argc, char** argv) {
    FILE* f = std::fopen(argv[1], "rb");
    FILE* g = std::fopen(argv[2], "wb");
    int64_t rows;
    std::fread(&rows, 8, 1, f);
    for (int64_t r = 0; r < rows; ++r) {
        int64_t n;
        std::fread(&n, 8, 1, f);
        std::vector<double> x(n), y(n);
        std::fread(x.data(), 8, n, f);
        std::fread(y.data(), 8, n, f);   // the same values, shuffled
        XAcc a{0, 0, 0}, b{0, 0, 0};
        for (int64_t j = 0; j < n; ++j) xacc_add_abs(a, bits_of(x[j]));
        for (int64_t j = 0; j < n; ++j) xacc_add_abs(b, bits_of(y[j]));
        XAcc lane[32];
        for (int l = 0; l < 32; ++l) {
            lane[l] = XAcc{0, 0, 0};
            for (int64_t j = l; j < n; j += 32) xacc_add_abs(lane[l], bits_of(x[j]));
        }
        for (int o = 16; o > 0; o >>= 1) {
            XAcc nxt[32];
            for (int l = 0; l < 32; ++l) { nxt[l] = lane[l]; xacc_merge(nxt[l], lane[l ^ o]); }
            for (int l = 0; l < 32; ++l) lane[l] = nxt[l];
        }
        double out[3] = {xacc_to_double(a), xacc_to_double(b), xacc_to_double(lane[0])};
        int same = 1;
        for (int l = 1; l < 32; ++l)
            same &= lane[l].lo == lane[0].lo && lane[l].hi == lane[0].hi && lane[l].e == lane[0].e;
        std::fwrite(out, 8, 3, g);
        std::fwrite(&same, 4, 1, g);
    }
    std::fclose(f);
    std::fclose(g);
    return 0;
}
"""


def rows(seed):
    rng = np.random.default_rng(seed)
    out = []
    for kind in range(12):
        for _ in range(40):
            n = int(rng.integers(1, 3000))
            if kind == 0:      # H-like entries
                x = rng.normal(0.0, 1.0, n)
            elif kind == 1:    # a wide exponent range
                x = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-80, 80, n)
            elif kind == 2:    # the whole exponent range
                x = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-1070, 1000, n)
            elif kind == 3:    # subnormals and the smallest normals
                x = rng.integers(0, 2 ** 53, n).astype(np.uint64).view(np.float64)
            elif kind == 4:    # sparse: mostly zeros
                x = np.where(rng.random(n) < 0.9, 0.0, rng.normal(0, 3, n))
            elif kind == 5:    # near the largest finite value (sums may round to +inf)
                x = rng.uniform(0.5, 1.0, n) * 1.7e308 / max(1, n // 2)
            elif kind == 6:    # one large value, many tiny ones (the dropped-bits case)
                x = rng.normal(0, 1e-30, n)
                x[rng.integers(0, n)] = 1e10
            elif kind == 7:    # ties: small integers times a power of two
                x = rng.integers(-4, 5, n) * 2.0 ** -60
            elif kind == 8:    # exact halves at the 53-bit boundary
                x = np.full(n, 2.0 ** 52)
                x[0] = 0.5
                x[-1] = 0.5 if n > 1 else x[-1]
            elif kind == 9:    # random bit patterns (finite)
                u = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
                x = u.view(np.float64)
                x = np.where(np.isfinite(x), x, 1.0)
            elif kind == 10:   # exponents in increasing order (every term rescales)
                x = np.sort(2.0 ** rng.uniform(-200, 200, n))
            else:              # tight-binding-like rows: a few large, many small
                x = rng.normal(0, 1e-3, n)
                x[rng.integers(0, n, 8)] = rng.normal(0, 2.0, 8)
            out.append(np.ascontiguousarray(x, dtype=np.float64))
    return out


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_exact_sums_match_fsum(tmp_path):
    src, exe = tmp_path / "xs.cpp", tmp_path / "xs"
    src.write_text(PROGRAM)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    data = rows(2306)
    rng = np.random.default_rng(1)
    with open(tmp_path / "in.bin", "wb") as f:
        f.write(np.int64(len(data)).tobytes())
        for x in data:
            f.write(np.int64(x.size).tobytes())
            f.write(x.tobytes())
            f.write(rng.permutation(x).tobytes())
    subprocess.run([str(exe), str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], check=True, timeout=600)
    raw = (tmp_path / "out.bin").read_bytes()
    rec = np.dtype([("s", "<f8", 3), ("same", "<i4")])
    res = np.frombuffer(raw, dtype=rec)
    assert res.size == len(data)
    for x, r in zip(data, res):
        try:
            want = math.fsum(np.abs(x))
        except OverflowError:
            want = math.inf
        assert r["same"] == 1
        for got in r["s"]:
            assert got == want or (math.isinf(want) and math.isinf(got)), (got, want, x[:4])
