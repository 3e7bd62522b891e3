"""Index arithmetic of the contraction kernel, checked on the CPU.

k_contract_f32 walks the upper triangle of an n_pad x n_pad matrix as 16-byte quads: row r
holds the quads starting at columns 4 floor(r / 4), ..., n_pad - 4. Quad q of the flattened
order lies in the row group b = floor(r / 4) with C(b) <= q < C(b + 1),
C(b) = b n_pad - 2 b (b - 1); the kernel estimates b with a float32 square root and
corrects it exactly. This test restates that arithmetic (float32 where the kernel uses
float32) and checks that it enumerates every upper quad exactly once and that the estimate
is never more than a few steps off, so that the kernel's correction loops stay short.
"""
import numpy as np
import pytest


def locate(q, npad):
    g = npad // 4
    d = np.float32(np.float32(npad + 2) * np.float32(npad + 2) - np.float32(8.0) * np.float32(q))
    b = int(np.float32((np.float32(npad + 2) - np.sqrt(max(d, np.float32(0.0)))) * np.float32(0.25)))
    b = max(0, min(b, g - 1))
    c_of = lambda x: x * npad - 2 * x * (x - 1)
    steps = 0
    while b > 0 and c_of(b) > q:
        b -= 1
        steps += 1
    while b + 1 < g and c_of(b + 1) <= q:
        b += 1
        steps += 1
    length = g - b
    off = q - c_of(b)
    return 4 * b + off // length, 4 * b + 4 * (off % length), steps


def quads(npad):
    return npad * (npad + 4) // 8   # ct_quads


@pytest.mark.parametrize("npad", [128, 256, 640, 1024])
def test_every_upper_quad_once(npad):
    seen = set()
    for q in range(quads(npad)):
        r, c, steps = locate(q, npad)
        assert steps <= 1
        assert 0 <= r < npad and c % 4 == 0 and 4 * (r // 4) <= c <= npad - 4
        seen.add((r, c))
    want = {(r, c) for r in range(npad) for c in range(4 * (r // 4), npad, 4)}
    assert seen == want


@pytest.mark.parametrize("npad", [5120, 32768, 65536])
def test_group_boundaries_large(npad):
    g = npad // 4
    c_of = lambda x: x * npad - 2 * x * (x - 1)
    groups = list(range(0, 40)) + list(range(g // 2 - 20, g // 2 + 20)) + list(range(g - 40, g))
    for b in groups:
        for q in (c_of(b), c_of(b) + 1, c_of(b + 1) - 1):
            if q >= quads(npad):
                continue
            r, c, steps = locate(q, npad)
            assert r // 4 == b and steps <= 4
    # the last quad is the last row's only one
    assert locate(quads(npad) - 1, npad)[:2] == (npad - 1, npad - 4)


def test_indices_fit_32_bits_at_the_largest_size():
    """The kernel locates quads in 32-bit integers: at the largest n_pad (65536, the library's
    size limit) the quad index, C(b) and b n_pad stay below 2^31."""
    npad = 65536
    g = npad // 4
    assert quads(npad) < 2 ** 31
    b = np.arange(g, dtype=np.int64)
    assert int((b * npad).max()) < 2 ** 31
    assert int((b * npad - 2 * b * (b - 1)).max()) < 2 ** 31
    assert int((2 * b * (b - 1)).max()) < 2 ** 31
