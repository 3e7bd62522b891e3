"""Index arithmetic of the upper-triangle tile decode (csrc/internal.cuh, upper_tile), checked
on the CPU: block b of a kernel over the tiles on and above the diagonal of a tn x tn grid
(the scaling of H, the plane mirror of the last R, the float64 product tiles) takes tile
(bi, bj) with P(bi) <= b < P(bi + 1), P(x) = x tn - x (x - 1) / 2, bj = bi + b - P(bi). The
kernel estimates bi with a float32 square root and corrects it exactly; this test restates
that arithmetic (float32 where the kernel uses float32) and checks that every upper tile is
taken exactly once, in row-major order, with at most a few correction steps.
"""
import numpy as np
import pytest


def upper_tile(b, tn):
    e = np.float32(2.0) * np.float32(tn) + np.float32(1.0)
    d = np.float32(e * e - np.float32(8.0) * np.float32(b))
    r = int(np.float32((e - np.sqrt(max(d, np.float32(0.0)))) * np.float32(0.5)))
    r = max(0, min(r, tn - 1))
    p = lambda x: x * tn - x * (x - 1) // 2
    steps = 0
    while r > 0 and p(r) > b:
        r -= 1
        steps += 1
    while r + 1 < tn and p(r + 1) <= b:
        r += 1
        steps += 1
    return r, r + (b - p(r)), steps


@pytest.mark.parametrize("tn", [1, 2, 3, 8, 33, 160, 1024])
def test_every_upper_tile_once_in_order(tn):
    want = [(i, j) for i in range(tn) for j in range(i, tn)]
    got = []
    for b in range(tn * (tn + 1) // 2):
        bi, bj, steps = upper_tile(b, tn)
        assert steps <= 2
        got.append((bi, bj))
    assert got == want


@pytest.mark.parametrize("tn", [2048, 4096])
def test_row_boundaries_large(tn):
    """The largest grids: 32-wide tiles at n_pad = 65536 (tn = 2048) and beyond."""
    p = lambda x: x * tn - x * (x - 1) // 2
    rows = list(range(0, 30)) + list(range(tn // 2 - 15, tn // 2 + 15)) + list(range(tn - 30, tn))
    for r in rows:
        for b in (p(r), p(r) + 1, p(r + 1) - 1):
            if b < p(r) or b >= tn * (tn + 1) // 2:
                continue
            bi, bj, steps = upper_tile(b, tn)
            assert (bi, bj) == (r, r + b - p(r)) and steps <= 4
    assert tn * (tn + 1) // 2 < 2 ** 31 and p(tn - 1) < 2 ** 31
