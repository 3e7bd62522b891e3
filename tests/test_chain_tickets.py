"""Host-side check of the chain launch's work list (no GPU): the ticket decode of the chained
product kernel, restated, over batches of instances of different sizes and window budgets.

Every (step, instance, tile) must be decoded from exactly one ticket, and every tile's
dependencies -- the tiles of the previous step of the same instance -- must hold smaller
tickets. A CTA takes its ticket when it starts, so every ticket a tile waits on belongs to a
CTA that is already running: the chain cannot deadlock. The per-instance counter index stays
inside the counters of the launch.
"""
import numpy as np
import pytest


def tiles_128(np_):
    """Symmetric 128-wide tiles of an n_pad x n_pad product (row blocks I, J >= I)."""
    nb = np_ // 128
    return nb * (nb + 1) // 2


def tiles_256(np_):
    """Symmetric 256-wide tiles: column tiles J >= (128 I) / 256 in each 128-row block I."""
    tm, tn = np_ // 128, (np_ + 255) // 256
    return sum(tn - (128 * i) // 256 for i in range(tm))


def windows(pre, i0, i1, nsteps, win_tiles, max_win=64):
    """The window table: consecutive instances with at least win_tiles tiles per step."""
    base, j, out = 0, i0, []
    while j < i1:
        k = j + 1
        if win_tiles > 0:
            while k < i1 and pre[k] - pre[j] < win_tiles:
                k += 1
        else:
            k = i1
        if len(out) == max_win - 1:
            k = i1
        out.append((base, j))
        base += nsteps * (pre[k] - pre[j])
        j = k
    out.append((base, i1))
    return out


def decode(t, win, pre):
    w = 0
    while w + 1 < len(win) - 1 and win[w + 1][0] <= t:
        w += 1
    wi0, wi1 = win[w][1], win[w + 1][1]
    tw = pre[wi1] - pre[wi0]
    local = t - win[w][0]
    s = local // tw
    gtile = pre[wi0] + local - s * tw
    inst = int(np.searchsorted(pre, gtile, side="right") - 1)
    assert wi0 <= inst < wi1
    return s, inst, gtile - pre[inst]


@pytest.mark.parametrize("tiles", [tiles_128, tiles_256])
@pytest.mark.parametrize("win_tiles", [0, 1, 7, 40, 500])
def test_tickets_cover_each_tile_once_and_respect_dependencies(tiles, win_tiles):
    rng = np.random.default_rng(3)
    n = 4 * np.round(np.exp(rng.uniform(np.log(64), np.log(1024), 90)) / 4).astype(int)
    npad = np.sort(-(-n // 128) * 128)[::-1]                 # sorted largest first
    per = np.array([tiles(int(x)) for x in npad])
    pre = np.concatenate([[0], np.cumsum(per)])
    i0, i1, nsteps = 5, 80, 9                                 # a group inside the batch
    win = windows(pre, i0, i1, nsteps, win_tiles)
    total = win[-1][0]
    assert total == nsteps * (pre[i1] - pre[i0])
    seen = {}
    for t in range(total):
        s, inst, tile = decode(t, win, pre)
        assert 0 <= s < nsteps and 0 <= tile < per[inst]
        assert 0 <= inst - i0 < i1 - i0                       # counter index in range
        key = (s, inst, tile)
        assert key not in seen
        seen[key] = t
    assert len(seen) == total
    for (s, inst, tile), t in seen.items():
        if s > 0:
            assert max(seen[(s - 1, inst, q)] for q in range(per[inst])) < t


def test_window_table_is_bounded():
    pre = np.arange(0, 1001)                                  # 1000 one-tile instances
    win = windows(pre, 0, 1000, 3, 1)
    assert len(win) - 1 == 64 and win[-1] == (3000, 1000)
