"""Pins of the Lanczos-bounds oracle (oracle/lanczos.py): the published splitmix64 sequence,
exactness of Lanczos on small matrices (eigenvalues of T_n = those of H, by LAPACK), the
residual bound on a diagonal matrix, and enclosure of the model spectra."""
import numpy as np
import pytest

import oracle as O
import oracle.lanczos as L
import synth


def test_splitmix64_published_sequence():
    # splitmix64 seeded with 0: 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f
    u = L.splitmix64_uniform(0, 3)
    raw = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert np.array_equal(u, np.array([(r >> 11) * 2.0 ** -53 for r in raw]))


def test_full_lanczos_reproduces_the_spectrum():
    rng = np.random.default_rng(0)
    g = rng.normal(size=(8, 8))
    h = (g + g.T) / 2
    alpha, beta = L.lanczos_tridiagonal(h, 8)
    K = len(alpha)
    assert K == 8
    t = np.diag(alpha) + np.diag(beta[1:K], 1) + np.diag(beta[1:K], -1)
    assert np.allclose(np.linalg.eigvalsh(t), np.linalg.eigvalsh(h), atol=1e-10)
    assert beta[K] < 1e-8


def test_known_spectrum_bounds_are_the_extremes_plus_margin():
    # Q diag(d) Q^T: Gershgorin is loose, full Lanczos finds the extremes with zero residual
    d = np.linspace(-3.0, 5.0, 12)
    q, _ = np.linalg.qr(np.random.default_rng(2).normal(size=(12, 12)))
    h = q @ np.diag(d) @ q.T
    lo, hi = L.lanczos_bounds(h, steps=12)
    w = 8.0
    assert lo == pytest.approx(-3.0 - L.MARGIN * w, abs=1e-9)
    assert hi == pytest.approx(5.0 + L.MARGIN * w, abs=1e-9)


@pytest.mark.parametrize("kind,n", [("tb", 200), ("tb", 600), ("rand", 128)])
def test_bounds_enclose_and_tighten(kind, n):
    h = synth.tight_binding(n, 70 + n) if kind == "tb" else synth.random_symmetric(n, 3)
    ev = np.linalg.eigvalsh(h)
    lo, hi = L.lanczos_bounds(h, steps=40)
    ga, gb = O.gershgorin_bounds(h)
    assert lo <= ev[0] and hi >= ev[-1]
    assert ga <= lo and hi <= gb
    if kind == "tb":
        assert (hi - lo) < 0.5 * (gb - ga)


def test_planted_lanczos_mistake_is_caught(monkeypatch):
    """Dropping the beta q_{j-1} term breaks the three-term recurrence: the tridiagonal no
    longer carries the spectrum of H."""
    rng = np.random.default_rng(1)
    g = rng.normal(size=(8, 8))
    h = (g + g.T) / 2

    def broken(hh, steps, seed=L.LANCZOS_SEED):
        n = hh.shape[0]
        q = L.start_vector(n, seed)
        alpha, beta = [], [0.0]
        for _ in range(min(steps, n)):
            w = hh @ q
            a = float(w @ q)
            w = w - a * q
            b = float(np.linalg.norm(w))
            alpha.append(a)
            beta.append(b)
            q = w / b
        return np.array(alpha), np.array(beta)

    alpha, beta = broken(h, 8)
    t = np.diag(alpha) + np.diag(beta[1:8], 1) + np.diag(beta[1:8], -1)
    assert not np.allclose(np.linalg.eigvalsh(t), np.linalg.eigvalsh(h), atol=1e-6)
