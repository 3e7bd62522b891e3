"""Pins of the learned-mu oracle (oracle/mlp.py) against mathematics it does not share code
with: central finite differences, closed forms of special cases, brute force, and library
routines (numpy's Chebyshev series)."""
import math

import numpy as np
import pytest

import oracle.mlp as M


def small_batch(seed=0, B=3):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, M.N_IN))
    t = rng.normal(size=(B, M.N_OUT))
    return x, t


def test_silu_derivative_matches_finite_differences():
    z = np.linspace(-8, 8, 401)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.silu_grad(z))) < 1e-8
    # silu(0) = 0, silu'(0) = 1/2, silu(z) -> z for large z
    assert M.silu(np.array(0.0)) == 0.0 and M.silu_grad(np.array(0.0)) == 0.5
    assert abs(M.silu(np.array(40.0)) - 40.0) < 1e-12


def test_zero_weights_give_the_output_bias():
    p = {k: np.zeros(s) for k, s in M.param_shapes()}
    p["b3"] = np.array([0.3, -1.2])
    x, t = small_batch()
    y, _ = M.forward(p, x)
    assert np.array_equal(y, np.tile(p["b3"], (3, 1)))
    w = [1.0, 0.1]
    L, g = M.gradients(p, x, t, w)
    assert L == pytest.approx(np.sum(np.array(w) * (p["b3"] - t) ** 2) / 3)
    assert np.allclose(g["b3"], 2 * np.array(w) * np.mean(p["b3"] - t, axis=0))
    # with a2 = silu(0) = 0 nothing upstream of W3 moves
    for k in ("W1", "b1", "W2", "b2", "W3"):
        assert not np.any(g[k])


@pytest.mark.parametrize("seed", [1, 2])
def test_gradients_match_central_differences(seed):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 10)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    x, t = small_batch(seed)
    w = [1.0, 0.1]
    _, g = M.gradients(p, x, t, w)
    h = 1e-6
    for k, shp in M.param_shapes():
        flat = p[k].ravel()
        idx = rng.choice(flat.size, size=min(flat.size, 40), replace=False)
        for i in idx:
            orig = flat[i]
            flat[i] = orig + h
            lp = M.loss(p, x, t, w)
            flat[i] = orig - h
            lm = M.loss(p, x, t, w)
            flat[i] = orig
            fd = (lp - lm) / (2 * h)
            an = g[k].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (k, i, fd, an)


def test_adam_first_steps_closed_form():
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.2, -3.0, 0.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    lr, eps = 0.01, 1e-8
    M.adam_step(p, g, m, v, 1, lr, eps=eps)
    # bias-corrected first step: mhat = g, vhat = g^2 -> update lr g / (|g| + eps)
    assert np.allclose(p["a"], [1.0 - lr * 0.2 / (0.2 + eps), -2.0 + lr * 3.0 / (3.0 + eps), 0.5])
    # second step with the same gradient: still lr per unit of sign(g)
    M.adam_step(p, g, m, v, 2, lr, eps=eps)
    assert np.allclose(p["a"], [1.0 - 2 * lr, -2.0 + 2 * lr, 0.5], atol=1e-9)


def test_features_of_a_diagonal_hamiltonian():
    # X = diag(x): tau_n = sum_i T_n(x_i), by numpy's Chebyshev series
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, 50)
    tau = np.array([np.sum(np.polynomial.chebyshev.chebval(x, np.eye(70)[j])) for j in range(70)])
    f = M.features(tau, 50, 25.0, 0.1, -4.0, 6.0, k=10)
    assert np.allclose(f[:20], tau[1:21] / 50)
    assert not np.any(f[20:M.N_MOM])              # beyond 2k = 20 moments
    assert f[M.N_MOM] == 0.5 and f[M.N_MOM + 1] == pytest.approx(0.02)
    assert (f[M.N_MOM + 2], f[M.N_MOM + 3]) == (-0.04, 0.06)


def test_order_from_coefficients_brute_force():
    rng = np.random.default_rng(4)
    for trial in range(50):
        nt = int(rng.integers(5, 40))
        c = rng.normal(size=nt) * np.exp(-0.3 * np.arange(nt))
        L = M.order_from_coefficients(c, eps=1e-3)

        def ok(L0):
            return np.sum(np.abs(c[L0:])) <= 1e-3

        assert ok(L) and 1 <= L <= nt
        assert min(j for j in range(1, nt + 1) if ok(j)) == L


def test_order_from_coefficients_geometric_closed_form():
    # c_j = r^j: the tail from L is (r^L - r^nt) / (1 - r); the order is the smallest L >= 1
    # with that at most eps
    for r, nt, eps in ((0.5, 60, 1e-6), (0.9, 400, 2.5e-7), (0.97, 300, 1e-3)):
        c = r ** np.arange(nt, dtype=np.float64)
        L = M.order_from_coefficients(c, eps)
        expect = next(j for j in range(1, nt + 1) if (r ** j - r ** nt) / (1 - r) <= eps * (1 + 1e-12))
        assert L == expect


def test_order_cut_bounds_the_change_of_p():
    # the bound behind the target: the expansion cut at L* differs from the full one by at
    # most sum_{j >= L*} |c_j| on every eigenvalue of X in [-1, 1]
    rng = np.random.default_rng(9)
    x = np.sort(rng.uniform(-1, 1, 200))
    c = rng.normal(size=120) * np.exp(-0.08 * np.arange(120))
    L = M.order_from_coefficients(c, eps=1e-4)
    full = np.polynomial.chebyshev.chebval(x, c)
    cut = np.polynomial.chebyshev.chebval(x, c[:L])
    assert np.max(np.abs(full - cut)) <= np.sum(np.abs(c[L:])) <= 1e-4


def test_targets_scale_mu_onto_the_chebyshev_axis():
    c = np.array([0.5, 0.1, 0.0, 0.0])
    t = M.targets(1.0, -3.0, 7.0, c)
    assert t[0] == pytest.approx((2 * 1.0 - 4.0) / 10.0)
    mid, half = 2.0, 5.0
    assert mid + half * t[0] == pytest.approx(1.0)
    assert t[1] == pytest.approx(0.5)    # c_1 = 0.1 > eps: L* = 2 terms; log2(2) / log2(4)


def test_planted_backprop_mistake_is_caught(monkeypatch):
    """A sign slip in the activation derivative fails the finite-difference pin."""
    p = M.init_params(5)
    x, t = small_batch(5)
    w = [1.0, 0.1]
    monkeypatch.setattr(M, "silu_grad", lambda z: (1 / (1 + np.exp(-z))) * (1 - z * (1 - 1 / (1 + np.exp(-z)))))
    _, g = M.gradients(p, x, t, w)
    monkeypatch.undo()
    h = 1e-6
    flat = p["W1"].ravel()
    bad = 0
    for i in range(0, flat.size, 997):
        o = flat[i]
        flat[i] = o + h
        lp = M.loss(p, x, t, w)
        flat[i] = o - h
        lm = M.loss(p, x, t, w)
        flat[i] = o
        if abs((lp - lm) / (2 * h) - g["W1"].ravel()[i]) > 1e-6 * max(1e-3, abs((lp - lm) / (2 * h))):
            bad += 1
    assert bad > 0
