"""Plant plausible mistakes in the CPU oracle and check that a pin catches each one.

Each mutation replaces one oracle function by a copy with a single slip (a dropped term, a
wrong sign, a transposed index). The pins in test_oracle_pins.py are then re-run against
the mutated oracle and must fail. Everything runs on the CPU.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.fermi as OF
import test_oracle_pins as pins


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(OF, name, fn)
    monkeypatch.setattr(O, name, fn)


def test_fermi_dirac_closed_form_values():
    mu, kT = 0.3, 0.07
    assert O.fermi_dirac(mu, mu, kT) == 0.5
    assert abs(O.fermi_dirac(mu + kT * math.log(3.0), mu, kT) - 0.25) < 1e-15
    assert abs(O.fermi_dirac(mu - kT * math.log(3.0), mu, kT) - 0.75) < 1e-15
    assert O.fermi_dirac(mu + 100.0, mu, kT) == 0.0


MUTATIONS = []


def mutation(fn):
    MUTATIONS.append(fn)
    return fn


@mutation
def a_recursion_drops_half(monkeypatch):
    orig = OF.power_matrix_A

    def bad(m):
        a = orig(m).copy()
        for j in range(2, m):                # l = 1 case without the 1/2 on a_{j-1,2}
            a[j, 1] = (a[j - 1, 0] if j - 1 >= 0 else 0) + (a[j - 1, 2] if j - 1 >= 2 else 0.0)
        return a
    _patch(monkeypatch, "power_matrix_A", bad)
    return pins.test_A_matches_worked_example


@mutation
def g_transposed_index(monkeypatch):
    def bad(c, k, m):
        cc = np.zeros(k * m)
        cc[: len(c)] = c
        g = np.zeros((k, m))
        for l in range(m - 1, -1, -1):
            g[0, l] = cc[l * k]
            for i in range(1, k):
                ci = cc[l * k + i]
                if m == 1:
                    g[i, l] = ci
                elif l == m - 1:
                    g[i, l] = 2.0 * ci
                elif l == 0:
                    g[i, l] = ci - 0.5 * g[i, 1]          # should be g[k - i, 1]
                else:
                    g[i, l] = 2.0 * ci - g[k - i, l + 1]
        return g
    _patch(monkeypatch, "liang_g", bad)
    return lambda: pins.test_four_routes_agree(26)


@mutation
def giant_step_sign(monkeypatch):
    def bad(x, g):
        k, m = g.shape
        t = OF.chebyshev_matrices(x, k + 1)
        r = [sum(g[i, l] * t[i] for i in range(k)) for l in range(m)]
        giant = [t[0], t[k]]
        for _ in range(2, m):
            giant.append(2.0 * t[k] @ giant[-1] + giant[-2])
        return sum(giant[l] @ r[l] for l in range(m))
    _patch(monkeypatch, "liang_cheb_eval", bad)
    return lambda: pins.test_four_routes_agree(26)


@mutation
def naive_recursion_missing_factor_two(monkeypatch):
    def bad(x, c):
        n = x.shape[0]
        t_prev, t_cur = np.eye(n), x.copy()
        p = c[0] * t_prev + (c[1] * t_cur if len(c) > 1 else 0)
        for j in range(2, len(c)):
            t_prev, t_cur = t_cur, x @ t_cur - t_prev
            p = p + c[j] * t_cur
        return p
    _patch(monkeypatch, "chebyshev_naive", bad)
    return lambda: pins.test_four_routes_agree(17)


@mutation
def c0_without_half(monkeypatch):
    orig = OF.chebyshev_interp

    def bad(fun, n_terms, n_quad):
        c = orig(fun, n_terms, n_quad)
        c[0] *= 2.0
        return c
    _patch(monkeypatch, "chebyshev_interp", bad)
    return pins.test_interp_of_constants_and_polynomials


@mutation
def scaling_sign_flip(monkeypatch):
    def bad(h, ea, eb):
        return ((ea + eb) * np.eye(h.shape[0]) - 2.0 * h) / (eb - ea)
    _patch(monkeypatch, "scale_hamiltonian", bad)
    return pins.test_diagonal_hamiltonian_gives_diagonal_fermi_values


@mutation
def gershgorin_without_abs(monkeypatch):
    def bad(h):
        d = np.diag(h)
        r = np.sum(h, axis=1) - d
        return float(np.min(d - r)), float(np.max(d + r))
    _patch(monkeypatch, "gershgorin_bounds", bad)
    return pins.test_gershgorin_cases


@mutation
def bisection_wrong_direction(monkeypatch):
    orig = OF.bisect_mu

    def bad(trace_fn, n_e, ea, eb, kT, max_iter=200, widen_steps=8):
        return orig(lambda mu: 2 * n_e - trace_fn(mu), n_e, ea, eb, kT, max_iter, widen_steps)
    _patch(monkeypatch, "bisect_mu", bad)
    return lambda: pins.test_invariants_tight_binding("naive")


@mutation
def fermi_sign_flip(monkeypatch):
    def bad(e, mu, kT):
        with np.errstate(over="ignore"):
            return 1.0 / (1.0 + np.exp(-(np.asarray(e, dtype=np.float64) - mu) / kT))
    _patch(monkeypatch, "fermi_dirac", bad)
    return test_fermi_dirac_closed_form_values


@mutation
def moments_off_by_one(monkeypatch):
    def bad(x_evals, count):
        xs = np.clip(np.asarray(x_evals, dtype=np.float64), -1.0, 1.0)
        return np.cos(np.outer(np.arange(1, count + 1), np.arccos(xs))).sum(axis=1)
    _patch(monkeypatch, "moments_eig", bad)
    return pins.test_moments_two_routes_and_low_order_identities


@mutation
def x_system_missing_half(monkeypatch):
    orig = OF.liang_system_X

    def bad(k, m):
        x = orig(k, m)
        r0 = (m - 1) * k
        for i in range(1, k):
            x[r0 + i, r0 + i] *= 2.0                 # last block row without the 1/2
        return x
    _patch(monkeypatch, "liang_system_X", bad)
    return lambda: pins.test_four_routes_agree(25)


@pytest.mark.parametrize("mut", MUTATIONS, ids=[f.__name__ for f in MUTATIONS])
def test_pin_catches_planted_mistake(mut, monkeypatch):
    check = mut(monkeypatch)
    with pytest.raises(AssertionError):
        check()
