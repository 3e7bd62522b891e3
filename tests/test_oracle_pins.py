"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own formulas: worked examples printed in
the paper (tests/golden), textbook closed forms, library routines, brute force and
invariants. None of these tests needs a GPU.
"""
import math

import numpy as np
import pytest
from scipy.special import comb

import oracle as O
import synth
from conftest import load_golden


# ------------------------------------------------------------------ matrix A (Eq. 7-9)

def test_A_matches_worked_example():
    gold = load_golden("A_m5.txt")
    np.testing.assert_array_equal(O.power_matrix_A(5), gold)


def test_A_rows_match_printed_powers_of_Tk():
    gold = load_golden("powers_Tk.txt")
    a = O.power_matrix_A(5)
    for row in gold:
        j = int(row[0])
        np.testing.assert_array_equal(a[j, :5], row[1:])


def test_A_binomial_closed_form():
    # cos^j(t) = 2^{1-j} sum_{r < j/2} C(j, r) cos((j - 2r) t) + 2^{-j} C(j, j/2) [j even]
    m = 14
    a = O.power_matrix_A(m)
    ref = np.zeros((m, m))
    for j in range(m):
        for r in range(j + 1):
            l = j - 2 * r
            if l < 0:
                break
            ref[j, l] = 2.0 ** (-j) * comb(j, j // 2) if l == 0 else 2.0 ** (1 - j) * comb(j, r)
    ref[0, 0] = 1.0
    np.testing.assert_allclose(a, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_A_scalar_identity(k):
    # T_k(x)^j = sum_l a_{j,l} T_{lk}(x)  (Eq. power_of_Tk) on a grid, via cos(n arccos x)
    m = 10
    a = O.power_matrix_A(m)
    th = np.linspace(0.0, np.pi, 57)
    for j in range(m):
        lhs = np.cos(k * th) ** j
        rhs = sum(a[j, l] * np.cos(l * k * th) for l in range(m))
        np.testing.assert_allclose(rhs, lhs, atol=1e-14)


def test_A_lower_triangular_with_parity_zeros():
    a = O.power_matrix_A(9)
    for j in range(9):
        for l in range(9):
            if l > j or (j - l) % 2:
                assert a[j, l] == 0.0


# ------------------------------------------------------------ system X (Eq. X, Appendix)

def test_X_upper_triangular_and_first_row_exception():
    k, m = 4, 5
    x = O.liang_system_X(k, m)
    assert np.all(np.tril(x, -1) == 0.0)
    assert np.all(np.diag(x) != 0.0)
    a = O.power_matrix_A(m)
    # first block row: I blocks carry a_{j,0} without 1/2, J blocks carry a_{j,1}/2
    for i in range(1, k):
        for j in range(m):
            assert x[i, j * k + i] == a[j, 0] + (0.5 * a[j, 1] if i == k - i else 0.0)
    # last block row: a_{m-1,m-1} for i = 0 and a_{m-1,m-1}/2 on the I block
    r0 = (m - 1) * k
    assert x[r0, r0] == a[m - 1, m - 1]
    for i in range(1, k):
        assert x[r0 + i, r0 + i] == 0.5 * a[m - 1, m - 1]


def test_d_and_g_related_by_A():
    # g_{i,l} = d_i^T a_l (the bracket of the derivation): G = D A
    rng = np.random.default_rng(5)
    for k, m in [(3, 4), (5, 5), (6, 2), (2, 7)]:
        c = rng.standard_normal(k * m)
        d = O.liang_d(c, k, m)
        g = O.liang_g(c, k, m)
        np.testing.assert_allclose(d @ O.power_matrix_A(m), g, atol=1e-10)


# ----------------------------------------------------------------- coefficients

def test_interp_of_constants_and_polynomials():
    c = O.chebyshev_interp(lambda x: np.ones_like(x), 8, 64)
    np.testing.assert_allclose(c, [1, 0, 0, 0, 0, 0, 0, 0], atol=1e-15)
    c = O.chebyshev_interp(lambda x: x, 8, 64)
    np.testing.assert_allclose(c, [0, 1, 0, 0, 0, 0, 0, 0], atol=1e-15)
    c = O.chebyshev_interp(lambda x: 16 * x**5 - 20 * x**3 + 5 * x, 8, 64)   # T_5
    np.testing.assert_allclose(c, [0, 0, 0, 0, 0, 1, 0, 0], atol=1e-14)


def test_interp_matches_numpy_chebinterpolate():
    f = lambda x: O.fermi_dirac(x, 0.1, 0.07)
    for deg in (5, 17, 40):
        ref = np.polynomial.chebyshev.chebinterpolate(f, deg)
        np.testing.assert_allclose(O.chebyshev_interp(f, deg + 1, deg + 1), ref, atol=1e-14)


def test_fermi_coeffs_midpoint_symmetry():
    # mu at the centre of [e_a, e_b]: f - 1/2 is odd, so c_0 = 1/2 and even c_n = 0
    c = O.chebyshev_coeffs(0.3, 1.5, -2.0, 5.0, 64)
    assert abs(c[0] - 0.5) < 1e-15
    assert np.max(np.abs(c[2::2])) < 1e-15


def test_fermi_coeffs_step_limit():
    # kT -> 0: f is the step 1[x < mu_x]; c_0 = 1 - phi/pi, c_n = -2 sin(n phi)/(n pi), phi = acos(mu_x)
    ea, eb, mu = -3.0, 1.0, -0.4
    mu_x = (2 * mu - (ea + eb)) / (eb - ea)
    phi = math.acos(mu_x)
    c = O.chebyshev_coeffs(1e-9, mu, ea, eb, 12, n_quad=1 << 17)
    n = np.arange(1, 12)
    ref = np.concatenate([[1 - phi / math.pi], -2 * np.sin(n * phi) / (n * math.pi)])
    np.testing.assert_allclose(c, ref, atol=5e-5)


def test_fermi_coeffs_endpoint_sums():
    ea, eb, mu, kT = -2.0, 3.0, 0.7, 0.4
    c = O.chebyshev_coeffs(kT, mu, ea, eb, 200)
    assert abs(c.sum() - O.fermi_dirac(eb, mu, kT)) < 1e-13
    assert abs((c * (-1.0) ** np.arange(200)).sum() - O.fermi_dirac(ea, mu, kT)) < 1e-13


def test_fermi_expansion_converges_pointwise():
    ea, eb, mu, kT = -1.0, 1.0, 0.2, 0.05
    c = O.chebyshev_coeffs(kT, mu, ea, eb, 256)
    x = np.linspace(-1, 1, 101)
    np.testing.assert_allclose(np.polynomial.chebyshev.chebval(x, c),
                               O.fermi_dirac(x, mu, kT), atol=1e-13)


# ---------------------------------------------------------- routes agree (brute force)

@pytest.mark.parametrize("n_terms", [1, 2, 3, 8, 15, 16, 17, 24, 25, 26, 50])
def test_four_routes_agree(n_terms):
    h = synth.random_symmetric(24, 11)
    ea, eb = O.gershgorin_bounds(h)
    x = O.scale_hamiltonian(h, ea, eb)
    c = O.chebyshev_coeffs(0.05 * (eb - ea), 0.05, ea, eb, n_terms)
    k, m = O.plan_km(n_terms)
    ref = O.poly_eig(h, c, ea, eb)
    for p in (O.chebyshev_naive(x, c), O.liang_cheb_eval(x, O.liang_g(c, k, m)),
              O.liang_power_eval(x, O.liang_d(c, k, m))):
        assert np.abs(p - ref).max() < 1e-13


def test_chebyshev_apply_is_columns_of_naive():
    h = synth.tight_binding(32, 3)
    ea, eb = O.gershgorin_bounds(h)
    x = O.scale_hamiltonian(h, ea, eb)
    c = O.chebyshev_coeffs(0.1, -6.0, ea, eb, 40)
    p = O.chebyshev_naive(x, c)
    cols = [0, 5, 31]
    np.testing.assert_allclose(O.chebyshev_apply(x, c, np.eye(32)[:, cols]), p[:, cols], atol=1e-14)


def test_staged_baby_steps_match_recurrence_and_printed_stages():
    h = synth.random_symmetric(12, 2)
    ea, eb = O.gershgorin_bounds(h)
    x = O.scale_hamiltonian(h, ea, eb)
    t = O.chebyshev_matrices(x, 20)
    for kk in (2, 3, 5, 8, 13, 19):
        staged = O.baby_steps_staged(x, kk)
        assert sorted(staged) == list(range(kk + 1))
        for i, ti in staged.items():
            assert np.abs(ti - t[i]).max() < 1e-13
    for _, n, a, b, cc in load_golden("staged_baby_steps.txt"):
        assert np.abs(2 * t[int(a)] @ t[int(b)] - t[int(cc)] - t[int(n)]).max() < 1e-14


# -------------------------------------------------------------- special cases

def test_diagonal_hamiltonian_gives_diagonal_fermi_values():
    e = np.linspace(-3, 2, 9)
    h = np.diag(e)
    ea, eb = O.gershgorin_bounds(h)
    assert (ea, eb) == (-3.0, 2.0)
    mu, kT = -0.3, 0.5
    res = O.density_matrix(h, None, kT, 120, mu=mu, route="naive")
    assert np.abs(res.p - np.diag(np.diag(res.p))).max() == 0.0
    np.testing.assert_allclose(np.diag(res.p), O.fermi_dirac(e, mu, kT), atol=1e-12)


def test_two_by_two_closed_form():
    a, b, d = 0.3, -0.8, -0.5
    h = np.array([[a, b], [b, d]])
    mu, kT = 0.1, 0.2
    s = math.sqrt(((a - d) / 2) ** 2 + b * b)
    lp, lm = (a + d) / 2 + s, (a + d) / 2 - s
    fp, fm = O.fermi_dirac(lp, mu, kT), O.fermi_dirac(lm, mu, kT)
    ref = (fp * (h - lm * np.eye(2)) - fm * (h - lp * np.eye(2))) / (lp - lm)   # Sylvester
    np.testing.assert_allclose(O.fermi_exact(h, mu, kT), ref, atol=1e-15)
    res = O.density_matrix(h, None, kT, 200, mu=mu, route="liang")
    np.testing.assert_allclose(res.p, ref, atol=1e-13)


def test_known_spectrum_and_truncation_bound():
    rng = np.random.default_rng(9)
    n = 30
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-2, 2, n))
    h = (q * lam) @ q.T
    mu, kT = 0.0, 0.15
    exact = (q * O.fermi_dirac(lam, mu, kT)) @ q.T
    np.testing.assert_allclose(O.fermi_exact(h, mu, kT), exact, atol=1e-13)
    for n_terms in (20, 60, 150):
        res = O.density_matrix(h, None, kT, n_terms, mu=mu, route="naive")
        ea, eb = res.ea, res.eb
        p_lam = np.polynomial.chebyshev.chebval(O.spectrum_scaled(lam, ea, eb), res.coeffs)
        bound = np.max(np.abs(p_lam - O.fermi_dirac(lam, mu, kT)))
        err2 = np.linalg.norm(res.p - exact, 2)
        assert abs(err2 - bound) < 1e-12 + 1e-9 * bound


# ------------------------------------------------------------------ bounds

def test_gershgorin_cases():
    j = np.ones((7, 7))
    assert O.gershgorin_bounds(j) == (1.0 - 6.0, 1.0 + 6.0)
    assert O.gershgorin_bounds(2.5 * np.eye(4)) == (1.5, 3.5)        # degenerate -> centre -+ 1
    h = synth.tight_binding(64, 4)
    ea, eb = O.gershgorin_bounds(h)
    w = np.linalg.eigvalsh(h)
    assert ea <= w[0] and w[-1] <= eb


# --------------------------------------------------------------- moments and mu

def test_moments_two_routes_and_low_order_identities():
    h = synth.tight_binding(40, 8)
    ea, eb = O.gershgorin_bounds(h)
    x = O.scale_hamiltonian(h, ea, eb)
    t_eig = O.moments_eig(O.spectrum_scaled(np.linalg.eigvalsh(h), ea, eb), 30)
    t_mat = O.moments_naive(x, 30)
    np.testing.assert_allclose(t_eig, t_mat, atol=1e-11)
    assert t_eig[0] == 40.0
    assert abs(t_eig[1] - np.trace(x)) < 1e-12
    assert abs(t_eig[2] - (2 * np.sum(x * x) - 40)) < 1e-11


def test_bisection_symmetric_spectrum_gives_zero_mu():
    n = 40
    h = np.diag(-np.ones(n - 1), 1) + np.diag(-np.ones(n - 1), -1)    # bipartite chain
    res = O.density_matrix(h, n / 2, 0.1, 64, route="naive")
    assert res.status == "ok"
    assert abs(res.mu) < 1e-12
    assert abs(np.trace(res.p) - n / 2) < 1e-10


@pytest.mark.parametrize("route", ["eig", "naive", "liang"])
def test_invariants_tight_binding(route):
    n = 96
    h = synth.tight_binding(n, 2000 + n)
    res = O.density_matrix(h, n / 2, 0.1, 400, route=route)
    p = res.p
    assert res.status == "ok"
    assert abs(np.trace(p) - n / 2) < 1e-9
    assert np.abs(p - p.T).max() < 1e-12
    comm = np.linalg.norm(h @ p - p @ h) / (np.linalg.norm(h) * np.linalg.norm(p))
    assert comm < 1e-12
    ev = np.linalg.eigvalsh(p)
    assert ev.min() > -0.05 and ev.max() < 1.05       # Gibbs overshoot of a truncated expansion


def test_idempotent_for_gapped_hamiltonian():
    rng = np.random.default_rng(1)
    n = 20
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-2, -1, n // 2), rng.uniform(1, 2, n // 2)])
    h = (q * lam) @ q.T
    res = O.density_matrix(h, n / 2, 0.05, 400, route="liang", bounds=(-2.1, 2.1))
    assert abs(res.mu) < 1.0
    assert np.abs(res.p @ res.p - res.p).max() < 1e-8


def test_no_bracket_reported():
    h = synth.random_symmetric(16, 1)
    res = O.density_matrix(h, 40.0, 0.05, 32, route="naive", want_p=False)
    assert res.status == "no_bracket"


# ------------------------------------------------------------------ generators

def test_tight_binding_generator_structure():
    n = 64
    h = synth.tight_binding(n, 7)
    assert np.array_equal(h, h.T)
    onsite = np.diag(h).reshape(-1, 4)
    assert np.all(np.abs(onsite - np.array([-10, -5, -5, -5])) < 0.6)
    blocks = h.reshape(16, 4, 16, 4).transpose(0, 2, 1, 3)
    for a in range(16):
        off = blocks[a, a] - np.diag(np.diag(blocks[a, a]))
        assert np.all(off == 0.0)                        # no intra-atom coupling
    mags = np.abs(h[np.triu_indices(n, 1)])
    nz = mags[mags > 0]
    assert nz.max() <= 2.0 and nz.min() >= 2.0 * math.exp(-6.0 / 1.5)
