"""GPU parity: every stage of the CUDA path against the CPU FP64 oracle, through the C ABI.

Tolerances (stated per test):
* float64 path: ||P - P_ref||_F / sqrt(N) <= 1e-10 and |tr P - N_e| <= 1e-8;
* split-precision paths: ||P - P_ref||_F / sqrt(N) <= 1e-6 for BF16x3 (FP16x2 and BF16x1 are
  measured and bounded by their own looser arithmetic limits);
* scalars (bounds, coefficients): relative 1e-13 / absolute 1e-13.
The oracle P is evaluated at the bounds and mu the GPU reports, which isolates the expansion
from the mu search; mu itself is compared with the oracle's own bisection separately.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
import paper_2306_12616_gb300 as fo

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def to_dev(h):
    return torch.from_numpy(np.ascontiguousarray(h)).to(DEV)


def rel_frob(p, ref):
    return float(np.linalg.norm(p - ref) / math.sqrt(p.shape[0]))


# --------------------------------------------------------------------- bounds

@pytest.mark.parametrize("n", [1, 3, 17, 64, 129, 256, 1000])
def test_bounds_match_oracle(solver, n):
    h = synth.random_symmetric(n, 100 + n)
    b = solver.spectral_bounds(to_dev(h)).cpu().numpy()
    ea, eb = O.gershgorin_bounds(h)
    assert abs(b[0] - ea) <= 1e-13 * max(1, abs(ea))
    assert abs(b[1] - eb) <= 1e-13 * max(1, abs(eb))
    assert b[2] == 0.0


@pytest.mark.parametrize("n,kind", [(1, "rand"), (33, "rand"), (1000, "rand"), (776, "tb"), (2048, "tb")])
def test_bounds_are_correctly_rounded_row_sums(solver, n, kind):
    """The Gershgorin radii are the row sums of |h_ij| rounded once (exact integer sums on the
    device): the bounds equal, bit for bit, min/max of h_ii -/+ math.fsum(|h_ij|, j != i) with
    the float64 subtraction and addition, for any order of the terms."""
    h = synth.random_symmetric(n, 300 + n) if kind == "rand" else synth.tight_binding(n, 300 + n)
    if kind == "rand":
        h[0, -1] = h[-1, 0] = 1e-200   # a far smaller entry and a large one in the same rows
        h[0, 0] = 3e5
    b = solver.spectral_bounds(to_dev(h)).cpu().numpy()
    r = np.array([math.fsum(np.abs(np.delete(h[i], i))) for i in range(n)])
    d = np.diag(h)
    lo, hi = np.min(d - r), np.max(d + r)
    if n == 1:
        lo, hi = d[0] - 1.0, d[0] + 1.0   # a single entry: the degenerate interval is widened
    assert b[0] == lo and b[1] == hi and b[2] == 0.0


def test_bounds_flag_nonfinite(solver):
    h = synth.random_symmetric(40, 1)
    h[3, 7] = np.nan
    b = solver.spectral_bounds(to_dev(h)).cpu().numpy()
    assert b[2] == 1.0


def test_bounds_tight_binding_and_strided(solver):
    h = synth.tight_binding(300, 7)
    big = np.zeros((300, 333))
    big[:, :300] = h
    d = to_dev(big)[:, :300]
    b = solver.spectral_bounds(d).cpu().numpy()
    ea, eb = O.gershgorin_bounds(h)
    assert abs(b[0] - ea) <= 1e-13 * abs(ea) and abs(b[1] - eb) <= 1e-13 * abs(eb)


# --------------------------------------------------------------- coefficients

@pytest.mark.parametrize("n_terms,kT,mu", [(1, 0.5, 0.0), (16, 0.3, -1.0), (400, 0.1, -6.0),
                                           (1000, 0.01, 0.0), (257, 2.0, 3.0)])
def test_coefficients_match_oracle(solver, n_terms, kT, mu):
    ea, eb = -20.0, 12.0
    c = solver.chebyshev_coeffs(kT, mu, ea, eb, n_terms).cpu().numpy()
    ref = O.chebyshev_coeffs(kT, mu, ea, eb, n_terms)
    np.testing.assert_allclose(c, ref, rtol=0, atol=1e-13)


# --------------------------------------------------------------------- moments

@pytest.mark.parametrize("n,n_mom", [(64, 10), (200, 33), (256, 64)])
def test_moments_float64(solver, n, n_mom):
    h = synth.tight_binding(n, 3 + n)
    dh = to_dev(h)
    b = solver.spectral_bounds(dh)
    tau = solver.moments(dh, b, n_mom, "fp64").cpu().numpy()
    ea, eb = b[0].item(), b[1].item()
    ref = O.moments_eig(O.spectrum_scaled(np.linalg.eigvalsh(h), ea, eb), n_mom)
    np.testing.assert_allclose(tau, ref, rtol=0, atol=1e-9 * n)


# ------------------------------------------------------- float64 density matrix

@pytest.mark.parametrize("n,n_terms", [(1, 5), (3, 2), (17, 1), (17, 16), (64, 17), (129, 50),
                                       (256, 256), (300, 101)])
def test_fp64_fixed_mu_matches_oracle(solver, n, n_terms):
    h = synth.random_symmetric(n, 7 + n)
    ea, eb = O.gershgorin_bounds(h)
    kT, mu = 0.05 * (eb - ea), 0.1 * ea + 0.9 * (0.5 * (ea + eb))
    prm = solver.params(n_terms, kT, mu=mu, precision="fp64", mu_mode="fixed")
    p, res = solver.density_matrix(to_dev(h), n / 2, prm)
    p = p.cpu().numpy()
    assert res["status"] == 0
    assert (res["emin"], res["emax"]) == pytest.approx((ea, eb), rel=1e-13)
    ref = O.density_matrix(h, None, kT, n_terms, mu=mu, bounds=(res["emin"], res["emax"]),
                           route="eig").p
    assert rel_frob(p, ref) <= 1e-10
    k, m = O.plan_km(n_terms)
    assert (res["k"], res["m"]) == (k, m)
    assert res["n_gemm"] == (k - 1) + (m - 1)


def test_fp64_given_bounds_and_strided_output(solver):
    n, n_terms = 100, 64
    h = synth.tight_binding(n, 11)
    kT, mu = 0.2, -6.0
    prm = solver.params(n_terms, kT, mu=mu, precision="fp64", mu_mode="fixed", bounds=(-40.0, 30.0))
    out = torch.zeros((n, n + 9), dtype=torch.float64, device=DEV)
    p, res = solver.density_matrix(to_dev(h), n / 2, prm, out=out[:, :n])
    ref = O.density_matrix(h, None, kT, n_terms, mu=mu, bounds=(-40.0, 30.0), route="naive").p
    assert rel_frob(out[:, :n].cpu().numpy(), ref) <= 1e-10
    assert float(out[:, n:].abs().max()) == 0.0


def test_fp64_random_config_bisection(solver):
    # N = 256 random symmetric H, N_e = 128, kT = 0.05 (e_b - e_a), 256 terms (k = m = 16)
    n, n_terms = 256, 256
    h = synth.random_symmetric(n, 1)
    ea, eb = O.gershgorin_bounds(h)
    kT = 0.05 * (eb - ea)
    prm = solver.params(n_terms, kT, precision="fp64", mu_mode="bisect")
    p, res = solver.density_matrix(to_dev(h), 128.0, prm)
    p = p.cpu().numpy()
    assert res["status"] == 0 and (res["k"], res["m"]) == (16, 16)
    orc = O.density_matrix(h, 128.0, kT, n_terms, route="eig")
    assert abs(res["mu"] - orc.mu) <= 1e-9 * (eb - ea)
    ref = O.density_matrix(h, None, kT, n_terms, mu=res["mu"], bounds=(res["emin"], res["emax"]),
                           route="eig").p
    assert rel_frob(p, ref) <= 1e-10
    assert abs(np.trace(p) - 128.0) <= 1e-8
    assert abs(res["trace"] - 128.0) <= 1e-8
    assert res["n_gemm"] == 15 + 14 + 15


@pytest.mark.parametrize("n", [100, 1000, 2000])
def test_fp64_tight_binding_bisection(solver, n):
    h = synth.tight_binding(n, 2000 + n)
    prm = solver.params(400, 0.1, precision="fp64", mu_mode="bisect")
    p, res = solver.density_matrix(to_dev(h), n / 2, prm)
    p = p.cpu().numpy()
    assert res["status"] == 0
    orc = O.density_matrix(h, n / 2, 0.1, 400, route="eig", want_p=False)
    assert abs(res["mu"] - orc.mu) <= 1e-9
    ref = O.density_matrix(h, None, 0.1, 400, mu=res["mu"], bounds=(res["emin"], res["emax"]),
                           route="eig").p
    assert rel_frob(p, ref) <= 1e-10
    assert abs(np.trace(p) - n / 2) <= 1e-8


def test_fp64_full_size_sampled_columns(solver):
    """The float64 path at the largest bench size (N = 5000, 400 terms): sampled columns of P
    against the oracle polynomial at the GPU's bounds and mu (from the oracle's
    eigendecomposition), mu against the oracle's bisection on the eigenvalues, the trace."""
    from conftest import poly_columns, tb_eig
    n = 5000
    h, w, _ = tb_eig(n)
    p, res = solver.density_matrix(to_dev(h), n / 2, solver.params(400, 0.1, precision="fp64", mu_mode="bisect"))
    assert res["status"] == 0 and (res["k"], res["m"]) == (20, 20)
    cols = np.arange(7, n, n // 8)
    c = O.chebyshev_coeffs(0.1, res["mu"], res["emin"], res["emax"], 400)
    ref = poly_columns(n, cols, c, res["emin"], res["emax"])
    err = math.sqrt(np.mean(np.sum((p[:, cols].cpu().numpy() - ref) ** 2, axis=0)))
    assert err <= 1e-10, err
    assert abs(res["trace"] - n / 2) <= 1e-8
    ga, gb = O.gershgorin_bounds(h)
    taus = O.moments_eig(O.spectrum_scaled(w, ga, gb), 400)
    br = O.bisect_mu(lambda mu: O.poly_trace(mu, taus, 0.1, ga, gb, 400), n / 2, ga, gb, 0.1)
    assert br.status == "ok" and abs(res["mu"] - br.mu) <= 1e-9


def test_fp64_host_buffers(solver):
    n = 200
    h = synth.tight_binding(n, 5)
    ht = torch.from_numpy(h).pin_memory()
    out = torch.empty((n, n), dtype=torch.float64).pin_memory()
    prm = solver.params(144, 0.1, precision="fp64", mu_mode="bisect")
    res = solver.density_matrix_host(ht, n / 2, prm, out)
    ref = O.density_matrix(h, None, 0.1, 144, mu=res["mu"], bounds=(res["emin"], res["emax"]),
                           route="eig").p
    assert rel_frob(out.numpy(), ref) <= 1e-10


def test_nonfinite_input_reported(solver):
    h = synth.random_symmetric(32, 2)
    h[0, 0] = np.inf
    prm = solver.params(16, 0.1, precision="fp64", mu_mode="bisect")
    with pytest.raises(fo.FermiError) as e:
        solver.density_matrix(to_dev(h), 16.0, prm)
    assert e.value.status == fo.FO_ERR_NONFINITE


def test_argument_errors(solver):
    h = to_dev(synth.random_symmetric(8, 1))
    prm = solver.params(0, 0.1, precision="fp64", mu_mode="fixed")
    with pytest.raises(fo.FermiError) as e:
        solver.density_matrix(h, 4.0, prm)
    assert e.value.status == fo.FO_ERR_ARG
    prm = solver.params(8, -1.0, precision="fp64", mu_mode="fixed")
    with pytest.raises(fo.FermiError):
        solver.density_matrix(h, 4.0, prm)


@pytest.mark.parametrize("prec,tol", [("bf16x3", 2e-6), ("fp64", 1e-10)])
@pytest.mark.parametrize("n_terms,k", [(160, 8), (400, 8)])
def test_forced_baby_step_count(solver, prec, tol, n_terms, k):
    """A forced k changes the split of the n_terms coefficients between baby and giant steps
    (k = 8 at 160 terms: 19 giants x 7 babies in the Frobenius products, 5 x 4 tiles; at 400
    terms: m = 50, 49 x 7 pairs over two launches of 4 x 4 tiles, and two contraction launches
    for R_0..R_49), not the polynomial: P stays the oracle's expansion at the reported mu.
    The float64 form pins those paths (measured ~1e-14). In a split form, k below sqrt(n_terms)
    makes the Clenshaw chain in Y = T_k run m = 20 and 50 steps instead of 13 and 20, and its
    float32 rounding grows with m (measured 1.05e-6, 1.36e-6): beyond the 1e-6 bar, so the
    library refuses it unless FO_FLAG_ALLOW_LOOSE asks for it; then it is checked at 2e-6."""
    n = 600
    h = synth.tight_binding(n, 4242)
    flags = 0
    if prec != "fp64":
        with pytest.raises(fo.FermiError) as e:
            solver.density_matrix(to_dev(h), n / 2, solver.params(n_terms, 0.1, precision=prec, k=k))
        assert e.value.status == fo.FO_ERR_UNSUPPORTED
        flags = fo.FO_FLAG_ALLOW_LOOSE
    p, r = solver.density_matrix(to_dev(h), n / 2, solver.params(n_terms, 0.1, precision=prec, mu_mode="bisect",
                                                                 k=k, flags=flags))
    assert r["status"] == 0 and (r["k"], r["m"]) == (k, -(-n_terms // k))
    c = O.chebyshev_coeffs(0.1, r["mu"], r["emin"], r["emax"], n_terms)
    ref = O.poly_eig(h, c, r["emin"], r["emax"])
    assert rel_frob(p.cpu().numpy(), ref) <= tol
