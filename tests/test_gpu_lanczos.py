"""Lanczos spectral bounds on the GPU against the float64 oracle (oracle/lanczos.py), and what
they buy: the same number of terms resolves the Fermi function on a ~7x narrower interval.

Tolerances: the bounds agree with the oracle's Lanczos to 1e-8 of the width (both float64,
different summation orders; 1e-6 when the steps reach half the dimension); P at the Lanczos bounds meets the usual bars against the oracle
polynomial at the same bounds and mu.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import oracle.lanczos as L
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def to_dev(h):
    return torch.from_numpy(np.ascontiguousarray(h)).to(DEV)


@pytest.mark.parametrize("kind,n", [("tb", 300), ("tb", 1000), ("rand", 256)])
def test_bounds_match_oracle_and_enclose(solver, kind, n):
    h = synth.tight_binding(n, 900 + n) if kind == "tb" else synth.random_symmetric(n, 8)
    prm = solver.params(64, 0.1, precision="fp64", mu_mode="fixed", mu=0.0, lanczos_steps=40)
    _, r = solver.density_matrix(to_dev(h), 0.0, prm)
    lo, hi = L.lanczos_bounds(h, steps=40)
    w = hi - lo
    assert abs(r["emin"] - lo) <= 1e-8 * w and abs(r["emax"] - hi) <= 1e-8 * w, (r["emin"], lo, r["emax"], hi)
    ev = np.linalg.eigvalsh(h)
    assert r["emin"] <= ev[0] and r["emax"] >= ev[-1]
    ga, gb = O.gershgorin_bounds(h)
    print(f"{kind} N={n}: Gershgorin [{ga:.2f}, {gb:.2f}], Lanczos [{r['emin']:.2f}, {r['emax']:.2f}], "
          f"spectrum [{ev[0]:.2f}, {ev[-1]:.2f}]")


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-6), ("fp64", 1e-10)])
def test_density_matrix_at_lanczos_bounds(solver, prec, tol):
    n = 500
    h = synth.tight_binding(n, 33)
    prm = solver.params(400, 0.1, precision=prec, mu_mode="bisect", lanczos_steps=40)
    p, r = solver.density_matrix(to_dev(h), n / 2, prm)
    c = O.chebyshev_coeffs(0.1, r["mu"], r["emin"], r["emax"], 400)
    ref = O.poly_eig(h, c, r["emin"], r["emax"])
    assert np.linalg.norm(p.cpu().numpy() - ref) / math.sqrt(n) <= tol
    assert abs(r["trace"] - n / 2) <= 1e-8


def test_tighter_bounds_resolve_the_fermi_function(solver):
    """Against the exact Fermi operator U f(Lambda) U^T at the same mu: 400 terms on the
    Lanczos interval are much closer than 400 terms on the Gershgorin interval."""
    n = 600
    h = synth.tight_binding(n, 44)
    mu = -6.0
    exact = O.fermi_exact(h, mu, 0.1)
    errs = {}
    for steps in (0, 40):
        prm = solver.params(400, 0.1, precision="fp64", mu_mode="fixed", mu=mu, lanczos_steps=steps)
        p, r = solver.density_matrix(to_dev(h), 0.0, prm)
        errs[steps] = np.linalg.norm(p.cpu().numpy() - exact) / math.sqrt(n)
    print(f"||P - f(H)||_F/sqrt(N) at 400 terms: Gershgorin {errs[0]:.2e}, Lanczos {errs[40]:.2e}")
    assert errs[40] < 0.25 * errs[0]


def test_lanczos_bounds_in_a_batch(solver):
    ns = [64, 200, 452]
    hs = [synth.tight_binding(nn, 5 + nn) for nn in ns]
    prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="bisect", lanczos_steps=32)
    ps, res = solver.density_matrix_batched([to_dev(h) for h in hs], [nn / 2 for nn in ns], prm)
    for h, nn, p, r in zip(hs, ns, ps, res):
        lo, hi = L.lanczos_bounds(h, steps=32)
        # N = 64 with 32 steps: past convergence, Lanczos without reorthogonalisation carries
        # the rounding of either summation order further (5.6e-7 eV on a 20 eV width)
        assert abs(r["emin"] - lo) <= 1e-6 * (hi - lo) and abs(r["emax"] - hi) <= 1e-6 * (hi - lo)
        c = O.chebyshev_coeffs(0.1, r["mu"], r["emin"], r["emax"], 300)
        ref = O.poly_eig(h, c, r["emin"], r["emax"])
        assert np.linalg.norm(p.cpu().numpy() - ref) / math.sqrt(nn) <= 1e-6
