"""The paper's literal power-basis evaluation (FO_FLAG_POWER_BASIS: d_{i,j}, S_j and the
nested Horner scheme of Eq. (ansatz)) against the oracle, and its instability against the
Chebyshev-basis form (g_{i,l} with the Clenshaw recurrence) as m grows.

The power-basis coefficients grow like 2^j (reading R10), so the evaluation error grows with m:
in float64 it stays small for moderate m; in the split forms (float32 masters) it grows to
O(1e-2 .. 1) while the Chebyshev form keeps ~1e-7.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2306_12616_gb300 import FO_FLAG_ALLOW_LOOSE, FO_FLAG_POWER_BASIS

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def to_dev(h):
    return torch.from_numpy(np.ascontiguousarray(h)).to(DEV)


def run(solver, h, n_terms, kT, prec, flags, mu=0.0):
    # the split forms' power basis is beyond their 1e-6 bar: it runs on request only
    if prec != "fp64" and flags:
        flags |= FO_FLAG_ALLOW_LOOSE
    prm = solver.params(n_terms, kT, precision=prec, mu_mode="fixed", mu=mu, flags=flags)
    p, r = solver.density_matrix(to_dev(h), 0.0, prm)
    return p.cpu().numpy(), r


def test_power_basis_matches_oracle_literal_form(solver):
    n = 128
    h = synth.random_symmetric(n, 12)
    ea, eb = O.gershgorin_bounds(h)
    kT = 0.02 * (eb - ea)
    p, r = run(solver, h, 64, kT, "fp64", FO_FLAG_POWER_BASIS)
    assert (r["k"], r["m"]) == (8, 8)
    c = O.chebyshev_coeffs(kT, 0.0, ea, eb, 64)
    x = O.scale_hamiltonian(h, ea, eb)
    lit = O.liang_power_eval(x, O.liang_d(c, 8, 8))
    ref = O.poly_eig(h, c, ea, eb)
    assert np.linalg.norm(p - lit) / math.sqrt(n) <= 1e-10
    assert np.linalg.norm(p - ref) / math.sqrt(n) <= 1e-10


def test_power_basis_instability_grows_with_m(solver):
    """kT_x = 2 kT / (e_b - e_a) = 0.002: the error of the power basis against the exact
    polynomial, next to the Chebyshev basis, for m = 8, 16, 32."""
    n = 128
    h = synth.random_symmetric(n, 13)
    ea, eb = O.gershgorin_bounds(h)
    kT = 0.001 * (eb - ea)
    ev = np.linalg.eigh(h)
    rows = []
    for n_terms in (64, 256, 1024):
        c = O.chebyshev_coeffs(kT, 0.0, ea, eb, n_terms)
        ref = O.poly_eig(h, c, ea, eb, eig=ev)
        errs = {}
        for prec in ("fp64", "bf16x3"):
            for flags in (0, FO_FLAG_POWER_BASIS):
                p, r = run(solver, h, n_terms, kT, prec, flags)
                errs[(prec, flags)] = np.linalg.norm(p - ref) / math.sqrt(n)
        rows.append((r["m"], errs))
        print(f"m={r['m']}: fp64 cheb {errs[('fp64', 0)]:.1e} power {errs[('fp64', FO_FLAG_POWER_BASIS)]:.1e}; "
              f"bf16x3 cheb {errs[('bf16x3', 0)]:.1e} power {errs[('bf16x3', FO_FLAG_POWER_BASIS)]:.1e}")
    for m, e in rows:
        assert e[("fp64", 0)] <= 1e-10 and e[("bf16x3", 0)] <= 1e-6     # Chebyshev basis: stable
    # power basis: the error grows with m, and in the split form it is orders above the
    # Chebyshev form at m = 32
    p_fp64 = [e[("fp64", FO_FLAG_POWER_BASIS)] for _, e in rows]
    p_bf16 = [e[("bf16x3", FO_FLAG_POWER_BASIS)] for _, e in rows]
    assert p_fp64[2] > p_fp64[0] and p_bf16[2] > p_bf16[0]
    assert p_bf16[2] > 100 * rows[2][1][("bf16x3", 0)]


def test_power_basis_rejects_fp16x2_and_needs_the_request(solver):
    import paper_2306_12616_gb300 as fo
    h = to_dev(synth.random_symmetric(64, 1))
    with pytest.raises(Exception):
        solver.density_matrix(h, 0.0, solver.params(64, 0.1, precision="fp16x2", mu_mode="fixed",
                                                     flags=FO_FLAG_POWER_BASIS | FO_FLAG_ALLOW_LOOSE))
    with pytest.raises(fo.FermiError) as e:
        solver.density_matrix(h, 0.0, solver.params(64, 0.1, precision="bf16x3", mu_mode="fixed",
                                                     flags=FO_FLAG_POWER_BASIS))
    assert e.value.status == fo.FO_ERR_UNSUPPORTED
