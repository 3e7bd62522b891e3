"""Algorithm 1 (staged baby and giant steps, the independent products of a stage in one
launch, FO_FLAG_STAGED) against the oracle and against the default three-term recurrence.

The staged and the sequential chains are the same polynomials computed in a different order.
In float64 both meet the 1e-10 bar. In the split forms the staged chain is less accurate:
a doubling stage U_{2v} = 2 U_v U_v - I multiplies the error of U_v by up to 4 |U_v|, so
log2(k) stages amplify the float32-level rounding that the three-term recurrence lets grow only
linearly; its bar here is 1e-4 (measured ~2e-5), the default recurrence keeps 1e-6.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2306_12616_gb300 import FO_ERR_UNSUPPORTED, FO_FLAG_ALLOW_LOOSE, FO_FLAG_STAGED, FermiError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def to_dev(h):
    return torch.from_numpy(np.ascontiguousarray(h)).to(DEV)


@pytest.mark.parametrize("prec,tol_seq,tol_staged", [("bf16x3", 1e-6, 1e-4), ("fp64", 1e-10, 1e-10)])
@pytest.mark.parametrize("n", [200, 700])
def test_staged_and_sequential_match_oracle(solver, prec, tol_seq, tol_staged, n):
    h = synth.tight_binding(n, 500 + n)
    errs = {}
    for flags, tol in ((0, tol_seq), (FO_FLAG_STAGED, tol_staged)):
        if prec != "fp64" and flags:
            # beyond the split forms' 1e-6 bar: refused unless requested
            with pytest.raises(FermiError) as e:
                solver.density_matrix(to_dev(h), n / 2, solver.params(400, 0.1, precision=prec, flags=flags))
            assert e.value.status == FO_ERR_UNSUPPORTED
            flags |= FO_FLAG_ALLOW_LOOSE
        prm = solver.params(400, 0.1, precision=prec, mu_mode="bisect", flags=flags)
        p, r = solver.density_matrix(to_dev(h), n / 2, prm)
        c = O.chebyshev_coeffs(0.1, r["mu"], r["emin"], r["emax"], 400)
        ref = O.poly_eig(h, c, r["emin"], r["emax"])
        err = np.linalg.norm(p.cpu().numpy() - ref) / math.sqrt(n)
        assert err <= tol, (flags, err)
        # + the trace correction's product in the split forms
        assert r["n_gemm"] == 19 + 18 + 19 + (prec != "fp64")
        errs[flags & FO_FLAG_STAGED] = err
    print(f"{prec} N={n}: ||dP||/sqrt(N) three-term {errs[0]:.2e}, staged {errs[FO_FLAG_STAGED]:.2e}")


def test_stage_launch_counts(solver):
    """k = m = 20: staged baby steps T_2..T_20 take 5 launches (T_2 | T_3..T_4 | T_5..T_8 |
    T_9..T_16 | T_17..T_20), the giant chain U_2..U_19 also 5, Clenshaw 19 one by one."""
    n = 300
    h = to_dev(synth.tight_binding(n, 3))
    for flags, launches in ((FO_FLAG_STAGED | FO_FLAG_ALLOW_LOOSE, 5 + 5 + 19 + 1), (0, 19 + 18 + 19 + 1)):
        prm = solver.params(400, 0.1, precision="bf16x3", mu_mode="bisect", flags=flags)
        solver.density_matrix(h, n / 2, prm)            # plan and autotuning outside the profile
        solver.profile_enable(True)
        _, r = solver.density_matrix(h, n / 2, prm)
        prof = solver.profile_read(reset=True)
        solver.profile_enable(False)
        assert prof["products"]["launches"] == launches
        # 56 products in BF16x3 (6 split products each) and the trace correction's in BF16x1
        assert prof["products"]["flops"] == pytest.approx((56 * 6 + 1) * n * n * (n + 1))


def test_staged_moments_match_oracle(solver):
    """fo_moments runs the staged baby steps: tau_j against the eigenvalue moments."""
    n = 256
    h = synth.random_symmetric(n, 4)
    hd = to_dev(h)
    b = solver.spectral_bounds(hd)
    ea, eb = float(b[0]), float(b[1])
    tau = solver.moments(hd, b, 40, precision="fp64").cpu().numpy()
    ref = O.moments_eig(np.linalg.eigvalsh(O.scale_hamiltonian(h, ea, eb)), 40)
    assert np.max(np.abs(tau - ref)) <= 1e-10 * n
