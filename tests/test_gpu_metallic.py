"""A high density of states at the Fermi level: the metallic model (tight-binding hopping,
25 % of the onsite energies ~ N(0, 0.02 eV)), N = 1024, kT = 0.01 eV, 1000 Chebyshev terms
(k = m = 32), N_e = 0.775 N (Fermi level at 0 eV), BF16x3 split products.

Both ways of fixing mu are judged against the float64 oracle (oracle/fermi.py) at the
GPU's bounds and mu: ||P - P_ref||_F / sqrt(N) <= 1e-6, and |tr P - N_e| <= 1e-8 after the
trace correction (bisection: always; an accepted learned proposal: where the correction is
rounding-sized, else its trace stays within the acceptance tolerance). The network of the
learned form is trained here on pairs the exact method generates from device-drawn matrices
of the same family.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from synth.device import metallic_batch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N, TERMS, KT = 1024, 1000, 0.01


def held_out(count, seed0=5000):
    return [synth.metallic(N, seed0 + i) for i in range(count)]


def judge(h, p, r, n_e, tol):
    assert r["status"] == 0
    c = O.chebyshev_coeffs(KT, r["mu"], r["emin"], r["emax"], TERMS)
    ref = O.poly_eig(h, c, r["emin"], r["emax"])
    assert np.linalg.norm(p.cpu().numpy() - ref) / math.sqrt(N) <= 1e-6
    assert abs(r["trace_raw"] - n_e) <= tol
    assert abs(r["trace"] - n_e) <= (1e-8 if r["trace_gamma"] != 0.0 else tol)
    # the polynomial trace at the reported mu agrees with the trace of the returned P
    assert abs(np.trace(ref) - r["trace"]) <= 2e-6 * N


def test_metallic_bisection_matches_oracle(solver):
    hs = held_out(4)
    ne = synth.metallic_electrons(N)
    prm = solver.params(TERMS, KT, precision="bf16x3", mu_mode="bisect")
    ps, rs = solver.density_matrix_batched([torch.from_numpy(h).to(DEV) for h in hs], [ne] * 4, prm)
    # 31 baby, 30 giant, 31 Clenshaw products and the trace correction's
    assert all(r["k"] == 32 and r["m"] == 32 and r["n_gemm"] == 31 + 30 + 31 + 1 for r in rs)
    for i in (0, 3):
        judge(hs[i], ps[i], rs[i], ne, 1e-7 * N)
    assert all(r["trace_gamma"] != 0.0 and abs(r["trace"] - ne) <= 1e-8 for r in rs)
    # mu near the intended Fermi level (0 eV) for the whole batch
    assert all(abs(r["mu"]) < 0.5 for r in rs)


def test_metallic_learned_mu_judged(solver):
    prm = solver.params(TERMS, KT, precision="bf16x3")
    rng = np.random.default_rng(77)
    feats, tgts = [], []
    for b in range(16):                                 # 1024 method-generated pairs
        hb = metallic_batch(64, N, 9000 + b, DEV)
        f, t, res = solver.learned_features([hb[i] for i in range(64)], rng.uniform(0.74, 0.81, 64) * N, prm)
        assert all(r["status"] == 0 for r in res)
        feats.append(f)
        tgts.append(t)
        del hb
    solver.mlp_init(3)
    losses = solver.mlp_train(torch.cat(feats), torch.cat(tgts), epochs=60, batch=128, lr=1e-3, seed=3)
    assert losses[-1] < 0.2 * losses[0]
    hs = held_out(6, 5100)
    ne = synth.metallic_electrons(N)
    dh = [torch.from_numpy(h).to(DEV) for h in hs]
    for tol in (0.5, 0.0):                              # 0: the default, 1e-7 N
        pl, rl = solver.density_matrix_batched(
            dh, [ne] * 6, solver.params(TERMS, KT, precision="bf16x3", mu_mode="learned", tr_tol=tol,
                                        max_newton=3))
        band = tol if tol > 0 else 1e-7 * N
        for i in (0, 5):
            judge(hs[i], pl[i], rl[i], ne, band if rl[i]["learned_accepted"] else 1e-7 * N)
        for r in rl:
            assert r["status"] == 0 and abs(r["trace_raw"] - ne) <= (band if r["learned_accepted"] else 1e-7 * N)
            assert abs(r["trace"] - ne) <= (1e-8 if r["trace_gamma"] != 0.0 else band)
            if not r["learned_accepted"]:
                assert r["trace_gamma"] != 0.0
            # products: 31 baby steps, 31 per evaluation of P (the fallback's included), 30
            # giant steps for the exact moments of the fallback, and the trace correction's
            assert r["n_gemm"] == 31 + 31 * r["evals"] + (0 if r["learned_accepted"] else 30) + 1
