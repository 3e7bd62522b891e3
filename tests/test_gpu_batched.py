"""Batched density matrices (one grouped launch per stage over instances of different sizes)
against the CPU FP64 oracle, and the batch machinery against itself.

Workload: tight-binding Hamiltonians with N log-uniform in [64, 1024] (multiples of 4),
N_e = N/2, kT ~ U(0.05, 0.2) eV, 300 terms (k = 18, m = 17), BF16x3 products, mu by
bisection on exact moments. Tolerances as for single instances: ||P - P_ref||_F / sqrt(N)
<= 1e-6 against the oracle polynomial at the bounds and mu the GPU used, |mu_gpu - mu_oracle|
<= 1e-5, |tr P - N_e| <= 1e-8 after the trace correction (before it, within the 1e-7 N band
of the split form's rounding); FP64 batches <= 1e-10 and |tr P - N_e| <= 1e-8.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2306_12616_gb300 import FO_FLAG_GRAPH, FO_FLAG_NO_RESULT_SYNC, FoParams

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def to_dev(h):
    return torch.from_numpy(np.ascontiguousarray(h)).to(DEV)


def batch(count, seed, lo=64, hi=1024):
    ns = synth.batch_sizes(count, seed, lo, hi)
    kts = synth.batch_temperatures(count, seed)
    hs = [synth.tight_binding(int(n), 4000 + seed * 1000 + i) for i, n in enumerate(ns)]
    return ns, kts, hs


def ref_at(h, r, kT, n_terms):
    c = O.chebyshev_coeffs(kT, r["mu"], r["emin"], r["emax"], n_terms)
    return O.poly_eig(h, c, r["emin"], r["emax"])


@pytest.mark.parametrize("prec,tol,split", [("bf16x3", 1e-6, True), ("fp64", 1e-10, False)])
def test_batch_matches_oracle(solver, prec, tol, split):
    ns, kts, hs = batch(10, 1, 64, 640)
    prm = solver.params(300, 0.1, precision=prec, mu_mode="bisect")
    ps, res = solver.density_matrix_batched([to_dev(h) for h in hs], [n / 2 for n in ns], prm, kT=kts)
    for h, n, kT, p, r in zip(hs, ns, kts, ps, res):
        assert r["status"] == 0 and (r["k"], r["m"]) == (18, 17)
        p = p.cpu().numpy()
        err = np.linalg.norm(p - ref_at(h, r, kT, 300)) / math.sqrt(n)
        assert err <= tol, (n, err)
        assert np.array_equal(p, p.T)
        orc = O.density_matrix(h, n / 2, kT, 300, route="eig", want_p=False)
        assert abs(r["mu"] - orc.mu) <= (1e-5 if split else 1e-9 * (orc.eb - orc.ea)), n
        assert abs(np.trace(p) - n / 2) <= 1e-8 and abs(r["trace"] - n / 2) <= 1e-8, n
        assert abs(r["trace_raw"] - n / 2) <= 1e-7 * n, n


def test_batch_equals_single_calls(solver):
    ns, kts, hs = batch(6, 2, 64, 512)
    prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="bisect")
    hd = [to_dev(h) for h in hs]
    ps, res = solver.density_matrix_batched(hd, [n / 2 for n in ns], prm, kT=kts)
    for h, n, kT, p, r in zip(hd, ns, kts, ps, res):
        p1, r1 = solver.density_matrix(h, n / 2, solver.params(300, float(kT), precision="bf16x3",
                                                               mu_mode="bisect"))
        # same products; the moment partial sums are split differently in a batch
        assert abs(r1["mu"] - r["mu"]) <= 1e-9 * (r["emax"] - r["emin"])
        assert torch.max(torch.abs(p1 - p)).item() <= 1e-9


def test_more_buckets_than_one_launch_group(solver):
    """18 distinct padded sizes (n_pad = 128 .. 2304): more buckets than one grouped launch
    carries tensor maps for (16), so the products and the Frobenius products run one launch per
    group of buckets; each instance against its single call, and the trace bar."""
    ns = [100 + 128 * i for i in range(18)]
    hs = [synth.tight_binding(n, 900 + n) for n in ns]
    hd = [to_dev(h) for h in hs]
    prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="bisect")
    ps, res = solver.density_matrix_batched(hd, [n / 2 for n in ns], prm)
    for h, n, p, r in zip(hd, ns, ps, res):
        assert r["status"] == 0 and abs(r["trace"] - n / 2) <= 1e-8
        p1, r1 = solver.density_matrix(h, n / 2, prm)
        assert abs(r1["mu"] - r["mu"]) <= 1e-9 * (r["emax"] - r["emin"])
        assert torch.max(torch.abs(p1 - p)).item() <= 1e-9


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2", "bf16x1"])
def test_tile_configs_bit_identical(solver, prec):
    """Every tile configuration and plane storage the autotuner may pick gives the same bits."""
    ns, kts, hs = batch(5, 3, 100, 700)
    hd = [to_dev(h) for h in hs]
    out = {}
    for t, c, d in ((256, 1, 8), (256, 1, 16), (128, 1, 8), (128, 2, 8)):
        for st in (1, 2):
            prm = solver.params(300, 0.1, precision=prec, mu_mode="bisect", tile_n=t, tile_ctas=c, tile_drain=d,
                                tile_store=st)
            ps, res = solver.density_matrix_batched(hd, [n / 2 for n in ns], prm, kT=kts)
            assert all(r["tile_n"] == t and r["tile_ctas"] == c and r["tile_drain"] == d and r["tile_store"] == st
                       for r in res)
            out[(t, c, d, st)] = ps
    for key in out:
        for a, b in zip(out[(256, 1, 8, 1)], out[key]):
            assert torch.equal(a, b), key
    # the autotuner's pick is one of them
    _, res = solver.density_matrix_batched(hd, [n / 2 for n in ns],
                                           solver.params(300, 0.1, precision=prec, mu_mode="bisect"), kT=kts)
    assert all(r["tile_store"] in (1, 2) for r in res)


def test_graph_replay_equals_eager(solver):
    ns, kts, hs = batch(4, 4, 64, 400)
    hd = [to_dev(h) for h in hs]
    eager, r0 = solver.density_matrix_batched(hd, [n / 2 for n in ns],
                                              solver.params(300, 0.1, precision="bf16x3"), kT=kts)
    prm = solver.params(300, 0.1, precision="bf16x3", flags=FO_FLAG_GRAPH)
    for _ in range(2):   # capture, then replay
        g, r1 = solver.density_matrix_batched(hd, [n / 2 for n in ns], prm, kT=kts)
        for a, b in zip(eager, g):
            assert torch.equal(a, b)
        assert [x["mu"] for x in r0] == [x["mu"] for x in r1]
    # replay into new output buffers and new inputs of the same sizes
    hd2 = [to_dev(synth.tight_binding(int(n), 77 + i)) for i, n in enumerate(ns)]
    g2, r2 = solver.density_matrix_batched(hd2, [n / 2 for n in ns], prm, kT=kts)
    e2, r3 = solver.density_matrix_batched(hd2, [n / 2 for n in ns],
                                           solver.params(300, 0.1, precision="bf16x3"), kT=kts)
    for a, b in zip(g2, e2):
        assert torch.equal(a, b)


def test_fixed_mu_and_given_bounds_batch(solver):
    ns = [96, 200, 332]
    hs = [synth.tight_binding(n, 11 + n) for n in ns]
    prm = solver.params(120, 0.15, precision="bf16x3", mu_mode="fixed", mu=-6.0, bounds=(-90.0, 80.0))
    ps, res = solver.density_matrix_batched([to_dev(h) for h in hs], [0.0] * 3, prm)
    for h, n, p, r in zip(hs, ns, ps, res):
        assert (r["mu"], r["emin"], r["emax"]) == (-6.0, -90.0, 80.0)
        err = np.linalg.norm(p.cpu().numpy() - ref_at(h, r, 0.15, 120)) / math.sqrt(n)
        assert err <= 1e-6, (n, err)


def test_full_c4_batch_sampled(solver):
    """The 512-instance batch: every instance converges; sampled instances match the oracle
    (small ones in full, the largest on sampled columns)."""
    count = 512
    ns = synth.batch_sizes(count, 4000)
    kts = synth.batch_temperatures(count, 4000)
    hs = [synth.tight_binding(int(n), 4000 + i) for i, n in enumerate(ns)]
    prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="bisect", flags=FO_FLAG_GRAPH)
    ps, res = solver.density_matrix_batched([to_dev(h) for h in hs], [n / 2 for n in ns], prm, kT=kts)
    assert all(r["status"] == 0 for r in res)
    for r, n in zip(res, ns):
        assert abs(r["trace"] - n / 2) <= 1e-8 and abs(r["trace_raw"] - n / 2) <= 1e-7 * n
    order = np.argsort(ns)
    for i in list(order[:3]) + list(order[count // 2:count // 2 + 2]):
        h, n, kT, r = hs[i], ns[i], kts[i], res[i]
        err = np.linalg.norm(ps[i].cpu().numpy() - ref_at(h, r, kT, 300)) / math.sqrt(n)
        assert err <= 1e-6, (n, err)
    i = int(order[-1])
    h, n, kT, r = hs[i], int(ns[i]), kts[i], res[i]
    cols = np.arange(3, n, n // 6)
    c = O.chebyshev_coeffs(kT, r["mu"], r["emin"], r["emax"], 300)
    ref = O.chebyshev_apply(O.scale_hamiltonian(h, r["emin"], r["emax"]), c, np.eye(n)[:, cols])
    err = math.sqrt(np.mean(np.sum((ps[i][:, cols].cpu().numpy() - ref) ** 2, axis=0)))
    assert err <= 1e-6, err


def test_batch_argument_errors(solver):
    h = to_dev(synth.tight_binding(64, 1))
    with pytest.raises(Exception):
        solver.density_matrix_batched([h], [100.0], solver.params(64, 0.1))   # n_e > n
    with pytest.raises(Exception):
        solver.density_matrix_batched([h], [32.0], solver.params(64, 0.1, tile_n=64))
    with pytest.raises(Exception):
        solver.density_matrix_batched([h], [32.0], solver.params(64, 0.1, tile_n=256, tile_ctas=2))


def test_batched_host_buffers_equal_device_buffers(solver):
    ns, kts, hs = batch(4, 6, 64, 500)
    prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="bisect")
    pd, rd = solver.density_matrix_batched([to_dev(h) for h in hs], [n / 2 for n in ns], prm, kT=kts)
    hin = [torch.from_numpy(h).pin_memory() for h in hs]
    # one instance with a row pitch larger than n (a 2-D copy)
    wide = torch.zeros((ns[0], ns[0] + 3), dtype=torch.float64).pin_memory()
    wide[:, :ns[0]] = hin[0]
    hin[0] = wide[:, :ns[0]]
    outs = [torch.empty((n, n), dtype=torch.float64).pin_memory() for n in ns]
    rh = solver.density_matrix_batched_host(hin, [n / 2 for n in ns], prm, outs, kT=kts)
    for a, b, x, y in zip(pd, outs, rd, rh):
        assert torch.equal(a.cpu(), b) and x["mu"] == y["mu"]


def test_pipelined_host_calls_equal_synchronous_calls(solver):
    """Host-buffer calls enqueued back to back (FO_FLAG_NO_RESULT_SYNC: the copies of
    neighbouring calls overlap the solves, on two staging slots used in turn) give the same
    bits as synchronous calls; four calls cycle both slots twice, with different inputs."""
    prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="bisect")
    prm_async = FoParams.from_buffer_copy(prm)
    prm_async.flags |= FO_FLAG_NO_RESULT_SYNC
    calls = []
    for seed in (11, 12, 13, 14):
        ns, kts, hs = batch(3, seed, 64, 400)
        hin = [torch.from_numpy(h).pin_memory() for h in hs]
        ref = [torch.empty((n, n), dtype=torch.float64).pin_memory() for n in ns]
        solver.density_matrix_batched_host(hin, [n / 2 for n in ns], prm, ref, kT=kts)
        calls.append((ns, kts, hin, ref))
    outs = []
    for ns, kts, hin, _ in calls:
        out = [torch.full((n, n), float("nan"), dtype=torch.float64).pin_memory() for n in ns]
        solver.density_matrix_batched_host(hin, [n / 2 for n in ns], prm_async, out, kT=kts)
        outs.append(out)
    solver.host_wait()
    for (_, _, _, ref), out in zip(calls, outs):
        for a, b in zip(ref, out):
            assert torch.equal(a, b)
