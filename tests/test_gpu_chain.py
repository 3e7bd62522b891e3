"""Chain launches (each chain of dependent products -- baby steps, giant steps, Clenshaw
recurrence -- as one launch over the whole batch, tiles ordered by ticket and waiting per
instance for the previous step) against one launch per product: the same tiles compute the
same sums, so every result must be bit-identical, for single instances and ragged batches,
every tile configuration, instance windows, graph replay and the learned form's parked
instances. The timeout path is exercised by withholding one tile's completion count.
"""
import math
import os
import time

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


def ragged(count=12, seed=5, lo=64, hi=640):
    ns = [int(n) for n in synth.batch_sizes(count, seed, lo, hi)]
    kts = [float(t) for t in synth.batch_temperatures(count, seed)]
    return ns, kts, [to_dev(synth.tight_binding(n, 7100 + i)) for i, n in enumerate(ns)]


def same(a, b):
    pa, ra = a
    pb, rb = b
    for x, y in zip(pa, pb):
        assert torch.equal(x, y)
    for x, y in zip(ra, rb):
        for k in ("mu", "trace", "trace_raw", "frob2", "n_gemm"):
            assert x[k] == y[k], k


def test_single_instance_chain_equals_per_product(solver):
    n = 1000
    h = to_dev(synth.tight_binding(n, 2000 + n))
    ref = solver.density_matrix(h, n / 2, solver.params(400, 0.1, precision="bf16x3", chain=1))
    got = solver.density_matrix(h, n / 2, solver.params(400, 0.1, precision="bf16x3", chain=2))
    same(([ref[0]], [ref[1]]), ([got[0]], [got[1]]))
    assert got[1]["n_launches"] < ref[1]["n_launches"] - 40     # 57 product launches -> 4
    assert abs(got[1]["trace"] - n / 2) <= 1e-8


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
@pytest.mark.parametrize("tile", [(128, 2, 8, 1), (128, 1, 8, 2), (256, 1, 16, 1), (256, 1, 8, 2)])
@pytest.mark.parametrize("window", [0, 9])
def test_batch_chain_equals_per_product(solver, prec, tile, window):
    ns, kts, hs = ragged()
    kw = dict(tile_n=tile[0], tile_ctas=tile[1], tile_drain=tile[2], tile_store=tile[3])
    ne = [n / 2 for n in ns]
    ref = solver.density_matrix_batched(hs, ne, solver.params(300, 0.1, precision=prec, chain=1, **kw), kT=kts)
    got = solver.density_matrix_batched(hs, ne, solver.params(300, 0.1, precision=prec, chain=2,
                                                              chain_window=window, **kw), kT=kts)
    same(ref, got)
    assert all(r["status"] == 0 for r in got[1])


def test_chain_against_oracle_and_graph_replay(solver):
    ns, kts, hs = ragged(8, 6, 64, 512)
    ne = [n / 2 for n in ns]
    prm = solver.params(300, 0.1, precision="bf16x3", chain=2, chain_window=5, flags=fo.FO_FLAG_GRAPH)
    ps, rs = solver.density_matrix_batched(hs, ne, prm, kT=kts)
    ps2, rs2 = solver.density_matrix_batched(hs, ne, prm, kT=kts)          # replay
    same((ps, rs), (ps2, rs2))
    for h, n, kT, p, r in zip(hs, ns, kts, ps, rs):
        c = O.chebyshev_coeffs(kT, r["mu"], r["emin"], r["emax"], 300)
        ref = O.poly_eig(h.cpu().numpy(), c, r["emin"], r["emax"])
        assert np.linalg.norm(p.cpu().numpy() - ref) / math.sqrt(n) <= 1e-6
        assert abs(r["trace"] - n / 2) <= 1e-8


def test_chain_with_parked_instances(solver):
    """The learned form parks accepted instances (their tiles skip and count as done): with a
    network that sends every proposal far off, all fall back to bisection, whose products run
    as chains after rounds in which the instances were active; chain == per product."""
    import oracle.mlp as M
    p = {k: np.zeros(s) for k, s in M.param_shapes()}
    p["b3"] = np.array([0.9, 0.0])
    solver.mlp_set_params(M.flatten(p).astype(np.float32))
    ns, kts, hs = ragged(6, 8, 64, 400)
    ne = [n / 2 for n in ns]
    out = {}
    for chain in (1, 2):
        prm = solver.params(300, 0.1, precision="bf16x3", mu_mode="learned", max_newton=1, chain=chain)
        out[chain] = solver.density_matrix_batched(hs, ne, prm, kT=kts)
    same(out[1], out[2])


def test_chain_timeout_is_reported_and_the_context_recovers(solver):
    """One tile withholds its completion count (FERMI_CHAIN_DROP_SIGNAL): the tiles of the
    next step of its instance give up after their bounded wait, every other tile of the chain
    stops, and the call fails with FO_ERR_DEVICE_TIMEOUT within seconds; the next call of the
    same context succeeds with the same result as before."""
    n = 300
    h = to_dev(synth.tight_binding(n, 41))
    prm = solver.params(200, 0.1, precision="bf16x3", chain=2)
    p0, r0 = solver.density_matrix(h, n / 2, prm)
    os.environ["FERMI_CHAIN_DROP_SIGNAL"] = "0"
    try:
        t0 = time.monotonic()
        with pytest.raises(fo.FermiError) as e:
            solver.density_matrix(h, n / 2, prm)
        elapsed = time.monotonic() - t0
    finally:
        del os.environ["FERMI_CHAIN_DROP_SIGNAL"]
    assert e.value.status == fo.FO_ERR_DEVICE_TIMEOUT
    assert elapsed < 30.0
    p1, r1 = solver.density_matrix(h, n / 2, prm)
    assert torch.equal(p0, p1) and r0["mu"] == r1["mu"] and r1["status"] == 0
