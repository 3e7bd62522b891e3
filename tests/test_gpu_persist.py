"""The persistent product kernel (one CTA per SM walking the tiles, separate epilogue warps)
against the one-tile-per-CTA kernel with the same 128-wide tiles: every tile is the same sum
of the same products in the same order and goes through the same epilogue arithmetic, so
every result must be bit-identical -- in every split precision, both plane storages, single
instances and ragged batches, the float64-output products (final Clenshaw step, trace
correction), graph replay and the learned form's parked instances -- and P matches the
oracle.
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


def same(a, b):
    for x, y in zip(a[0], b[0]):
        assert torch.equal(x, y)
    for x, y in zip(a[1], b[1]):
        for k in ("mu", "trace", "trace_raw", "frob2", "n_gemm", "status"):
            assert x[k] == y[k], k


def tiles(store, persist):
    return dict(tile_n=128, tile_ctas=1, tile_drain=8, tile_store=store, tile_persist=persist)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2", "bf16x1"])
@pytest.mark.parametrize("store", [1, 2])
def test_batch_persistent_equals_one_tile_per_cta(solver, prec, store):
    ns = [int(n) for n in synth.batch_sizes(14, 21, 64, 900)]
    kts = [float(t) for t in synth.batch_temperatures(14, 21)]
    hs = [to_dev(synth.tight_binding(n, 8100 + i)) for i, n in enumerate(ns)]
    ne = [n / 2 for n in ns]
    ref = solver.density_matrix_batched(hs, ne, solver.params(300, 0.1, precision=prec, **tiles(store, 1)), kT=kts)
    got = solver.density_matrix_batched(hs, ne, solver.params(300, 0.1, precision=prec, **tiles(store, 2)), kT=kts)
    same(ref, got)
    assert all(r["tile_persist"] == 2 for r in got[1]) and all(r["tile_persist"] == 1 for r in ref[1])


def test_single_instance_persistent_matches_oracle(solver):
    n = 1000
    h = synth.tight_binding(n, 2000 + n)
    p, r = solver.density_matrix(to_dev(h), n / 2, solver.params(400, 0.1, precision="bf16x3", **tiles(1, 2)))
    q, rq = solver.density_matrix(to_dev(h), n / 2, solver.params(400, 0.1, precision="bf16x3", **tiles(1, 1)))
    same(([p], [r]), ([q], [rq]))
    c = O.chebyshev_coeffs(0.1, r["mu"], r["emin"], r["emax"], 400)
    ref = O.poly_eig(h, c, r["emin"], r["emax"])
    assert np.linalg.norm(p.cpu().numpy() - ref) / math.sqrt(n) <= 1e-6
    assert abs(r["trace"] - n / 2) <= 1e-8


def test_persistent_graph_replay_and_parked_instances(solver):
    import oracle.mlp as M
    ns = [int(n) for n in synth.batch_sizes(6, 22, 64, 500)]
    kts = [float(t) for t in synth.batch_temperatures(6, 22)]
    hs = [to_dev(synth.tight_binding(n, 8200 + i)) for i, n in enumerate(ns)]
    ne = [n / 2 for n in ns]
    prm = solver.params(300, 0.1, precision="bf16x3", flags=fo.FO_FLAG_GRAPH, **tiles(2, 2))
    a = solver.density_matrix_batched(hs, ne, prm, kT=kts)
    b = solver.density_matrix_batched(hs, ne, prm, kT=kts)
    same(a, b)
    ref = solver.density_matrix_batched(hs, ne, solver.params(300, 0.1, precision="bf16x3", **tiles(2, 1)), kT=kts)
    same(a, ref)
    # a network whose proposals are far off: every instance falls back after a round in which
    # the others were parked
    p = {k: np.zeros(s) for k, s in M.param_shapes()}
    p["b3"] = np.array([0.9, 0.0])
    solver.mlp_set_params(M.flatten(p).astype(np.float32))
    out = [solver.density_matrix_batched(hs, ne, solver.params(300, 0.1, precision="bf16x3", mu_mode="learned",
                                                               max_newton=1, **tiles(1, pp)), kT=kts)
           for pp in (1, 2)]
    same(out[0], out[1])


def test_persistent_is_a_tuning_candidate(solver):
    """With the tile autotuned the persistent kernel is among the candidates, and whatever
    is picked gives the one-tile-per-CTA 128-wide kernel's bits."""
    n = 640
    h = to_dev(synth.tight_binding(n, 99))
    p, r = solver.density_matrix(h, n / 2, solver.params(200, 0.1, precision="bf16x3", tile_persist=2))
    assert r["tile_persist"] == 2 and r["tile_n"] == 128
    q, rq = solver.density_matrix(h, n / 2, solver.params(200, 0.1, precision="bf16x3",
                                                          tile_n=128, tile_store=r["tile_store"], tile_persist=1))
    same(([p], [r]), ([q], [rq]))
