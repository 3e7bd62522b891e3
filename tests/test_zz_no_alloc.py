"""The allocation-free spectral-bounds entry point against the context-based one.

fo_spectral_bounds_noalloc serves callers that cannot allocate device memory when they need
the bounds; it keeps its partial results in a fixed device array of the library. This file
is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

import paper_2306_12616_gb300 as fo
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def noalloc_bounds(h):
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=DEV)
    st = fo.fo_spectral_bounds_noalloc(h.data_ptr(), h.shape[0], h.stride(0), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert st == fo.FO_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_context_entry_point_twice(solver):
    # two calls in a row on different matrices: the shared array must not leak between them
    cases = [synth.tight_binding(1000, 3), synth.random_symmetric(257, 9)]
    for h in cases:
        d = torch.from_numpy(h).to(DEV)
        ref = solver.spectral_bounds(d).cpu().numpy()
        got = noalloc_bounds(d)
        # both sum each row exactly and round once: the same bits
        assert got[0] == ref[0] and got[1] == ref[1]
        assert got[2] == ref[2] == 0.0


def test_noalloc_flags_nonfinite_and_rejects_oversize():
    h = synth.random_symmetric(64, 2)
    h[5, 9] = np.inf
    got = noalloc_bounds(torch.from_numpy(h).to(DEV))
    assert got[2] == 1.0
    big = torch.zeros((1, 1), dtype=torch.float64, device=DEV)
    st = fo.fo_spectral_bounds_noalloc(big.data_ptr(), fo.FO_NOALLOC_MAX_N + 1,
                                       fo.FO_NOALLOC_MAX_N + 1, big.data_ptr(), 0)
    assert st == fo.FO_ERR_ARG
