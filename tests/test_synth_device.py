"""The batched device generator draws from the same families as the numpy generator (it
feeds training data of the learned chemical potential); checked on the CPU device."""
import numpy as np
import torch

import synth
from synth.device import metallic_batch, tight_binding_batch


def test_tight_binding_batch_structure():
    h = tight_binding_batch(3, 64, 5, "cpu")
    assert h.shape == (3, 64, 64) and h.dtype == torch.float64
    a = h.numpy()
    for x in a:
        assert np.array_equal(x, x.T)
        d = np.diag(x)
        # onsite {-10, -5, -5, -5} + N(0, 0.1)
        assert np.all(np.abs(d - np.tile([-10.0, -5.0, -5.0, -5.0], 16)) < 0.6)
        off = x - np.diag(d)
        # hopping magnitudes 2 exp(-r / 1.5) with r < 6 A; zero inside an atom's 4 x 4 block
        nz = np.abs(off[off != 0.0])
        assert np.all(nz <= 2.0) and np.all(nz >= 2.0 * np.exp(-6.0 / 1.5) - 1e-12)
        for i in range(16):
            assert not np.any(off[4 * i:4 * i + 4, 4 * i:4 * i + 4])
    # same seed, same matrices; another seed, others
    assert torch.equal(h, tight_binding_batch(3, 64, 5, "cpu"))
    assert not torch.equal(h, tight_binding_batch(3, 64, 6, "cpu"))


def test_metallic_batch_matches_numpy_family():
    h = metallic_batch(3, 512, 11, "cpu").numpy()
    ref = synth.metallic(512, 11)
    for x in h:
        assert np.array_equal(x, x.T)
        d = np.diag(x)
        assert np.sum(np.abs(d) < 0.2) == 128                 # 25 % redrawn around 0 eV
        # the same density of couplings and the same spectral range as the numpy family
        assert abs(np.count_nonzero(x) - np.count_nonzero(ref)) < 0.1 * np.count_nonzero(ref)
        ev = np.linalg.eigvalsh(x)
        evr = np.linalg.eigvalsh(ref)
        for q in (0.1, 0.5, 0.9):
            assert abs(np.quantile(ev, q) - np.quantile(evr, q)) < 1.0
        # the electron count of the family puts the Fermi level near mu0 = 0 eV
        ne = int(synth.metallic_electrons(512))
        assert -0.6 < 0.5 * (ev[ne - 1] + ev[ne]) < 0.6
