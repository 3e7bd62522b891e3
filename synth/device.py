"""Batched, seeded generators of the same Hamiltonian families on a torch device.

Training the learned chemical potential takes tens of thousands of method-generated
(H, mu) pairs at N = 1024; drawing them one by one with numpy costs ~50 ms per matrix,
so this module draws whole batches with torch's generator on the device instead. The
recipe is the one of ``synth.hamiltonians`` (same densities, radii, onsite energies,
hopping and sign rules); the random streams differ (torch's Philox instead of numpy's
PCG64), so these matrices are other members of the same families, used for training
data only. Like the rest of ``synth`` this module holds none of the method's arithmetic.
"""
from __future__ import annotations

import torch

from .hamiltonians import ONSITE_EV, tight_binding_box


def tight_binding_batch(count: int, n: int, seed: int, device, density: float = 0.1,
                        r0: float = 1.5, rcut: float = 6.0, t0: float = -2.0,
                        onsite_sigma: float = 0.1) -> torch.Tensor:
    """``count`` dense tight-binding Hamiltonians of size n (a multiple of 4), float64,
    shape (count, n, n), in eV."""
    if n % 4 != 0 or n <= 0 or count < 1:
        raise ValueError("tight-binding size must be a positive multiple of 4")
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(device=device, dtype=torch.float64)
    na = n // 4
    box = tight_binding_box(n, density)
    pos = torch.rand((count, na, 3), generator=g, **f64) * box
    d = pos[:, :, None, :] - pos[:, None, :, :]
    d = d - box * torch.round(d / box)                 # minimum image, one term per pair
    r = torch.sqrt((d * d).sum(-1))
    del d
    hop = torch.where(r < rcut, t0 * torch.exp(-r / r0), torch.zeros((), **f64))
    hop.diagonal(dim1=1, dim2=2).zero_()               # no intra-atom coupling
    sign = torch.randint(0, 2, (count, n, n), generator=g, device=device).to(torch.float64)
    sign = torch.triu(sign * 2.0 - 1.0, 1)
    sign = sign + sign.transpose(1, 2)                 # independent symmetric sign per pair
    h = hop.repeat_interleave(4, dim=1).repeat_interleave(4, dim=2) * sign
    del sign
    onsite = torch.tensor(ONSITE_EV, **f64).repeat(na)[None, :] \
        + onsite_sigma * torch.randn((count, n), generator=g, **f64)
    h.diagonal(dim1=1, dim2=2).copy_(onsite)
    return h


def metallic_batch(count: int, n: int, seed: int, device, fraction: float = 0.25,
                   mu0: float = 0.0, sigma: float = 0.02) -> torch.Tensor:
    """Tight-binding batch with ``fraction`` of each matrix's onsite energies redrawn from
    N(mu0, sigma) (distinct orbitals per matrix)."""
    h = tight_binding_batch(count, n, seed, device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) + 7919)
    k = int(round(fraction * n))
    idx = torch.argsort(torch.rand((count, n), generator=g, device=device), dim=1)[:, :k]
    vals = mu0 + sigma * torch.randn((count, k), generator=g, device=device, dtype=torch.float64)
    diag = h.diagonal(dim1=1, dim2=2)
    diag.scatter_(1, idx, vals)
    return h
