"""Seeded generators for the workloads the solver is measured on.

The paper benchmarks model Hamiltonians from an external Fortran module that is not
available (Section "Model tight-binding Hamiltonian matrices"), so these generators stand
in for it with the same sizes (N = 256 ... 5000), dense storage and a metallic density of
states at the Fermi level:

* ``random_symmetric``: H = (G + G^T) / (2 sqrt(N)) + diag(U(-1, 1)), G_ij ~ N(0, 1).
* ``tight_binding``: N/4 atoms uniform in a periodic cube at 0.1 atoms / A^3, four
  orbitals per atom with onsite energies {-10, -5, -5, -5} eV + N(0, 0.1 eV); hopping
  -2 exp(-r / 1.5 A) times an independent symmetric random sign per orbital pair,
  between orbitals of different atoms closer than 6 A (minimum image), stored dense.
* ``metallic``: the tight-binding hopping with 25 % of the onsite energies redrawn
  from N(0, 0.02 eV), which piles states up at 0 eV.

Every generator takes an explicit seed and uses numpy's PCG64 (``default_rng``).
"""
from __future__ import annotations

import numpy as np

ONSITE_EV = (-10.0, -5.0, -5.0, -5.0)


def random_symmetric(n: int, seed: int = 1) -> np.ndarray:
    """Dense random symmetric H = (G+G^T)/(2 sqrt N) + diag(U(-1,1)), float64."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n))
    h = (g + g.T) / (2.0 * np.sqrt(n))
    h[np.diag_indices(n)] += rng.uniform(-1.0, 1.0, n)
    return np.ascontiguousarray(h)


def tight_binding_box(n: int, density: float = 0.1) -> float:
    """Edge (A) of the periodic cube holding n/4 atoms at the given atom density."""
    return float((n // 4 / density) ** (1.0 / 3.0))


def _hopping(rng: np.random.Generator, n: int, density: float, r0: float,
             rcut: float, t0: float) -> np.ndarray:
    if n % 4 != 0 or n <= 0:
        raise ValueError("tight-binding size must be a positive multiple of 4")
    n_atoms = n // 4
    box = tight_binding_box(n, density)
    pos = rng.uniform(0.0, box, (n_atoms, 3))
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.round(d / box)                     # minimum image, one term per pair
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    hop = np.where(r < rcut, t0 * np.exp(-r / r0), 0.0)
    np.fill_diagonal(hop, 0.0)                       # no intra-atom coupling
    sign = rng.integers(0, 2, size=(n, n)).astype(np.float64) * 2.0 - 1.0
    sign = np.triu(sign, 1)
    sign = sign + sign.T
    h = np.kron(hop, np.ones((4, 4))) * sign
    return h


def tight_binding(n: int, seed: int, density: float = 0.1, r0: float = 1.5,
                  rcut: float = 6.0, t0: float = -2.0,
                  onsite_sigma: float = 0.1) -> np.ndarray:
    """Dense tight-binding Hamiltonian in eV (N a multiple of 4), float64."""
    rng = np.random.default_rng(seed)
    h = _hopping(rng, n, density, r0, rcut, t0)
    onsite = np.tile(np.asarray(ONSITE_EV), n // 4) + rng.normal(0.0, onsite_sigma, n)
    h[np.diag_indices(n)] = onsite
    return np.ascontiguousarray(h)


def metallic(n: int, seed: int, fraction: float = 0.25, mu0: float = 0.0,
             sigma: float = 0.02) -> np.ndarray:
    """Tight-binding hopping with ``fraction`` of the onsite energies ~ N(mu0, sigma)."""
    h = tight_binding(n, seed)
    rng = np.random.default_rng(seed + 7919)
    idx = rng.choice(n, size=int(round(fraction * n)), replace=False)
    h[idx, idx] = rng.normal(mu0, sigma, idx.size)
    return h


# Fraction of the states of the metallic family below mu0 = 0 eV: 0.770-0.778 of N over
# seeds 5100-5107 at N = 1024 (eigenvalue count). With N_e = METALLIC_FILLING * N the
# Fermi level sits at mu0, among the redrawn onsite energies.
METALLIC_FILLING = 0.775


def metallic_electrons(n: int) -> float:
    """Electron count that puts the Fermi level of a metallic Hamiltonian of size n at mu0."""
    return float(round(METALLIC_FILLING * n))


def batch_sizes(count: int, seed: int, lo: int = 64, hi: int = 1024) -> np.ndarray:
    """Log-uniform sizes in [lo, hi], rounded to multiples of 4."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), count))
    n = (4 * np.round(n / 4)).astype(np.int64)
    return np.clip(n, lo, hi)


def batch_temperatures(count: int, seed: int, lo: float = 0.05, hi: float = 0.2) -> np.ndarray:
    """Electronic temperatures kT ~ U(lo, hi) eV."""
    rng = np.random.default_rng(seed + 1)
    return rng.uniform(lo, hi, count)
