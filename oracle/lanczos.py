"""Plain FP64 oracle of the Lanczos spectral bounds (the tighter alternative to Gershgorin).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the library path.

The paper maps H onto [-1, 1] with its lowest and highest eigenvalues (Sec. "Chebyshev
expansions with O(sqrt L) number of matrix multiplications") without saying how they are
found. Gershgorin discs enclose the spectrum but are wide for the tight-binding model (about
7x the true width), which costs resolution per term. This module restates the textbook
Lanczos process (Lanczos 1950; Golub and Van Loan, Sec. 10.1) for the two extreme
eigenvalues, step by step:

1. start vector v_i = u_i - 1/2, u_i the i-th splitmix64 output of `seed` (Steele, Lea and
   Flood 2014) scaled to [0, 1); q_1 = v / ||v||;
2. for j = 1..K: w = H q_j - beta_j q_{j-1}; alpha_j = w . q_j; w = w - alpha_j q_j;
   beta_{j+1} = ||w||; stop early if beta_{j+1} <= 1e-12 (|alpha_j| + beta_j);
   q_{j+1} = w / beta_{j+1} (no reorthogonalisation: only the extreme Ritz values are used);
3. theta_min, theta_max = the extreme eigenvalues of the tridiagonal T_K, y their unit
   eigenvectors; the residual of a Ritz pair is r = beta_{K+1} |y_K| (an eigenvalue of H
   lies within r of theta);
4. bounds [theta_min - r_min - 0.01 w, theta_max + r_max + 0.01 w], w = theta_max -
   theta_min, intersected with the Gershgorin interval.

The bounds are not a guaranteed enclosure (a start vector almost orthogonal to an extreme
eigenvector would hide it); the tests check enclosure on the model Hamiltonians.
"""
from __future__ import annotations

import numpy as np

from .fermi import gershgorin_bounds

__all__ = ["splitmix64_uniform", "start_vector", "lanczos_tridiagonal", "lanczos_bounds",
           "MARGIN", "LANCZOS_SEED"]

MARGIN = 0.01
LANCZOS_SEED = 0x4C414E43
_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of splitmix64 started at `seed`, as (z >> 11) 2^-53."""
    out = np.empty(count)
    x = seed & _M64
    for i in range(count):
        x = (x + _GAMMA) & _M64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        z = z ^ (z >> 31)
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def start_vector(n: int, seed: int = LANCZOS_SEED) -> np.ndarray:
    v = splitmix64_uniform(seed, n) - 0.5
    return v / np.linalg.norm(v)


def lanczos_tridiagonal(h: np.ndarray, steps: int, seed: int = LANCZOS_SEED):
    """alpha (K), beta (K + 1: beta[0] = 0, beta[j] couples q_j and q_{j+1}, beta[K] the
    residual coupling) after K <= steps Lanczos steps."""
    h = np.asarray(h, dtype=np.float64)
    n = h.shape[0]
    q_prev = np.zeros(n)
    q = start_vector(n, seed)
    alpha, beta = [], [0.0]
    for _ in range(min(steps, n)):
        w = h @ q - beta[-1] * q_prev
        a = float(w @ q)
        w = w - a * q
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        if b <= 1e-12 * (abs(a) + beta[-2]):
            break
        q_prev, q = q, w / b
    return np.array(alpha), np.array(beta)


def lanczos_bounds(h: np.ndarray, steps: int = 40, seed: int = LANCZOS_SEED,
                   margin: float = MARGIN) -> tuple[float, float]:
    alpha, beta = lanczos_tridiagonal(h, steps, seed)
    K = len(alpha)
    t = np.diag(alpha) + np.diag(beta[1:K], 1) + np.diag(beta[1:K], -1)
    theta, y = np.linalg.eigh(t)
    r_min = beta[K] * abs(y[K - 1, 0])
    r_max = beta[K] * abs(y[K - 1, K - 1])
    width = theta[-1] - theta[0]
    lo = theta[0] - r_min - margin * width
    hi = theta[-1] + r_max + margin * width
    ga, gb = gershgorin_bounds(h)
    lo, hi = max(lo, ga), min(hi, gb)
    if not (hi - lo > 1e-12 * max(1.0, abs(lo), abs(hi))):
        c = 0.5 * (lo + hi)
        lo, hi = c - 1.0, c + 1.0
    return float(lo), float(hi)
