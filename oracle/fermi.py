"""Plain FP64 oracle of the dense Chebyshev Fermi-operator expansion (arXiv 2306.12616).

TEST INFRASTRUCTURE ONLY: imported by tests, smoke() and the bench CPU baseline, never by
the library path.

Paper sections and equations are cited by their LaTeX labels:

* Sec. "Density Matrix", Eq. (D from diag) and Eq. (fermifunc): D = V f(E) V^T with the
  Fermi-Dirac function f(e) = 1 / (1 + exp(beta (e - mu))).
* Sec. "Chebyshev expansions with O(sqrt L) ...", Eq. (fermi): D = f(H), approximated by
  sum_{n=0}^{L} c_n T_n with H mapped onto [-1, 1] by the lowest/highest eigenvalue bounds.
* Eq. (ansatz), (ansatz2), (ansatz3): Liang's nested form with k baby steps and m giant
  steps, L = km - 1.
* Eq. (identity): 2 T_n T_m = T_{n+m} + T_{|n-m|}.
* Eq. (power_of_Tk), (coeff recursion), (example A): T_k^j = sum_l a_{j,l} T_{lk}, the
  lower-triangular matrix A.
* Eq. (formula for d0), (formula for d), (X): the coefficient-matching equations and the
  block upper-triangular system solved by back substitution (Appendix).
* Sec. "Speed up with multiple GPU streams": the S_j grouping and the staged baby steps
  T_{i+u} = 2 T_i T_u - T_{i-u} (Algorithm 1).

Readings where the paper is silent or garbled (each also listed in the design notes):

R1 scaling: the paper prints T_0 = (H - e_a)/(e_b - e_a); read as T_0 = I and
   T_1 = X = (2H - (e_a + e_b) I) / (e_b - e_a), which maps the spectrum onto [-1, 1].
R2 bounds: e_a, e_b are Gershgorin bounds (a guaranteed enclosure); if the interval is
   degenerate (width <= 1e-12 max(1, |e_a|, |e_b|)) it becomes centre -+ 1.
R3 term count: n_terms coefficients c_0 .. c_{n_terms-1}; k = ceil(sqrt(n_terms)),
   m = ceil(n_terms / k); c is zero-padded to km.
R4 coefficients: Chebyshev-Gauss interpolation of f on M = max(2048, 4 n_terms) nodes,
   c_0 = (1/M) sum_j f_j, c_n = (2/M) sum_j f_j cos(n theta_j), theta_j = pi (j + 1/2) / M,
   no damping kernel.
R5 recursion edge: in Eq. (coeff recursion) a_{j-1, l} outside 0 <= l <= j-1 is zero.
R6 m = 1: the l = 0 case of Eq. (formula for d) holds (c_i = d_i^T a_0, no 1/2 factor).
R7 Algorithm 1 stage 1 computes only T_2; stages s >= 2 use u = 2^{s-2}, v = 2^{s-1}.
R8 chemical potential: mu solves sum_n c_n(mu) tau_n = N_e, tau_n = tr T_n(X), by the
   bisection in ``bisect_mu`` (bracket [e_a, e_b] widened by 10 kT steps, stop when
   |F| <= 1e-12 max(1, N_e) or the bracket is narrower than 1e-15 (e_b - e_a), at most
   max_iter halvings, return the last midpoint).
R9 occupation: tr P = N_e with spinless occupations in [0, 1].
R10 hot-path coefficients: the giant-step coefficients g_{i,l} = d_i^T a_l (the bracket in
   the derivation leading to Eq. (formula for d)), i.e. the same equations with A = I,
   evaluated as P = sum_l T_l(T_k) R_l, R_l = sum_i g_{i,l} T_i.

Parity pins live in tests/test_oracle_*.py; every function below is pinned there against
the paper's worked examples, closed forms, library routines or brute force.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

__all__ = [
    "fermi_dirac", "gershgorin_bounds", "scale_hamiltonian", "plan_km", "n_quadrature",
    "chebyshev_coeffs", "chebyshev_interp", "chebyshev_naive", "chebyshev_apply",
    "chebyshev_matrices", "poly_eig", "fermi_exact", "power_matrix_A", "liang_system_X",
    "liang_d", "liang_power_eval", "liang_g", "liang_cheb_eval", "baby_steps_staged",
    "moments_eig", "moments_naive", "poly_trace", "bisect_mu", "density_matrix",
    "OracleResult", "spectrum_scaled",
]


# ----------------------------------------------------------------------------- basics

def fermi_dirac(e, mu: float, kT: float):
    """Eq. (fermifunc): f(e) = 1 / (1 + exp(beta (e - mu))), beta = 1 / kT."""
    beta = 1.0 / kT
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(beta * (np.asarray(e, dtype=np.float64) - mu)))


def gershgorin_bounds(h: np.ndarray) -> tuple[float, float]:
    """Reading R2: e_a = min_i (h_ii - sum_{j!=i} |h_ij|), e_b = max_i (h_ii + sum_{j!=i} |h_ij|).

    The paper needs the lowest and highest eigenvalue (Sec. "Chebyshev expansions"); the
    Gershgorin discs enclose every eigenvalue. A degenerate interval becomes centre -+ 1.
    """
    h = np.asarray(h, dtype=np.float64)
    d = np.diag(h)
    r = np.sum(np.abs(h), axis=1) - np.abs(d)
    ea = float(np.min(d - r))
    eb = float(np.max(d + r))
    if not (eb - ea > 1e-12 * max(1.0, abs(ea), abs(eb))):
        c = 0.5 * (ea + eb)
        ea, eb = c - 1.0, c + 1.0
    return ea, eb


def scale_hamiltonian(h: np.ndarray, ea: float, eb: float) -> np.ndarray:
    """Reading R1: X = (2 H - (e_a + e_b) I) / (e_b - e_a), spectrum inside [-1, 1]."""
    n = h.shape[0]
    return (2.0 * h - (ea + eb) * np.eye(n)) / (eb - ea)


def spectrum_scaled(evals: np.ndarray, ea: float, eb: float) -> np.ndarray:
    """Eigenvalues of X for eigenvalues of H (the same affine map as ``scale_hamiltonian``)."""
    return (2.0 * np.asarray(evals) - (ea + eb)) / (eb - ea)


def plan_km(n_terms: int, k: int = 0) -> tuple[int, int]:
    """Reading R3: k baby steps, m giant steps with km >= n_terms (k = m = sqrt(L+1) when square)."""
    if n_terms < 1:
        raise ValueError("n_terms must be >= 1")
    if k <= 0:
        k = int(math.ceil(math.sqrt(n_terms)))
    m = int(math.ceil(n_terms / k))
    return k, m


def n_quadrature(n_terms: int) -> int:
    """Reading R4: number of Chebyshev-Gauss nodes."""
    return max(2048, 4 * n_terms)


def chebyshev_interp(fun, n_terms: int, n_quad: int) -> np.ndarray:
    """Chebyshev-Gauss interpolation coefficients of fun on [-1, 1] (reading R4).

    c_n = (2 - delta_{n0}) / M sum_{j<M} fun(cos theta_j) cos(n theta_j), theta_j = pi (j+1/2)/M.
    """
    theta = np.pi * (np.arange(n_quad) + 0.5) / n_quad
    fj = np.asarray(fun(np.cos(theta)), dtype=np.float64)
    n = np.arange(n_terms)
    c = (2.0 / n_quad) * (np.cos(np.outer(n, theta)) @ fj)
    c[0] *= 0.5
    return c


def chebyshev_coeffs(kT: float, mu: float, ea: float, eb: float, n_terms: int,
                     n_quad: int = 0) -> np.ndarray:
    """Chebyshev coefficients c_0..c_{n_terms-1} of the Fermi operator on [e_a, e_b].

    Eq. (fermi) expanded as sum_n c_n T_n(X) (Sec. "Chebyshev expansions"); the paper does
    not say how c_n is obtained, reading R4 applies.
    """
    m_q = n_quad if n_quad > 0 else n_quadrature(n_terms)
    half, mid = 0.5 * (eb - ea), 0.5 * (eb + ea)
    return chebyshev_interp(lambda x: fermi_dirac(mid + half * x, mu, kT), n_terms, m_q)


# ------------------------------------------------------------------ reference routes

def chebyshev_matrices(x: np.ndarray, count: int) -> list[np.ndarray]:
    """T_0 .. T_{count-1} of X by the three-term recurrence T_{n+1} = 2 X T_n - T_{n-1}."""
    n = x.shape[0]
    out = [np.eye(n)]
    if count > 1:
        out.append(x.copy())
    for _ in range(2, count):
        out.append(2.0 * x @ out[-1] - out[-2])
    return out[:count]


def chebyshev_naive(x: np.ndarray, c: np.ndarray) -> np.ndarray:
    """sum_n c_n T_n(X) by the plain three-term recurrence (len(c) - 1 matrix products)."""
    n = x.shape[0]
    t_prev, t_cur = np.eye(n), x.copy()
    p = c[0] * t_prev
    if len(c) > 1:
        p = p + c[1] * t_cur
    for j in range(2, len(c)):
        t_prev, t_cur = t_cur, 2.0 * x @ t_cur - t_prev
        p = p + c[j] * t_cur
    return p


def chebyshev_apply(x: np.ndarray, c: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(sum_n c_n T_n(X)) V by the three-term recurrence on the block of vectors V."""
    t_prev, t_cur = v.copy(), x @ v
    p = c[0] * t_prev
    if len(c) > 1:
        p = p + c[1] * t_cur
    for j in range(2, len(c)):
        t_prev, t_cur = t_cur, 2.0 * (x @ t_cur) - t_prev
        p = p + c[j] * t_cur
    return p


def poly_eig(h: np.ndarray, c: np.ndarray, ea: float, eb: float, eig=None) -> np.ndarray:
    """U p(Lambda) U^T with p(x) = sum_n c_n T_n(x) evaluated on the scaled eigenvalues."""
    w, u = eig if eig is not None else np.linalg.eigh(h)
    p = np.polynomial.chebyshev.chebval(spectrum_scaled(w, ea, eb), c)
    return (u * p) @ u.T


def fermi_exact(h: np.ndarray, mu: float, kT: float, eig=None) -> np.ndarray:
    """Eq. (D from diag): D = V f(E) V^T."""
    w, u = eig if eig is not None else np.linalg.eigh(h)
    return (u * fermi_dirac(w, mu, kT)) @ u.T


# ------------------------------------------------------------- Liang sqrt(n) scheme

def power_matrix_A(m: int) -> np.ndarray:
    """Eq. (coeff recursion): A_{j,l} = a_{j,l} with T_k^j = sum_l a_{j,l} T_{lk} (Eq. power_of_Tk).

    a_{0,0} = 1, a_{1,0} = 0, a_{1,1} = 1; for j > 1 the four cases of the recursion, with
    entries outside 0 <= l <= j-1 of row j-1 read as zero (reading R5).
    """
    a = np.zeros((max(m, 2), max(m, 2)))
    a[0, 0] = 1.0
    a[1, 1] = 1.0

    def prev(j, l):
        return a[j - 1, l] if 0 <= l <= j - 1 else 0.0

    for j in range(2, m):
        for l in range(0, j + 1):
            if l == 0:
                a[j, l] = 0.5 * prev(j, 1)
            elif l == 1:
                a[j, l] = prev(j, 0) + 0.5 * prev(j, 2)
            elif l < j:
                a[j, l] = 0.5 * (prev(j, l - 1) + prev(j, l + 1))
            else:
                a[j, l] = 0.5 * prev(j, l - 1)
    return a[:m, :m]


def liang_system_X(k: int, m: int) -> np.ndarray:
    """The km x km upper-triangular matrix X of Eq. (X), built row by row from
    Eq. (formula for d0) and Eq. (formula for d).

    Unknowns are ordered d_{0,0}, d_{1,0}, ..., d_{k-1,0}, d_{0,1}, ... (index j k + i);
    equations c_{l k + i} in the same order.
    """
    a = power_matrix_A(m)
    x = np.zeros((k * m, k * m))
    for l in range(m):
        for i in range(k):
            row = l * k + i
            if i == 0:                                   # Eq. (formula for d0)
                for j in range(m):
                    x[row, j * k] += a[j, l]
                continue
            if l == 0:                                   # first case of Eq. (formula for d)
                for j in range(m):
                    x[row, j * k + i] += a[j, 0]
                    if m > 1:
                        x[row, j * k + (k - i)] += 0.5 * a[j, 1]
            elif l <= m - 2:                             # middle case
                for j in range(m):
                    x[row, j * k + i] += 0.5 * a[j, l]
                    x[row, j * k + (k - i)] += 0.5 * a[j, l + 1]
            else:                                        # l = m - 1
                for j in range(m):
                    x[row, j * k + i] += 0.5 * a[j, m - 1]
    return x


def liang_d(c: np.ndarray, k: int, m: int) -> np.ndarray:
    """Power-basis coefficients d_{i,j} (returned as a k x m array) by back substitution in Eq. (X)."""
    cc = np.zeros(k * m)
    cc[: len(c)] = c
    sol = sla.solve_triangular(liang_system_X(k, m), cc, lower=False)
    return sol.reshape(m, k).T.copy()


def liang_power_eval(x: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Eq. (ansatz): S_j = sum_i d_{i,j} T_i, then nested Horner Y = S_j + T_k Y."""
    k, m = d.shape
    t = chebyshev_matrices(x, k + 1)
    s = [sum(d[i, j] * t[i] for i in range(k)) for j in range(m)]
    y = s[m - 1]
    for j in range(m - 2, -1, -1):
        y = s[j] + t[k] @ y
    return y


def liang_g(c: np.ndarray, k: int, m: int) -> np.ndarray:
    """Giant-step coefficients g_{i,l} = d_i^T a_l (k x m) from Eq. (formula for d0) and
    Eq. (formula for d) read with A replaced by the identity (reading R10):

    c_{lk} = g_{0,l};  c_i = g_{i,0} + g_{k-i,1}/2;  c_{lk+i} = (g_{i,l} + g_{k-i,l+1})/2
    for 1 <= l <= m-2;  c_{(m-1)k+i} = g_{i,m-1}/2 (and c_i = g_{i,0} when m = 1).
    Solved from l = m-1 downwards.
    """
    cc = np.zeros(k * m)
    cc[: len(c)] = c
    g = np.zeros((k, m))
    for l in range(m - 1, -1, -1):
        g[0, l] = cc[l * k]
        for i in range(1, k):
            ci = cc[l * k + i]
            if m == 1:
                g[i, l] = ci
            elif l == m - 1:
                g[i, l] = 2.0 * ci
            elif l == 0:
                g[i, l] = ci - 0.5 * g[k - i, 1]
            else:
                g[i, l] = 2.0 * ci - g[k - i, l + 1]
    return g


def liang_cheb_eval(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """P = sum_l T_{lk} R_l with R_l = sum_i g_{i,l} T_i; T_{lk} = T_l(T_k) built by
    T_{(l+1)k} = 2 T_k T_{lk} - T_{(l-1)k} (Eq. identity with n = lk, m = k)."""
    k, m = g.shape
    t = chebyshev_matrices(x, k + 1)
    r = [sum(g[i, l] * t[i] for i in range(k)) for l in range(m)]
    giant = [t[0], t[k]]
    for _ in range(2, m):
        giant.append(2.0 * t[k] @ giant[-1] - giant[-2])
    return sum(giant[l] @ r[l] for l in range(m))


def baby_steps_staged(x: np.ndarray, k: int) -> dict[int, np.ndarray]:
    """Algorithm 1: T_2 .. T_k in ceil(log2 k) stages with T_{i+u} = 2 T_i T_u - T_{i-u}
    and T_{i+v} = 2 T_v T_i - T_{v-i} (reading R7 for stage 1). Returns {index: T_index}."""
    n = x.shape[0]
    t = {0: np.eye(n), 1: x.copy()}
    if k < 2:
        return t
    stages = int(math.ceil(math.log2(k)))
    for s in range(1, stages + 1):
        new = {}
        if s == 1:
            new[2] = 2.0 * t[1] @ t[1] - t[0]
        else:
            u, v = 2 ** (s -2), 2 ** (s - 1)
            for i in range(u + 1, v + 1):
                if i + u <= k:
                    new[i + u] = 2.0 * t[i] @ t[u] - t[i - u]
            for i in range(u + 1, v + 1):
                if i + v <= k:
                    new[i + v] = 2.0 * t[v] @ t[i] - t[v - i]
        t.update(new)
    return t


# -------------------------------------------------------------- moments and mu search

def moments_eig(x_evals: np.ndarray, count: int) -> np.ndarray:
    """tau_n = tr T_n(X) = sum_i T_n(x_i) for the eigenvalues x_i of X, n < count."""
    xs = np.clip(np.asarray(x_evals, dtype=np.float64), -1.0, 1.0)
    ang = np.arccos(xs)
    return np.cos(np.outer(np.arange(count), ang)).sum(axis=1)


def moments_naive(x: np.ndarray, count: int) -> np.ndarray:
    """tau_n = tr T_n(X) from the matrices of the three-term recurrence, n < count."""
    return np.array([np.trace(t) for t in chebyshev_matrices(x, count)])


def poly_trace(mu: float, taus: np.ndarray, kT: float, ea: float, eb: float,
               n_terms: int, n_quad: int = 0) -> float:
    """tr p(X) = sum_n c_n(mu) tau_n for the expansion with n_terms coefficients."""
    c = chebyshev_coeffs(kT, mu, ea, eb, n_terms, n_quad)
    return float(np.dot(c, taus[:n_terms]))


@dataclass
class BisectResult:
    mu: float
    iterations: int
    status: str          # "ok", "no_bracket" or "not_converged"
    lo: float
    hi: float


def bisect_mu(trace_fn, n_e: float, ea: float, eb: float, kT: float,
              max_iter: int = 200, widen_steps: int = 8) -> BisectResult:
    """Reading R8: bisection for F(mu) = trace_fn(mu) - N_e = 0 (F increases with mu)."""
    lo, hi = ea, eb
    for _ in range(widen_steps):
        if trace_fn(lo) - n_e <= 0.0:
            break
        lo -= 10.0 * kT
    for _ in range(widen_steps):
        if trace_fn(hi) - n_e >= 0.0:
            break
        hi += 10.0 * kT
    if trace_fn(lo) - n_e > 0.0 or trace_fn(hi) - n_e < 0.0:
        return BisectResult(0.5 * (lo + hi), 0, "no_bracket", lo, hi)
    tol_f = 1e-12 * max(1.0, abs(n_e))
    tol_w = 1e-15 * (eb - ea)
    mid = 0.5 * (lo + hi)
    for it in range(1, max_iter + 1):
        mid = 0.5 * (lo + hi)
        f = trace_fn(mid) - n_e
        if abs(f) <= tol_f:
            return BisectResult(mid, it, "ok", lo, hi)
        if f < 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= tol_w:
            return BisectResult(0.5 * (lo + hi), it, "ok", lo, hi)
    return BisectResult(0.5 * (lo + hi), max_iter, "not_converged", lo, hi)


# ------------------------------------------------------------------- full pipeline

@dataclass
class OracleResult:
    p: np.ndarray | None
    mu: float
    ea: float
    eb: float
    k: int
    m: int
    coeffs: np.ndarray
    iterations: int = 0
    status: str = "ok"
    taus: np.ndarray | None = field(default=None, repr=False)


def density_matrix(h: np.ndarray, n_e: float | None, kT: float, n_terms: int, *,
                   mu: float | None = None, bounds: tuple[float, float] | None = None,
                   route: str = "eig", k: int = 0, n_quad: int = 0,
                   max_iter: int = 200, want_p: bool = True) -> OracleResult:
    """Density matrix P = sum_n c_n(mu) T_n(X) (Eq. fermi, Sec. "Chebyshev expansions").

    * bounds: Gershgorin (reading R2) unless given;
    * mu: given, or by ``bisect_mu`` on the exact polynomial trace (reading R8), with the
      moments tau_n taken from the eigenvalues of X;
    * route "eig": U p(Lambda) U^T; "naive": three-term recurrence; "liang": the giant-step
      (g) form; "liang_d": the paper's power-basis (d) form.
    """
    ea, eb = bounds if bounds is not None else gershgorin_bounds(h)
    kk, mm = plan_km(n_terms, k)
    eig = None
    taus = None
    iters, status = 0, "ok"
    if mu is None:
        eig = np.linalg.eigh(h) if (want_p and route == "eig") else (np.linalg.eigvalsh(h), None)
        taus = moments_eig(spectrum_scaled(eig[0], ea, eb), n_terms)
        br = bisect_mu(lambda mu_: poly_trace(mu_, taus, kT, ea, eb, n_terms, n_quad),
                       float(n_e), ea, eb, kT, max_iter=max_iter)
        mu, iters, status = br.mu, br.iterations, br.status
    c = chebyshev_coeffs(kT, mu, ea, eb, n_terms, n_quad)
    p = None
    if want_p:
        x = None if route == "eig" else scale_hamiltonian(h, ea, eb)
        if route == "eig":
            p = poly_eig(h, c, ea, eb, eig if (eig is not None and eig[1] is not None) else None)
        elif route == "naive":
            p = chebyshev_naive(x, c)
        elif route == "liang":
            p = liang_cheb_eval(x, liang_g(c, kk, mm))
        elif route == "liang_d":
            p = liang_power_eval(x, liang_d(c, kk, mm))
        else:
            raise ValueError(route)
    return OracleResult(p, float(mu), ea, eb, kk, mm, c, iters, status, taus)
