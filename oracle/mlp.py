"""Plain FP64 oracle of the learned chemical-potential model.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the library path.

The paper fixes mu by hand; the learned proposal of mu (and of the expansion order) is a
build-side addition whose every step this module writes out in float64:

* the input features of one Hamiltonian (``features``): the Chebyshev moments
  tau_n = tr T_n(X) of the scaled Hamiltonian, n = 1..64, divided by N (zero beyond the
  2k moments the k baby steps give), the electron fraction N_e / N, the temperature on the
  scaled axis kT_x = 2 kT / (e_b - e_a), and the bounds e_a / 100, e_b / 100;
* the regression targets (``targets``): mu on the scaled axis,
  mu_x = (2 mu - (e_a + e_b)) / (e_b - e_a), and the order target log2(L*) / log2(n_terms),
  L* the smallest number of terms whose coefficient tail sum_{j >= L*} |c_j| is at most
  2.5e-7 (``order_from_coefficients``): since |T_j(x)| <= 1 on [-1, 1], cutting the
  expansion there changes P by at most that much in the 2-norm, a quarter of the 1e-6 bar;
* a fully connected network 68 -> 256 -> 256 -> 2 with SiLU activations,
  silu(z) = z / (1 + exp(-z)) (Elfwing, Uchibe and Doya 2018), y = W3 a2 + b3;
* the weighted squared error L = (1/B) sum_b sum_j w_j (y_bj - t_bj)^2 and its gradients
  by the chain rule (``gradients``), pinned against central finite differences;
* Adam (Kingma and Ba 2015) with bias-corrected moments (``adam_step``).

Parameters are a dict of float64 arrays: W1 (256, 68), b1 (256,), W2 (256, 256), b2 (256,),
W3 (2, 256), b3 (2,), with W the (out, in) matrices of y = x W^T + b.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["N_IN", "N_HID", "N_OUT", "N_MOM", "silu", "silu_grad", "forward", "loss",
           "gradients", "adam_step", "features", "targets", "order_from_coefficients", "param_shapes",
           "flatten", "unflatten", "init_params"]

N_MOM = 64
N_IN = N_MOM + 4
N_HID = 256
N_OUT = 2
ORDER_EPS = 2.5e-7


def param_shapes() -> list[tuple[str, tuple[int, ...]]]:
    """Parameter names and shapes in the library's storage order."""
    return [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
            ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k, _ in param_shapes()])


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in param_shapes():
        size = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    assert o == flat.size
    return out


def init_params(seed: int, scale: float = 1.0) -> dict:
    """Uniform(-a, a) weights with a = scale sqrt(6 / (fan_in + fan_out)), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in param_shapes():
        if k.startswith("W"):
            a = scale * math.sqrt(6.0 / (shp[0] + shp[1]))
            p[k] = rng.uniform(-a, a, shp)
        else:
            p[k] = np.zeros(shp)
    return p


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    """d/dz [z sigma(z)] = sigma(z) (1 + z (1 - sigma(z)))."""
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params: dict, x: np.ndarray):
    """Returns (y, cache) for a batch x of shape (B, 68)."""
    z1 = x @ params["W1"].T + params["b1"]
    a1 = silu(z1)
    z2 = a1 @ params["W2"].T + params["b2"]
    a2 = silu(z2)
    y = a2 @ params["W3"].T + params["b3"]
    return y, (x, z1, a1, z2, a2)


def loss(params: dict, x: np.ndarray, t: np.ndarray, w) -> float:
    y, _ = forward(params, x)
    return float(np.sum(np.asarray(w) * (y - t) ** 2) / x.shape[0])


def gradients(params: dict, x: np.ndarray, t: np.ndarray, w) -> tuple[float, dict]:
    """Loss and its gradient with respect to every parameter (chain rule, layer by layer)."""
    y, (x0, z1, a1, z2, a2) = forward(params, x)
    B = x.shape[0]
    w = np.asarray(w, dtype=np.float64)
    L = float(np.sum(w * (y - t) ** 2) / B)
    dy = 2.0 * w * (y - t) / B                 # dL/dy
    g = {"W3": dy.T @ a2, "b3": dy.sum(axis=0)}
    da2 = dy @ params["W3"]
    dz2 = da2 * silu_grad(z2)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(axis=0)
    da1 = dz2 @ params["W2"]
    dz1 = da1 * silu_grad(z1)
    g["W1"] = dz1.T @ x0
    g["b1"] = dz1.sum(axis=0)
    return L, g


def adam_step(params: dict, grads: dict, m: dict, v: dict, step: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; step counts from 1."""
    for k in params:
        m[k] = beta1 * m[k] + (1.0 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * grads[k] ** 2
        mhat = m[k] / (1.0 - beta1 ** step)
        vhat = v[k] / (1.0 - beta2 ** step)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)


def features(tau: np.ndarray, n: int, n_e: float, kT: float, ea: float, eb: float, k: int) -> np.ndarray:
    """Input vector of one Hamiltonian: tau_1..tau_64 / n (tau_j with j > 2k set to 0),
    N_e / n, kT_x, e_a / 100, e_b / 100."""
    f = np.zeros(N_IN)
    avail = min(N_MOM, 2 * k, len(tau) - 1)
    f[:avail] = np.asarray(tau[1:avail + 1], dtype=np.float64) / n
    f[N_MOM] = n_e / n
    f[N_MOM + 1] = 2.0 * kT / (eb - ea)
    f[N_MOM + 2] = ea / 100.0
    f[N_MOM + 3] = eb / 100.0
    return f


def order_from_coefficients(c: np.ndarray, eps: float = ORDER_EPS) -> int:
    """Smallest L >= 1 such that sum_{j=L}^{n_terms-1} |c_j| <= eps: the expansion cut at L
    terms differs from the full one by at most eps in the 2-norm (|T_j| <= 1 on the scaled
    spectrum), whatever the Hamiltonian."""
    n_terms = len(c)
    tail = 0.0
    L = n_terms
    for j in range(n_terms - 1, 0, -1):
        tail += abs(c[j])
        if tail > eps:
            break
        L = j
    return L


def targets(mu: float, ea: float, eb: float, c: np.ndarray) -> np.ndarray:
    """(mu_x, log2(L*) / log2(n_terms)) for the coefficients c of the expansion at mu."""
    n_terms = len(c)
    L = order_from_coefficients(c)
    return np.array([(2.0 * mu - (ea + eb)) / (eb - ea),
                     math.log2(max(L, 1)) / math.log2(max(n_terms, 2))])
