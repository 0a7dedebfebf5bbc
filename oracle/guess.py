"""Initial electron densities for the SCF: plain FP64 CPU code.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

The paper starts each SCF from a density it does not specify.  Three
starting points are compared here:

* uniform: N_e / |Omega| everywhere;
* atomic superposition: a Gaussian per atom (periodic images summed),
  normalised to N_e, its width fitted to reference densities;
* learned: a small multilayer perceptron on Gaussian radial descriptors
  d_k(x) = sum_I sum_images exp(-|x - R_I|^2 / w_k^2), rho(x) =
  N_e softplus(z(x)) / (sum softplus(z) dV) with
  z = W2 . tanh(W1^T d(x) + b1) + b2, trained by L-BFGS on the squared
  density error against self-consistent densities of other cells.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize, minimize_scalar

WIDTHS = (0.8, 1.3, 2.0, 3.0)     # descriptor widths, bohr
HIDDEN = 8


def _gauss_1d(n: int, L: float, r0: float, w: float) -> np.ndarray:
    x = np.arange(n) * (L / n)
    kmax = int(np.ceil(27.0 * w / L)) + 1
    out = np.zeros(n)
    for m in range(-kmax, kmax + 1):
        d = x - r0 - m * L
        out += np.exp(-d * d / (w * w))
    return out


def radial_sum(n: int, L: float, positions: np.ndarray, w: float) -> np.ndarray:
    """sum over atoms and images of exp(-|x - R|^2 / w^2) on the grid."""
    tot = np.zeros((n, n, n))
    for R in positions:
        tot += np.einsum("l,j,i->lji", _gauss_1d(n, L, R[2], w), _gauss_1d(n, L, R[1], w),
                         _gauss_1d(n, L, R[0], w))
    return tot.ravel()


def descriptors(n: int, L: float, positions: np.ndarray, widths=WIDTHS) -> np.ndarray:
    """(N, len(widths)) features."""
    return np.stack([radial_sum(n, L, positions, w) for w in widths], axis=1)


def uniform(n: int, L: float, Ne: float) -> np.ndarray:
    return np.full(n ** 3, Ne / L ** 3)


def superposition(n: int, L: float, positions: np.ndarray, Ne: float, w: float) -> np.ndarray:
    r = radial_sum(n, L, positions, w)
    return r * Ne / (r.sum() * (L / n) ** 3)


def fit_superposition_width(samples, n: int, L: float, Ne: float) -> float:
    """Width minimising the mean L1 error over (positions, rho) samples."""
    dV = (L / n) ** 3

    def err(w):
        return np.mean([np.abs(superposition(n, L, p, Ne, w) - r).sum() * dV for p, r in samples])

    return float(minimize_scalar(err, bounds=(0.5, 5.0), method="bounded",
                                 options={"xatol": 1e-3}).x)


def _unpack(p: np.ndarray, K: int):
    W1 = p[:K * HIDDEN].reshape(K, HIDDEN)
    b1 = p[K * HIDDEN:K * HIDDEN + HIDDEN]
    W2 = p[K * HIDDEN + HIDDEN:K * HIDDEN + 2 * HIDDEN]
    return W1, b1, W2, p[-1]


def n_params(K: int = len(WIDTHS)) -> int:
    return K * HIDDEN + 2 * HIDDEN + 1


def predict(p: np.ndarray, X: np.ndarray, Ne: float, dV: float) -> np.ndarray:
    W1, b1, W2, b2 = _unpack(p, X.shape[1])
    y = np.logaddexp(0.0, np.tanh(X @ W1 + b1) @ W2 + b2)
    return y * Ne / (y.sum() * dV)


def loss_and_grad(p: np.ndarray, data, Ne: float, dV: float):
    """sum over (X, rho_ref) of int (rho_hat - rho_ref)^2 dx and its
    gradient in the parameters (back-propagation through the
    normalisation, the softplus and the tanh layer)."""
    K = data[0][0].shape[1]
    W1, b1, W2, b2 = _unpack(p, K)
    loss, g = 0.0, np.zeros_like(p)
    for X, r in data:
        A = np.tanh(X @ W1 + b1)
        z = A @ W2 + b2
        y = np.logaddexp(0.0, z)
        S = y.sum() * dV
        res = y * Ne / S - r
        loss += float(np.sum(res * res) * dV)
        drh = 2.0 * res * dV
        dy = (Ne / S) * drh - (Ne / S ** 2) * dV * float(np.sum(drh * y))
        dz = dy / (1.0 + np.exp(-z))
        dA = np.outer(dz, W2) * (1.0 - A * A)
        g += np.concatenate([(X.T @ dA).ravel(), dA.sum(0), A.T @ dz, [dz.sum()]])
    return loss, g


def train(data, Ne: float, dV: float, seed: int = 0, maxiter: int = 500) -> np.ndarray:
    p0 = np.random.default_rng(seed + 32452843).normal(size=n_params(data[0][0].shape[1])) * 0.3
    res = minimize(loss_and_grad, p0, args=(data, Ne, dV), jac=True, method="L-BFGS-B",
                   options={"maxiter": maxiter})
    return res.x
