"""The learned starting density as a plain FP64 CPU model: forward pass,
loss, back-propagated gradient and Adam, for checking the GPU's BF16
training and inference kernels.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

Not in the paper (which does not say how each SCF starts): the starting
density of a QMD step is predicted from the atom positions by a multilayer
perceptron over atom-centred Gaussian descriptors.

* Descriptors at grid point x: d_k(x) = sum_J sum_images
  exp(-|x - R_J|^2 / w_k^2) for the widths w_k of WIDTHS, divided by their
  mean over the cell, natoms pi^(3/2) w_k^3 / Omega (the same scale for any
  cell of the same atom density), and compressed as f_k = log(1 + d_k):
  near an atom the narrow widths reach a hundred times their mean, which
  would saturate the first tanh layer.
* Network: three hidden layers of HIDDEN units with tanh,
  h_1 = tanh(W_1 d + b_1), h_l = tanh(W_l h_{l-1} + b_l) (l = 2, 3), and an
  output y = softplus(w_4 . h_3 + b_4) > 0.
* Density: rho(x) = Ne y(x) / (sum_x y dV), so it holds exactly Ne electrons.
* Loss of one cell: L = sum_x (rho(x) - rho*(x))^2 dV against the
  self-consistent density rho*.
* Gradient by back-propagation through the normalisation, the softplus and
  the tanh layers (chain rule, written out below); pinned against central
  finite differences of L.
* Adam (Kingma and Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

from .guess import radial_sum

WIDTHS = (0.6, 0.8, 1.0, 1.3, 1.6, 2.0, 2.5, 3.0)    # bohr
HIDDEN = 128
LAYER_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")


def descriptors(n: int, L: float, positions: np.ndarray, widths=WIDTHS) -> np.ndarray:
    """(N, len(widths)) features log(1 + d_k / mean_k)."""
    natoms = len(positions)
    cols = []
    for w in widths:
        mean = natoms * np.pi ** 1.5 * w ** 3 / L ** 3
        cols.append(np.log1p(radial_sum(n, L, positions, w) / mean))
    return np.stack(cols, axis=1)


def init_params(n_in: int = len(WIDTHS), hidden: int = HIDDEN, seed: int = 0) -> dict:
    """Seeded initial weights: W_l ~ N(0, 1 / fan_in), biases 0, output 0."""
    rng = np.random.default_rng(seed + 7368787)
    p = {"W1": rng.normal(size=(hidden, n_in)) / np.sqrt(n_in), "b1": np.zeros(hidden),
         "W2": rng.normal(size=(hidden, hidden)) / np.sqrt(hidden), "b2": np.zeros(hidden),
         "W3": rng.normal(size=(hidden, hidden)) / np.sqrt(hidden), "b3": np.zeros(hidden),
         "w4": rng.normal(size=hidden) / np.sqrt(hidden), "b4": np.zeros(1)}
    return p


def forward(p: dict, X: np.ndarray) -> dict:
    """Activations of every layer for features X (P, n_in)."""
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    z = h3 @ p["w4"] + p["b4"][0]
    y = np.logaddexp(0.0, z)
    return {"h1": h1, "h2": h2, "h3": h3, "z": z, "y": y}


def predict(p: dict, X: np.ndarray, Ne: float, dV: float) -> np.ndarray:
    y = forward(p, X)["y"]
    return y * Ne / (y.sum() * dV)


def loss(p: dict, X: np.ndarray, rho_ref: np.ndarray, Ne: float, dV: float) -> float:
    r = predict(p, X, Ne, dV) - rho_ref
    return float(np.sum(r * r) * dV)


def loss_and_grad(p: dict, X: np.ndarray, rho_ref: np.ndarray, Ne: float, dV: float):
    """L and dL/dp (a dict shaped like p)."""
    a = forward(p, X)
    y = a["y"]
    S = y.sum() * dV
    res = y * Ne / S - rho_ref
    L = float(np.sum(res * res) * dV)
    g_rho = 2.0 * res * dV                           # dL/drho
    # rho = Ne y / S, S = sum y dV: dL/dy_q = (Ne / S)(g_q - dV sum_p g_p y_p / S)
    dy = (Ne / S) * (g_rho - dV * float(np.dot(g_rho, y)) / S)
    dz = dy / (1.0 + np.exp(-a["z"]))               # softplus' = sigmoid
    g = {"w4": a["h3"].T @ dz, "b4": np.array([dz.sum()])}
    dh3 = np.outer(dz, p["w4"])
    dz3 = dh3 * (1.0 - a["h3"] ** 2)
    g["W3"], g["b3"] = dz3.T @ a["h2"], dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * (1.0 - a["h2"] ** 2)
    g["W2"], g["b2"] = dz2.T @ a["h1"], dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - a["h1"] ** 2)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(0)
    return L, g


class Adam:
    def __init__(self, p: dict, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = {k: np.zeros_like(v) for k, v in p.items()}
        self.v = {k: np.zeros_like(v) for k, v in p.items()}
        self.t = 0

    def step(self, p: dict, g: dict) -> None:
        self.t += 1
        for k in p:
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * g[k]
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * g[k] * g[k]
            mh = self.m[k] / (1.0 - self.b1 ** self.t)
            vh = self.v[k] / (1.0 - self.b2 ** self.t)
            p[k] = p[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
