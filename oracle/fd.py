"""Finite-difference Laplacian on a periodic grid (oracle, FP64).

The paper discretises with a twelfth-order accurate central finite-difference
scheme on a periodic cell (Sec. 5, simulation setup).  The central weights of
order 2n for the second derivative have the closed form (Fornberg)

    w_p = 2 (-1)^(p+1) (n!)^2 / (p^2 (n-p)! (n+p)!),   p = 1..n
    w_0 = -2 sum_{p=1}^{n} 1/p^2

so that u''(x) ~ (w_0 u(x) + sum_p w_p (u(x+ph) + u(x-ph))) / h^2.
"""
from math import factorial

import numpy as np
import scipy.sparse as sp


def fd_weights(order: int = 12) -> np.ndarray:
    """Weights w_0..w_n of the central second derivative of the given order."""
    if order % 2 or order < 2:
        raise ValueError("order must be even and >= 2")
    n = order // 2
    w = np.zeros(n + 1)
    for p in range(1, n + 1):
        w[p] = 2.0 * (-1) ** (p + 1) * factorial(n) ** 2 / (
            p * p * factorial(n - p) * factorial(n + p))
    w[0] = -2.0 * sum(1.0 / (p * p) for p in range(1, n + 1))
    return w


def laplacian_1d(n: int, h: float, order: int = 12) -> np.ndarray:
    """Dense periodic n x n second-derivative matrix (wraps mod n)."""
    w = fd_weights(order)
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] += w[0]
        for p in range(1, len(w)):
            A[i, (i + p) % n] += w[p]
            A[i, (i - p) % n] += w[p]
    return A / (h * h)


def laplacian_3d(nx: int, ny: int, nz: int, hx: float, hy: float, hz: float,
                 order: int = 12) -> sp.csr_matrix:
    """Sparse periodic 3-D Laplacian for grid index k = i + nx j + nx ny l.

    With that index order x is the fastest axis, so in Kronecker form
    Lap = Iz (x) Iy (x) Lx + Iz (x) Ly (x) Ix + Lz (x) Iy (x) Ix.
    """
    Lx = sp.csr_matrix(laplacian_1d(nx, hx, order))
    Ly = sp.csr_matrix(laplacian_1d(ny, hy, order))
    Lz = sp.csr_matrix(laplacian_1d(nz, hz, order))
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(Iz, sp.kron(Iy, Lx)) + sp.kron(Iz, sp.kron(Ly, Ix))
            + sp.kron(Lz, sp.kron(Iy, Ix))).tocsr()
