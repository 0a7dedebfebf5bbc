"""Hellmann-Feynman forces on the nuclei: plain FP64 CPU code.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

Eq. (force:NewForm) (Sec. 3; Eq. (ON:forces) in Sec. 2):

    f_I = sum_{I'} int grad b_{I'}(x, R_{I'}) phi(x) dx + f_sc,I
          - 4 sum_i sum_lm gamma_Il (int phi_i chi_Ilm dx)(int grad phi~_i chi_Ilm dx),

I' running over atom I and its periodic images, phi the electrostatic
potential of rho + b, phi_i the orthonormal subspace functions and
phi~_i = sum_j phi_j (Ds)_ji their transforms by the density kernel.
With the Gaussian pseudocharges used here E_self is a constant and E_c = 0,
so f_sc = 0.  On the grid every integral is a sum times dV; with Euclidean
vectors u = phi sqrt(dV) and c = chi sqrt(dV), the nonlocal term is
-4 sum gamma (c . u_i)(c . grad_h u~_i), grad_h the central
finite-difference first derivative of the same order as the Laplacian.
"""
from __future__ import annotations

import numpy as np


def fd_first_weights(order: int = 12) -> np.ndarray:
    """a_1..a_n (n = order/2) of the central first derivative
    f'(x) ~ sum_p a_p (f(x + p h) - f(x - p h)) / h, Fornberg's closed form
    a_p = (-1)^(p+1) (n!)^2 / (p (n-p)! (n+p)!)."""
    from math import factorial
    n = order // 2
    return np.array([(-1) ** (p + 1) * factorial(n) ** 2 /
                     (p * factorial(n - p) * factorial(n + p)) for p in range(1, n + 1)])


def gradient_fd(U: np.ndarray, n: int, L: float, order: int = 12) -> np.ndarray:
    """grad_h of grid functions: U is (n^3,) or (n^3, k) in grid order
    [z][y][x]; returns (3, n^3) or (3, n^3, k), components x, y, z."""
    h = L / n
    a = fd_first_weights(order)
    shape = U.shape
    V = U.reshape((n, n, n) + shape[1:])
    out = []
    for axis in (2, 1, 0):                      # x, y, z
        g = np.zeros_like(V)
        for p, w in enumerate(a, start=1):
            g += w * (np.roll(V, -p, axis=axis) - np.roll(V, p, axis=axis))
        out.append((g / h).reshape(shape))
    return np.stack(out)


def local_forces(grad_b: np.ndarray, phi: np.ndarray, dV: float) -> np.ndarray:
    """First term of Eq. (force:NewForm): (natoms, 3) from grad_x b_I on the
    grid (natoms, 3, N; images included) and phi (N)."""
    return np.einsum("iak,k->ia", grad_b, phi) * dV


def nonlocal_forces(X: np.ndarray, Ds: np.ndarray, proj, n: int, L: float, natoms: int,
                    atom_of: np.ndarray | None = None, order: int = 12) -> np.ndarray:
    """Last term of Eq. (force:NewForm): (natoms, 3).

    X: N x Ns orthonormal (Euclidean) subspace vectors; Ds: Ns x Ns density
    kernel; proj: table with ptr, idx, val (chi at idx, continuum values)
    and gamma; atom_of[p]: the atom of projector p (default p // 4)."""
    N = X.shape[0]
    dV = (L / n) ** 3
    Xt = X @ Ds                                  # u~_i
    G = gradient_fd(Xt, n, L, order)             # (3, N, Ns)
    nproj = len(proj.gamma)
    if atom_of is None:
        atom_of = np.arange(nproj) // 4
    f = np.zeros((natoms, 3))
    for p in range(nproj):
        sl = slice(proj.ptr[p], proj.ptr[p + 1])
        c = np.zeros(N)
        c[proj.idx[sl]] = proj.val[sl] * np.sqrt(dV)
        cu = c @ X                               # (Ns,)
        for a in range(3):
            f[atom_of[p], a] -= 4.0 * proj.gamma[p] * float(cu @ (c @ G[a]))
    return f
