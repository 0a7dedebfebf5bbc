"""Auxiliary-basis steps of one SQ3 iteration (oracle, FP64).

Sec. 4, first paragraph: Chebyshev filtering of the previous auxiliary
orbitals, then orthonormalisation, then projection Hs = X^T H X
(Sec. 3, Eq. (DsHsRelation)); after the kernel, the kernel-transformed
orbitals X Ds (Eq. (phi_tilde)) give rho = 2 sum_i phi~_i phi_i
(Eq. (density:NewForm)).  Vectors are Euclidean-normalised (u = psi sqrt(dV)),
so on the grid rho_k = (2/dV) sum_i X_ki (X Ds)_ki.

The paper does not name its orthonormalisation; the reading used here is
Cholesky QR: S = X^T X = R^T R with R upper triangular, X <- X R^{-1}.
"""
import numpy as np
import scipy.linalg as sla

from . import chebyshev, fermi


def cholqr(X: np.ndarray) -> np.ndarray:
    S = X.T @ X
    R = np.linalg.cholesky(S).T
    return sla.solve_triangular(R, X.T, trans="T", lower=False).T


def project(apply_H, X: np.ndarray) -> np.ndarray:
    Hs = X.T @ apply_H(X)
    return 0.5 * (Hs + Hs.T)


def exact_bounds(Hs: np.ndarray):
    """chi = (lambda_Ns + lambda_1)/2, xi = (lambda_Ns - lambda_1)/2 (Sec. 4)."""
    lam = np.linalg.eigvalsh(Hs)
    return 0.5 * (lam[-1] + lam[0]), 0.5 * (lam[-1] - lam[0])


def density_from_kernel(X: np.ndarray, D: np.ndarray, dV: float) -> np.ndarray:
    return (2.0 / dV) * np.sum(X * (X @ D), axis=1)


def sq3_iteration(apply_H, X, m, a, b, a0, npl, sigma, Ne, dV) -> dict:
    """One fixed-potential SQ3 iteration in the paper's order."""
    Y = chebyshev.filter_plain(apply_H, X, m, a, b, a0)
    Q = cholqr(Y)
    Hs = project(apply_H, Q)
    chi, xi = exact_bounds(Hs)
    out = chebyshev.foe_density_kernel(Hs, npl, sigma, Ne, chi, xi)
    out.update(X=Q, Hs=Hs, chi=chi, xi=xi,
               rho=density_from_kernel(Q, out["D"], dV))
    return out


def kernel_by_diagonalisation(Hs: np.ndarray, Ne: float, sigma: float) -> dict:
    """Ds = g(Hs) through the eigendecomposition of Hs (Eq. (DsHsRelation))."""
    lam, Q = np.linalg.eigh(Hs)
    mu = fermi.fermi_level(lam, Ne, sigma)
    g = fermi.fermi(lam, mu, sigma)
    return {"D": (Q * g) @ Q.T, "mu": mu, "lam": lam,
            "e_band": 2.0 * float(np.dot(g, lam)),
            "e_ent": 2.0 * sigma * float(np.sum(fermi.entropy_density(lam, mu, sigma)))}
