"""Discrete Kohn-Sham Hamiltonian (oracle, FP64).

Sec. 2, Eq. (KSeqn): H = -1/2 Lap + V_eff + V_nl, with the Kleinman-Bylander
nonlocal operator of Eq. (nonlocaloperator), V_nl = sum_J sum_lm gamma_Jl
|chi_Jlm><chi_Jlm|.  On the grid the vectors are Euclidean-normalised
(u = psi sqrt(dV)), so the projector enters as c = chi sqrt(dV) and
V_nl = sum_p gamma_p c_p c_p^T.  V_eff (= V_xc + phi) is an input here.
"""
import numpy as np
import scipy.sparse as sp

from .fd import laplacian_3d


def projector_vectors(N: int, dV: float, ptr, idx, val) -> sp.csc_matrix:
    """N x n_proj sparse matrix whose column p is c_p = chi_p sqrt(dV)."""
    ptr = np.asarray(ptr)
    cols = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    return sp.csc_matrix((np.asarray(val) * np.sqrt(dV), (np.asarray(idx), cols)),
                         shape=(N, len(ptr) - 1))


def hamiltonian_sparse(n: int, L: float, V, proj=None, order: int = 12):
    """H as a scipy sparse matrix (local part) plus low-rank projector part.

    Returns (Hloc, C, gamma) with H = Hloc + C diag(gamma) C^T.
    """
    h = L / n
    Hloc = (-0.5 * laplacian_3d(n, n, n, h, h, h, order)
            + sp.diags(np.asarray(V, dtype=float))).tocsr()
    if proj is None:
        return Hloc, None, None
    C = projector_vectors(n ** 3, h ** 3, proj.ptr, proj.idx, proj.val)
    return Hloc, C, np.asarray(proj.gamma, dtype=float)


def hamiltonian_dense(n: int, L: float, V, proj=None, order: int = 12) -> np.ndarray:
    Hloc, C, gamma = hamiltonian_sparse(n, L, V, proj, order)
    H = Hloc.toarray()
    if C is not None:
        Cd = C.toarray()
        H += (Cd * gamma) @ Cd.T
    return H


def apply(Hparts, X: np.ndarray) -> np.ndarray:
    """Y = H X for X of shape (N, k) using the (Hloc, C, gamma) triple."""
    Hloc, C, gamma = Hparts
    Y = Hloc @ X
    if C is not None:
        Y = Y + C @ (gamma[:, None] * (C.T @ X))
    return Y
