"""Fermi-Dirac occupations, Fermi level, density and energies by exact
diagonalisation (oracle, FP64).

This is the plain definition the SQ3 method converges to (Sec. 3: the
auxiliary basis spans the same N_s-dimensional subspace as the Kohn-Sham
orbitals, Eq. (SubspaceRotation), and Ds = g(Hs), Eq. (DsHsRelation)):

* g(lambda, mu, sigma) = 1 / (1 + exp((lambda - mu)/sigma))   (Sec. 2)
* mu fixed by 2 Tr D = 2 sum_n g_n = N_e                     (Eq. (TraceD))
* rho(x) = 2 D(x, x) = 2 sum_n g_n psi_n(x)^2                 (Eq. (rhoDensMat))
* E_band = 2 Tr(D H) = 2 sum_n g_n lambda_n                   (Eq. (ON:FreeEnergy))
* E_ent  = 2 sigma sum_n [g ln g + (1-g) ln(1-g)]            (Eq. (ON:FreeEnergy))

The N_s lowest states are kept (Sec. 2: the sum runs over N_s states).
"""
import numpy as np
import scipy.linalg as sla
from scipy.special import expit


def fermi(lam, mu: float, sigma: float):
    """g = 1/(1 + exp((lam - mu)/sigma)), evaluated without overflow."""
    return expit(-(np.asarray(lam, dtype=float) - mu) / sigma)


def entropy_density(lam, mu: float, sigma: float):
    """g ln g + (1-g) ln(1-g) at x = (lam - mu)/sigma.

    With ln g = -softplus(x) and ln(1-g) = x - softplus(x) this equals
    -softplus(x) + (1-g) x.  The expression is even in x (g(-x) = 1 - g(x)),
    so it is evaluated at t = -|x| <= 0, where both terms are negative and
    nothing cancels: -log1p(e^t) + t e^t / (1 + e^t).
    """
    t = -np.abs((np.asarray(lam, dtype=float) - mu) / sigma)
    et = np.exp(t)
    return -np.log1p(et) + t * et / (1.0 + et)


def fermi_level(lam, Ne: float, sigma: float, max_halvings: int = 200) -> float:
    """mu with 2 sum_n g(lam_n, mu, sigma) = Ne, by bisection.

    The count is strictly increasing in mu, so the root is unique; the
    bracket [lam_min - 40 sigma, lam_max + 40 sigma] contains it whenever
    0 < Ne < 2 len(lam).  Bisection runs until the bracket cannot shrink.
    """
    lam = np.asarray(lam, dtype=float)
    if not (0.0 < Ne < 2.0 * len(lam)):
        raise ValueError("need 0 < Ne < 2 Ns")
    lo, hi = lam.min() - 40.0 * sigma, lam.max() + 40.0 * sigma
    for _ in range(max_halvings):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if 2.0 * fermi(lam, mid, sigma).sum() < Ne:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def lowest_eigenpairs(H: np.ndarray, Ns: int):
    """The Ns lowest eigenpairs of a dense symmetric H (LAPACK via scipy)."""
    lam, U = sla.eigh(H, subset_by_index=[0, Ns - 1])
    return lam, U


def ks_fixed_potential(lam, U, Ne: float, sigma: float, dV: float) -> dict:
    """Occupations, mu, rho and the two energies from eigenpairs.

    U holds Euclidean-normalised eigenvectors (columns), so psi = U/sqrt(dV)
    and rho_k = (2/dV) sum_n g_n U_kn^2.
    """
    mu = fermi_level(lam, Ne, sigma)
    g = fermi(lam, mu, sigma)
    rho = (2.0 / dV) * (U * U) @ g
    return {
        "lam": lam, "mu": mu, "g": g, "rho": rho,
        "e_band": 2.0 * float(np.dot(g, lam)),
        "e_ent": 2.0 * sigma * float(np.sum(entropy_density(lam, mu, sigma))),
    }
