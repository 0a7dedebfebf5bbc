"""Degree of the Chebyshev Fermi-operator expansion: the plain definition.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

The expansion error of the occupations for a degree n_pl is the largest
|f(x) - sum'_j c_j T_j((x - chi) / xi)| over the spectral interval
[chi - xi, chi + xi], with f the Fermi function and c_j of Eq.
(ChebyshevCoeff) (Chebyshev-Gauss quadrature, as in ``chebyshev``).  The
minimal degree for a tolerance is the smallest n_pl whose error stays
below it for every Fermi level of a grid over the interval.  Sec. 5 reports
that this degree falls as the temperature rises; ``npl_sweep`` repeats its
accuracy study (free energy and forces against diagonalisation versus n_pl,
10,000 to 250,000 K) on a synthetic cell.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev
from .fermi import fermi


def max_error(npl: int, mu: float, sigma: float, chi: float, xi: float,
              npts: int = 2001) -> float:
    c = chebyshev.projection_coeffs(lambda l: fermi(xi * l + chi, mu, sigma), npl,
                                    chebyshev.quadrature_size(npl))
    x = np.linspace(-1.0, 1.0, npts)
    return float(np.abs(fermi(xi * x + chi, mu, sigma) - chebyshev.series_scalar(c, x)).max())


def min_degree(tol: float, sigma: float, chi: float, xi: float, n_mu: int = 21,
               nmax: int = 4000) -> int:
    """Smallest n_pl with max_error <= tol for every mu of an n_mu-point grid
    over the interval (bisection on the worst error, then a step down while
    the degree below still meets the tolerance)."""
    mus = chi + xi * np.linspace(-1.0, 1.0, n_mu)
    worst = lambda n: max(max_error(n, mu, sigma, chi, xi) for mu in mus)
    lo, hi = 0, 1
    while worst(hi) > tol:
        lo, hi = hi, 2 * hi
        if hi > nmax:
            raise ValueError("degree beyond nmax")
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if worst(mid) <= tol:
            hi = mid
        else:
            lo = mid
    while hi > 1 and worst(hi - 1) <= tol:
        hi -= 1
    return hi


def npl_sweep(n: int, L: float, positions: np.ndarray, Ns: int, temps_K, npls,
              Z: float, rc: float) -> dict:
    """Error of the free energy per atom and of the local forces against
    diagonalisation, as a function of the expansion degree, at several
    temperatures (the accuracy study of Sec. 5, on a synthetic cell).

    The potential is held fixed (the pseudocharges' electrostatic potential),
    the subspace is the exact lowest Ns eigenvectors, and only the density
    kernel changes: the exact Fermi occupations against the Chebyshev
    expansion of degree n_pl (``chebyshev.foe_density_kernel`` with the exact
    spectral bounds).  F follows Eq. (FreeEnergy:NewForm) and the forces the
    first term of Eq. (force:NewForm) (``scf``, ``forces``)."""
    from . import fermi, forces, hamiltonian, scf, subspace
    KB_HA = 8.617333262e-5 / 27.211386245988
    natoms = len(positions)
    Ne = Z * natoms
    dV = (L / n) ** 3
    b, tot = scf.pseudocharge(n, L, positions, Z, rc, Ne=Ne)
    grad_b = scf.pseudocharge_gradients(n, L, positions, Z, rc, scale=-Ne / tot)
    V = scf.poisson_fd(b, n, L)
    lam, U = fermi.lowest_eigenpairs(hamiltonian.hamiltonian_dense(n, L, V), Ns)
    chi, xi = subspace.exact_bounds(np.diag(lam))

    def f_and_forces(rho, e_band, e_ent):
        phi = scf.poisson_fd(rho + b, n, L)
        F = scf.free_energy(e_band, e_ent, rho, b, phi, dV, natoms, Z, rc)["F"]
        return F, forces.local_forces(grad_b, phi, dV)

    out = {}
    for T in temps_K:
        sigma = T * KB_HA
        ex = fermi.ks_fixed_potential(lam, U, Ne, sigma, dV)
        F0, f0 = f_and_forces(ex["rho"], ex["e_band"], ex["e_ent"])
        rows = []
        for npl in npls:
            k = chebyshev.foe_density_kernel(np.diag(lam), npl, sigma, Ne, chi, xi)
            rho = subspace.density_from_kernel(U, k["D"], dV)
            F, f = f_and_forces(rho, k["e_band"], k["e_ent"])
            rows.append((npl, abs(F - F0) / natoms, float(np.abs(f - f0).max())))
        out[T] = rows
    return out
