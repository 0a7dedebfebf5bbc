"""Degree of the Chebyshev Fermi-operator expansion: the plain definition.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

The expansion error of the occupations for a degree n_pl is the largest
|f(x) - sum'_j c_j T_j((x - chi) / xi)| over the spectral interval
[chi - xi, chi + xi], with f the Fermi function and c_j of Eq.
(ChebyshevCoeff) (Chebyshev-Gauss quadrature, as in ``chebyshev``).  The
minimal degree for a tolerance is the smallest n_pl whose error stays
below it for every Fermi level of a grid over the interval.  Sec. 5 reports
that this degree falls as the temperature rises.
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
