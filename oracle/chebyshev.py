"""Chebyshev machinery of the SQ3 method (oracle, FP64).

Sec. 4 of the paper:

* Eq. (ChebyshevExpansion): Ds ~ sum'_{j=0}^{npl} c_j T_j(Hhat),
  Hhat = (Hs - chi I)/xi, chi = (lambda_Ns + lambda_1)/2,
  xi = (lambda_Ns - lambda_1)/2; the prime halves the j = 0 term.
* Eq. (ChebyshevCoeff): c_j = (2/pi) int_{-1}^{1} g(xi l + chi) T_j(l)
  / sqrt(1 - l^2) dl.  The paper does not say how the integral is evaluated;
  the reading used here is Chebyshev-Gauss quadrature with M nodes
  theta_k = (k + 1/2) pi / M, which gives
  c_j = (2/M) sum_k f(cos theta_k) cos(j theta_k), M = max(1024, 8 (npl+1)).
* d_j and e_j: the same projection of (xi l + chi) g and of
  g ln g + (1-g) ln(1-g).
* Eq. (DMCFinal), (ThreeTermRecurrenceRelation): columns t^j_n of T_j(Hhat)
  from t^0 = e_n, t^1 = Hhat e_n, t^{j+1} = 2 Hhat t^j - t^{j-1}.
* Eq. (FermiLevelCalc): mu solves 2 sum_n sum'_j c_j(mu) e_n^T t^j_n = Ne.
* E_band ~ 2 sum_n sum'_j d_j e_n^T t^j_n and E_ent ~ 2 sigma sum_n sum'_j
  e_j e_n^T t^j_n.  The printed entropy expansion omits the factor sigma that
  Eq. (FreeEnergy:NewForm) carries; the reading used here restores it.

The Chebyshev filter of the CheFSI step (Sec. 4, first paragraph, after
Zhou et al. 2006) is given by its plain definition
p_m(t) = T_m((t - c)/e) / T_m((a0 - c)/e), c = (b+a)/2, e = (b-a)/2.
"""
import numpy as np

from .fermi import fermi, entropy_density


def quadrature_size(npl: int) -> int:
    return max(1024, 8 * (npl + 1))


def cheb_T(j: int, x):
    """T_j(x) for any real x: cos(j acos x) on [-1, 1], cosh outside."""
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(j * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** j * np.cosh(j * np.arccosh(np.abs(xo)))
    return out


def projection_coeffs(f, npl: int, M: int) -> np.ndarray:
    """(2/M) sum_k f(cos theta_k) cos(j theta_k), j = 0..npl."""
    theta = (np.arange(M) + 0.5) * np.pi / M
    fx = f(np.cos(theta))
    j = np.arange(npl + 1)
    return (2.0 / M) * np.cos(np.outer(j, theta)) @ fx


def fermi_coeffs(mu: float, sigma: float, chi: float, xi: float, npl: int,
                 M: int | None = None):
    """c_j, d_j, e_j of Eq. (ChebyshevCoeff) and the E_band / E_ent expansions."""
    M = quadrature_size(npl) if M is None else M
    eps = lambda l: xi * l + chi
    c = projection_coeffs(lambda l: fermi(eps(l), mu, sigma), npl, M)
    d = projection_coeffs(lambda l: eps(l) * fermi(eps(l), mu, sigma), npl, M)
    e = projection_coeffs(lambda l: entropy_density(eps(l), mu, sigma), npl, M)
    return c, d, e


def primed_sum(coeffs, terms) -> float:
    """sum'_j coeffs_j terms_j with the j = 0 term halved."""
    coeffs = np.asarray(coeffs, dtype=float)
    terms = np.asarray(terms, dtype=float)
    return float(np.dot(coeffs, terms) - 0.5 * coeffs[0] * terms[0])


def series_scalar(coeffs, x):
    """sum'_j c_j T_j(x) at scalar points x in [-1, 1]."""
    x = np.asarray(x, dtype=float)
    t_prev, t = np.ones_like(x), x.copy()
    acc = 0.5 * coeffs[0] * t_prev + (coeffs[1] * t if len(coeffs) > 1 else 0.0)
    for j in range(2, len(coeffs)):
        t_prev, t = t, 2.0 * x * t - t_prev
        acc = acc + coeffs[j] * t
    return acc


def filter_plain(apply_H, X: np.ndarray, m: int, a: float, b: float, a0: float):
    """p_m(H) X with p_m(t) = T_m((t-c)/e) / T_m((a0-c)/e).

    T_m((H - c)/e) X is built by the three-term recurrence on the
    unscaled Chebyshev polynomials and divided by the scalar at the end.
    """
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    z_prev = X
    z = (apply_H(X) - c * X) / e
    for _ in range(1, m):
        z_prev, z = z, 2.0 * (apply_H(z) - c * z) / e - z_prev
    return z / cheb_T(m, np.array([(a0 - c) / e]))[0]


def fermi_level_series(moments, sigma: float, Ne: float, chi: float, xi: float,
                       M: int | None = None, max_halvings: int = 200) -> float:
    """mu of Eq. (FermiLevelCalc): 2 sum'_j c_j(mu) m_j = Ne, by bisection on
    [chi - xi - 40 sigma, chi + xi + 40 sigma] with c_j(mu) re-evaluated by
    quadrature at every trial mu, until the bracket cannot shrink."""
    npl = len(moments) - 1

    def count(mu):
        c, _, _ = fermi_coeffs(mu, sigma, chi, xi, npl, M)
        return 2.0 * primed_sum(c, moments)

    lo, hi = chi - xi - 40.0 * sigma, chi + xi + 40.0 * sigma
    for _ in range(max_halvings):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if count(mid) < Ne:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def foe_density_kernel(Hs: np.ndarray, npl: int, sigma: float, Ne: float,
                       chi: float, xi: float, M: int | None = None,
                       max_halvings: int = 200) -> dict:
    """Density kernel by the Chebyshev Fermi-operator expansion, Sec. 4.

    Pass 1 runs the column recurrence for all columns at once (T_j as
    matrices) and keeps the moments e_n^T t^j_n summed over n; mu is then
    found by bisection on Eq. (FermiLevelCalc) with c_j(mu) re-evaluated by
    quadrature at every trial mu; pass 2 re-runs the recurrence and
    accumulates Ds = sum'_j c_j T_j.
    """
    Ns = Hs.shape[0]
    Hhat = (Hs - chi * np.eye(Ns)) / xi

    moments = np.empty(npl + 1)
    T_prev, T = np.eye(Ns), Hhat.copy()
    moments[0] = np.trace(T_prev)
    if npl >= 1:
        moments[1] = np.trace(T)
    for j in range(1, npl):
        T_prev, T = T, 2.0 * Hhat @ T - T_prev
        moments[j + 1] = np.trace(T)

    mu = fermi_level_series(moments, sigma, Ne, chi, xi, M, max_halvings)
    c, d, e = fermi_coeffs(mu, sigma, chi, xi, npl, M)

    D = 0.5 * c[0] * np.eye(Ns)
    T_prev, T = np.eye(Ns), Hhat.copy()
    if npl >= 1:
        D += c[1] * T
    for j in range(1, npl):
        T_prev, T = T, 2.0 * Hhat @ T - T_prev
        D += c[j + 1] * T
    return {
        "D": D, "mu": mu, "moments": moments, "c": c, "d": d, "e": e,
        "e_band": 2.0 * primed_sum(d, moments),
        "e_ent": 2.0 * sigma * primed_sum(e, moments),
    }
