"""Pins for the oracle's Chebyshev machinery (Sec. 4: Eq.
(ChebyshevExpansion), (ChebyshevCoeff), (DMCFinal),
(ThreeTermRecurrenceRelation), (FermiLevelCalc), the E_band/E_ent
expansions, and the Chebyshev filter of the CheFSI step)."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy import integrate
from scipy.stats import ortho_group

from oracle import chebyshev, fermi, subspace

SIGMA = 10.0 / 27.211386245988


def test_cheb_T_against_numpy_and_closed_form():
    x = np.linspace(-1, 1, 41)
    for j in (0, 1, 2, 7, 30):
        np.testing.assert_allclose(chebyshev.cheb_T(j, x), npcheb.chebval(x, [0] * j + [1]),
                                   atol=1e-12)
    xo = np.array([-1.3, 1.2, 2.5])
    for j in (3, 8):
        np.testing.assert_allclose(chebyshev.cheb_T(j, xo), npcheb.chebval(xo, [0] * j + [1]),
                                   rtol=1e-12)


def test_projection_of_polynomial_is_exact():
    c = chebyshev.projection_coeffs(lambda l: npcheb.chebval(l, [0.5, 0, 0, 1.5, -2]), 10, 64)
    # f = 0.5 T0 + 1.5 T3 - 2 T4 has coefficients c0 = 1 (primed), c3, c4.
    np.testing.assert_allclose(c, [1.0, 0, 0, 1.5, -2, 0, 0, 0, 0, 0, 0], atol=1e-14)


# quad reports roundoff when it nears its 1e-15 absolute request; the
# comparison below is at 1e-13
@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("j", [0, 1, 5, 17])
def test_fermi_coeffs_against_adaptive_quadrature(j):
    """c_j, d_j, e_j against (2/pi) int_0^pi f(cos t) cos(j t) dt by adaptive
    quadrature: the integral of Eq. (ChebyshevCoeff) after l = cos t."""
    mu, chi, xi = 0.9, 1.1, 2.3
    c, d, e = chebyshev.fermi_coeffs(mu, SIGMA, chi, xi, 20)
    eps = lambda t: xi * np.cos(t) + chi
    fs = (lambda t: fermi.fermi(eps(t), mu, SIGMA),
          lambda t: eps(t) * fermi.fermi(eps(t), mu, SIGMA),
          lambda t: fermi.entropy_density(eps(t), mu, SIGMA))
    for coef, f in zip((c, d, e), fs):
        ref = 2 / np.pi * integrate.quad(lambda t: f(t) * np.cos(j * t), 0, np.pi,
                                         epsabs=1e-15, epsrel=1e-13, limit=200)[0]
        assert abs(coef[j] - ref) < 1e-13


def test_scalar_series_matches_direct_functions():
    """sum' c_j T_j(x) reproduces g, eps*g and the entropy density on 10^4
    points for a spectral half-width ~1 Ha at kT = 10 eV, npl = 60."""
    chi, xi, mu, npl = 0.9, 0.98, 0.6, 60
    c, d, e = chebyshev.fermi_coeffs(mu, SIGMA, chi, xi, npl)
    x = np.linspace(-1, 1, 10000)
    eps = xi * x + chi
    np.testing.assert_allclose(chebyshev.series_scalar(c, x), fermi.fermi(eps, mu, SIGMA), atol=1e-13)
    np.testing.assert_allclose(chebyshev.series_scalar(d, x), eps * fermi.fermi(eps, mu, SIGMA), atol=1e-13)
    np.testing.assert_allclose(chebyshev.series_scalar(e, x), fermi.entropy_density(eps, mu, SIGMA),
                               atol=1e-13)


def test_series_error_falls_with_degree():
    chi, xi, mu = 3.0, 4.0, 1.0
    x = np.linspace(-1, 1, 2001)
    ref = fermi.fermi(xi * x + chi, mu, SIGMA)
    errs = [np.max(np.abs(chebyshev.series_scalar(chebyshev.fermi_coeffs(mu, SIGMA, chi, xi, n)[0], x) - ref))
            for n in (10, 20, 40)]
    assert errs[0] > errs[1] > errs[2]


def _random_hs(Ns=40, seed=0, lo=-1.0, hi=4.0):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(lo, hi, Ns))
    Q = ortho_group.rvs(Ns, random_state=seed + 1)
    return (Q * lam) @ Q.T, lam


def test_foe_matches_diagonalisation_at_high_degree():
    Hs, lam = _random_hs()
    chi, xi = subspace.exact_bounds(Hs)
    foe = chebyshev.foe_density_kernel(Hs, 120, SIGMA, 14.0, chi, xi)
    ref = subspace.kernel_by_diagonalisation(Hs, 14.0, SIGMA)
    np.testing.assert_allclose(foe["D"], ref["D"], atol=1e-12)
    assert abs(foe["mu"] - ref["mu"]) < 1e-11
    assert abs(foe["e_band"] - ref["e_band"]) < 1e-11
    assert abs(foe["e_ent"] - ref["e_ent"]) < 1e-11
    # E_band by the d_j series equals 2 tr(Ds Hs) (Eq. (FreeEnergy:NewForm)).
    assert abs(foe["e_band"] - 2 * np.sum(foe["D"] * Hs)) < 1e-11
    # Ds and Hs commute; eigenvalues of Ds lie in (0, 1).
    assert np.max(np.abs(foe["D"] @ Hs - Hs @ foe["D"])) < 1e-11
    ev = np.linalg.eigvalsh(foe["D"])
    assert ev.min() > 0 and ev.max() < 1


def test_foe_trace_constraint_holds_at_low_degree():
    """At npl = 8 the expansion is inexact, but mu is chosen from the same
    moments, so 2 tr Ds = Ne still holds to rounding (Eq. (FermiLevelCalc))."""
    Hs, _ = _random_hs(seed=5)
    chi, xi = subspace.exact_bounds(Hs)
    foe = chebyshev.foe_density_kernel(Hs, 8, SIGMA, 14.0, chi, xi)
    ref = subspace.kernel_by_diagonalisation(Hs, 14.0, SIGMA)
    assert abs(2 * np.trace(foe["D"]) - 14.0) < 1e-12
    assert np.max(np.abs(foe["D"] - ref["D"])) > 1e-6


def test_filter_acts_as_scalar_polynomial_on_eigenvectors():
    """p_m(H) v = p_m(lambda) v for an eigenpair, p_m(a0) = 1, and the result
    equals U p_m(Lambda) U^T X computed through the eigendecomposition."""
    Hs, lam = _random_hs(Ns=30, seed=2, lo=-1.0, hi=9.0)
    w, U = np.linalg.eigh(Hs)
    m, a, b, a0 = 12, 2.0, 9.5, w[0]
    apply_H = lambda X: Hs @ X
    Y = chebyshev.filter_plain(apply_H, U, m, a, b, a0)
    c, e = 0.5 * (b + a), 0.5 * (b - a)
    scal = chebyshev.cheb_T(m, (w - c) / e) / chebyshev.cheb_T(m, np.array([(a0 - c) / e]))[0]
    np.testing.assert_allclose(Y, U * scal, atol=1e-11 * np.abs(scal).max())
    assert abs(scal[0] - 1.0) < 1e-13
    X = np.random.default_rng(0).normal(size=(30, 5))
    np.testing.assert_allclose(chebyshev.filter_plain(apply_H, X, m, a, b, a0),
                               U @ (scal[:, None] * (U.T @ X)), atol=1e-10)
    # Components with eigenvalues in [a, b] are damped below 1 in magnitude.
    inside = (w >= a) & (w <= b)
    assert np.all(np.abs(scal[inside]) <= 1.0 / abs(chebyshev.cheb_T(m, np.array([(a0 - c) / e]))[0]) + 1e-15)
