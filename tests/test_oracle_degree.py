"""Pins of the degree oracle (``oracle.degree``) and of the library's degree
rule (sq3_fermi_degree, host arithmetic, called here through the C ABI on the
CPU).  The oracle's error decays at the rate the Bernstein ellipse through
the Fermi function's nearest pole fixes, ln rho with rho = a + sqrt(1 + a^2),
a = pi sigma / xi; the minimal degree falls as the temperature rises (the
trend Sec. 5 reports); the rule's degree meets the tolerance for every Fermi
level in the interval without being wasteful."""
import numpy as np
import pytest

from oracle import degree

KB_HA = 8.617333262e-5 / 27.211386245988      # Boltzmann constant, Ha / K
CHI, XI = 0.5, 1.5


def _rho(sigma, xi):
    a = np.pi * sigma / xi
    return a + np.sqrt(1.0 + a * a)


def test_error_decays_at_the_ellipse_rate():
    """Fermi level at the centre (the pole nearest the interval): the error
    of degrees 20..60 falls like rho^-n (fitted rate within 3 %)."""
    sigma = 0.1
    ns = np.arange(21, 61, 4)                    # odd degrees (f - 1/2 is odd here)
    e = [degree.max_error(n, CHI, sigma, CHI, XI) for n in ns]
    slope = -np.polyfit(ns, np.log(e), 1)[0]
    assert abs(slope / np.log(_rho(sigma, XI)) - 1) < 0.03
    assert degree.max_error(200, CHI, sigma, CHI, XI) < 1e-12     # rounding level (1.2e-14)


def test_min_degree_falls_as_temperature_rises():
    degs = [degree.min_degree(1e-4, T * KB_HA, CHI, XI) for T in (10_000, 50_000, 100_000, 250_000)]
    assert all(a > b for a, b in zip(degs, degs[1:])), degs


@pytest.fixture(scope="module")
def sq3_host():
    from paper_2112_08639_gb300 import build
    build.build()
    from paper_2112_08639_gb300 import sq3
    return sq3


@pytest.mark.parametrize("a", [0.05, 0.2, 0.8])
@pytest.mark.parametrize("tol", [1e-3, 1e-9])
def test_library_degree_rule_meets_the_tolerance(sq3_host, a, tol):
    sigma = a * XI / np.pi
    n_rule = sq3_host.fermi_degree(sigma, XI, tol)
    n_min = degree.min_degree(tol, sigma, CHI, XI)
    assert n_min <= n_rule <= 1.15 * n_min + 2, (n_min, n_rule)
    mus = CHI + XI * np.linspace(-1, 1, 21)
    assert max(degree.max_error(n_rule, mu, sigma, CHI, XI) for mu in mus) <= tol


def test_library_degree_rule_errors(sq3_host):
    for bad in ((0.0, 1.0, 1e-3), (0.1, 0.0, 1e-3), (0.1, 1.0, 0.0), (0.1, 1.0, 1.0),
                (float("nan"), 1.0, 1e-3)):
        with pytest.raises(sq3_host.SQ3Error):
            sq3_host.fermi_degree(*bad)
    assert sq3_host.fermi_degree(100.0, 1.0, 0.5) == 1
