"""Pins of the SCF oracle (``oracle.scf``): electrostatics, LDA, mixing and
the free energy, each checked against something other than itself (the
separately pinned FD operator, closed forms, textbook limits, finite
differences, a linear fixed point, and a second route to F)."""
import numpy as np
import pytest

from oracle import fd, fermi, scf
from paper_2112_08639_gb300 import inputs


def test_fd_symbol_is_minus_the_eigenvalue_of_the_fd_matrix():
    n = 11
    L1 = fd.laplacian_1d(n, 1.0, 12)
    s = scf.fd_symbol(n, 12)
    k = np.arange(n)
    for m in range(n):
        mode = np.exp(2j * np.pi * np.fft.fftfreq(n, d=1.0 / n)[m] * k / n)
        np.testing.assert_allclose(L1 @ mode, -s[m] * mode, atol=1e-12)
    assert abs(s[0]) < 1e-13 and np.all(s[1:] > 0)


def test_poisson_residual_through_the_real_space_laplacian():
    n, L = 10, 7.0
    rng = np.random.default_rng(1)
    rho = rng.normal(size=n ** 3)
    phi = scf.poisson_fd(rho, n, L)
    h = L / n
    Lap = fd.laplacian_3d(n, n, n, h, h, h, 12)
    np.testing.assert_allclose(-(Lap @ phi) / (4 * np.pi), rho - rho.mean(), atol=1e-11)
    assert abs(phi.mean()) < 1e-12


def test_poisson_single_mode_closed_form():
    n, L, m = 12, 9.0, 2
    h = L / n
    x = (np.arange(n ** 3) % n) * h
    rho = np.cos(2 * np.pi * m * x / L)
    phi = scf.poisson_fd(rho, n, L)
    s = -fd.fd_weights(12)[0] - 2 * sum(w * np.cos(p * 2 * np.pi * m / n)
                                        for p, w in enumerate(fd.fd_weights(12)) if p)
    np.testing.assert_allclose(phi, 4 * np.pi * rho / (s / h ** 2), atol=1e-12)


def test_pseudocharge_sums():
    cfg = inputs.C1
    pos = inputs.fcc_positions(cfg.ncell, disp_sigma=cfg.disp_sigma, seed=cfg.seed)
    b, total = scf.pseudocharge(cfg.n, cfg.L, pos, inputs.Z_VALENCE, inputs.RC_LOCAL, Ne=cfg.Ne)
    assert abs(total + 12.0) < 1e-12                      # periodic sum, unscaled (aliasing only)
    assert abs(b.sum() * cfg.dV + cfg.Ne) < 1e-12         # rescaled exactly
    assert np.all(b <= 0)


def test_potential_of_the_pseudocharges_matches_the_continuum_local_potential():
    """phi[b] by the FD Poisson solve against the continuum Coulomb potential
    of the same Gaussians (the fixed local potential of the inputs): they
    differ only by the FD symbol at high frequency and by grid sampling."""
    n, L = 24, inputs.A0_FCC
    pos = inputs.fcc_positions(1, disp_sigma=0.05, seed=0)
    b, _ = scf.pseudocharge(n, L, pos, inputs.Z_VALENCE, inputs.RC_LOCAL, Ne=12.0)
    phi = scf.poisson_fd(b, n, L)
    V = inputs.local_potential(n, L, pos)
    assert np.max(np.abs(phi - V)) < 2e-5 * np.max(np.abs(V))      # 1.8e-6 seen


def test_slater_exchange_closed_form():
    """eps_x in terms of rs is the textbook -(3/4) (9 / (4 pi^2))^(1/3) / rs
    = -0.458165 / rs (the function takes rho)."""
    rs = np.array([0.5, 1.0, 2.0, 5.0])
    ex, vx = scf.slater_exchange(3.0 / (4.0 * np.pi * rs ** 3))
    np.testing.assert_allclose(ex, -0.4581652932831429 / rs, rtol=1e-12)
    np.testing.assert_allclose(vx, -0.6108870577108572 / rs, rtol=1e-12)


def test_vxc_is_the_density_derivative_of_rho_eps_xc():
    rho = np.array([1e-4, 1e-3, 0.01, 0.1, 1.0, 10.0])
    _, v = scf.lda_xc(rho)
    d = 1e-6 * rho
    ep, _ = scf.lda_xc(rho + d)
    em, _ = scf.lda_xc(rho - d)
    fdv = ((rho + d) * ep - (rho - d) * em) / (2 * d)
    np.testing.assert_allclose(v, fdv, rtol=1e-8)


def test_pw92_high_density_limit_is_gell_mann_brueckner():
    """d eps_c / d ln rs -> (1 - ln 2) / pi^2 as rs -> 0; eps_c < 0."""
    rs = np.array([1e-8, 1e-8 * np.exp(1e-3)])
    ec, _ = scf.pw92_correlation(3.0 / (4.0 * np.pi * rs ** 3))
    slope = (ec[1] - ec[0]) / 1e-3
    gmb = (1 - np.log(2)) / np.pi ** 2
    assert abs(slope - gmb) < 1e-3 * gmb
    ec1, _ = scf.pw92_correlation(3.0 / (4.0 * np.pi * np.array([0.5, 1.0, 5.0, 20.0]) ** 3))
    assert np.all(ec1 < 0) and np.all(np.diff(ec1) > 0)    # weaker as the gas thins


def test_kerker_removes_the_mean_and_scales_a_mode():
    n, L, k0 = 8, 6.0, 0.8
    x = (np.arange(n ** 3) % n) * (L / n)
    mode = np.cos(2 * np.pi * x / L)
    out = scf.kerker(3.0 + mode, n, L, k0)
    g2 = (2 * np.pi / L) ** 2
    np.testing.assert_allclose(out, g2 / (g2 + k0 ** 2) * mode, atol=1e-12)


@pytest.mark.parametrize("period", [1, 2])
def test_pulay_solves_a_linear_fixed_point(period):
    rng = np.random.default_rng(3)
    dim = 6
    Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
    A = Q @ np.diag(np.linspace(-0.9, 0.9, dim)) @ Q.T
    c = rng.normal(size=dim)
    xstar = np.linalg.solve(np.eye(dim) - A, c)
    mix = scf.PulayMixer(beta=0.3, history=dim + 1, period=period)
    x = np.zeros(dim)
    for _ in range(40):
        x = mix.step(x, A @ x + c)
    assert np.linalg.norm(x - xstar) < 1e-10 * np.linalg.norm(xstar)


def test_scf_small_cell_converges_and_f_matches_the_direct_route():
    """A 4-atom cell on a 12^3 grid to self-consistency; F by the paper's
    double-counting form against the direct sum T_s + E_xc + the
    electrostatic energy of rho + b - E_self + E_ent (no projectors here, so
    no nonlocal energy)."""
    n, L = 12, inputs.A0_FCC
    pos = inputs.fcc_positions(1, disp_sigma=0.05, seed=0)
    sigma = inputs.ev_to_ha(10.0)
    res = scf.scf(n, L, pos, Ns=40, sigma=sigma, Z=inputs.Z_VALENCE, rc=inputs.RC_LOCAL,
                  tol=1e-9)
    dV = (L / n) ** 3
    assert res["errors"][-1] < 1e-9
    assert abs(res["rho"].sum() * dV - 12.0) < 1e-9
    # direct route: kinetic energy from the eigenvectors and occupations
    h = L / n
    Lap = fd.laplacian_3d(n, n, n, h, h, h, 12)
    g = fermi.fermi(res["lam"], res["mu"], sigma)
    U = res["U"]
    t_s = 2.0 * float(np.sum(g * np.einsum("ki,ki->i", U, -0.5 * (Lap @ U))))
    exc, _ = scf.lda_xc(res["rho"])
    phi = scf.poisson_fd(res["rho"] + res["b"], n, L)
    e_h = 0.5 * float(np.sum((res["rho"] + res["b"]) * phi) * dV)
    F_direct = (t_s + float(np.sum(exc * res["rho"]) * dV) + e_h - res["e_self"] + res["e_ent"])
    assert abs(res["F"] - F_direct) < 1e-9 * abs(res["F"])      # 2.6e-11 seen


def test_kerker_preconditioned_pulay_reaches_the_fixed_point():
    """A mean-preserving linear contraction on a grid, x -> x0_mean + S (x -
    mean) + c with c of zero mean, S a smoothing operator diagonal in Fourier
    space (eigenvalues in (-0.6, 0.9)): Kerker kills the mean of the
    residual, which is zero here, so the preconditioned Pulay iteration must
    reach the exact fixed point (period 2, history 7, beta 0.3)."""
    n, L, k0 = 8, 6.0, 0.8
    rng = np.random.default_rng(4)
    lam = rng.uniform(-0.6, 0.9, size=(n, n, n))
    lam = 0.5 * (lam + np.roll(np.flip(lam), 1, axis=(0, 1, 2)))   # lam(k) = lam(-k): S real
    lam[0, 0, 0] = 0.0
    c = rng.normal(size=n ** 3)
    c -= c.mean()

    def S(x):
        return np.fft.ifftn(lam * np.fft.fftn(x.reshape(n, n, n))).real.ravel()

    def G(x):
        return x.mean() + S(x - x.mean()) + c

    x0 = np.full(n ** 3, 0.7)
    chat = np.fft.fftn(c.reshape(n, n, n))
    den = 1.0 - lam
    den[0, 0, 0] = 1.0
    xstar = 0.7 + np.fft.ifftn(chat / den).real.ravel()
    np.testing.assert_allclose(G(xstar), xstar, atol=1e-12)
    mix = scf.PulayMixer(beta=0.3, history=7, period=2, precond=lambda f: scf.kerker(f, n, L, k0))
    x = x0
    for _ in range(60):
        x = mix.step(x, G(x))
    assert np.max(np.abs(x - xstar)) < 1e-9
    assert abs(x.mean() - 0.7) < 1e-12


def test_self_energy_is_the_gaussians_own_coulomb_energy():
    """E_self per atom = 1/2 int rho(r) phi(r) d^3r for the Gaussian charge
    rho = Z exp(-r^2/rc^2) / (pi^(3/2) rc^3), whose potential is
    Z erf(r/rc) / r: radial quadrature against the closed form used in F."""
    from scipy.integrate import quad
    from scipy.special import erf
    for Z, rc in ((3.0, 1.0), (1.0, 0.6), (4.0, 1.7)):
        rho = lambda r: Z * np.exp(-r * r / (rc * rc)) / (np.pi ** 1.5 * rc ** 3)
        e, _ = quad(lambda r: 0.5 * 4 * np.pi * r * rho(r) * Z * erf(r / rc), 0, 30 * rc,
                    epsabs=1e-14, epsrel=1e-13)
        assert abs(scf.self_energy(1, Z, rc) - e) < 1e-11 * e
        assert abs(scf.self_energy(5, Z, rc) - 5 * e) < 1e-10 * e


def test_scf_in_the_papers_order_reaches_the_diagonalisation_scf():
    """The SCF with the fixed-potential SQ3 iteration inside (filter, CholQR,
    Hs, Chebyshev kernel of degree 80) against the SCF by exact
    diagonalisation, at Ns = 57 (the largest gap between states 31 and 60 of
    the converged Hamiltonian; the filter cut sits in it): the method
    converges to the same fixed point (7.5e-13 in rho L1/Ne, 6e-14 Ha/atom
    in F measured)."""
    from oracle import hamiltonian
    n, L, Ns = 12, inputs.A0_FCC, 57
    pos = inputs.fcc_positions(1, disp_sigma=0.05, seed=0)
    sigma, Z, rc = inputs.ev_to_ha(10.0), inputs.Z_VALENCE, inputs.RC_LOCAL
    dV = (L / n) ** 3
    ref = scf.scf(n, L, pos, Ns=Ns, sigma=sigma, Z=Z, rc=rc, tol=1e-11)
    lam = np.linalg.eigvalsh(hamiltonian.hamiltonian_dense(n, L, ref["veff"]))
    filt = (0.5 * (lam[Ns - 1] + lam[Ns]), 1.5 * 7.0729 / (L / n) ** 2 + 10.0, lam[0] - 0.5)
    X0 = inputs.random_block(n ** 3, Ns, seed=0).T
    got = scf.scf_sq3(n, L, pos, X0, sigma, Z, rc, filt, npl=80)
    assert np.sum(np.abs(got["rho"] - ref["rho"])) * dV / 12.0 < 1e-10
    assert abs(got["F"] - ref["F"]) / 4 < 1e-10
    assert abs(got["mu"] - ref["mu"]) < 1e-10


def test_scf_in_the_papers_order_rejects_a_filter_bound_below_the_spectrum():
    """An upper filter bound below the top of H's spectrum (here the FD
    kinetic maximum alone is 24 Ha at 12^3) is caught at the first
    iteration instead of letting the filter amplify the top states."""
    n, L, Ns = 12, inputs.A0_FCC, 20
    pos = inputs.fcc_positions(1, disp_sigma=0.05, seed=0)
    X0 = inputs.random_block(n ** 3, Ns, seed=0).T
    with pytest.raises(ValueError, match="below the spectrum"):
        scf.scf_sq3(n, L, pos, X0, inputs.ev_to_ha(10.0), inputs.Z_VALENCE, inputs.RC_LOCAL,
                    (1.0, 5.0, -2.0), npl=40, max_iter=2)
