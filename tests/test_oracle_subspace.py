"""Pins for the oracle's auxiliary-basis steps (Sec. 4: filter,
orthonormalisation, projection; Sec. 3: Eq. (DsHsRelation),
(phi_tilde), (density:NewForm)) and for one end-to-end fixed-potential SQ3
iteration against exact diagonalisation."""
import numpy as np

from oracle import chebyshev, fermi, hamiltonian, subspace
from paper_2112_08639_gb300 import inputs


def test_cholqr_equals_qr_with_positive_diagonal():
    X = np.random.default_rng(0).normal(size=(300, 20)) @ np.diag(np.logspace(0, 3, 20))
    Q = subspace.cholqr(X)
    Qr, R = np.linalg.qr(X)
    Qr = Qr * np.sign(np.diag(R))
    np.testing.assert_allclose(Q, Qr, atol=1e-10)
    np.testing.assert_allclose(Q.T @ Q, np.eye(20), atol=1e-12)


def test_project_on_eigenvectors_is_diagonal():
    n, L = 6, 4.5
    pos = inputs.fcc_positions(1, a0=L, seed=2)
    V = inputs.local_potential(n, L, pos)
    H = hamiltonian.hamiltonian_dense(n, L, V)
    lam, U = np.linalg.eigh(H)
    parts = hamiltonian.hamiltonian_sparse(n, L, V)
    Hs = subspace.project(lambda X: hamiltonian.apply(parts, X), U[:, :15])
    np.testing.assert_allclose(Hs, np.diag(lam[:15]), atol=1e-11)


def test_end_to_end_fixed_potential_iteration_converges_to_diagonalisation():
    """Repeated filter + CholQR + projection + Chebyshev kernel (the paper's
    steps) reproduce the diagonalisation result when Ns sits at a spectral
    gap: rho to 1e-10 relative L2, energies to 1e-10 Ha/atom."""
    n, L, Ns, Ne, npl = 8, 5.0, 20, 8.0, 80
    sigma = 10.0 / 27.211386245988
    pos = inputs.fcc_positions(1, a0=L, seed=4)
    V = inputs.local_potential(n, L, pos)
    proj = inputs.projectors(n, L, pos, seed=4, rcut=2.0)
    dV = (L / n) ** 3
    H = hamiltonian.hamiltonian_dense(n, L, V, proj)
    lam_all, U_all = np.linalg.eigh(H)
    gaps = np.diff(lam_all[:40])
    Ns = int(np.argmax(gaps[10:30]) + 11)          # largest gap above 10 states
    ref = fermi.ks_fixed_potential(lam_all[:Ns], U_all[:, :Ns], Ne, sigma, dV)
    parts = hamiltonian.hamiltonian_sparse(n, L, V, proj)
    apply_H = lambda X: hamiltonian.apply(parts, X)
    a = 0.5 * (lam_all[Ns - 1] + lam_all[Ns])
    b = lam_all[-1] * 1.01
    X = inputs.random_block(n ** 3, Ns, seed=1).T
    for _ in range(40):
        out = subspace.sq3_iteration(apply_H, X, 16, a, b, lam_all[0], npl, sigma, Ne, dV)
        X = out["X"]
    err = np.linalg.norm(out["rho"] - ref["rho"]) / np.linalg.norm(ref["rho"])
    assert err < 1e-10
    assert abs(out["e_band"] - ref["e_band"]) / 4 < 1e-10
    assert abs(out["e_ent"] - ref["e_ent"]) / 4 < 1e-10
    assert abs(out["mu"] - ref["mu"]) < 1e-10
    assert abs(out["rho"].sum() * dV - Ne) < 1e-10
