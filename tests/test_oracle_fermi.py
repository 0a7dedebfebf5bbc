"""Pins for the oracle's occupations, Fermi level, density and energies
(Sec. 2: Eq. (TraceD), (rhoDensMat), (ON:FreeEnergy); Sec. 3: Eq.
(SubspaceRotation), (traceDs), (density:NewForm))."""
import numpy as np
import pytest
from scipy.stats import ortho_group

from oracle import fermi, hamiltonian, subspace
from paper_2112_08639_gb300 import inputs


def test_fermi_values_and_symmetry():
    assert fermi.fermi(0.3, 0.3, 0.1) == 0.5
    x = np.linspace(-50, 50, 101)
    g = fermi.fermi(x, 0.0, 1.0)
    np.testing.assert_allclose(g + fermi.fermi(-x, 0.0, 1.0), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g[60], 1.0 / (1.0 + np.exp(10.0)), rtol=1e-15)
    assert fermi.fermi(1e4, 0.0, 1.0) == 0.0 and fermi.fermi(-1e4, 0.0, 1.0) == 1.0


def test_entropy_density_against_naive_formula_and_limits():
    x = np.linspace(-8, 8, 81)
    g = 1.0 / (1.0 + np.exp(x))
    naive = g * np.log(g) + (1 - g) * np.log1p(-g)
    np.testing.assert_allclose(fermi.entropy_density(x, 0.0, 1.0), naive, rtol=1e-9, atol=1e-15)
    # g ln g + (1-g) ln(1-g) is even in x.
    xs = np.linspace(-40, 40, 161)
    np.testing.assert_allclose(fermi.entropy_density(xs, 0.0, 1.0),
                               fermi.entropy_density(-xs, 0.0, 1.0), rtol=1e-12, atol=1e-300)
    assert abs(fermi.entropy_density(0.0, 0.0, 1.0) + np.log(2.0)) < 1e-15
    assert abs(fermi.entropy_density(800.0, 0.0, 1.0)) < 1e-300
    assert abs(fermi.entropy_density(-800.0, 0.0, 1.0)) < 1e-300


def test_two_level_fermi_level_closed_form():
    # Two states, two electrons: g1 + g2 = 1 forces mu = midpoint.
    mu = fermi.fermi_level([0.2, 1.4], 2.0, 0.37)
    assert abs(mu - 0.8) < 1e-14


def test_fermi_level_count_and_errors():
    rng = np.random.default_rng(0)
    lam = np.sort(rng.uniform(-2, 5, 40))
    for Ne in (1.0, 12.0, 79.0):
        mu = fermi.fermi_level(lam, Ne, 0.3)
        assert abs(2 * fermi.fermi(lam, mu, 0.3).sum() - Ne) < 1e-12 * Ne
    with pytest.raises(ValueError):
        fermi.fermi_level(lam, 80.0, 0.3)


def _small_problem(n=8, L=6.0, seed=1, with_proj=False):
    pos = inputs.fcc_positions(1, a0=L, disp_sigma=0.05, seed=seed)
    V = inputs.local_potential(n, L, pos)
    proj = inputs.projectors(n, L, pos, seed=seed, rcut=2.0) if with_proj else None
    return n, L, V, proj


def test_density_integrates_to_ne_and_energy_trace():
    n, L, V, proj = _small_problem(with_proj=True)
    H = hamiltonian.hamiltonian_dense(n, L, V, proj)
    dV = (L / n) ** 3
    lam, U = fermi.lowest_eigenpairs(H, 30)
    r = fermi.ks_fixed_potential(lam, U, 12.0, 0.3675, dV)
    assert abs(r["rho"].sum() * dV - 12.0) < 1e-11
    # E_band = 2 Tr(D H) with D = U diag(g) U^T
    D = (U * r["g"]) @ U.T
    assert abs(2 * np.sum(D * H) - r["e_band"]) < 1e-10 * abs(r["e_band"])
    assert r["e_ent"] < 0


def test_constant_potential_shift():
    """Brute force: V -> V + v0 shifts every eigenvalue and mu by v0, leaves
    rho and E_ent unchanged and shifts E_band by Ne v0."""
    n, L, V, _ = _small_problem(n=6)
    dV = (L / n) ** 3
    a = fermi.ks_fixed_potential(*fermi.lowest_eigenpairs(hamiltonian.hamiltonian_dense(n, L, V), 20), 12.0, 0.4, dV)
    b = fermi.ks_fixed_potential(*fermi.lowest_eigenpairs(hamiltonian.hamiltonian_dense(n, L, V + 0.7), 20), 12.0, 0.4, dV)
    np.testing.assert_allclose(b["lam"], a["lam"] + 0.7, atol=1e-11)
    assert abs(b["mu"] - a["mu"] - 0.7) < 1e-11
    np.testing.assert_allclose(b["rho"], a["rho"], atol=1e-9 * a["rho"].max())
    assert abs(b["e_band"] - a["e_band"] - 12.0 * 0.7) < 1e-10
    assert abs(b["e_ent"] - a["e_ent"]) < 1e-11


def test_rank_one_projector_interlacing():
    """Adding gamma c c^T (gamma > 0) raises eigenvalues but not past the
    next unperturbed one (Cauchy interlacing for a rank-1 update)."""
    n, L, V, proj = _small_problem(n=6, with_proj=True)
    one = inputs.ProjectorTable(proj.ptr[:2].copy(), proj.idx[:proj.ptr[1]].copy(),
                                proj.val[:proj.ptr[1]].copy(), proj.gamma[:1].copy())
    l0 = np.linalg.eigvalsh(hamiltonian.hamiltonian_dense(n, L, V))
    l1 = np.linalg.eigvalsh(hamiltonian.hamiltonian_dense(n, L, V, one))
    assert np.all(l1 >= l0 - 1e-12)
    assert np.all(l1[:-1] <= l0[1:] + 1e-12)
    dV = (L / n) ** 3
    c = np.zeros(n ** 3)
    c[one.idx] = one.val * np.sqrt(dV)
    assert abs(np.linalg.norm(c) - 1.0) < 1e-12        # unit-norm projector
    assert abs(l1.sum() - l0.sum() - one.gamma[0]) < 1e-9   # trace shift


def test_subspace_invariance():
    """rho and energies from U equal those from the rotated basis X = U Q
    with kernel Ds = Q^T diag(g) Q (Eq. (SubspaceRotation), (traceDs),
    (density:NewForm))."""
    n, L, V, _ = _small_problem(n=7)
    dV = (L / n) ** 3
    lam, U = fermi.lowest_eigenpairs(hamiltonian.hamiltonian_dense(n, L, V), 25)
    r = fermi.ks_fixed_potential(lam, U, 12.0, 0.3675, dV)
    Q = ortho_group.rvs(25, random_state=4)
    X = U @ Q
    Ds = Q.T @ np.diag(r["g"]) @ Q
    np.testing.assert_allclose(subspace.density_from_kernel(X, Ds, dV), r["rho"],
                               atol=1e-12 * r["rho"].max())
    assert abs(2 * np.trace(Ds) - 12.0) < 1e-12
    Hs = Q.T @ np.diag(lam) @ Q
    k = subspace.kernel_by_diagonalisation(Hs, 12.0, 0.3675)
    np.testing.assert_allclose(k["D"], Ds, atol=1e-12)
    assert abs(k["mu"] - r["mu"]) < 1e-12
