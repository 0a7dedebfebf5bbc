"""GPU parity of the plain-FP64 path against the CPU oracle, through the C ABI.

Tolerances: the FP64 path must reproduce the oracle's rho to 1e-10 relative
L2 and the energies to 1e-10 Ha/atom end to end; the single steps are held to
1e-12..1e-13 relative (they differ from the oracle only in summation order).
"""
import numpy as np
import pytest
import torch
from scipy.stats import ortho_group

from oracle import chebyshev, fermi, hamiltonian, subspace
from paper_2112_08639_gb300 import inputs

from gpu_common import (apply_fn, c1_cell, c1_eigs, context_for, from_gpu_block,
                        need_gpu, oracle_parts, small_proj_cell, sq3, to_gpu_block)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("cellf,Ns", [(c1_cell, 7), (c1_cell, 64), (small_proj_cell, 13)])
def test_hamiltonian_apply(cellf, Ns):
    cell = cellf()
    ctx = context_for(cell)
    X = inputs.random_block(cell.cfg.N, Ns, seed=2).T
    Y = ctx.hamiltonian_apply(to_gpu_block(X))
    ref = hamiltonian.apply(oracle_parts(cell), X)
    assert _rel(from_gpu_block(Y), ref) < 1e-14


@pytest.mark.parametrize("fd_order", [2, 8])
def test_hamiltonian_apply_lower_orders(fd_order):
    cell = c1_cell()
    ctx = context_for(cell, fd_order)
    X = inputs.random_block(cell.cfg.N, 5, seed=4).T
    Y = ctx.hamiltonian_apply(to_gpu_block(X))
    parts = hamiltonian.hamiltonian_sparse(cell.cfg.n, cell.cfg.L, cell.V, None, fd_order)
    assert _rel(from_gpu_block(Y), hamiltonian.apply(parts, X)) < 1e-14


@pytest.mark.parametrize("cellf,Ns,m", [(c1_cell, 16, 20), (c1_cell, 3, 1),
                                        (small_proj_cell, 12, 16), (small_proj_cell, 9, 7)])
def test_chebyshev_filter(cellf, Ns, m):
    cell = cellf()
    ctx = context_for(cell)
    X = inputs.random_block(cell.cfg.N, Ns, seed=5).T
    a0, a, b = -1.8, 2.0, 60.0
    Xg = to_gpu_block(X)
    ctx.cheb_filter(Xg, m, a, b, a0)
    ref = chebyshev.filter_plain(apply_fn(oracle_parts(cell)), X, m, a, b, a0)
    assert _rel(from_gpu_block(Xg), ref) < 1e-13


@pytest.mark.parametrize("Ns", [1, 40, 67, 130])
def test_orthonormalise(Ns):
    cell = c1_cell()
    ctx = context_for(cell)
    rng = np.random.default_rng(Ns)
    X = rng.normal(size=(cell.cfg.N, Ns)) @ np.diag(np.logspace(0, 2, Ns))
    Xg = to_gpu_block(X)
    ctx.orthonormalise(Xg)
    got = from_gpu_block(Xg)
    ref = subspace.cholqr(X)
    assert np.max(np.abs(got - ref)) < 1e-11
    assert np.max(np.abs(got.T @ got - np.eye(Ns))) < 1e-12


def test_orthonormalise_reports_rank_deficiency():
    cell = c1_cell()
    ctx = context_for(cell)
    X = inputs.random_block(cell.cfg.N, 6, seed=1).T.copy()
    X[:, 3] = X[:, 1]
    with pytest.raises(sq3().SQ3Error) as e:
        ctx.orthonormalise(to_gpu_block(X))
    assert e.value.code == sq3().ENOTPD
    # the context stays usable afterwards
    Y = to_gpu_block(inputs.random_block(cell.cfg.N, 6, seed=2).T)
    ctx.orthonormalise(Y)


@pytest.mark.parametrize("cellf,Ns", [(c1_cell, 64), (small_proj_cell, 21)])
def test_project(cellf, Ns):
    cell = cellf()
    ctx = context_for(cell)
    X = subspace.cholqr(inputs.random_block(cell.cfg.N, Ns, seed=6).T)
    Hs = ctx.project(to_gpu_block(X)).cpu().numpy()
    ref = subspace.project(apply_fn(oracle_parts(cell)), X)
    assert np.max(np.abs(Hs - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(Hs, Hs.T)


def _random_hs(Ns, seed, lo=-0.6, hi=2.0):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(lo, hi, Ns))
    Q = ortho_group.rvs(Ns, random_state=seed)
    return (Q * lam) @ Q.T


@pytest.mark.parametrize("Ns,npl", [(64, 60), (75, 11), (130, 25), (5, 3)])
def test_kernel_from_hs_given_bounds_matches_foe_oracle(Ns, npl):
    """With the oracle's exact chi, xi passed in, the GPU's recurrence,
    moments, Fermi level, coefficients and sums reproduce the oracle's
    Chebyshev expansion, including its truncation error at low npl."""
    sigma = inputs.ev_to_ha(10.0)
    Ne = min(12.0, 1.2 * Ns)
    Hs = _random_hs(Ns, seed=Ns)
    chi, xi = subspace.exact_bounds(Hs)
    ref = chebyshev.foe_density_kernel(Hs, npl, sigma, Ne, chi, xi)
    ctx = context_for(c1_cell())
    D, out = ctx.kernel_from_hs(torch.from_numpy(Hs).cuda(), npl, sigma, Ne, bounds=(chi, xi))
    D = D.cpu().numpy()
    assert np.max(np.abs(D - ref["D"])) < 1e-12
    assert abs(out["mu"] - ref["mu"]) < 1e-11
    assert abs(out["e_band"] - ref["e_band"]) < 1e-11
    assert abs(out["e_ent"] - ref["e_ent"]) < 1e-11
    assert abs(out["two_tr_D"] - Ne) < 1e-11
    assert abs(2 * np.trace(D) - Ne) < 1e-10


def test_kernel_from_hs_lanczos_bounds_matches_diagonalisation():
    """With bounds estimated on the GPU (Lanczos), npl = 80 reaches g(Hs)."""
    sigma = inputs.ev_to_ha(10.0)
    Hs = _random_hs(64, seed=9)
    ref = subspace.kernel_by_diagonalisation(Hs, 12.0, sigma)
    lam = np.linalg.eigvalsh(Hs)
    ctx = context_for(c1_cell())
    D, out = ctx.kernel_from_hs(torch.from_numpy(Hs).cuda(), 80, sigma, 12.0)
    assert out["chi"] - out["xi"] <= lam[0] + 1e-12
    assert out["chi"] + out["xi"] >= lam[-1] - 1e-12
    assert np.max(np.abs(D.cpu().numpy() - ref["D"])) < 1e-11
    assert abs(out["mu"] - ref["mu"]) < 1e-10
    assert abs(out["e_band"] - ref["e_band"]) < 1e-10
    assert abs(out["e_ent"] - ref["e_ent"]) < 1e-10


def test_kernel_rejects_bad_arguments():
    ctx = context_for(c1_cell())
    Hs = torch.eye(4, dtype=torch.float64, device="cuda")
    with pytest.raises(sq3().SQ3Error) as e:
        ctx.kernel_from_hs(Hs, 10, 0.3, 8.0)          # Ne >= 2 Ns
    assert e.value.code == sq3().EINVAL


@pytest.mark.parametrize("Ns", [1, 64, 67])
def test_density(Ns):
    cell = c1_cell()
    ctx = context_for(cell)
    X = subspace.cholqr(inputs.random_block(cell.cfg.N, Ns, seed=7).T)
    rng = np.random.default_rng(Ns)
    D = rng.normal(size=(Ns, Ns))
    D = 0.5 * (D + D.T)
    rho = ctx.density(to_gpu_block(X), torch.from_numpy(D).cuda()).cpu().numpy()
    ref = subspace.density_from_kernel(X, D, cell.cfg.dV)
    assert _rel(rho, ref) < 1e-13


def test_kernel_and_density_on_exact_subspace_match_diagonalisation():
    """X = U Q spans the oracle's Ns lowest eigenvectors of the C1 cell; the
    GPU projection, density kernel and density reproduce the exact
    Ns-truncated Fermi density (rho rel-L2 <= 1e-10, energies <= 1e-10
    Ha/atom)."""
    cell = c1_cell()
    cfg = cell.cfg
    lam, U = c1_eigs()
    Ns = cfg.Ns
    ref = fermi.ks_fixed_potential(lam[:Ns], U[:, :Ns], cfg.Ne, cfg.sigma, cfg.dV)
    X = U[:, :Ns] @ ortho_group.rvs(Ns, random_state=1)
    ctx = context_for(cell)
    Xg = to_gpu_block(X)
    D, out = ctx.density_kernel(Xg, cfg.npl, cfg.sigma, cfg.Ne)
    rho = ctx.density(Xg, D).cpu().numpy()
    assert _rel(rho, ref["rho"]) < 1e-10
    assert abs(out["e_band"] - ref["e_band"]) / cfg.natoms < 1e-10
    assert abs(out["e_ent"] - ref["e_ent"]) / cfg.natoms < 1e-10
    assert abs(out["mu"] - ref["mu"]) < 1e-10
    assert abs(rho.sum() * cfg.dV - cfg.Ne) < 1e-10


@pytest.mark.parametrize("Ns", [57, 81])
def test_end_to_end_from_random_block(Ns):
    """Filter + CholQR from the seeded random X0 at a gap-aligned Ns of the
    C1 cell converge to the exact result (P9)."""
    cell = c1_cell()
    cfg = cell.cfg
    lam, U = c1_eigs()
    ref = fermi.ks_fixed_potential(lam[:Ns], U[:, :Ns], cfg.Ne, cfg.sigma, cfg.dV)
    ctx = context_for(cell)
    X = to_gpu_block(inputs.random_block(cfg.N, Ns, seed=0).T)
    a = 0.5 * (lam[Ns - 1] + lam[Ns])
    b = 1.5 * 7.0729 / cfg.h ** 2 + 1.0          # above the FD kinetic maximum
    for _ in range(40):
        ctx.cheb_filter(X, cfg.m, a, b, lam[0])
        ctx.orthonormalise(X)
    D, out = ctx.density_kernel(X, cfg.npl, cfg.sigma, cfg.Ne)
    rho = ctx.density(X, D).cpu().numpy()
    assert _rel(rho, ref["rho"]) < 1e-10
    assert abs(out["e_band"] - ref["e_band"]) / cfg.natoms < 1e-10
    assert abs(out["e_ent"] - ref["e_ent"]) / cfg.natoms < 1e-10


def test_errors_before_setup():
    m = sq3()
    ctx = m.Context(0)
    X = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(m.SQ3Error) as e:
        ctx.cheb_filter(X, 3, 1.0, 2.0, 0.0)
    assert e.value.code == m.ENOTSETUP
