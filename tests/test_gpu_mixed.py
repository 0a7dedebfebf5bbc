"""GPU parity of the mixed-precision path (FP32 block, BF16-split tcgen05
GEMMs with FP32 accumulation, FP64 Cholesky fallback, Fermi level and energies).

Single steps are compared with the FP64 oracle on the same inputs at
tolerances set by FP32 storage (2^-24 ~ 6e-8 per element) times the
operation's growth; the end-to-end mixed result is compared with the FP64
GPU path at the stated target: rho L1/Ne <= 1e-5 and energies <= 1e-5
Ha/atom.
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


def _f32(X):
    return X.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("cellf,Ns", [(c1_cell, 9), (small_proj_cell, 13)])
def test_hamiltonian_apply_fp32(cellf, Ns):
    cell = cellf()
    ctx = context_for(cell)
    X = _f32(inputs.random_block(cell.cfg.N, Ns, seed=3).T)
    Y = ctx.hamiltonian_apply(to_gpu_block(X, torch.float32), prec=sq3().MIXED)
    ref = hamiltonian.apply(oracle_parts(cell), X)
    assert _rel(from_gpu_block(Y), ref) < 1e-6


@pytest.mark.parametrize("cellf,Ns,m", [(c1_cell, 16, 20), (small_proj_cell, 12, 16)])
def test_chebyshev_filter_fp32(cellf, Ns, m):
    cell = cellf()
    ctx = context_for(cell)
    X = _f32(inputs.random_block(cell.cfg.N, Ns, seed=5).T)
    a0, a, b = -1.8, 2.0, 60.0
    Xg = to_gpu_block(X, torch.float32)
    ctx.cheb_filter(Xg, m, a, b, a0, prec=sq3().MIXED)
    ref = chebyshev.filter_plain(apply_fn(oracle_parts(cell)), X, m, a, b, a0)
    assert _rel(from_gpu_block(Xg), ref) < 1e-5


@pytest.mark.parametrize("cellf,Ns", [(c1_cell, 64), (c1_cell, 130), (small_proj_cell, 21),
                                      (c1_cell, 5)])
def test_project_tensor_core(cellf, Ns):
    """Hs = X^T (H X): FP32 stencil plus the split-K tcgen05 Gram (FP64
    atomics, upper tiles mirrored)."""
    cell = cellf()
    ctx = context_for(cell)
    X = _f32(subspace.cholqr(inputs.random_block(cell.cfg.N, Ns, seed=6).T))
    Hs = ctx.project(to_gpu_block(X, torch.float32), prec=sq3().MIXED).cpu().numpy()
    ref = subspace.project(apply_fn(oracle_parts(cell)), X)
    assert np.max(np.abs(Hs - ref)) < 2e-6 * np.max(np.abs(ref))
    assert np.array_equal(Hs, Hs.T)


@pytest.mark.parametrize("Ns", [1, 64, 67, 200])
def test_density_tensor_core(Ns):
    """rho = (2/dV) rowdot(X, X D) with X D on the tensor cores (ragged Ns,
    several 128-row tiles of the grid)."""
    cell = c1_cell()
    ctx = context_for(cell)
    X = _f32(subspace.cholqr(inputs.random_block(cell.cfg.N, Ns, seed=7).T))
    rng = np.random.default_rng(Ns)
    D = rng.normal(size=(Ns, Ns))
    D = 0.5 * (D + D.T)
    rho = ctx.density(to_gpu_block(X, torch.float32), torch.from_numpy(D).cuda(),
                      prec=sq3().MIXED).cpu().numpy()
    ref = subspace.density_from_kernel(X, D, cell.cfg.dV)
    assert _rel(rho, ref) < 2e-6


@pytest.mark.parametrize("Ns,cond", [(40, 1e1), (67, 1e3), (130, 1e4)])
def test_orthonormalise_mixed(Ns, cond):
    """Cholesky QR 2 (shifted when needed) on blocks of growing condition
    number: the result is orthonormal and spans the input's column space."""
    cell = c1_cell()
    ctx = context_for(cell)
    rng = np.random.default_rng(Ns)
    Q0 = subspace.cholqr(rng.normal(size=(cell.cfg.N, Ns)))
    X = _f32(Q0 @ np.diag(np.logspace(0, np.log10(cond), Ns)) @ ortho_group.rvs(Ns, random_state=1))
    Xg = to_gpu_block(X, torch.float32)
    ctx.orthonormalise(Xg, prec=sq3().MIXED)
    got = from_gpu_block(Xg)
    assert np.max(np.abs(got.T @ got - np.eye(Ns))) < 1e-5
    # same column space: the projector onto span(got) reproduces Q0
    resid = Q0 - got @ (got.T @ Q0)
    assert np.max(np.abs(resid)) < 1e-5 * cond


@pytest.mark.parametrize("Ns,cond", [(40, 1.0), (300, 1.0), (40, 3.0), (300, 10.0),
                                     (130, 1e2)])
def test_orthonormalise_mixed_matches_the_oracle_q(Ns, cond):
    """The orthonormal factor of a full-rank block is unique (Q = X R^-1 with
    R upper triangular, positive diagonal), so the mixed Cholesky QR 2 must
    reproduce the FP64 oracle's Q of the same FP32 input elementwise, to
    FP32 accuracy times the condition number.  Inputs from orthonormal (the
    last pass then corrects X by one BF16 piece of R^-1 - I) to cond 1e2
    (two pieces or the full product); Ns = 300 spans three tiles and a
    ragged one."""
    cell = c1_cell()
    ctx = context_for(cell)
    rng = np.random.default_rng(Ns + int(cond))
    Q0 = subspace.cholqr(rng.normal(size=(cell.cfg.N, Ns)))
    X = _f32(Q0 @ np.diag(np.logspace(0, np.log10(cond), Ns)) @ ortho_group.rvs(Ns, random_state=2)
             if cond > 1.0 else Q0)
    ref = subspace.cholqr(X)
    Xg = to_gpu_block(X, torch.float32)
    ctx.orthonormalise(Xg, prec=sq3().MIXED)
    got = from_gpu_block(Xg)
    assert np.max(np.abs(got.T @ got - np.eye(Ns))) < 2e-6
    assert np.max(np.abs(got - ref)) < 2e-6 * cond * np.max(np.abs(ref))


@pytest.mark.parametrize("Ns,npl", [(64, 60), (130, 25)])
def test_kernel_from_hs_mixed(Ns, npl):
    """The recurrence on the tensor cores (FP32 T_j, BF16-split products)
    against the FP64 oracle expansion with the same bounds."""
    sigma = inputs.ev_to_ha(10.0)
    Ne = 12.0
    rng = np.random.default_rng(Ns)
    lam = np.sort(rng.uniform(-0.6, 2.0, Ns))
    Q = ortho_group.rvs(Ns, random_state=Ns)
    Hs = (Q * lam) @ Q.T
    chi, xi = subspace.exact_bounds(Hs)
    ref = chebyshev.foe_density_kernel(Hs, npl, sigma, Ne, chi, xi)
    ctx = context_for(c1_cell())
    D, out = ctx.kernel_from_hs(torch.from_numpy(Hs).cuda(), npl, sigma, Ne, bounds=(chi, xi),
                                prec=sq3().MIXED)
    assert np.max(np.abs(D.cpu().numpy() - ref["D"])) < 2e-5
    assert abs(out["mu"] - ref["mu"]) < 1e-5
    assert abs(out["e_band"] - ref["e_band"]) < 1e-4
    assert abs(out["e_ent"] - ref["e_ent"]) < 1e-4
    assert abs(out["two_tr_D"] - Ne) < 1e-9


def test_mixed_matches_fp64_end_to_end():
    """Same seeded start, same filter bounds, a few SQ3 iterations in each
    precision on the C1 cell: rho L1/Ne <= 1e-5, energies <= 1e-5 Ha/atom."""
    cell = c1_cell()
    cfg = cell.cfg
    lam, U = c1_eigs()
    m = sq3()
    ctx64, ctx32 = context_for(cell), context_for(cell)
    X0 = inputs.random_block(cfg.N, cfg.Ns, seed=0)
    X64 = torch.from_numpy(X0).cuda()
    X32 = torch.from_numpy(X0).cuda().float()
    b = 1.5 * 7.0729 / cfg.h ** 2 + 1.0
    a0, a = lam[0] - 0.1, lam[cfg.Ns - 1] + 0.05
    for it in range(8):
        ctx64.cheb_filter(X64, cfg.m, a, b, a0)
        ctx64.orthonormalise(X64)
        ctx32.cheb_filter(X32, cfg.m, a, b, a0, prec=m.MIXED)
        ctx32.orthonormalise(X32, prec=m.MIXED)
    D64, o64 = ctx64.density_kernel(X64, cfg.npl, cfg.sigma, cfg.Ne)
    D32, o32 = ctx32.density_kernel(X32, cfg.npl, cfg.sigma, cfg.Ne, prec=m.MIXED)
    r64 = ctx64.density(X64, D64).cpu().numpy()
    r32 = ctx32.density(X32, D32, prec=m.MIXED).cpu().numpy()
    l1 = np.sum(np.abs(r32 - r64)) * cfg.dV / cfg.Ne
    assert l1 < 1e-5, l1
    assert abs(o32["e_band"] - o64["e_band"]) / cfg.natoms < 1e-5
    assert abs(o32["e_ent"] - o64["e_ent"]) / cfg.natoms < 1e-5
