"""GPU parity at the full 108-atom size (72^3 grid, Ns = 2200, the bench's
workload and launch configuration), mixed precision, on sampled outputs the
FP64 oracle computes one by one: filtered columns, pairs of the
orthonormalised block, entries of Hs, grid points of rho, and the density
kernel of a 2200 x 2200 Hs of known spectrum against the Chebyshev series
evaluated on that spectrum.

Tolerances: FP32 storage (6e-8 per element) times the growth of each step;
the filter's columns are compared relative to their norm (1e-5, the same as
the small-grid filter test), orthonormality and Hs to 2e-6 of their scale,
rho to 2e-6 relative, Ds to 2e-5 absolute (as for Ns = 64, 130)."""
import functools

import numpy as np
import pytest
import torch

from oracle import chebyshev, hamiltonian
from paper_2112_08639_gb300 import inputs

from gpu_common import context_for, need_gpu, sq3

pytestmark = pytest.mark.gpu

SAMPLE_COLS = (0, 1099, 2199)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@functools.lru_cache(maxsize=None)
def c3():
    cell = inputs.make_cell(inputs.C3)
    parts = hamiltonian.hamiltonian_sparse(cell.cfg.n, cell.cfg.L, cell.V, cell.proj)
    return cell, parts


def filter_bounds(cell):
    # the bench's first-iteration interval (kinetic maximum + potential +
    # projector range as b, the lowest 5 % of [V_min - 1, b] as the kept part)
    cfg = cell.cfg
    b = 0.5 * 3 * 7.0729 / cfg.h ** 2 + float(cell.V.max()) + 4 * float(np.max(cell.proj.gamma))
    a0 = float(cell.V.min()) - 1.0
    return a0, a0 + 0.05 * (b - a0), b


@pytest.fixture(scope="module")
def filtered():
    need_gpu()
    cell, parts = c3()
    cfg = cell.cfg
    ctx = context_for(cell)
    X = inputs.random_block_device(cfg.N, cfg.Ns, seed=11)
    X0 = X[list(SAMPLE_COLS)].double().cpu().numpy().T          # (N, 3)
    a0, a, b = filter_bounds(cell)
    ctx.cheb_filter(X, cfg.m, a, b, a0, prec=sq3().MIXED)
    torch.cuda.synchronize()
    return ctx, X, X0, (a0, a, b)


def test_filter_fullsize_sampled_columns(filtered):
    ctx, X, X0, (a0, a, b) = filtered
    cell, parts = c3()
    ref = chebyshev.filter_plain(lambda Z: hamiltonian.apply(parts, Z), X0, cell.cfg.m, a, b, a0)
    got = X[list(SAMPLE_COLS)].double().cpu().numpy().T
    for j in range(len(SAMPLE_COLS)):
        err = np.linalg.norm(got[:, j] - ref[:, j]) / np.linalg.norm(ref[:, j])
        assert err < 1e-5, (SAMPLE_COLS[j], err)


@pytest.fixture(scope="module")
def orthonormal(filtered):
    ctx, X, _, _ = filtered
    Q = X.clone()
    ctx.orthonormalise(Q, prec=sq3().MIXED)
    torch.cuda.synchronize()
    return ctx, Q


def test_orthonormalise_fullsize_sampled_pairs(orthonormal):
    _, Q = orthonormal
    rng = np.random.default_rng(3)
    cols = np.unique(np.concatenate([rng.integers(0, Q.shape[0], 40), [0, Q.shape[0] - 1]]))
    C = Q[torch.from_numpy(cols).cuda()].double().cpu().numpy()   # (k, N)
    G = C @ C.T
    assert np.max(np.abs(G - np.eye(len(cols)))) < 2e-6


def test_project_fullsize_sampled_entries(orthonormal):
    ctx, Q = orthonormal
    cell, parts = c3()
    Hs = ctx.project(Q, prec=sq3().MIXED).cpu().numpy()
    rng = np.random.default_rng(4)
    cols = np.unique(rng.integers(0, Q.shape[0], 6))
    C = Q[torch.from_numpy(cols).cuda()].double().cpu().numpy().T   # (N, k)
    ref = C.T @ hamiltonian.apply(parts, C)
    got = Hs[np.ix_(cols, cols)]
    assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(Hs))
    assert np.array_equal(Hs, Hs.T)


def test_density_fullsize_sampled_points(orthonormal):
    ctx, Q = orthonormal
    cell, _ = c3()
    Ns = Q.shape[0]
    rng = np.random.default_rng(5)
    D = rng.normal(size=(Ns, Ns)) / Ns
    D = 0.5 * (D + D.T)
    rho = ctx.density(Q, torch.from_numpy(D).cuda(), prec=sq3().MIXED).cpu().numpy()
    pts = rng.integers(0, cell.cfg.N, 300)
    Xk = Q[:, torch.from_numpy(pts).cuda()].double().cpu().numpy()   # (Ns, k)
    ref = (2.0 / cell.cfg.dV) * np.einsum("ik,ij,jk->k", Xk, D, Xk)
    assert np.max(np.abs(rho[pts] - ref)) < 2e-6 * np.max(np.abs(ref))


def test_kernel_fullsize_known_spectrum():
    """Ns = 2200, n_pl = 120: mu against the oracle's Fermi level of the
    same expansion on the known eigenvalues (1e-6 Ha), D against
    sum'_j c_j(mu) T_j evaluated there (the exact value of the expansion),
    2 tr D = Ne."""
    cell, _ = c3()
    cfg = cell.cfg
    Ns = cfg.Ns
    rng = np.random.default_rng(7)
    lam = np.sort(rng.uniform(-0.4, 1.6, Ns))
    Q, _ = np.linalg.qr(rng.normal(size=(Ns, Ns)))
    Hs = (Q * lam) @ Q.T
    Hs = 0.5 * (Hs + Hs.T)
    chi, xi = 0.6, 1.05
    Ne = float(cfg.Ne)
    ctx = context_for(inputs.make_cell(inputs.C1))
    D, out = ctx.kernel_from_hs(torch.from_numpy(Hs).cuda(), cfg.npl, cfg.sigma, Ne,
                                bounds=(chi, xi), prec=sq3().MIXED)
    # the Fermi level of the same expansion, independent of the GPU: the
    # moments m_j = sum_n T_j(x_n) of the known spectrum and the oracle's
    # bisection on Eq. (FermiLevelCalc)
    x = (lam - chi) / xi
    moments = np.array([np.sum(chebyshev.cheb_T(j, x)) for j in range(cfg.npl + 1)])
    mu_ref = chebyshev.fermi_level_series(moments, cfg.sigma, Ne, chi, xi)
    assert abs(out["mu"] - mu_ref) < 1e-6
    c, _, _ = chebyshev.fermi_coeffs(mu_ref, cfg.sigma, chi, xi, cfg.npl)
    g = chebyshev.series_scalar(c, x)
    Dref = (Q * g) @ Q.T
    assert np.max(np.abs(D.cpu().numpy() - Dref)) < 2e-5
    assert abs(2.0 * np.sum(g) - Ne) < 1e-9 * Ne
    assert abs(out["two_tr_D"] - Ne) < 1e-6 * Ne
