"""Hellmann-Feynman forces on the GPU (sq3_forces) against the oracle
(oracle.forces): the local term from the Gaussian pseudocharges and phi,
the nonlocal term of Eq. (force:NewForm) from an orthonormal block and a
density kernel, element by element in FP64 (1e-10 relative to the largest
component); the FP32 block of the mixed path within 1e-5; and, on a cell
without projectors, the force against central differences of the
self-consistent free energy through the SCF driver (the oracle's own pin,
repeated on the GPU path)."""
import numpy as np
import pytest
import torch

from oracle import forces, scf, subspace
from paper_2112_08639_gb300 import inputs

from gpu_common import need_gpu, small_proj_cell, sq3, to_gpu_block

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _inputs(seed=0, Ns=24):
    cell = small_proj_cell()
    cfg = cell.cfg
    pos = cell.positions
    rng = np.random.default_rng(seed)
    X = subspace.cholqr(rng.normal(size=(cfg.N, Ns)))
    D = rng.normal(size=(Ns, Ns)) / Ns
    D = 0.5 * (D + D.T)
    b, _ = scf.pseudocharge(cfg.n, cfg.L, pos, inputs.Z_VALENCE, inputs.RC_LOCAL, Ne=cfg.Ne)
    rho = np.exp(0.2 * rng.normal(size=cfg.N))
    rho *= cfg.Ne / (rho.sum() * cfg.dV)
    phi = scf.poisson_fd(rho + b, cfg.n, cfg.L)
    return cell, X, D, b, phi


def _ctx(cell):
    cfg = cell.cfg
    ctx = sq3().Context(0)
    ctx.setup_grid(cfg.n, cfg.n, cfg.n, cfg.L, cfg.L, cfg.L, 12)
    pr = cell.proj
    ctx.set_projectors(pr.ptr, pr.idx, pr.val, pr.gamma)
    return ctx


def _oracle(cell, X, D, b, phi):
    cfg = cell.cfg
    _, total = scf.pseudocharge(cfg.n, cfg.L, cell.positions, inputs.Z_VALENCE, inputs.RC_LOCAL)
    gb = scf.pseudocharge_gradients(cfg.n, cfg.L, cell.positions, inputs.Z_VALENCE,
                                    inputs.RC_LOCAL, scale=-cfg.Ne / total)
    floc = forces.local_forces(gb, phi, cfg.dV)
    fnl = forces.nonlocal_forces(X, D, cell.proj, cfg.n, cfg.L, cfg.natoms)
    return floc, fnl


def test_forces_fp64_match_oracle():
    cell, X, D, b, phi = _inputs(0)
    cfg = cell.cfg
    ctx = _ctx(cell)
    atom_of = np.arange(cell.proj.n_proj) // 4
    f, floc, fnl = ctx.forces(cell.positions, inputs.Z_VALENCE, inputs.RC_LOCAL, cfg.Ne,
                              torch.from_numpy(phi).cuda(), to_gpu_block(X),
                              torch.from_numpy(D).cuda(), atom_of=atom_of)
    rloc, rnl = _oracle(cell, X, D, b, phi)
    scale = np.max(np.abs(rloc + rnl))
    assert np.max(np.abs(floc - rloc)) < 1e-10 * np.max(np.abs(rloc))
    assert np.max(np.abs(fnl - rnl)) < 1e-10 * np.max(np.abs(rnl))
    assert np.max(np.abs(f - (rloc + rnl))) < 1e-10 * scale
    # a second call reuses the gradient tables
    f2, _, _ = ctx.forces(cell.positions, inputs.Z_VALENCE, inputs.RC_LOCAL, cfg.Ne,
                          torch.from_numpy(phi).cuda(), to_gpu_block(X),
                          torch.from_numpy(D).cuda(), atom_of=atom_of)
    np.testing.assert_array_equal(f, f2)


def test_forces_mixed_block_within_fp32_rounding():
    cell, X, D, b, phi = _inputs(1)
    cfg = cell.cfg
    ctx = _ctx(cell)
    atom_of = np.arange(cell.proj.n_proj) // 4
    args = (cell.positions, inputs.Z_VALENCE, inputs.RC_LOCAL, cfg.Ne, torch.from_numpy(phi).cuda())
    Dg = torch.from_numpy(D).cuda()
    f64, _, n64 = ctx.forces(*args, to_gpu_block(X), Dg, atom_of=atom_of)
    f32, _, n32 = ctx.forces(*args, to_gpu_block(X, torch.float32), Dg, prec=sq3().MIXED,
                             atom_of=atom_of)
    assert np.max(np.abs(n32 - n64)) < 1e-5 * np.max(np.abs(n64))


def test_force_is_minus_the_derivative_of_the_scf_free_energy():
    """4 atoms, 12^3 grid, no projectors: F(R) by the FP64 SCF driver at
    R +- delta along one coordinate; (F(-) - F(+)) / (2 delta) equals the
    force at R within 1e-7 Ha/bohr (central-difference and SCF tolerance;
    the oracle's pin measured 5e-10 - 1.2e-9)."""
    n, L, Ns, Ne = 12, inputs.A0_FCC, 57, 12.0
    sigma, Z, rc = inputs.ev_to_ha(10.0), inputs.Z_VALENCE, inputs.RC_LOCAL
    pos0 = inputs.fcc_positions(1, disp_sigma=0.05, seed=0)
    ctx = sq3().Context(0)
    ctx.setup_grid(n, n, n, L, L, L, 12)
    e_self = scf.self_energy(4, Z, rc)
    X0 = to_gpu_block(inputs.random_block(n ** 3, Ns, seed=0).T)

    def solve(pos):
        b, _ = ctx.pseudocharge(pos, Z, rc)
        rho = torch.full((n ** 3,), Ne / L ** 3, dtype=torch.float64, device="cuda:0")
        X = X0.clone()
        res, _ = ctx.scf_solve(b, rho, X, degree=16, npl=80, kT=sigma, Ne=Ne, e_self=e_self,
                               tol=1e-11, first_passes=12, passes=3, max_iter=100,
                               cut_shift=0.07)
        return res, rho, b

    res, rho, b = solve(pos0)
    phi = torch.empty_like(rho)
    ctx.effective_potential(rho, b, phi=phi)
    f, _, _ = ctx.forces(pos0, Z, rc, Ne, phi)
    d = 1e-3
    for (I, a) in ((1, 0), (2, 2)):
        pp, pm = pos0.copy(), pos0.copy()
        pp[I, a] += d
        pm[I, a] -= d
        Fp = solve(pp)[0]["F"]
        Fm = solve(pm)[0]["F"]
        assert abs((Fm - Fp) / (2 * d) - f[I, a]) < 1e-7, (I, a)
