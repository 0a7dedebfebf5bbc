"""GPU parity of the FP32 nonlocal pass (the Kleinman-Bylander term of
Sec. 2, Eq. (nonlocaloperator), applied and projected per 8 x 8 x 4 brick
and group of 16 vectors) against the oracle's Hamiltonian, on a 4-atom cell
(bricks in up to 4 balls) and the 32-atom cell (up to 9 balls per brick),
with vector counts that are not multiples of the 16-vector group.  Smooth
columns (long-wavelength plane waves) keep the kinetic term small, so the
nonlocal term itself is checked to 1e-5 rather than hidden in the rounding
of H X."""
import numpy as np
import pytest
import torch

from oracle import chebyshev, hamiltonian
from paper_2112_08639_gb300 import inputs

from gpu_common import (apply_fn, context_for, from_gpu_block, need_gpu, oracle_parts,
                        small_proj_cell, sq3, to_gpu_block)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _f32(X):
    return X.astype(np.float32).astype(np.float64)


_C2 = None


def _c2_cell():
    global _C2
    if _C2 is None:
        _C2 = inputs.make_cell(inputs.C2)
    return _C2


def _smooth_block(cell, Ns, seed):
    """Columns that are sums of four long-wavelength plane waves (wave
    numbers -2..2 per axis): -1/2 Lap X stays O(X), so the nonlocal term is
    a sizeable part of H X and its error is not hidden by the rounding of
    the kinetic term."""
    n, L = cell.cfg.n, cell.cfg.L
    r = np.arange(n) * (2 * np.pi / n)
    x, y, z = np.meshgrid(r, r, r, indexing="ij")
    x, y, z = (a.transpose(2, 1, 0).ravel() for a in (x, y, z))   # x fastest
    rng = np.random.default_rng(seed)
    X = np.zeros((n ** 3, Ns))
    for j in range(Ns):
        for _ in range(4):
            k = rng.integers(-2, 3, size=3)
            X[:, j] += rng.normal() * np.cos(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 6.3))
    return _f32(X)


def _context(cell):
    return context_for(cell)


def _cell(name):
    return small_proj_cell() if name == "al4" else _c2_cell()


def test_the_32_atom_cell_has_bricks_in_many_balls():
    cell = _c2_cell()
    cfg = cell.cfg
    info = sq3().projector_table_info((cfg.n,) * 3, (cfg.L / cfg.n) ** 3, cell.proj.ptr,
                                      cell.proj.idx, cell.proj.val, cell.proj.gamma)
    assert info["max_brick_balls"] >= 6


@pytest.mark.parametrize("name,Ns", [("al4", 5), ("al4", 16), ("al4", 37), ("al32", 21),
                                     ("al32", 70)])
def test_hamiltonian_apply_fp32_matches_the_oracle(name, Ns):
    cell = _cell(name)
    X = _f32(inputs.random_block(cell.cfg.N, Ns, seed=11).T)
    ref = hamiltonian.apply(oracle_parts(cell), X)
    ctx = _context(cell)
    Y = from_gpu_block(ctx.hamiltonian_apply(to_gpu_block(X, torch.float32),
                                             prec=sq3().MIXED))
    assert _rel(Y, ref) < 1e-6
    # the nonlocal term alone on smooth columns, against the oracle's
    Xs = _smooth_block(cell, Ns, seed=14)
    Hloc, C, gamma = oracle_parts(cell)
    nl_ref = C @ (gamma[:, None] * (C.T @ Xs))
    Ys = from_gpu_block(ctx.hamiltonian_apply(to_gpu_block(Xs, torch.float32),
                                              prec=sq3().MIXED))
    nl = Ys - Hloc @ Xs
    assert np.linalg.norm(nl_ref) > 0.05 * np.linalg.norm(Ys)
    assert _rel(nl, nl_ref) < 1e-5


@pytest.mark.parametrize("name,Ns,m", [("al4", 19, 12), ("al32", 40, 8)])
def test_chebyshev_filter_fp32_matches_the_oracle(name, Ns, m):
    # every step: the apply with the previous step's projections, then the
    # projections of the result (and the projection-only pass of the input)
    cell = _cell(name)
    X = _f32(inputs.random_block(cell.cfg.N, Ns, seed=13).T)
    a0, a, b = -1.8, 2.0, 60.0
    Xg = to_gpu_block(X, torch.float32)
    _context(cell).cheb_filter(Xg, m, a, b, a0, prec=sq3().MIXED)
    ref = chebyshev.filter_plain(apply_fn(oracle_parts(cell)), X, m, a, b, a0)
    assert _rel(from_gpu_block(Xg), ref) < 1e-5
