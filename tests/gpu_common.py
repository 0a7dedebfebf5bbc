"""Shared set-up for the GPU parity tests: builds the library, creates a
context on cuda:0 and evaluates the CPU oracle on the same seeded inputs."""
import functools

import numpy as np
import pytest
import torch

from oracle import fermi, hamiltonian
from paper_2112_08639_gb300 import inputs


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@functools.lru_cache(maxsize=None)
def sq3():
    from paper_2112_08639_gb300 import build
    build.build()
    from paper_2112_08639_gb300 import sq3 as mod
    return mod


def context_for(cell: inputs.Cell, fd_order: int = 12):
    m = sq3()
    ctx = m.Context(0)
    cfg = cell.cfg
    ctx.setup_grid(cfg.n, cfg.n, cfg.n, cfg.L, cfg.L, cfg.L, fd_order)
    ctx.set_potential(torch.from_numpy(cell.V))
    if cell.proj is not None:
        ctx.set_projectors(cell.proj.ptr, cell.proj.idx, cell.proj.val, cell.proj.gamma)
    return ctx


def oracle_parts(cell: inputs.Cell):
    cfg = cell.cfg
    return hamiltonian.hamiltonian_sparse(cfg.n, cfg.L, cell.V, cell.proj)


def apply_fn(parts):
    return lambda X: hamiltonian.apply(parts, X)


@functools.lru_cache(maxsize=None)
def c1_cell():
    return inputs.make_cell(inputs.C1)


@functools.lru_cache(maxsize=None)
def c1_eigs(nstates: int = 100):
    cell = c1_cell()
    H = hamiltonian.hamiltonian_dense(cell.cfg.n, cell.cfg.L, cell.V)
    return fermi.lowest_eigenpairs(H, nstates)


@functools.lru_cache(maxsize=None)
def small_proj_cell():
    """A 4-atom cell on a 16^3 grid with s/p projectors truncated at 3 bohr,
    small enough for dense diagonalisation, with every projector code path."""
    cfg = inputs.CellConfig("al4_16_proj", ncell=1, n=16, Ns=40, m=16, npl=60,
                            projectors=True, seed=3)
    pos = inputs.fcc_positions(1, disp_sigma=0.05, seed=3)
    V = inputs.local_potential(cfg.n, cfg.L, pos)
    pr = inputs.projectors(cfg.n, cfg.L, pos, seed=3, rcut=3.0)
    return inputs.Cell(cfg, pos, V, pr)


def to_gpu_block(X_np: np.ndarray, dtype=torch.float64):
    """numpy (N, Ns) -> contiguous torch (Ns, N) on cuda:0."""
    return torch.from_numpy(np.ascontiguousarray(X_np.T)).to("cuda:0", dtype)


def from_gpu_block(X: torch.Tensor) -> np.ndarray:
    return X.double().cpu().numpy().T
