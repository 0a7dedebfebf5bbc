"""Seeded synthetic inputs for the SQ3 hot path.

This module generates the *inputs* of the method and nothing else: atom
positions of an FCC Al-like cell, the local potential on the grid, the
Kleinman-Bylander projector table, and the random starting block X0.  It holds
none of the method's arithmetic (no stencil, no Hamiltonian apply, no Fermi
function, no Chebyshev expansion), so that both the CPU oracle (through the
tests) and the CUDA path can be fed from it without sharing method code.

Recipe (stand-in for the paper's Al workloads, Sec. 5 of the paper, whose
ONCV pseudopotential and QMD initial conditions are not available):

* FCC basis (0,0,0), (0,1/2,1/2), (1/2,0,1/2), (1/2,1/2,0) times a0 = 7.78
  bohr, replicated ncell^3 times (4, 32, 108 atoms), each atom displaced by
  N(0, disp_sigma) bohr from ``numpy.random.default_rng(seed)``.
* Local potential: the periodic electrostatic potential of one Gaussian
  pseudocharge of charge -Z (Z = 3, width r_c = 1.0 bohr) per atom on a
  neutralising background, i.e. the periodic sum of -Z erf(r/r_c)/r with its
  G = 0 component removed, evaluated on the grid by a Fourier sum.
* Projectors (optional): per atom one s and three p Gaussian projectors,
  chi_s = exp(-r^2/rc^2), chi_p = (x_a - R_a) exp(-r^2/rc^2), rc = 1.2 bohr,
  truncated at 4.2 bohr (minimum image), each scaled so that the
  Euclidean-normalised vector c = chi * sqrt(dV) has unit norm.  Energies
  gamma_J0 (s) and gamma_J1 (p, shared by m = x, y, z) ~ U(0.1, 1.0) Ha.
* Grid index k = i + nx*j + nx*ny*l (x fastest); arrays are returned with
  shape (nz, ny, nx) flattened in C order, which is that ordering.
"""
from __future__ import annotations

import dataclasses
import numpy as np

HARTREE_EV = 27.211386245988
A0_FCC = 7.78
Z_VALENCE = 3.0
RC_LOCAL = 1.0
RC_PROJ = 1.2
RCUT_PROJ = 4.2


def ev_to_ha(kT_ev: float) -> float:
    return kT_ev / HARTREE_EV


@dataclasses.dataclass(frozen=True)
class CellConfig:
    """One synthetic cell: geometry, grid and method parameters."""
    name: str
    ncell: int          # FCC supercell repeats per axis (atoms = 4 ncell^3)
    n: int              # grid points per axis
    Ns: int             # number of auxiliary vectors
    m: int              # Chebyshev filter degree
    npl: int            # Fermi-operator Chebyshev degree
    kT_ev: float = 10.0
    projectors: bool = False
    disp_sigma: float = 0.05
    seed: int = 0

    @property
    def natoms(self) -> int:
        return 4 * self.ncell ** 3

    @property
    def L(self) -> float:
        return A0_FCC * self.ncell

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def N(self) -> int:
        return self.n ** 3

    @property
    def dV(self) -> float:
        return self.h ** 3

    @property
    def Ne(self) -> float:
        return Z_VALENCE * self.natoms

    @property
    def sigma(self) -> float:
        return ev_to_ha(self.kT_ev)


# The three single-cell workloads: 4-atom 18^3 (Ns 64), 32-atom 48^3 (Ns 640)
# and 108-atom 72^3 (Ns 2200).
C1 = CellConfig("al4_18", ncell=1, n=18, Ns=64, m=20, npl=60, projectors=False)
C2 = CellConfig("al32_48", ncell=2, n=48, Ns=640, m=25, npl=100, projectors=True)
C3 = CellConfig("al108_72", ncell=3, n=72, Ns=2200, m=30, npl=120, projectors=True)
CONFIGS = {c.name: c for c in (C1, C2, C3)}

AL_MASS_AMU = 26.9815385


@dataclasses.dataclass(frozen=True)
class QMDConfig:
    """A QMD run of one cell (Sec. 5: Al at 116,045 K, i.e. kT = 10 eV, in
    the isokinetic ensemble): velocity Verlet with dt_fs, nsteps steps, the
    learned start trained on the first train_steps steps' densities."""
    name: str
    cell: CellConfig
    dt_fs: float
    nsteps: int
    train_steps: int
    mass_amu: float = AL_MASS_AMU
    seed: int = 0


# C5: the 32-atom cell of C2, 0.5 fs steps, 300 steps, trained on 0 .. 99
C5 = QMDConfig("al32_48_qmd", cell=C2, dt_fs=0.5, nsteps=300, train_steps=100)


def batch_cells(ncells: int = 64, seed: int = 0):
    """C4, the batched workload: uneven Al-like cells of 4 to 32 atoms (FCC
    supercells 1x1x1, 2x1x1, 2x2x1, 2x2x2 on 0.324-bohr grids of 24 to 48
    points per side), seeded thermal displacements (0.3 bohr), kT drawn
    from 5 to 20 eV, Ns = 20 x atoms (80 to 640), filter degree 20."""
    rng = np.random.default_rng(seed)
    shapes = [(1, 1, 1), (2, 1, 1), (2, 2, 1), (2, 2, 2)]
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    cells = []
    for c in range(ncells):
        sx, sy, sz = shapes[rng.integers(0, 4)]
        L = np.array([sx, sy, sz], dtype=float) * A0_FCC
        n = tuple(int(24 * s) for s in (sx, sy, sz))
        pos = np.array([(np.array([i, j, k]) + b) * A0_FCC
                        for i in range(sx) for j in range(sy) for k in range(sz) for b in basis])
        pos = np.mod(pos + rng.normal(0.0, 0.3, size=pos.shape), L)
        kT = float(rng.uniform(5.0, 20.0))
        cells.append({"n": n, "L": tuple(L), "pos": pos, "natoms": len(pos),
                      "Ns": 20 * len(pos), "m": 20, "kT": kT, "seed": seed * 1000 + c})
    return cells


def small_cells(ncells: int = 64, seed: int = 1):
    """Many small cells: 4-atom FCC cells on 24^3 grids, Ns = 80, degree 20
    (each cell's filter alone fills a small part of the GPU)."""
    return [c for c in batch_cells(4 * ncells, seed=seed) if c["natoms"] == 4][:ncells]


def fcc_positions(ncell: int, a0: float = A0_FCC, disp_sigma: float = 0.05,
                  seed: int = 0) -> np.ndarray:
    """Atom positions (natoms, 3) in bohr, wrapped into [0, L)."""
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    cells = np.array([[i, j, k] for i in range(ncell) for j in range(ncell)
                      for k in range(ncell)], dtype=float)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a0
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, disp_sigma, size=pos.shape)
    return np.mod(pos, a0 * ncell)


def grid_points(n: int, L: float) -> np.ndarray:
    """Coordinates (N, 3) of the periodic grid, index k = i + n j + n^2 l."""
    h = L / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) * h


def local_potential(n: int, L: float, positions: np.ndarray,
                    Z: float = Z_VALENCE, rc: float = RC_LOCAL) -> np.ndarray:
    """Periodic potential of Gaussian charges -Z (width rc), zero mean.

    V(G) = -(4 pi Z / (Omega G^2)) exp(-G^2 rc^2 / 4) sum_J exp(-i G.R_J) for
    G != 0 and V(0) = 0, summed over the grid's reciprocal vectors.  Returns
    float64 of length n^3 in grid order.
    """
    omega = L ** 3
    m = np.fft.fftfreq(n, d=1.0 / n)            # integer frequencies
    g1 = 2.0 * np.pi * m / L
    gz, gy, gx = np.meshgrid(g1, g1, g1, indexing="ij")
    g2 = gx ** 2 + gy ** 2 + gz ** 2
    sf = np.zeros_like(g2, dtype=complex)
    for R in positions:
        sf += np.exp(-1j * (gx * R[0] + gy * R[1] + gz * R[2]))
    with np.errstate(divide="ignore", invalid="ignore"):
        vg = -(4.0 * np.pi * Z / omega) * np.exp(-g2 * rc * rc / 4.0) / g2 * sf
    vg[0, 0, 0] = 0.0
    V = np.fft.ifftn(vg).real * n ** 3
    return np.ascontiguousarray(V.ravel())


@dataclasses.dataclass
class ProjectorTable:
    """CSR projector table: projector p covers grid indices idx[ptr[p]:ptr[p+1]]
    with continuum values val (chi at those points) and energy gamma[p]."""
    ptr: np.ndarray     # int32 (n_proj + 1)
    idx: np.ndarray     # int32 (nnz)
    val: np.ndarray     # float64 (nnz)
    gamma: np.ndarray   # float64 (n_proj)

    @property
    def n_proj(self) -> int:
        return len(self.gamma)


def projectors(n: int, L: float, positions: np.ndarray, seed: int = 0,
               rc: float = RC_PROJ, rcut: float = RCUT_PROJ) -> ProjectorTable:
    """Seeded s/p Gaussian projectors, 4 per atom, minimum image."""
    h = L / n
    dV = h ** 3
    rng = np.random.default_rng(seed + 7919)
    ptr, idx, val, gam = [0], [], [], []
    for R in positions:
        # the grid points of the cube of half-width rcut around R (wrapped,
        # each index once), in ascending grid order
        ax = []
        for a in range(3):
            lo, hi = int(np.floor((R[a] - rcut) / h)), int(np.ceil((R[a] + rcut) / h))
            ax.append(np.unique(np.mod(np.arange(lo, hi + 1), n)))
        kz, ky, kx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        cand = (kx + n * ky + n * n * kz).ravel()
        order = np.argsort(cand, kind="stable")
        cand = cand[order]
        d = np.stack([kx.ravel()[order], ky.ravel()[order], kz.ravel()[order]], axis=1) * h - R
        d -= L * np.round(d / L)
        r2 = np.einsum("ij,ij->i", d, d)
        keep = np.nonzero(r2 < rcut * rcut)[0]
        sel, d, r2 = cand[keep], d[keep], r2[keep]
        env = np.exp(-r2 / (rc * rc))
        g_s, g_p = rng.uniform(0.1, 1.0, size=2)
        for chi, g in ((env, g_s), (d[:, 0] * env, g_p),
                       (d[:, 1] * env, g_p), (d[:, 2] * env, g_p)):
            chi = chi / np.sqrt(np.sum(chi * chi) * dV)
            idx.append(sel.astype(np.int32))
            val.append(chi)
            gam.append(g)
            ptr.append(ptr[-1] + len(sel))
    return ProjectorTable(np.asarray(ptr, np.int32), np.concatenate(idx),
                          np.concatenate(val), np.asarray(gam, float))


def random_block(N: int, Ns: int, seed: int = 0) -> np.ndarray:
    """X0 ~ N(0, 1), shape (Ns, N) in C order == N x Ns column-major."""
    rng = np.random.default_rng(seed + 104729)
    return rng.standard_normal((Ns, N))


def random_block_device(N: int, Ns: int, seed: int = 0, dtype=None, device="cuda:0"):
    """X0 ~ N(0, 1) drawn on the device by torch's seeded generator, shape
    (Ns, N) (N x Ns column-major); for full-size blocks that are too large to
    draw on the host.  Tests hand the oracle copies of sampled columns."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed + 104729)
    return torch.randn((Ns, N), generator=g, device=device,
                       dtype=torch.float32 if dtype is None else dtype)


@dataclasses.dataclass
class Cell:
    cfg: CellConfig
    positions: np.ndarray
    V: np.ndarray
    proj: ProjectorTable | None


def make_cell(cfg: CellConfig) -> Cell:
    pos = fcc_positions(cfg.ncell, disp_sigma=cfg.disp_sigma, seed=cfg.seed)
    V = local_potential(cfg.n, cfg.L, pos)
    pr = projectors(cfg.n, cfg.L, pos, seed=cfg.seed) if cfg.projectors else None
    return Cell(cfg, pos, V, pr)
