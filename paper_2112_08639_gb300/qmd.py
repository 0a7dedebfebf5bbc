"""Quantum molecular dynamics of the nuclei on the library's forces (the QMD
of Sec. 5: velocity Verlet, isokinetic ensemble), one converged SCF solve
per step through the SCF driver, with a choice of starting density per
step: the atomic superposition, the previous step's density, or the
learned model (``learned.LearnedStart``).

This module orders library calls: the projector table of each step comes
from the inputs module (the synthetic pseudopotential's projectors at the
new positions), and the pseudocharges, the SCF solve, the forces and the
Verlet halves run in the library.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import inputs, sq3

AMU_IN_ME = 1822.888486209             # atomic mass unit / electron mass
FS_IN_AU = 1.0 / 0.02418884326585747    # femtoseconds in hbar / Ha
MASS_AL = inputs.AL_MASS_AMU * AMU_IN_ME
# width (bohr) of the atomic-superposition start: the best single width on
# self-consistent densities of 32-atom cells at kT = 10 eV (L1 error per
# electron 0.10 at 2.3 bohr against 0.25 at 1.9 and 0.62 at 1.5)
SUPERPOSITION_WIDTH = 2.3


def maxwell_boltzmann(natoms: int, kT: float, seed: int = 0, mass: float = MASS_AL) -> np.ndarray:
    """Seeded velocities with zero total momentum and kinetic energy
    (3 natoms - 3) kT / 2 (the equipartition value of the free degrees)."""
    rng = np.random.default_rng(seed + 15485863)
    V = rng.normal(size=(natoms, 3)) * np.sqrt(kT / mass)
    V -= V.mean(axis=0)
    ke = 0.5 * mass * float(np.sum(V * V))
    return np.ascontiguousarray(V * np.sqrt(0.5 * (3 * natoms - 3) * kT / ke))


class Cell:
    """One periodic cell on a context: grid, pseudopotential parameters and
    the per-step state (block X, density, last spectral bounds)."""

    def __init__(self, cfg: inputs.CellConfig, device: int = 0, prec=sq3.MIXED,
                 proj_seed: int | None = None, kernel_eval: int = sq3.EVAL_RECURRENCE):
        self.cfg = cfg
        self.prec = prec
        self.kernel_eval = kernel_eval
        self.ctx = sq3.Context(device)
        self.ctx.setup_grid(cfg.n, cfg.n, cfg.n, cfg.L, cfg.L, cfg.L, 12)
        self.proj_seed = cfg.seed if proj_seed is None else proj_seed
        dtype = torch.float64 if prec == sq3.FP64 else torch.float32
        self.X = inputs.random_block_device(cfg.N, cfg.Ns, seed=cfg.seed, dtype=dtype)
        self.rho = torch.empty(cfg.N, dtype=torch.float64, device=self.ctx.device)
        self.b = torch.empty_like(self.rho)
        self.phi = torch.empty_like(self.rho)
        self.D = torch.empty((cfg.Ns, cfg.Ns), dtype=torch.float64, device=self.ctx.device)
        self.bounds = None
        self.rho_prev = None
        self.pos_prev = None
        self._ma = torch.empty_like(self.rho)
        self._mb = torch.empty_like(self.rho)
        self.e_self = cfg.natoms * inputs.Z_VALENCE ** 2 / np.sqrt(2 * np.pi) / inputs.RC_LOCAL

    def set_positions(self, pos):
        cfg = self.cfg
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.proj = None
        self.atom_of = None
        if cfg.projectors:
            pr = inputs.projectors(cfg.n, cfg.L, self.pos, seed=self.proj_seed)
            self.ctx.set_projectors(pr.ptr, pr.idx, pr.val, pr.gamma)
            self.proj = pr
            self.atom_of = np.arange(pr.n_proj) // 4
        self.ctx.pseudocharge(self.pos, inputs.Z_VALENCE, inputs.RC_LOCAL, out=self.b)

    def _model(self, kind: str, pos, learned, out):
        if kind == "learned":
            return learned.predict(self.ctx, pos, self.cfg.Ne, out=out)
        return self.ctx.atom_gaussians(pos, SUPERPOSITION_WIDTH, total=self.cfg.Ne, out=out)[0]

    def start_density(self, start: str, learned=None):
        """The starting density of the next solve:
        superposition   atomic superposition at the current positions;
        learned-direct  the learned model at the current positions;
        previous        the previous step's converged density;
        learned         previous + learned(R) - learned(R_prev) (the model's
                        systematic error cancels, its response to the motion
                        remains; the learned model alone on the first step);
        extrapolated    the same with the atomic superposition as the model."""
        cfg = self.cfg
        have_prev = self.rho_prev is not None and self.pos_prev is not None
        if start == "previous" and self.rho_prev is not None:
            self.rho.copy_(self.rho_prev)
        elif start in ("learned", "extrapolated") and have_prev:
            kind = "learned" if start == "learned" else "superposition"
            a = self._model(kind, self.pos, learned, self._ma)
            b = self._model(kind, self.pos_prev, learned, self._mb)
            self.ctx.extrapolate_density(self.rho_prev, a, b, cfg.Ne, out=self.rho)
        elif start in ("learned", "learned-direct"):
            self._model("learned", self.pos, learned, self.rho)
        else:
            self._model("superposition", self.pos, learned, self.rho)

    def solve(self, tol: float = 1e-6, **kw):
        cfg = self.cfg
        first = self.bounds is None
        # mixing: a Pulay step every iteration (Kerker-preconditioned) with
        # beta 0.5 for a solve from scratch and 0.8 for a QMD step that starts
        # near the previous step's state (at 108 atoms, two consecutive QMD
        # steps: 6 iterations with beta 0.5 or 0.6, 5 with 0.7 .. 1.0, 7 with
        # k0 = 0.5 or 1.2; every second Pulay step with beta 0.3 took 9); from
        # a random block the first iteration runs four filter passes, later
        # ones one
        args = dict(degree=cfg.m, npl=cfg.npl, kT=cfg.sigma, Ne=cfg.Ne, e_self=self.e_self,
                    tol=tol, prec=self.prec, first_passes=4 if first else 1, passes=1,
                    max_iter=100, bounds0=self.bounds, D=self.D, mix_history=7,
                    mix_period=1, mix_beta=0.5 if first else 0.8,
                    kernel_eval=self.kernel_eval)
        args.update(kw)
        res, hist = self.ctx.scf_solve(self.b, self.rho, self.X, **args)
        self.bounds = (res["chi"], res["xi"])
        self.rho_prev = self.rho.clone()
        self.pos_prev = self.pos.copy()
        return res, hist

    def forces(self):
        cfg = self.cfg
        self.ctx.effective_potential(self.rho, self.b, phi=self.phi)
        f, _, _ = self.ctx.forces(self.pos, inputs.Z_VALENCE, inputs.RC_LOCAL, cfg.Ne, self.phi,
                                  self.X if cfg.projectors else None,
                                  self.D if cfg.projectors else None, self.prec, self.atom_of)
        return np.ascontiguousarray(f)


def save_checkpoint(path: str, cell: Cell, step: int, R, V, F, ke0: float, traj: dict) -> None:
    """Everything a QMD run needs to continue after `step`: the nuclei (R, V
    and the forces F at R), the target kinetic energy, the trajectory so
    far, and the SCF state a step hands to the next (the block X, the
    density kernel D, the converged density with its positions, the last
    spectral bounds).  Written to path + '.tmp' and renamed, so an existing
    checkpoint is replaced only by a complete one."""
    state = {
        "version": 1, "config": cell.cfg.name, "prec": int(cell.prec), "step": int(step),
        "R": np.array(R, dtype=np.float64), "V": np.array(V, dtype=np.float64),
        "F": np.array(F, dtype=np.float64), "ke0": float(ke0),
        "traj": {k: list(v) for k, v in traj.items()},
        "X": cell.X.detach().cpu(), "D": cell.D.detach().cpu(),
        "rho_prev": None if cell.rho_prev is None else cell.rho_prev.detach().cpu(),
        "pos_prev": None if cell.pos_prev is None else np.array(cell.pos_prev),
        "bounds": None if cell.bounds is None else tuple(float(b) for b in cell.bounds),
    }
    tmp = path + ".tmp"
    torch.save(state, tmp)
    os.replace(tmp, path)


def load_checkpoint(path: str, cell: Cell) -> dict:
    """Restores the SCF state of `cell` from a checkpoint written by
    save_checkpoint for the same configuration and precision; returns the
    checkpoint (its step, R, V, F, ke0 and trajectory)."""
    state = torch.load(path, map_location="cpu", weights_only=False)
    if state.get("version") != 1 or state["config"] != cell.cfg.name or \
            state["prec"] != int(cell.prec) or tuple(state["X"].shape) != tuple(cell.X.shape):
        raise ValueError(f"checkpoint {path} is not for this cell ({cell.cfg.name}, prec "
                         f"{int(cell.prec)}, X {tuple(cell.X.shape)})")
    cell.X.copy_(state["X"].to(cell.X.device, cell.X.dtype))
    cell.D.copy_(state["D"].to(cell.D.device))
    cell.rho_prev = None if state["rho_prev"] is None else state["rho_prev"].to(cell.rho.device)
    cell.pos_prev = state["pos_prev"]
    cell.bounds = state["bounds"]
    return state


def write_metrics(f, step: int, res: dict, hist: list, E_kin: float) -> None:
    """One JSON line per SCF iteration of the step (its history: change of
    rho, mu, energies, expansion degree, milliseconds, spectral centre and
    half-width) and one for the step itself."""
    for i, h in enumerate(hist):
        f.write(json.dumps({"kind": "scf", "step": step, "iteration": i + 1,
                            **{k: float(v) for k, v in h.items()}}) + "\n")
    f.write(json.dumps({"kind": "step", "step": step, "iterations": int(res["iterations"]),
                        "converged": int(res["converged"]), "F": float(res["F"]),
                        "mu": float(res["mu"]), "err": float(res["err"]),
                        "E_kin": float(E_kin)}) + "\n")
    f.flush()


def run(cell: Cell, R0, V0, dt_fs: float, nsteps: int, start: str = "previous",
        learned=None, isokinetic: bool = True, tol: float = 1e-6, on_step=None,
        checkpoint: str | None = None, checkpoint_every: int = 1, resume: str | None = None,
        metrics: str | None = None) -> dict:
    """nsteps of velocity Verlet from (R0, V0) with dt_fs femtoseconds per
    step; returns per-step positions, SCF iterations, F and kinetic energy.
    on_step(step, cell, result) is called after each converged solve (for
    example to collect training densities).  checkpoint: a file rewritten
    after every checkpoint_every-th step (and the last); resume: a
    checkpoint to continue from instead of (R0, V0) (the trajectory then
    holds the steps before it as well); metrics: a JSON-lines file that gets
    the SCF history and a summary of every step (appended)."""
    dt = dt_fs * FS_IN_AU
    mf = open(metrics, "a") if metrics else None
    try:
        if resume:
            st = load_checkpoint(resume, cell)
            R, V, F, ke0, first = st["R"], st["V"], st["F"], st["ke0"], st["step"] + 1
            traj = st["traj"]
            masses = np.full(len(R), MASS_AL)
        else:
            masses = np.full(len(R0), MASS_AL)
            R = np.array(R0, dtype=np.float64)
            V = np.array(V0, dtype=np.float64)
            ke0 = 0.5 * float(np.sum(masses[:, None] * V * V))
            cell.set_positions(R)
            cell.start_density(start, learned)
            res, hist = cell.solve(tol)
            if on_step:
                on_step(0, cell, res)
            F = cell.forces()
            traj = {"R": [R.copy()], "iterations": [res["iterations"]], "F": [res["F"]],
                    "E_kin": [ke0], "converged": [res["converged"]]}
            if mf:
                write_metrics(mf, 0, res, hist, ke0)
            if checkpoint:
                save_checkpoint(checkpoint, cell, 0, R, V, F, ke0, traj)
            first = 1
        for step in range(first, nsteps + 1):
            sq3.verlet(masses, dt, R, V, F, 0)
            cell.set_positions(R)
            cell.start_density(start, learned)
            res, hist = cell.solve(tol)
            if on_step:
                on_step(step, cell, res)
            F = cell.forces()
            sq3.verlet(masses, dt, R, V, F, 1, ke0 if isokinetic else 0.0)
            ek = 0.5 * float(np.sum(masses[:, None] * V * V))
            traj["R"].append(R.copy())
            traj["iterations"].append(res["iterations"])
            traj["F"].append(res["F"])
            traj["E_kin"].append(ek)
            traj["converged"].append(res["converged"])
            if mf:
                write_metrics(mf, step, res, hist, ek)
            if checkpoint and (step % max(checkpoint_every, 1) == 0 or step == nsteps):
                save_checkpoint(checkpoint, cell, step, R, V, F, ke0, traj)
    finally:
        if mf:
            mf.close()
    return {k: np.asarray(v) for k, v in traj.items()}
