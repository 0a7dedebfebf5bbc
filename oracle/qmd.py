"""Quantum molecular dynamics of the nuclei: plain FP64 CPU code.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

Sec. 5 runs Kohn-Sham QMD of aluminium with the Hellmann-Feynman forces of
Eq. (force:NewForm) at a time step of 0.15 fs, in the isokinetic ensemble
(Gaussian thermostat).  The integrator is velocity Verlet:

    R(t + dt) = R + dt V + dt^2 F / (2 m)
    V(t + dt) = V + dt (F(t) + F(t + dt)) / (2 m),

with F(t + dt) from a new self-consistent solution at R(t + dt).  The
isokinetic constraint is kept by rescaling the velocities to the target
kinetic energy after every step (a reading: the paper names the thermostat,
not its discretisation).  Atomic units throughout: bohr, electron masses,
hbar / Ha for time.
"""
from __future__ import annotations

import numpy as np

AMU_IN_ME = 1822.888486209            # atomic mass unit / electron mass
FS_IN_AU = 1.0 / 0.02418884326585747   # femtoseconds in hbar / Ha
MASS_AL = 26.9815385 * AMU_IN_ME


def kinetic_energy(V: np.ndarray, masses: np.ndarray) -> float:
    """sum_I m_I |V_I|^2 / 2; V (natoms, 3), masses (natoms,)."""
    return 0.5 * float(np.sum(masses[:, None] * V * V))


def rescale_isokinetic(V: np.ndarray, masses: np.ndarray, ke_target: float) -> np.ndarray:
    ke = kinetic_energy(V, masses)
    return V if ke == 0.0 else V * np.sqrt(ke_target / ke)


def velocity_verlet_step(R, V, F, masses, dt, force_fn):
    """One step; force_fn(R) -> (forces (natoms, 3), potential energy).
    Returns R, V, F, E_pot at t + dt."""
    m = masses[:, None]
    R1 = R + dt * V + (0.5 * dt * dt) * F / m
    F1, E1 = force_fn(R1)
    V1 = V + (0.5 * dt) * (F + F1) / m
    return R1, V1, F1, E1


def run(R0, V0, masses, dt, nsteps, force_fn, isokinetic: bool = False) -> dict:
    """nsteps of velocity Verlet from (R0, V0); with `isokinetic` the kinetic
    energy is held at its initial value.  Returns the trajectory of
    positions, velocities, potential and kinetic energies (nsteps + 1 each)."""
    R, V = np.array(R0, dtype=float), np.array(V0, dtype=float)
    F, E = force_fn(R)
    ke0 = kinetic_energy(V, masses)
    Rs, Vs, Es, Ks = [R.copy()], [V.copy()], [E], [ke0]
    for _ in range(nsteps):
        R, V, F, E = velocity_verlet_step(R, V, F, masses, dt, force_fn)
        if isokinetic:
            V = rescale_isokinetic(V, masses, ke0)
        Rs.append(R.copy())
        Vs.append(V.copy())
        Es.append(E)
        Ks.append(kinetic_energy(V, masses))
    return {"R": np.array(Rs), "V": np.array(Vs), "E_pot": np.array(Es), "E_kin": np.array(Ks)}


def maxwell_boltzmann(natoms: int, masses: np.ndarray, kT: float, seed: int = 0) -> np.ndarray:
    """Seeded velocities with zero total momentum, scaled so that the
    kinetic energy is exactly (3 natoms - 3) kT / 2."""
    rng = np.random.default_rng(seed + 15485863)
    V = rng.normal(size=(natoms, 3)) * np.sqrt(kT / masses)[:, None]
    V -= np.sum(masses[:, None] * V, axis=0) / masses.sum()
    return rescale_isokinetic(V, masses, 0.5 * (3 * natoms - 3) * kT)
