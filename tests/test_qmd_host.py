"""The library's velocity-Verlet halves (sq3_verlet, host arithmetic, no
GPU) against the oracle's integrator (oracle.qmd) on a harmonic force
field: the same trajectory to rounding, with and without the isokinetic
rescaling."""
import numpy as np

from oracle import qmd


def _lib():
    from paper_2112_08639_gb300 import build
    build.build()
    from paper_2112_08639_gb300 import sq3
    return sq3


def _force(K):
    return lambda R: (-(R @ K), 0.0)


def test_verlet_matches_oracle_on_a_harmonic_field():
    sq3 = _lib()
    rng = np.random.default_rng(0)
    n = 5
    A = rng.normal(size=(3, 3))
    K = A @ A.T + 3 * np.eye(3)
    masses = rng.uniform(1e4, 5e4, size=n)
    R0 = rng.normal(size=(n, 3))
    V0 = rng.normal(size=(n, 3)) * 1e-3
    dt = 40.0
    for iso in (False, True):
        ref = qmd.run(R0, V0, masses, dt, 25, _force(K), isokinetic=iso)
        R, V = R0.copy(), V0.copy()
        F = -(R @ K)
        ke0 = qmd.kinetic_energy(V0, masses)
        for step in range(25):
            sq3.verlet(masses, dt, R, V, F, 0)
            F = np.ascontiguousarray(-(R @ K))
            sq3.verlet(masses, dt, R, V, F, 1, ke0 if iso else 0.0)
            np.testing.assert_allclose(R, ref["R"][step + 1], rtol=1e-13, atol=1e-15)
            np.testing.assert_allclose(V, ref["V"][step + 1], rtol=1e-12, atol=1e-17)
        if iso:
            assert abs(qmd.kinetic_energy(V, masses) - ke0) < 1e-14 * ke0
