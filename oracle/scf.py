"""Self-consistent field around the fixed-potential SQ3 iteration: plain FP64
CPU code for the electrostatics, exchange-correlation, density mixing and
the free energy of one cell.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only ``tests/``
(and the entry points named in the package docstring) may use it.

* ``pseudocharge``  -- b = sum_J b_J with b_J(r) = -Z exp(-r^2/rc^2) /
                       (pi^(3/2) rc^3), the pseudocharge whose potential is
                       the local pseudopotential (Sec. 2, Eq. (poisson)),
                       summed over each atom and its periodic images (as
                       the force expression of Eq. (ON:forces) sums them),
                       rescaled so that sum b dV = -N_e; and its gradients
                       grad_x b_J for the forces.
* ``poisson_fd``    -- phi with -L_h phi / (4 pi) = rho + b (Sec. 2,
                       Eq. (poisson)), L_h the finite-difference Laplacian of
                       the Hamiltonian, solved in Fourier space through its
                       symbol s(theta) = -w_0 - 2 sum_p w_p cos(p theta) per
                       direction; the zero mode is set to 0 (the total charge
                       is zero, so the gauge drops out of F).
* ``lda_xc``        -- the LDA of Sec. 2 (named, not specified): Slater
                       exchange and the Perdew-Wang 1992 correlation of the
                       spin-unpolarised electron gas, restated from their
                       published forms; densities below 1e-14 are clamped.
* ``free_energy``   -- F = E_band + E_xc - int V_xc rho + 1/2 int (b - rho) phi
                       - E_self + E_c + E_ent (Sec. 2, Eq. (ON:FreeEnergy);
                       Sec. 3, Eq. (FreeEnergy:NewForm)), with the analytic
                       self energy of the Gaussian pseudocharges and E_c = 0
                       (the nuclei are the Gaussian charges themselves).
* ``kerker`` and ``PulayMixer`` -- density mixing (Sec. 5 cites periodic
                       Pulay with a Kerker preconditioner): Anderson/Pulay
                       extrapolation every second step over a history of 7,
                       linear mixing with beta = 0.3 otherwise, the residual
                       preconditioned by K(G) = G^2 / (G^2 + k0^2).
* ``scf``           -- the loop: V_eff = phi[rho + b] + V_xc[rho], the
                       occupied subspace by exact diagonalisation
                       (``fermi``), mixing, until the L1 change of rho per
                       electron falls below a tolerance.
* ``scf_sq3``       -- the same loop in the paper's algorithm order, the
                       fixed-potential SQ3 iteration (``subspace``) in
                       place of the diagonalisation.
"""
from __future__ import annotations

import numpy as np

import scipy.sparse.linalg as sla

from . import fd, fermi, hamiltonian


def _as_operator(parts):
    """H of hamiltonian_sparse as a scipy LinearOperator."""
    Hloc = parts[0]
    return sla.LinearOperator(Hloc.shape, matvec=lambda v: hamiltonian.apply(parts, v[:, None])[:, 0],
                              dtype=float)

# Perdew-Wang 1992 parameters of the spin-unpolarised correlation energy
# (A, alpha1, beta1..beta4; p = 1)
PW92_A = 0.031091
PW92_ALPHA1 = 0.21370
PW92_BETA = (7.5957, 3.5876, 1.6382, 0.49294)
RHO_FLOOR = 1e-14


def _grid3(n: int):
    """Integer Fourier indices of an n^3 grid in array order [l][j][i]."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return np.meshgrid(m, m, m, indexing="ij")


def _periodic_gaussian_1d(n: int, L: float, r0: float, rc: float, deriv: bool = False):
    """sum over images m of exp(-(x - r0 - m L)^2 / rc^2) at the n grid
    points x = k L / n (or its x-derivative); images while the term can
    exceed 1e-300 of the peak."""
    x = np.arange(n) * (L / n)
    kmax = int(np.ceil(27.0 * rc / L)) + 1
    g = np.zeros(n)
    for m in range(-kmax, kmax + 1):
        d = x - r0 - m * L
        e = np.exp(-d * d / (rc * rc))
        g += (-2.0 * d / (rc * rc)) * e if deriv else e
    return g


def pseudocharge(n: int, L: float, positions: np.ndarray, Z: float, rc: float,
                 Ne: float | None = None) -> tuple[np.ndarray, float]:
    """Gaussian pseudocharges on the grid (length n^3, grid order), summed
    over every atom and all its periodic images (the Gaussian factorises by
    axis, so each axis is summed over images), and the sum b dV before
    rescaling.  With Ne the array is rescaled so that its sum times dV is
    exactly -Ne (the factor differs from 1 by the grid's aliasing of the
    Gaussian, below 1e-9 for h < 0.7 rc)."""
    h = L / n
    b = np.zeros((n, n, n))
    norm = -Z / (np.pi ** 1.5 * rc ** 3)
    for R in positions:
        gx, gy, gz = (_periodic_gaussian_1d(n, L, R[a], rc) for a in range(3))
        b += norm * np.einsum("l,j,i->lji", gz, gy, gx)
    b = b.ravel()
    dV = h ** 3
    total = float(b.sum() * dV)
    if Ne is not None:
        b *= -Ne / total
    return b, total


def pseudocharge_gradients(n: int, L: float, positions: np.ndarray, Z: float, rc: float,
                           scale: float = 1.0) -> np.ndarray:
    """grad_x b_I on the grid for each atom I (with its periodic images):
    array (natoms, 3, n^3), times `scale` (the rescaling factor of
    ``pseudocharge``)."""
    norm = scale * -Z / (np.pi ** 1.5 * rc ** 3)
    out = np.zeros((len(positions), 3, n ** 3))
    for I, R in enumerate(positions):
        g = [_periodic_gaussian_1d(n, L, R[a], rc) for a in range(3)]
        dg = [_periodic_gaussian_1d(n, L, R[a], rc, deriv=True) for a in range(3)]
        out[I, 0] = norm * np.einsum("l,j,i->lji", g[2], g[1], dg[0]).ravel()
        out[I, 1] = norm * np.einsum("l,j,i->lji", g[2], dg[1], g[0]).ravel()
        out[I, 2] = norm * np.einsum("l,j,i->lji", dg[2], g[1], g[0]).ravel()
    return out


def fd_symbol(n: int, order: int = 12) -> np.ndarray:
    """s(theta_m) = -w_0 - 2 sum_p w_p cos(p theta_m), theta_m = 2 pi m / n,
    for the integer frequencies m of np.fft.fftfreq: minus the eigenvalue of
    the 1-D periodic FD second derivative (h = 1) on the mode exp(i theta k)."""
    w = fd.fd_weights(order)
    theta = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / n
    s = -w[0] * np.ones(n)
    for p in range(1, len(w)):
        s -= 2.0 * w[p] * np.cos(p * theta)
    return s


def poisson_fd(rho_tot: np.ndarray, n: int, L: float, order: int = 12) -> np.ndarray:
    """phi with -L_h phi = 4 pi (rho_tot - mean(rho_tot)), zero mean."""
    h = L / n
    s = fd_symbol(n, order) / (h * h)
    sz, sy, sx = np.meshgrid(s, s, s, indexing="ij")
    denom = sx + sy + sz
    rhat = np.fft.fftn(rho_tot.reshape(n, n, n))
    with np.errstate(divide="ignore", invalid="ignore"):
        phat = 4.0 * np.pi * rhat / denom
    phat[0, 0, 0] = 0.0
    return np.fft.ifftn(phat).real.ravel()


def slater_exchange(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(eps_x, v_x): eps_x = -(3/4) (3 rho / pi)^(1/3), v_x = (4/3) eps_x."""
    r = np.maximum(np.asarray(rho, dtype=float), RHO_FLOOR)
    ex = -0.75 * (3.0 * r / np.pi) ** (1.0 / 3.0)
    return ex, (4.0 / 3.0) * ex


def pw92_correlation(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(eps_c, v_c) of the spin-unpolarised gas (Perdew-Wang 1992):
    eps_c(rs) = -2A (1 + alpha1 rs) ln(1 + 1 / (2A (b1 rs^(1/2) + b2 rs
                + b3 rs^(3/2) + b4 rs^2))), v_c = eps_c - (rs / 3) d eps_c / d rs,
    rs = (3 / (4 pi rho))^(1/3)."""
    r = np.maximum(np.asarray(rho, dtype=float), RHO_FLOOR)
    rs = (3.0 / (4.0 * np.pi * r)) ** (1.0 / 3.0)
    A, a1 = PW92_A, PW92_ALPHA1
    b1, b2, b3, b4 = PW92_BETA
    sq = np.sqrt(rs)
    q0 = -2.0 * A * (1.0 + a1 * rs)
    q1 = 2.0 * A * (b1 * sq + b2 * rs + b3 * rs * sq + b4 * rs * rs)
    q1p = A * (b1 / sq + 2.0 * b2 + 3.0 * b3 * sq + 4.0 * b4 * rs)
    lg = np.log1p(1.0 / q1)
    ec = q0 * lg
    dec = -2.0 * A * a1 * lg - q0 * q1p / (q1 * q1 + q1)
    return ec, ec - rs * dec / 3.0


def lda_xc(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(eps_xc, v_xc) per point: Slater exchange plus PW92 correlation."""
    ex, vx = slater_exchange(rho)
    ec, vc = pw92_correlation(rho)
    return ex + ec, vx + vc


def self_energy(natoms: int, Z: float, rc: float) -> float:
    """Self energy of the Gaussian pseudocharges: Z^2 / (sqrt(2 pi) rc) each."""
    return natoms * Z * Z / (np.sqrt(2.0 * np.pi) * rc)


def free_energy(e_band: float, e_ent: float, rho: np.ndarray, b: np.ndarray, phi: np.ndarray,
                dV: float, natoms: int, Z: float, rc: float) -> dict:
    """The terms of F and their sum (E_c = 0)."""
    exc_pt, vxc = lda_xc(rho)
    e_xc = float(np.sum(exc_pt * rho) * dV)
    vxc_rho = float(np.sum(vxc * rho) * dV)
    e_es = 0.5 * float(np.sum((b - rho) * phi) * dV)
    e_self = self_energy(natoms, Z, rc)
    F = e_band + e_xc - vxc_rho + e_es - e_self + e_ent
    return {"F": F, "e_band": e_band, "e_ent": e_ent, "e_xc": e_xc, "vxc_rho": vxc_rho,
            "e_es": e_es, "e_self": e_self}


def kerker(res: np.ndarray, n: int, L: float, k0: float = 0.8) -> np.ndarray:
    """K(G) res with K(G) = G^2 / (G^2 + k0^2), applied in Fourier space
    (K(0) = 0: the preconditioned residual carries no charge)."""
    mz, my, mx = _grid3(n)
    g2 = (2.0 * np.pi / L) ** 2 * (mx * mx + my * my + mz * mz)
    rhat = np.fft.fftn(res.reshape(n, n, n))
    return np.fft.ifftn(rhat * g2 / (g2 + k0 * k0)).real.ravel()


class PulayMixer:
    """Periodic Pulay / Anderson mixing of the density: x_in -> x_out = G(x_in).

    Residual f = x_out - x_in.  Every `period`-th step the next input is the
    Anderson extrapolation x_bar + beta P f_bar, with x_bar = x - dX c,
    f_bar = f - dF c and c the least-squares solution of dF c ~ f over the
    last `history` differences; the other steps mix linearly, x + beta P f.
    P is the preconditioner (identity when None)."""

    def __init__(self, beta: float = 0.3, history: int = 7, period: int = 2, precond=None):
        self.beta, self.history, self.period = beta, history, period
        self.precond = precond if precond is not None else (lambda f: f)
        self.x_prev = self.f_prev = None
        self.dX, self.dF = [], []
        self.k = 0

    def step(self, x: np.ndarray, x_out: np.ndarray) -> np.ndarray:
        f = x_out - x
        if self.x_prev is not None:
            self.dX.append(x - self.x_prev)
            self.dF.append(f - self.f_prev)
            if len(self.dX) > self.history:
                self.dX.pop(0)
                self.dF.pop(0)
        self.x_prev, self.f_prev = x.copy(), f.copy()
        self.k += 1
        if self.dX and self.k % self.period == 0:
            DX = np.stack(self.dX, axis=1)
            DF = np.stack(self.dF, axis=1)
            c, *_ = np.linalg.lstsq(DF, f, rcond=None)
            xb = x - DX @ c
            fb = f - DF @ c
            return xb + self.beta * self.precond(fb)
        return x + self.beta * self.precond(f)


def scf(n: int, L: float, positions: np.ndarray, Ns: int, sigma: float, Z: float, rc: float,
        proj=None, rho0: np.ndarray | None = None, tol: float = 1e-9, max_iter: int = 200,
        order: int = 12, k0: float = 0.8) -> dict:
    """Self-consistent density of one cell by exact diagonalisation per
    iteration (cells small enough for a dense eigensolver)."""
    natoms = len(positions)
    Ne = Z * natoms
    dV = (L / n) ** 3
    b, _ = pseudocharge(n, L, positions, Z, rc, Ne=Ne)
    rho = np.full(n ** 3, Ne / (n ** 3 * dV)) if rho0 is None else rho0.copy()
    mixer = PulayMixer(precond=lambda f: kerker(f, n, L, k0))
    hist = []
    for it in range(max_iter):
        phi = poisson_fd(rho + b, n, L, order)
        _, vxc = lda_xc(rho)
        veff = phi + vxc
        H = hamiltonian.hamiltonian_dense(n, L, veff, proj, order)
        lam, U = fermi.lowest_eigenpairs(H, Ns)
        out = fermi.ks_fixed_potential(lam, U, Ne, sigma, dV)
        err = float(np.sum(np.abs(out["rho"] - rho)) * dV / Ne)
        hist.append(err)
        if err < tol:
            phi_out = poisson_fd(out["rho"] + b, n, L, order)
            terms = free_energy(out["e_band"], out["e_ent"], out["rho"], b, phi_out, dV, natoms,
                                Z, rc)
            return {"rho": out["rho"], "mu": out["mu"], "lam": lam, "U": U, "veff": veff,
                    "phi": phi, "b": b, "iterations": it + 1, "errors": hist, **terms}
        rho = mixer.step(rho, out["rho"])
    raise RuntimeError(f"SCF did not converge in {max_iter} iterations (last {hist[-1]:.3e})")


def scf_sq3(n: int, L: float, positions: np.ndarray, X0: np.ndarray, sigma: float, Z: float,
            rc: float, filt: tuple, npl: int, degree: int = 16, passes: tuple = (12, 3),
            proj=None, tol: float = 1e-10, max_iter: int = 200, order: int = 12,
            k0: float = 0.8) -> dict:
    """The SCF in the paper's algorithm order: each iteration builds V_eff
    from the mixed density, then runs the fixed-potential SQ3 iteration
    (``subspace.sq3_iteration``: Chebyshev filter, Cholesky QR, Hs, the
    Chebyshev density kernel with exact spectral bounds, rho) `passes[0]`
    times in the first iteration and `passes[1]` times after, from the
    starting block X0 (N x Ns, e.g. seeded random); filt = (a, b, a0) are the
    filter's cutoff, upper bound and lower estimate; every iteration checks
    that b lies above the spectrum of its H (a ValueError otherwise: the
    filter would amplify the top of the spectrum).  Stops when the L1 change
    of rho per electron is below `tol`; F by Eq. (FreeEnergy:NewForm) from
    the last output density."""
    from . import subspace
    natoms = len(positions)
    Ne = Z * natoms
    dV = (L / n) ** 3
    a, b_up, a0 = filt
    b, _ = pseudocharge(n, L, positions, Z, rc, Ne=Ne)
    rho = np.full(n ** 3, Ne / (n ** 3 * dV))
    mixer = PulayMixer(precond=lambda f: kerker(f, n, L, k0))
    X = np.array(X0, dtype=float)
    hist = []
    for it in range(max_iter):
        phi = poisson_fd(rho + b, n, L, order)
        _, vxc = lda_xc(rho)
        parts = hamiltonian.hamiltonian_sparse(n, L, phi + vxc, proj, order)
        apply_H = lambda Y: hamiltonian.apply(parts, Y)
        # the filter needs b_up above the spectrum of this iteration's H: the
        # largest eigenvalue of the sparse H by a few Lanczos steps of scipy
        lam_max = float(sla.eigsh(_as_operator(parts), k=1, which="LA", tol=1e-6,
                                  return_eigenvectors=False)[0])
        if lam_max > b_up:
            raise ValueError(f"filter upper bound {b_up} below the spectrum of H "
                             f"({lam_max}) at SCF iteration {it}")
        for _ in range(passes[0] if it == 0 else passes[1]):
            out = subspace.sq3_iteration(apply_H, X, degree, a, b_up, a0, npl, sigma, Ne, dV)
            X = out["X"]
        err = float(np.sum(np.abs(out["rho"] - rho)) * dV / Ne)
        hist.append(err)
        if err < tol:
            phi_out = poisson_fd(out["rho"] + b, n, L, order)
            terms = free_energy(out["e_band"], out["e_ent"], out["rho"], b, phi_out, dV, natoms,
                                Z, rc)
            return {"rho": out["rho"], "mu": out["mu"], "X": X, "D": out["D"], "b": b,
                    "iterations": it + 1, "errors": hist, **terms}
        rho = mixer.step(rho, out["rho"])
    raise RuntimeError(f"SCF did not converge in {max_iter} iterations (last {hist[-1]:.3e})")
