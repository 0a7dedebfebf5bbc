"""Thin ctypes binding of the libsq3 C ABI (``include/sq3.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays are torch CUDA tensors; a block of Ns vectors is a
contiguous tensor of shape (Ns, N), which is the library's N x Ns
column-major layout.  Importing this module loads ``_build/libsq3.so`` and
raises if it has not been built (``paper_2112_08639_gb300.build.build()``):
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

FP64 = 0
MIXED = 1
EVAL_RECURRENCE = 0
EVAL_PATERSON_STOCKMEYER = 1

OK, EINVAL, ENOTSETUP, ECUDA, ENOTPD, ENOCONV, ETIMEOUT, ENONFINITE, ENOMEM = \
    0, -1, -2, -3, -4, -5, -6, -7, -8

if not os.path.exists(_build.LIB):
    raise ImportError(f"libsq3.so is not built ({_build.LIB}); run "
                      "paper_2112_08639_gb300.build.build() first")
lib = ctypes.CDLL(_build.LIB)

_p = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_sigs = {
    "sq3_create": (_i, [ctypes.POINTER(_p), _i, _p]),
    "sq3_destroy": (None, [_p]),
    "sq3_setup_grid": (_i, [_p, _i, _i, _i, _d, _d, _d, _i]),
    "sq3_set_potential": (_i, [_p, _p]),
    "sq3_set_projectors": (_i, [_p, _i, _p, _p, _p, _p]),
    "sq3_projector_table_info": (_i, [_i, _i, _i, _d, _i, _p, _p, _p, _p, _p, _p]),
    "sq3_hamiltonian_apply": (_i, [_p, _p, _p, _i, _i]),
    "sq3_cheb_filter": (_i, [_p, _p, _i, _i, _d, _d, _d, _i]),
    "sq3_cheb_filter_from_host": (_i, [_p, _p, _p, _i, _i, _d, _d, _d, _i]),
    "sq3_orthonormalise": (_i, [_p, _p, _i, _i]),
    "sq3_project": (_i, [_p, _p, _i, _i, _p]),
    "sq3_kernel_from_hs": (_i, [_p, _p, _i, _i, _d, _d, _i, _p, _p, _p]),
    "sq3_kernel_from_hs_ex": (_i, [_p, _p, _i, _i, _d, _i, _d, _d, _i, _p, _p, _p, _p]),
    "sq3_density_kernel": (_i, [_p, _p, _i, _i, _d, _d, _i, _p, _p, _p, _p]),
    "sq3_density": (_i, [_p, _p, _p, _i, _i, _p]),
    "sq3_status_string": (ctypes.c_char_p, [_i]),
    "sq3_version": (ctypes.c_char_p, []),
    "sq3_last_cuda_error": (ctypes.c_char_p, []),
    "sq3_profile_enable": (_i, [_p, _i]),
    "sq3_lanczos_bounds_noalloc": (_i, [_p, _i, _p, _p]),
    "sq3_selftest_timeout": (_i, [_p]),
    "sq3_profile_read": (_i, [_p, _p, _p, _i]),
    "sq3_poisson": (_i, [_p, _p, _p, _p]),
    "sq3_effective_potential": (_i, [_p, _p, _p, _p, _p, _p]),
    "sq3_free_energy": (_i, [_p, _p, _p, _d, _d, _d, _p]),
    "sq3_kerker": (_i, [_p, _p, _p, _d]),
    "sq3_mixer_setup": (_i, [_p, _i, _i, _d, _d]),
    "sq3_mixer_step": (_i, [_p, _p, _p, _p]),
    "sq3_fermi_degree": (_i, [_d, _d, _d]),
    "sq3_hamiltonian_bounds": (_i, [_p, _p]),
    "sq3_scf_solve": (_i, [_p, _p, _p, _p, _p, _i, _p, _p, _p]),
    "sq3_atom_gaussians": (_i, [_p, _i, _p, _p, _d, _i, _d, _p, _p]),
    "sq3_verlet": (_i, [_i, _p, _d, _p, _p, _p, _i, _d]),
    "sq3_forces": (_i, [_p, _i, _p, _d, _d, _d, _p, _p, _p, _i, _i, _p, _p, _p]),
    "sq3_extrapolate_density": (_i, [_p, _p, _p, _p, _d, _p]),
    "sq3_batch_create": (_i, [_i, _p, ctypes.POINTER(_p)]),
    "sq3_batch_destroy": (None, [_p]),
    "sq3_batch_add_cell": (_i, [_p, _i, _i, _i, _d, _d, _d, _p, _p, _i, _i]),
    "sq3_batch_set_bounds": (_i, [_p, _i, _d, _d, _d]),
    "sq3_batch_filter": (_i, [_p]),
    "sq3_batch_autotune": (_i, [_p, _p, _p]),
    "sq3_mlp_create": (_i, [_p, _i, _p, _i, ctypes.POINTER(_p)]),
    "sq3_mlp_destroy": (None, [_p]),
    "sq3_mlp_num_params": (_i, [_p]),
    "sq3_mlp_set_params": (_i, [_p, _p]),
    "sq3_mlp_get_params": (_i, [_p, _p]),
    "sq3_mlp_features": (_i, [_p, _i, _p]),
    "sq3_mlp_predict": (_i, [_p, _d, _p]),
    "sq3_mlp_gradient": (_i, [_p, _p, _d, _p, _p, _p]),
    "sq3_mlp_train_step": (_i, [_p, _p, _d, _d, _p, _p]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class ScfParams(ctypes.Structure):
    """sq3_scf_params (include/sq3.h)."""
    _fields_ = [("Ns", _i), ("degree", _i), ("npl", _i), ("first_passes", _i), ("passes", _i),
                ("max_iter", _i), ("mix_history", _i), ("mix_period", _i), ("kT", _d), ("Ne", _d),
                ("tol", _d), ("e_self", _d), ("mix_beta", _d), ("kerker_k0", _d),
                ("fermi_tol", _d), ("filter_cut", _d), ("chi0", _d), ("xi0", _d),
                ("cut_shift", _d), ("kernel_eval", _i), ("reserved", _i)]


class ScfResult(ctypes.Structure):
    """sq3_scf_result (include/sq3.h)."""
    _fields_ = [("iterations", _i), ("converged", _i), ("npl_last", _i), ("reserved", _i),
                ("F", _d), ("e_band", _d), ("e_ent", _d), ("mu", _d), ("e_xc", _d),
                ("vxc_rho", _d), ("e_es", _d), ("err", _d), ("chi", _d), ("xi", _d),
                ("b_up", _d)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


SCF_HIST = 9
SCF_HIST_KEYS = ("err", "mu", "e_band", "e_ent", "F", "npl", "ms", "chi", "xi")


class SQ3Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {lib.sq3_status_string(code).decode()} ({code})"
        if code == ECUDA:
            msg += f" [{lib.sq3_last_cuda_error().decode()}]"
        super().__init__(msg)


def _check(code: int, where: str):
    if code != OK:
        raise SQ3Error(code, where)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _prec_dtype(prec: int):
    return torch.float64 if prec == FP64 else torch.float32


def version() -> str:
    return lib.sq3_version().decode()


def fermi_degree(sigma: float, xi: float, tol: float) -> int:
    """Chebyshev degree for the Fermi function of width sigma on a spectrum of
    half-width xi with occupation error below tol (host arithmetic only)."""
    n = lib.sq3_fermi_degree(sigma, xi, tol)
    if n < 0:
        raise SQ3Error(n, "sq3_fermi_degree")
    return n


def projector_table_info(grid, dV: float, ptr, idx, val, gamma) -> dict:
    """The tables a context would build from this projector table on the
    grid (nx, ny, nz) (sq3_projector_table_info; host only, no device)."""
    p = np.ascontiguousarray(ptr, dtype=np.int32)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    info = (ctypes.c_int * 6)()
    bounds = (ctypes.c_double * 2)()
    _check(lib.sq3_projector_table_info(int(grid[0]), int(grid[1]), int(grid[2]), float(dV),
                                        len(g), p.ctypes.data, ix.ctypes.data, v.ctypes.data,
                                        g.ctypes.data, info, bounds),
           "sq3_projector_table_info")
    keys = ("balls", "entries", "bricks", "max_brick_balls", "max_brick_entries", "smem_bytes")
    out = dict(zip(keys, list(info)))
    out["vnl_lo"], out["vnl_hi"] = bounds[0], bounds[1]
    return out


def verlet(masses, dt: float, R: np.ndarray, V: np.ndarray, F: np.ndarray, phase: int,
           ke_target: float = 0.0):
    """One velocity-Verlet half step in place on float64 (natoms, 3) arrays
    (sq3_verlet): phase 0 kicks V by F/2 and drifts R, phase 1 kicks V."""
    m = np.ascontiguousarray(masses, dtype=np.float64)
    for a in (R, V, F):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("float64 C-contiguous arrays expected")
    _check(lib.sq3_verlet(len(m), m.ctypes.data, dt, R.ctypes.data, V.ctypes.data,
                          F.ctypes.data, phase, ke_target), "sq3_verlet")


NOALLOC_MAX_NS = 8192


def lanczos_bounds_noalloc(Hs: torch.Tensor, bounds: torch.Tensor | None = None,
                           stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Spectral bounds {chi, xi} of a symmetric device matrix through the
    allocation-free entry point (its scratch is a fixed array inside the
    library; see include/sq3.h).  `bounds` is a caller-owned device tensor of
    2 doubles; one is created here when it is not given."""
    if bounds is None:
        bounds = torch.empty(2, dtype=torch.float64, device=Hs.device)
    st = stream if stream is not None else torch.cuda.current_stream(Hs.device)
    _check(lib.sq3_lanczos_bounds_noalloc(_ptr(Hs), Hs.shape[0], _ptr(bounds),
                                          ctypes.c_void_p(st.cuda_stream)),
           "sq3_lanczos_bounds_noalloc")
    return bounds


class Context:
    """Owns one sq3_ctx bound to a device and a stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(lib.sq3_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream)),
               "sq3_create")
        self._h = h
        self.N = 0

    def close(self):
        if getattr(self, "_h", None):
            lib.sq3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup_grid(self, nx, ny, nz, Lx, Ly, Lz, fd_order=12):
        _check(lib.sq3_setup_grid(self._h, nx, ny, nz, Lx, Ly, Lz, fd_order), "sq3_setup_grid")
        self.N = nx * ny * nz
        self.dV = (Lx / nx) * (Ly / ny) * (Lz / nz)

    def set_potential(self, V: torch.Tensor):
        V = V.to(device=self.device, dtype=torch.float64).contiguous()
        _check(lib.sq3_set_potential(self._h, _ptr(V)), "sq3_set_potential")

    def set_projectors(self, ptr, idx, val, gamma):
        ptr = np.ascontiguousarray(ptr, dtype=np.int32)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        gamma = np.ascontiguousarray(gamma, dtype=np.float64)
        n = len(gamma)
        _check(lib.sq3_set_projectors(self._h, n, ptr.ctypes.data, idx.ctypes.data,
                                      val.ctypes.data, gamma.ctypes.data),
               "sq3_set_projectors")

    def hamiltonian_apply(self, X: torch.Tensor, Y: torch.Tensor | None = None, prec=FP64):
        if Y is None:
            Y = torch.empty_like(X)
        _check(lib.sq3_hamiltonian_apply(self._h, _ptr(X), _ptr(Y), X.shape[0], prec),
               "sq3_hamiltonian_apply")
        return Y

    def cheb_filter(self, X: torch.Tensor, degree: int, a: float, b: float, a0: float, prec=FP64):
        _check(lib.sq3_cheb_filter(self._h, _ptr(X), X.shape[0], degree, a, b, a0, prec),
               "sq3_cheb_filter")
        return X

    def cheb_filter_from_host(self, X_host: torch.Tensor, X: torch.Tensor, degree: int, a: float,
                              b: float, a0: float, prec=FP64):
        """Filter the host block X_host into the device block X (same shape
        and dtype); the upload overlaps the filtering of earlier chunks."""
        if X_host.is_cuda or not X.is_cuda or X_host.shape != X.shape or X_host.dtype != X.dtype:
            raise ValueError("X_host: host tensor, X: device tensor of the same shape and dtype")
        if not (X_host.is_contiguous() and X.is_contiguous()):
            raise ValueError("contiguous blocks expected")
        _check(lib.sq3_cheb_filter_from_host(self._h, ctypes.c_void_p(X_host.data_ptr()), _ptr(X),
                                             X.shape[0], degree, a, b, a0, prec),
               "sq3_cheb_filter_from_host")
        return X

    def orthonormalise(self, X: torch.Tensor, prec=FP64):
        _check(lib.sq3_orthonormalise(self._h, _ptr(X), X.shape[0], prec), "sq3_orthonormalise")
        return X

    def project(self, X: torch.Tensor, prec=FP64, Hs: torch.Tensor | None = None):
        Ns = X.shape[0]
        if Hs is None:
            Hs = torch.empty((Ns, Ns), dtype=torch.float64, device=self.device)
        _check(lib.sq3_project(self._h, _ptr(X), Ns, prec, _ptr(Hs)), "sq3_project")
        return Hs

    @staticmethod
    def _unpack(out):
        return {"mu": out[0], "e_band": out[1], "e_ent": out[2], "chi": out[3],
                "xi": out[4], "two_tr_D": out[5]}

    def kernel_from_hs(self, Hs: torch.Tensor, npl: int, kT: float, Ne: float,
                       bounds=None, D: torch.Tensor | None = None, want_D=True, prec=FP64):
        Ns = Hs.shape[0]
        if D is None and want_D:
            D = torch.empty((Ns, Ns), dtype=torch.float64, device=self.device)
        out = (ctypes.c_double * 6)()
        b = (ctypes.c_double * 2)(*bounds) if bounds is not None else None
        _check(lib.sq3_kernel_from_hs(self._h, _ptr(Hs), Ns, npl, kT, Ne, prec, b, _ptr(D), out),
               "sq3_kernel_from_hs")
        return D, self._unpack(out)

    def kernel_from_hs_ex(self, Hs: torch.Tensor, npl: int, kT: float, Ne: float, prec=FP64,
                          fermi_tol: float = 0.0, eval_mode: int = EVAL_RECURRENCE, bounds=None,
                          D: torch.Tensor | None = None):
        """(D, outputs, degree used): the density kernel with the adaptive
        degree (npl < 1) and/or the Paterson-Stockmeyer evaluation."""
        Ns = Hs.shape[0]
        if D is None:
            D = torch.empty((Ns, Ns), dtype=torch.float64, device=self.device)
        out = (ctypes.c_double * 6)()
        used = ctypes.c_int()
        b = (ctypes.c_double * 2)(*bounds) if bounds is not None else None
        _check(lib.sq3_kernel_from_hs_ex(self._h, _ptr(Hs), Ns, npl, fermi_tol, eval_mode, kT, Ne,
                                         prec, b, _ptr(D), out, ctypes.byref(used)),
               "sq3_kernel_from_hs_ex")
        return D, self._unpack(out), used.value

    def density_kernel(self, X: torch.Tensor, npl: int, kT: float, Ne: float, prec=FP64,
                       bounds=None, Hs: torch.Tensor | None = None,
                       D: torch.Tensor | None = None):
        Ns = X.shape[0]
        if D is None:
            D = torch.empty((Ns, Ns), dtype=torch.float64, device=self.device)
        out = (ctypes.c_double * 6)()
        b = (ctypes.c_double * 2)(*bounds) if bounds is not None else None
        _check(lib.sq3_density_kernel(self._h, _ptr(X), Ns, npl, kT, Ne, prec, b, _ptr(Hs),
                                      _ptr(D), out), "sq3_density_kernel")
        return D, self._unpack(out)

    def density(self, X: torch.Tensor, D: torch.Tensor, prec=FP64, rho: torch.Tensor | None = None):
        if rho is None:
            rho = torch.empty(X.shape[1], dtype=torch.float64, device=self.device)
        _check(lib.sq3_density(self._h, _ptr(X), _ptr(D), X.shape[0], prec, _ptr(rho)),
               "sq3_density")
        return rho

    def _grid_vec(self, t: torch.Tensor | None):
        if t is not None and (t.dtype != torch.float64 or t.numel() != self.N):
            raise ValueError("expected a float64 CUDA tensor of N grid points")
        return _ptr(t)

    def poisson(self, rho: torch.Tensor, b: torch.Tensor | None = None,
                phi: torch.Tensor | None = None) -> torch.Tensor:
        """phi of rho + b (b optional) on the grid, zero mean."""
        if phi is None:
            phi = torch.empty_like(rho)
        _check(lib.sq3_poisson(self._h, self._grid_vec(rho), self._grid_vec(b),
                               self._grid_vec(phi)), "sq3_poisson")
        return phi

    def effective_potential(self, rho: torch.Tensor, b: torch.Tensor | None = None,
                            veff: torch.Tensor | None = None, phi: torch.Tensor | None = None):
        """(veff, terms): V_eff = phi[rho + b] + V_xc[rho] and the terms
        {e_xc, vxc_rho, e_es} of the free energy."""
        if veff is None:
            veff = torch.empty_like(rho)
        t = (ctypes.c_double * 3)()
        _check(lib.sq3_effective_potential(self._h, self._grid_vec(rho), self._grid_vec(b),
                                           self._grid_vec(veff), self._grid_vec(phi), t),
               "sq3_effective_potential")
        return veff, {"e_xc": t[0], "vxc_rho": t[1], "e_es": t[2]}

    def free_energy(self, rho: torch.Tensor, b: torch.Tensor, e_band: float, e_ent: float,
                    e_self: float) -> dict:
        out = (ctypes.c_double * 4)()
        _check(lib.sq3_free_energy(self._h, self._grid_vec(rho), self._grid_vec(b), e_band,
                                   e_ent, e_self, out), "sq3_free_energy")
        return {"F": out[0], "e_xc": out[1], "vxc_rho": out[2], "e_es": out[3]}

    def kerker(self, r: torch.Tensor, k0: float = 0.8,
               out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(r)
        _check(lib.sq3_kerker(self._h, self._grid_vec(r), self._grid_vec(out), k0), "sq3_kerker")
        return out

    def mixer_setup(self, history: int = 7, period: int = 2, beta: float = 0.3,
                    k0: float = 0.8):
        _check(lib.sq3_mixer_setup(self._h, history, period, beta, k0), "sq3_mixer_setup")

    def mixer_step(self, x_in: torch.Tensor, x_out: torch.Tensor,
                   x_next: torch.Tensor | None = None) -> torch.Tensor:
        if x_next is None:
            x_next = torch.empty_like(x_in)
        _check(lib.sq3_mixer_step(self._h, self._grid_vec(x_in), self._grid_vec(x_out),
                                  self._grid_vec(x_next)), "sq3_mixer_step")
        return x_next

    def atom_gaussians(self, positions, width: float, q=None, normalised: bool = True,
                       total: float = 0.0, out: torch.Tensor | None = None):
        """(out, sum dV before rescaling) of sum_J q_J Gaussians of the given
        width around the atoms (periodic images included)."""
        pos = np.ascontiguousarray(positions, dtype=np.float64)
        qa = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device=self.device)
        s = ctypes.c_double()
        _check(lib.sq3_atom_gaussians(self._h, pos.shape[0], pos.ctypes.data,
                                      None if qa is None else qa.ctypes.data, width,
                                      int(normalised), total, self._grid_vec(out),
                                      ctypes.byref(s)), "sq3_atom_gaussians")
        return out, s.value

    def pseudocharge(self, positions, Z: float, rc: float, out: torch.Tensor | None = None):
        """Gaussian pseudocharges b (sum b dV = -Z natoms) and the sum before
        rescaling."""
        n = len(positions)
        return self.atom_gaussians(positions, rc, q=np.full(n, -Z), normalised=True,
                                   total=-Z * n, out=out)

    def forces(self, positions, Z: float, rc: float, Ne: float, phi: torch.Tensor,
               X: torch.Tensor | None = None, D: torch.Tensor | None = None, prec=FP64,
               atom_of=None):
        """(forces (natoms, 3), local part, nonlocal part) in Ha/bohr."""
        pos = np.ascontiguousarray(positions, dtype=np.float64)
        n = pos.shape[0]
        f = np.empty((n, 3))
        parts = np.empty((n, 3, 2))
        ao = None if atom_of is None else np.ascontiguousarray(atom_of, dtype=np.int32)
        Ns = 0 if X is None else X.shape[0]
        _check(lib.sq3_forces(self._h, n, pos.ctypes.data, Z, rc, Ne, self._grid_vec(phi),
                              _ptr(X), _ptr(D), Ns, prec, None if ao is None else ao.ctypes.data,
                              f.ctypes.data, parts.ctypes.data), "sq3_forces")
        return f, parts[..., 0], parts[..., 1]

    def extrapolate_density(self, prev: torch.Tensor, a: torch.Tensor, b: torch.Tensor,
                            Ne: float, out: torch.Tensor | None = None) -> torch.Tensor:
        """max(prev + a - b, 0) rescaled to Ne electrons."""
        if out is None:
            out = torch.empty_like(prev)
        _check(lib.sq3_extrapolate_density(self._h, self._grid_vec(prev), self._grid_vec(a),
                                           self._grid_vec(b), Ne, self._grid_vec(out)),
               "sq3_extrapolate_density")
        return out

    def hamiltonian_bounds(self) -> tuple[float, float]:
        """Rigorous (lower, upper) bounds of the spectrum of H."""
        out = (ctypes.c_double * 2)()
        _check(lib.sq3_hamiltonian_bounds(self._h, out), "sq3_hamiltonian_bounds")
        return out[0], out[1]

    def scf_solve(self, b: torch.Tensor, rho: torch.Tensor, X: torch.Tensor, *, degree: int,
                  npl: int, kT: float, Ne: float, e_self: float, tol: float = 1e-6,
                  prec=FP64, first_passes: int = 4, passes: int = 1, max_iter: int = 100,
                  mix_history: int = 7, mix_period: int = 2, mix_beta: float = 0.3,
                  kerker_k0: float = 0.8, fermi_tol: float = 0.0, filter_cut: float = 0.0,
                  cut_shift: float = 0.0, kernel_eval: int = 0, bounds0=None, D: torch.Tensor | None = None, raise_on_noconv: bool = True):
        """Converged SCF solve (sq3_scf_solve).  rho (in: start, out: the
        converged density) and X (in: starting block, out: last block) are
        updated in place.  Returns (result dict, list of per-iteration dicts)."""
        if X.dtype != _prec_dtype(prec):
            raise ValueError("X dtype does not match the precision")
        p = ScfParams(Ns=X.shape[0], degree=degree, npl=npl, first_passes=first_passes,
                      passes=passes, max_iter=max_iter, mix_history=mix_history,
                      mix_period=mix_period, kT=kT, Ne=Ne, tol=tol, e_self=e_self,
                      mix_beta=mix_beta, kerker_k0=kerker_k0, fermi_tol=fermi_tol,
                      filter_cut=filter_cut,
                      chi0=bounds0[0] if bounds0 is not None else 0.0,
                      xi0=bounds0[1] if bounds0 is not None else 0.0, cut_shift=cut_shift,
                      kernel_eval=kernel_eval)
        r = ScfResult()
        hist = (ctypes.c_double * (max_iter * SCF_HIST))()
        code = lib.sq3_scf_solve(self._h, ctypes.byref(p), self._grid_vec(b), self._grid_vec(rho),
                                 _ptr(X), prec, _ptr(D), ctypes.byref(r), hist)
        rows = [dict(zip(SCF_HIST_KEYS, hist[i * SCF_HIST:(i + 1) * SCF_HIST]))
                for i in range(r.iterations)]
        if code != OK and not (code == ENOCONV and not raise_on_noconv):
            raise SQ3Error(code, "sq3_scf_solve")
        return r.as_dict(), rows

    STAGES = ("stencil", "nl_project", "gram", "cholesky", "tri_inverse", "x_rinv",
              "hs_gemm", "lanczos", "cheb_gemm", "fermi", "d_accum", "rho", "split", "copy", "nl_pass")

    def selftest_timeout(self) -> int:
        """Runs the bounded-wait failure path; returns the status code
        (ETIMEOUT when it works)."""
        return lib.sq3_selftest_timeout(self._h)

    def profile(self, enable: bool = True):
        _check(lib.sq3_profile_enable(self._h, int(enable)), "sq3_profile_enable")

    def profile_read(self) -> dict:
        n = len(self.STAGES)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_longlong * n)()
        r = lib.sq3_profile_read(self._h, ms, la, n)
        if r < 0:
            raise SQ3Error(r, "sq3_profile_read")
        return {s: (ms[i], la[i]) for i, s in enumerate(self.STAGES)}


class MLP:
    """Learned starting density (sq3_mlp_*): a 3 x 128 tanh perceptron over
    atom-centred Gaussian descriptors of the given widths, bound to a
    context's grid.  Parameters are one float32 array (W1 [128][F], b1, W2,
    b2, W3, b3, w4, b4)."""

    def __init__(self, ctx: Context, widths, seed: int = 0):
        self.ctx = ctx
        self.widths = np.ascontiguousarray(widths, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib.sq3_mlp_create(ctx._h, len(self.widths), self.widths.ctypes.data, seed,
                                  ctypes.byref(h)), "sq3_mlp_create")
        self._h = h
        self.n_params = lib.sq3_mlp_num_params(h)
        self._scratch = None

    def close(self):
        if getattr(self, "_h", None):
            lib.sq3_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(lib.sq3_mlp_set_params(self._h, a.ctypes.data), "sq3_mlp_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        _check(lib.sq3_mlp_get_params(self._h, a.ctypes.data), "sq3_mlp_get_params")
        return a

    def features(self, positions):
        pos = np.ascontiguousarray(positions, dtype=np.float64)
        _check(lib.sq3_mlp_features(self._h, pos.shape[0], pos.ctypes.data), "sq3_mlp_features")

    def predict(self, Ne: float, rho: torch.Tensor | None = None) -> torch.Tensor:
        if rho is None:
            rho = torch.empty(self.ctx.N, dtype=torch.float64, device=self.ctx.device)
        _check(lib.sq3_mlp_predict(self._h, Ne, self.ctx._grid_vec(rho)), "sq3_mlp_predict")
        return rho

    def _rho_scratch(self):
        if self._scratch is None or self._scratch.numel() != self.ctx.N:
            self._scratch = torch.empty(self.ctx.N, dtype=torch.float64, device=self.ctx.device)
        return self._scratch

    def gradient(self, rho_ref: torch.Tensor, Ne: float):
        """(loss, gradient as a float64 array) against rho_ref."""
        g = np.empty(self.n_params, dtype=np.float64)
        loss = ctypes.c_double()
        _check(lib.sq3_mlp_gradient(self._h, self.ctx._grid_vec(rho_ref), Ne,
                                    self.ctx._grid_vec(self._rho_scratch()), ctypes.byref(loss),
                                    g.ctypes.data), "sq3_mlp_gradient")
        return loss.value, g

    def train_step(self, rho_ref: torch.Tensor, Ne: float, lr: float) -> float:
        loss = ctypes.c_double()
        _check(lib.sq3_mlp_train_step(self._h, self.ctx._grid_vec(rho_ref), Ne, lr,
                                      self.ctx._grid_vec(self._rho_scratch()),
                                      ctypes.byref(loss)), "sq3_mlp_train_step")
        return loss.value


class Batch:
    """Many independent cells filtered together (sq3_batch_*): one persistent
    launch takes every vector of every cell through all its filter steps,
    replayed from a captured CUDA graph."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(lib.sq3_batch_create(device, ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), "sq3_batch_create")
        self._h = h
        self.blocks = []

    def close(self):
        if getattr(self, "_h", None):
            lib.sq3_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_cell(self, n: tuple, L: tuple, V: torch.Tensor, X: torch.Tensor, degree: int) -> int:
        """Adds a cell (grid n = (nx, ny, nz), lengths L); X (Ns, N) float32 is
        filtered in place by filter()."""
        if X.dtype != torch.float32:
            raise ValueError("the batched filter takes float32 blocks")
        V = V.to(device=self.device, dtype=torch.float64).contiguous()
        idx = lib.sq3_batch_add_cell(self._h, n[0], n[1], n[2], L[0], L[1], L[2], _ptr(V),
                                     _ptr(X), X.shape[0], degree)
        if idx < 0:
            raise SQ3Error(idx, "sq3_batch_add_cell")
        self.blocks.append(X)
        return idx

    def set_bounds(self, cell: int, a: float, b: float, a0: float):
        _check(lib.sq3_batch_set_bounds(self._h, cell, a, b, a0), "sq3_batch_set_bounds")

    def filter(self):
        _check(lib.sq3_batch_filter(self._h), "sq3_batch_filter")

    def autotune(self) -> tuple[int, int]:
        c, t = ctypes.c_int(), ctypes.c_int()
        _check(lib.sq3_batch_autotune(self._h, ctypes.byref(c), ctypes.byref(t)),
               "sq3_batch_autotune")
        return c.value, t.value
