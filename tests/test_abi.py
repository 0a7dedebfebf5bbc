"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
and exports every entry point that include/sq3.h declares.  No compute call
is made (there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sq3.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sq3_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2112_08639_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    syms = declared_symbols()
    for s in ("sq3_create", "sq3_destroy", "sq3_setup_grid", "sq3_set_potential",
              "sq3_set_projectors", "sq3_hamiltonian_apply", "sq3_cheb_filter",
              "sq3_orthonormalise", "sq3_project", "sq3_kernel_from_hs",
              "sq3_density_kernel", "sq3_density", "sq3_status_string"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\b(sq3_[a-z0-9_]+)\b", out))
    assert set(declared_symbols()) <= exported


def test_status_strings_and_version(libpath):
    lib = ctypes.CDLL(libpath)
    lib.sq3_status_string.restype = ctypes.c_char_p
    lib.sq3_version.restype = ctypes.c_char_p
    assert lib.sq3_status_string(0) == b"ok"
    assert b"Cholesky" in lib.sq3_status_string(-4)
    assert b"sm_103a" in lib.sq3_version()


def test_built_for_sm_103a():
    from paper_2112_08639_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_argument_errors_before_any_device_work(libpath):
    """Every entry point checks its context and arguments before touching
    the device: with a NULL context, NULL arrays or out-of-range sizes each
    returns its documented status, here on a host without a GPU."""
    lib = ctypes.CDLL(libpath)
    p, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    EINVAL, ENOTSETUP, ECUDA = -1, -2, -3
    h = ctypes.c_void_p(1)
    lib.sq3_create.argtypes = [ctypes.POINTER(p), i, p]
    assert lib.sq3_create(None, 0, None) == EINVAL
    assert lib.sq3_create(ctypes.byref(h), -1, None) == EINVAL and h.value is None
    assert lib.sq3_create(ctypes.byref(h), 0, None) == ECUDA and h.value is None   # no GPU here
    lib.sq3_destroy.argtypes = [p]
    lib.sq3_destroy(None)
    calls = {
        "sq3_setup_grid": ([p, i, i, i, d, d, d, i], (None, 8, 8, 8, 1.0, 1.0, 1.0, 12), EINVAL),
        "sq3_set_potential": ([p, p], (None, None), ENOTSETUP),
        "sq3_set_projectors": ([p, i, p, p, p, p], (None, 0, None, None, None, None), ENOTSETUP),
        "sq3_projector_table_info": ([i, i, i, d, i, p, p, p, p, p, p],
                                     (8, 8, 8, 0.1, 4, None, None, None, None, None, None),
                                     EINVAL),
        "sq3_hamiltonian_apply": ([p, p, p, i, i], (None, None, None, 4, 0), ENOTSETUP),
        "sq3_cheb_filter": ([p, p, i, i, d, d, d, i], (None, None, 4, 3, 1.0, 2.0, 0.0, 0),
                            ENOTSETUP),
        "sq3_cheb_filter_from_host": ([p, p, p, i, i, d, d, d, i],
                                      (None, None, None, 4, 3, 1.0, 2.0, 0.0, 0), ENOTSETUP),
        "sq3_orthonormalise": ([p, p, i, i], (None, None, 4, 0), ENOTSETUP),
        "sq3_project": ([p, p, i, i, p], (None, None, 4, 0, None), ENOTSETUP),
        "sq3_kernel_from_hs": ([p, p, i, i, d, d, i, p, p, p],
                               (None, None, 4, 10, 0.3, 2.0, 0, None, None, None), EINVAL),
        "sq3_density_kernel": ([p, p, i, i, d, d, i, p, p, p, p],
                               (None, None, 4, 10, 0.3, 2.0, 0, None, None, None, None), ENOTSETUP),
        "sq3_density": ([p, p, p, i, i, p], (None, None, None, 4, 0, None), ENOTSETUP),
        "sq3_selftest_timeout": ([p], (None,), EINVAL),
        "sq3_profile_enable": ([p, i], (None, 1), EINVAL),
        "sq3_profile_read": ([p, p, p, i], (None, None, None, 0), EINVAL),
        "sq3_lanczos_bounds_noalloc": ([p, i, p, p], (None, 4, None, None), EINVAL),
        "sq3_poisson": ([p, p, p, p], (None, None, None, None), EINVAL),
        "sq3_effective_potential": ([p, p, p, p, p, p], (None,) * 6, EINVAL),
        "sq3_free_energy": ([p, p, p, d, d, d, p], (None, None, None, 0.0, 0.0, 0.0, None), EINVAL),
        "sq3_kerker": ([p, p, p, d], (None, None, None, 0.8), EINVAL),
        "sq3_mixer_setup": ([p, i, i, d, d], (None, 7, 2, 0.3, 0.8), EINVAL),
        "sq3_mixer_step": ([p, p, p, p], (None, None, None, None), EINVAL),
        "sq3_hamiltonian_bounds": ([p, p], (None, None), EINVAL),
        "sq3_atom_gaussians": ([p, i, p, p, d, i, d, p, p], (None, 1, None, None, 1.0, 1, 0.0,
                                                            None, None), EINVAL),
        "sq3_mlp_create": ([p, i, p, i, p], (None, 8, None, 0, None), EINVAL),
        "sq3_batch_create": ([i, p, p], (-1, None, None), EINVAL),
        "sq3_extrapolate_density": ([p, p, p, p, d, p], (None, None, None, None, 1.0, None), EINVAL),
        "sq3_batch_add_cell": ([p, i, i, i, d, d, d, p, p, i, i],
                               (None, 24, 24, 24, 1.0, 1.0, 1.0, None, None, 8, 10), EINVAL),
        "sq3_batch_set_bounds": ([p, i, d, d, d], (None, 0, 1.0, 2.0, 0.0), EINVAL),
        "sq3_batch_filter": ([p], (None,), EINVAL),
        "sq3_batch_autotune": ([p, p, p], (None, None, None), EINVAL),
        "sq3_kernel_from_hs_ex": ([p, p, i, i, d, i, d, d, i, p, p, p, p],
                                  (None, None, 4, 10, 0.0, 0, 0.3, 2.0, 0, None, None, None, None),
                                  EINVAL),
        "sq3_verlet": ([i, p, d, p, p, p, i, d], (0, None, 1.0, None, None, None, 0, 0.0), EINVAL),
        "sq3_forces": ([p, i, p, d, d, d, p, p, p, i, i, p, p, p],
                       (None, 1, None, 3.0, 1.0, 3.0, None, None, None, 0, 0, None, None, None),
                       EINVAL),
        "sq3_mlp_num_params": ([p], (None,), EINVAL),
        "sq3_mlp_set_params": ([p, p], (None, None), EINVAL),
        "sq3_mlp_get_params": ([p, p], (None, None), EINVAL),
        "sq3_mlp_features": ([p, i, p], (None, 1, None), EINVAL),
        "sq3_mlp_predict": ([p, d, p], (None, 1.0, None), EINVAL),
        "sq3_mlp_gradient": ([p, p, d, p, p, p], (None, None, 1.0, None, None, None), EINVAL),
        "sq3_mlp_train_step": ([p, p, d, d, p, p], (None, None, 1.0, 1e-3, None, None), EINVAL),
        "sq3_scf_solve": ([p, p, p, p, p, i, p, p, p], (None,) * 5 + (0, None, None, None),
                          EINVAL),
    }
    for name, (argtypes, args, want) in calls.items():
        f = getattr(lib, name)
        f.argtypes = argtypes
        f.restype = i
        assert f(*args) == want, name
    missing = set(declared_symbols()) - set(calls) - {
        "sq3_create", "sq3_destroy", "sq3_status_string", "sq3_version", "sq3_last_cuda_error",
        "sq3_fermi_degree", "sq3_mlp_destroy", "sq3_batch_destroy"}
    assert not missing, missing
