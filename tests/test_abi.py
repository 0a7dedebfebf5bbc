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
