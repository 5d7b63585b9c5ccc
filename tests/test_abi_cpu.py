"""CPU-side checks of the C-ABI library: it loads and exports every entry
point that include/nir.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2606_20917_gb300", "libnir.so")


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(nir_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import importlib.util
        spec = importlib.util.spec_from_file_location("nb", os.path.join(ROOT, "paper_2606_20917_gb300", "build.py"))
        m = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(m)
        m.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_operator_set():
    names = declared_functions()
    for n in ("nir_bwd_trans", "nir_iproduct_wrt_base", "nir_phys_deriv", "nir_iproduct_wrt_deriv_base",
              "nir_mass", "nir_helmholtz", "nir_helmholtz_host", "nir_block_set_geometry", "nir_mesh_create",
              "nir_mesh_helmholtz", "nir_cg_solve", "nir_tune", "nir_probe_fp64_peak", "nir_strerror",
              "nir_asm_create", "nir_asm_gather", "nir_asm_assemble", "nir_asm_apply", "nir_asm_cg_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version_without_gpu(lib):
    lib.nir_strerror.restype = ctypes.c_char_p
    lib.nir_strerror.argtypes = [ctypes.c_int]
    assert lib.nir_strerror(0) == b"success"
    assert b"geometry" in lib.nir_strerror(-8) or b"Jacobian" in lib.nir_strerror(-7)
    lib.nir_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.nir_version()


def test_null_arguments_rejected_without_gpu(lib):
    lib.nir_helmholtz.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    lib.nir_helmholtz.restype = ctypes.c_int
    assert lib.nir_helmholtz(None, 0, 1.0, None, None) == -1
    lib.nir_block_num_modes.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.nir_block_num_modes(None, None) == -1
    lib.nir_cg_solve.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p]
    assert lib.nir_cg_solve(None, 1.0, None, None, None, None) < 0


def test_python_binding_imports_and_fails_loudly_without_gpu():
    import torch
    import paper_2606_20917_gb300 as nir
    assert "sm_103a" in nir.version()
    if not torch.cuda.is_available():
        with pytest.raises(Exception):
            nir.Context(0)
