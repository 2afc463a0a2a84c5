"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gem_fdtd.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|void|int64_t|const char\s*\*)\s*\**\s*(fdtd_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_00814_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fdtd_create", "fdtd_set_source", "fdtd_step", "fdtd_step_edgelist", "fdtd_add_probe",
                 "fdtd_add_dft_monitor", "fdtd_read_probe", "fdtd_read_dft", "fdtd_export_graph",
                 "fdtd_destroy", "fdtd_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.fdtd_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.fdtd_step(None, 1) == -1
    lib.fdtd_last_error.restype = ctypes.c_char_p
    lib.fdtd_last_error.argtypes = [ctypes.c_void_p]
    assert lib.fdtd_last_error(None) == b"NULL context"
    lib.fdtd_create.argtypes = [ctypes.c_void_p] * 9
    lib.fdtd_create.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double] + [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 2
    assert lib.fdtd_create(None, 1e-3, 0.0, 0.99, None, None, 1, None, None) == -1
