"""The C-ABI library loads and exports every entry point include/sgml.h declares (no GPU needed:
no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_1703_07206_gb300 import build, sgml

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "sgml.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgml_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(sgml.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("sgml_create_grid", "sgml_set_coeffs", "sgml_set_source", "sgml_set_bc", "sgml_run_cycle",
                     "sgml_solve_to_tol", "sgml_residual_norm"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) == set(sgml._SIGNATURES)


def test_argument_errors_need_no_gpu():
    lib = sgml.load()
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 1)(5)
    assert lib.sgml_create_grid(4, 1, n, 0, None, ctypes.byref(h)) == sgml.ERR_ARG
    assert b"dim" in lib.sgml_last_error()
    assert lib.sgml_create_grid(2, 1, n, 7, None, ctypes.byref(h)) == sgml.ERR_ARG
    bad = (ctypes.c_int * 1)(0)
    assert lib.sgml_create_grid(2, 1, bad, 0, None, ctypes.byref(h)) == sgml.ERR_ARG
    assert lib.sgml_run_cycle(None, 1) == sgml.ERR_ARG
    assert lib.sgml_destroy(None) == sgml.OK
