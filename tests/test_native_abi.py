"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/frpmg.h declares; argument validation rejects bad calls before touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "frpmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:(?:const|unsigned|long)\s+)*\w+(?:\s+|\s*\*\s*)(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_09733_gb300 import build as B, _native as N
    B.build()
    return N.load()


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ["fr_residual", "fr_jvp", "pmg_precondition", "gmres_solve", "esdirk_step", "row_step"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2202_09733_gb300 import _native as N
    names = _declared()
    assert sorted(names) == sorted(N.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2202_09733_gb300 import _native as N
    h = C.c_void_p()
    assert lib.fr_create(C.byref(h), None, None) == -1
    assert b"NULL" in lib.fr_last_error()
    md = N.MeshDesc(4, 1, 2, None, 0, None, 1, None)
    ph = N.Physics(1.4, 0.72, 0.0, 2.0)
    assert lib.fr_create(C.byref(h), C.byref(md), C.byref(ph)) == -1
    assert b"dim" in lib.fr_last_error()
    assert lib.fr_residual(None, 0, None, None, None) == -1
    assert lib.gmres_solve(None, None, None, None, None, None, None, None) == -1
