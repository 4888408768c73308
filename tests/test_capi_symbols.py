"""The C-ABI library loads and exports every function declared in
include/p4d.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "p4d.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(p4d_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_boundary():
    syms = declared_symbols()
    for name in ("p4d_setup", "p4d_jacobian_update", "p4d_precond_apply", "p4d_fgmres_solve",
                 "p4d_adjoint_solve", "p4d_jvp", "p4d_residual", "p4d_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    from paper_2602_07225_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2602_07225_gb300 import _native
    assert set(declared_symbols()) == set(_native.SIGNATURES)


def test_status_strings():
    from paper_2602_07225_gb300 import build, _native
    build.build()
    lib = _native.load()
    for code in range(9):
        assert lib.p4d_status_string(code).decode() == _native.STATUS[code]
