"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/dsasa.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dsasa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(dsasa_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("dsasa_create", "dsasa_compute", "dsasa_destroy", "dsasa_compute_vjp", "dsasa_compute_batch",
                 "dsasa_status_sync", "dsasa_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2401_10462_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.dsasa_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.dsasa_version()
    # host-only diagnostics: no kernel has been launched by this process
    lib.dsasa_kernel_launches.restype = ctypes.c_int64
    assert lib.dsasa_kernel_launches() == 0
