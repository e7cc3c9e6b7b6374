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


class _Cfg(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skin", ctypes.c_double), ("max_atoms", ctypes.c_int64),
                ("max_cells", ctypes.c_int64), ("carry", ctypes.c_int)]


def test_host_side_contract_without_a_gpu():
    """What the library decides on the host: the default configuration, invalid
    configurations refused before any CUDA call, NULL handles tolerated; with no usable GPU,
    context creation fails with a code, not a crash."""
    from paper_2401_10462_gb300 import build
    lib = ctypes.CDLL(build.build())
    vp = ctypes.c_void_p
    lib.dsasa_default_config.argtypes = [ctypes.POINTER(_Cfg)]
    lib.dsasa_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(_Cfg)]
    lib.dsasa_destroy.argtypes = [vp]
    lib.dsasa_status_sync.argtypes = [vp]
    cfg = _Cfg()
    lib.dsasa_default_config(ctypes.byref(cfg))
    assert (cfg.precision, cfg.skin, cfg.max_atoms, cfg.max_cells, cfg.carry) == (0, 0.0, 0, 0, 1)
    h = vp()
    for field, bad in (("precision", 7), ("skin", -1.0), ("carry", 3), ("max_atoms", -5), ("max_cells", -1)):
        c = _Cfg()
        lib.dsasa_default_config(ctypes.byref(c))
        setattr(c, field, bad)
        assert lib.dsasa_create(ctypes.byref(h), 0, None, ctypes.byref(c)) == 1   # DSASA_ERR_ARG
        assert not h.value
    assert lib.dsasa_create(None, 0, None, None) == 1
    lib.dsasa_destroy(None)                                  # tolerated
    assert lib.dsasa_status_sync(None) == 1
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:   # noqa: BLE001
        has_gpu = False
    if not has_gpu:
        st = lib.dsasa_create(ctypes.byref(h), 0, None, None)
        assert st == 5 and not h.value                        # DSASA_ERR_CUDA, no context
