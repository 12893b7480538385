"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/rr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rr_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_1902_01458_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for n in ("rr_create_operator", "rr_destroy_operator", "rr_factor",
              "rr_destroy_factors", "rr_sketch", "rr_modes", "rr_solve", "rr_apply",
              "rr_phi", "rr_gaussian", "rr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in _declared_symbols() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1902_01458_gb300 import _lib
    declared = _declared_symbols()
    assert set(_lib.SIGNATURES) <= declared
    # every declared entry point has a binding
    assert declared <= set(_lib.SIGNATURES) | {"rr_status_string"}


def test_status_strings_and_argument_errors(built_lib):
    """Host-side argument checks run without touching a device."""
    from paper_1902_01458_gb300 import _lib
    lib = _lib.load()
    assert lib.rr_status_string(0) == b"ok"
    assert lib.rr_status_string(3) == b"singular pivot"
    out = ctypes.c_void_p()
    st = lib.rr_create_operator(None, None, None, 0, ctypes.byref(out))
    assert st == 1 and b"null" in lib.rr_last_error()
    g = _lib.rr_grid(2, 8, 8, 0, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.1)
    fl = _lib.rr_baseflow(None, None, None)
    st = lib.rr_create_operator(ctypes.byref(g), ctypes.byref(fl), None, 0,
                                ctypes.byref(out))
    assert st == 1 and b"kind" in lib.rr_last_error()


def test_product_path_refuses_to_run_without_library(tmp_path):
    from paper_1902_01458_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
