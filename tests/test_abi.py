"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/sfx.h (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sfx_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2605_27534_gb300 import build, _lib
    so = build.build()
    L = ctypes.CDLL(so)
    declared = _declared()
    assert len(declared) >= 12
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(_lib.EXPORTS)


def test_binding_loads_and_reports_status_text():
    import paper_2605_27534_gb300 as m
    L = m.lib()
    assert b"sm_103a" in L.sfx_version()
    assert L.sfx_status_string(0) == b"ok"
    assert L.sfx_status_string(1) == b"invalid argument"


def test_context_rejects_bad_grid_before_touching_the_device():
    import paper_2605_27534_gb300 as m
    L = m.lib()
    h = ctypes.c_void_p()
    g = m.Grid(0, 0, 8, 1, 0.1)
    assert L.sfx_ctx_create(ctypes.byref(g), 0, ctypes.byref(h)) == 1
    g = m.Grid(2, 8, 8, 8, -1.0)
    assert L.sfx_ctx_create(ctypes.byref(g), 0, ctypes.byref(h)) == 1
    assert L.sfx_ctx_create(None, 0, ctypes.byref(h)) == 1


def test_product_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2605_27534_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "sfx_oracle" not in txt, fn
