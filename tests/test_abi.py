"""The C-ABI library builds, loads on the CPU, and exports every entry point
include/phisplit.h declares (no compute call: there may be no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2304_02327_gb300 import api, build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"MM_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libso():
    build_mod.build()
    return ctypes.CDLL(api.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("phi_plan_create", "mumode_phi_apply", "expint_step", "phi_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libso):
    missing = [n for n in declared_entry_points() if not hasattr(libso, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = set(declared_entry_points()) - set(api.EXPORTS)
    assert not missing, missing


def test_host_side_status_strings(libso):
    L = api.lib()
    assert L.mm_status_str(0) == b"ok"
    assert L.mm_status_str(-8) == b"workspace missing or too small"
    assert L.mm_version() >= 100


def test_host_side_argument_errors_need_no_gpu(libso):
    """Argument checks run on the host before any CUDA call."""
    L = api.lib()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 1)(4)
    a = (ctypes.c_void_p * 1)(None)
    assert L.phi_plan_create(None, 1, n, a, 0.1, 1, 0, None) == -1          # out NULL
    assert L.phi_plan_create(ctypes.byref(h), 0, n, a, 0.1, 1, 0, None) == -1   # d = 0
    assert L.phi_plan_create(ctypes.byref(h), 1, n, a, 0.1, 9, 0, None) == -1   # ell_max
    assert L.phi_plan_create(ctypes.byref(h), 1, n, a, 0.1, 1, 7, None) == -1   # prec
    n0 = (ctypes.c_int64 * 1)(0)
    a1 = (ctypes.c_void_p * 1)(8)
    assert L.phi_plan_create(ctypes.byref(h), 1, n0, a1, 0.1, 1, 0, None) == -2  # n = 0
    assert L.mumode_phi_apply(None, 0, None, None, 1.0, None, 0, None) == -1
    assert L.expint_step(None, 0, None, None, 0.0, 1, None, 0, None) == -1
    assert L.phi_plan_status(None, 0, None) == -1
    assert L.phi_plan_destroy(None) == 0
