"""The C ABI library builds, loads and exports every entry point that
include/glemur.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(glemur_[A-Za-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("glemur_init_grid", "glemur_set_B0", "glemur_step", "glemur_energy",
                     "glemur_forcefree_err"):
        assert required in names


def test_every_environment_switch_is_documented():
    """Each GLEMUR_* variable the library reads is described in the header."""
    csrc = os.path.join(ROOT, "paper_1405_0942_gb300", "csrc")
    used = set()
    for fn in os.listdir(csrc):
        if fn.endswith((".cu", ".cuh")):
            used |= set(re.findall(r'getenv\("(GLEMUR_[A-Z0-9_]+)"\)',
                                   open(os.path.join(csrc, fn)).read()))
    header = open(os.path.join(ROOT, "include", "glemur.h")).read()
    assert used, "no switches found"
    assert not [v for v in sorted(used) if v + "=" not in header]


def test_library_exports_every_declared_symbol():
    from paper_1405_0942_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    """Calls that touch no device: defaults, workspace sizing, argument
    checks and status strings."""
    import paper_1405_0942_gb300.glemur as g
    L = g.lib()
    o = g.default_opts()
    assert o.precision == g.FP64 and o.curl == g.MIMETIC and o.lambda0 == 1e-7
    n = 16
    b64 = g.workspace_bytes(n, n, n, g.FP64)
    b32 = g.workspace_bytes(n, n, n, g.MIXED)
    assert b64 % 256 == 0 and b32 % 256 == 0 and b64 > b32 >= 8 * 3 * n ** 3 * 4
    assert g.workspace_bytes(2, n, n, g.FP64) == 0
    assert g.workspace_bytes(n, n, n, 7) == 0
    # the largest grid: kernels index 3N components with 32-bit ints
    assert g.workspace_bytes(894, 894, 894, g.MIXED) > 0          # 3N < 2^31
    assert g.workspace_bytes(895, 895, 895, g.MIXED) == 0
    assert g.workspace_bytes(1 << 20, 1 << 20, 3, g.FP64) == 0    # no int overflow
    assert L.glemur_strerror(-8) == b"a device-side wait for a tile load timed out"
    h = ctypes.c_void_p()
    lo = (ctypes.c_double * 3)(-1, -1, -1)
    hi = (ctypes.c_double * 3)(1, 1, 1)
    # invalid sizes / boxes / workspace are rejected before any device work
    assert L.glemur_init_grid(ctypes.byref(h), 2, 4, 4, lo, hi, None, None, None, 0) == -1
    bad_hi = (ctypes.c_double * 3)(1, -2, 1)
    assert L.glemur_init_grid(ctypes.byref(h), 4, 4, 4, lo, bad_hi, None, None, None, 0) == -1
    assert L.glemur_init_grid(ctypes.byref(h), 4, 4, 4, lo, hi, None, None, None, 0) == -6
    assert L.glemur_strerror(-3) == b"grid collapsed (det dx/dX <= 0)"
    assert L.glemur_step(None, 1, None) == -1
    assert L.glemur_kernels_per_attempt(None) == 0
