"""The C-ABI library loads and exports every entry point include/pdfx.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1006_0532_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pdfx_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("pdfx_create", "pdfx_set_grid", "pdfx_set_fields", "pdfx_init_particles",
              "pdfx_step", "pdfx_get_nodal_stats", "pdfx_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    """Calls that need no device: defaults, error strings."""
    from paper_1006_0532_gb300 import _binding as B
    p = B.make_params({"bins": (5, 5, 5)})
    assert abs(p.C1 - 1.85) < 1e-15 and abs(p.Cw2 - 0.73) < 1e-15 and p.bins[2] == 5
    lib.pdfx_strerror.restype = ctypes.c_char_p
    assert lib.pdfx_strerror(0) == b"ok"
    assert b"element" in lib.pdfx_strerror(-6)


def test_host_only_argument_checks(lib):
    """Entry points refuse a null context or bad arguments before touching the device, and
    the defaults of the newer parameters are those documented (model 0, alpha 0.5 for Eq.
    47, CFL 0.7 for Eq. 26)."""
    from paper_1006_0532_gb300 import _binding as B
    p = B.make_params({})
    assert p.model == 0 and abs(p.alpha - 0.5) < 1e-15 and abs(p.cfl - 0.7) < 1e-15
    assert p.cond_mode == 0 and p.fox_bins == 5 and p.acc64 == 0
    ERR_ARG = -1
    L = B.lib()
    d = ctypes.c_double()
    assert L.pdfx_last_dt(None, ctypes.byref(d)) == ERR_ARG
    assert L.pdfx_batch_step(None, 0, 1e-3, None) == ERR_ARG
    assert L.pdfx_derive_fields(None, None) == ERR_ARG
    assert L.pdfx_get_fields(None, None, None) == ERR_ARG
    assert L.pdfx_correct_velocity(None, None, 1e-3, None) == ERR_ARG
    assert L.pdfx_scalar_stats(None, 1, None, 10, None, None, None, None, None, 0, None) == ERR_ARG


def test_host_only_argument_checks_of_the_eulerian_calls(lib):
    """The coupled loop's entry points refuse a null context, null arrays or a bad
    tolerance before touching the device; the new error code has its own message."""
    from paper_1006_0532_gb300 import _binding as B
    ERR_ARG = -1
    L = B.lib()
    it = ctypes.c_int32()
    assert L.pdfx_wp_rhs(None, None, None, None) == ERR_ARG
    assert L.pdfx_wp_solve(None, None, None, None, 1e-10, 10, ctypes.byref(it), None) == ERR_ARG
    assert L.pdfx_update_wp(None, 1e-10, 10, ctypes.byref(it), None) == ERR_ARG
    assert L.pdfx_pressure_rhs(None, None, None, 1e-3, 1e-3, None, None, None) == ERR_ARG
    assert L.pdfx_pressure_solve(None, None, None, None, 1e-10, 10, ctypes.byref(it), None) == ERR_ARG
    assert L.pdfx_set_pressure(None, None, None) == ERR_ARG
    assert L.pdfx_get_pressure(None, None, None, None) == ERR_ARG
    assert L.pdfx_coupled_step(None, 1e-3, 1e-3, 1e-10, 10, None, None) == ERR_ARG
    assert L.pdfx_strerror(-9) == b"an iterative solve did not converge within its iteration limit"
