"""The C-ABI library builds, loads and exports every entry point that
include/fcrkpm.h declares (no GPU needed: nothing here calls into compute)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "fcrkpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rk_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2403_19854_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("rk_setup", "rk_apply_K", "rk_solve", "rk_rhs", "rk_eval_u", "rk_solve_adjoint", "rk_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rk_\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_reports_sizes(libpath):
    from paper_2403_19854_gb300 import rk
    L = rk.lib()
    for n in rk.EXPORTED:
        assert hasattr(L, n)
    assert rk.supported_length(256) and rk.supported_length(16)
    assert not rk.supported_length(17)
    assert L.rk_status_string(5) == b"RK_ERR_NOT_CONVERGED"
    o = rk.default_opts()
    assert o.tol == 1e-10 and o.precision == rk.RK_PREC_MIXED


def test_invalid_arguments_rejected_without_gpu(libpath):
    """Argument checks run before any device work: a NULL grid / bad degree / odd or
    unbuilt size returns an error code, never a crash."""
    import ctypes

    from paper_2403_19854_gb300 import rk
    L = rk.lib()
    out = ctypes.c_void_p()
    assert L.rk_setup(None, None, None, None, 1, 2.0, None, ctypes.byref(out)) == 1
    g = rk.Grid()
    for k in range(3):
        g.n[k] = 16
        g.h[k] = 0.1
    dummy = (ctypes.c_uint8 * 8)()
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 3, 2.0, None, ctypes.byref(out)) == 1
    g.n[0] = 17
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 1, 2.0, None, ctypes.byref(out)) == 8
    assert not out.value


def test_grid_dimension_checks_without_gpu(libpath):
    """A box one node thick in z is two-dimensional, one node thick in y and z
    one-dimensional; a y axis of one node under a longer z axis, or a first axis of
    one node, is invalid; a side that is not built, or a 1D side that is not a
    multiple of 4, is unsupported -- all decided before any device work."""
    import ctypes

    from paper_2403_19854_gb300 import rk
    L = rk.lib()
    out = ctypes.c_void_p()
    dummy = (ctypes.c_uint8 * 8)()
    g = rk.Grid()
    for k in range(3):
        g.h[k] = 0.1
    g.n[0], g.n[1], g.n[2] = 32, 1, 4        # n[1] == 1 < n[2]
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 1, 1.5, None, ctypes.byref(out)) == 1
    g.n[0], g.n[1], g.n[2] = 20, 1, 1        # 1D, a side that is not built
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 1, 1.5, None, ctypes.byref(out)) == 8
    g.n[0], g.n[1], g.n[2] = 162, 1, 1       # 1D, built but not a multiple of 4
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 1, 1.5, None, ctypes.byref(out)) == 8
    assert b"multiple of 4" in L.rk_last_error_message()
    g.n[0], g.n[1], g.n[2] = 1, 32, 32
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 1, 1.5, None, ctypes.byref(out)) == 1
    g.n[0], g.n[1], g.n[2] = 32, 20, 1       # 2D, but a y side that is not built
    assert L.rk_setup(ctypes.byref(g), dummy, None, dummy, 1, 1.5, None, ctypes.byref(out)) == 8
    assert not out.value
