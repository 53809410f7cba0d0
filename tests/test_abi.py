"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
symbol include/rcx.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2408_14425_b300 import build as rbuild
from paper_2408_14425_b300 import rcx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(rc[a-z_0-9]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    rbuild.build()
    return rcx.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert {"rc_plan", "rc_formal_solve", "rc_last_error"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert set(rcx.EXPORTS) <= declared


def test_status_strings(lib):
    assert lib.rc_status_string(0) == b"RC_OK"
    assert lib.rc_status_string(-1) == b"RC_ERR_ARG"
    assert lib.rc_status_string(-6) == b"RC_ERR_UNSUPPORTED"


def _plan(lib, nx=8, nz=8, C=3, W0=4, B=4, L0=1.0, voxel=1.0, **kw):
    g = rcx.rc_grid(nx, nz, voxel)
    o = rcx.rc_options()
    lib.rc_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    st = lib.rc_plan(ctypes.byref(g), C, W0, B, L0, ctypes.byref(o), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=0), -1), (dict(nz=-3), -1), (dict(C=0), -1), (dict(C=17), -1), (dict(W0=0), -1),
    (dict(L0=0.0), -1), (dict(L0=float("inf")), -1), (dict(voxel=0.0), -1),
    (dict(B=2), -6), (dict(precision=3), -1), (dict(interval_rule=2), -1),
    (dict(lambda_block=3), -1), (dict(n_incl=0), -1), (dict(n_incl=17), -1),
    (dict(strips=17), -1), (dict(strips=-1), -1),
    (dict(nx=16384, nz=16384), -1),          # nx * nz * lambda_block must stay below 2^31
])
def test_plan_rejects_bad_arguments(lib, kw, expect):
    st, h = _plan(lib, **kw)
    assert st == expect
    assert h.value is None
    assert len(lib.rc_last_error()) > 0


def test_null_arguments(lib):
    g = rcx.rc_grid(8, 8, 1.0)
    assert lib.rc_plan(None, 3, 4, 4, 1.0, None, ctypes.byref(ctypes.c_void_p())) == -1
    assert lib.rc_plan(ctypes.byref(g), 3, 4, 4, 1.0, None, None) == -1
    assert lib.rc_formal_solve(None, None, None, 1, None, None, None) == -1
    assert lib.rc_formal_solve_host(None, None, None, 1, None, None) == -1
    assert lib.rc_plan_reserve(None, 4) == -1
    lib.rc_plan_destroy(None)  # no-op
    assert lib.rc_plan_scratch_bytes(None) == 0


def test_march_mode_setter_rejects_bad_arguments(lib):
    assert lib.rc_plan_set_march(None, 1) == -1
    assert lib.rc_plan_get_march(None, None) == -1


def test_top_list_calls_reject_a_null_plan(lib):
    assert lib.rc_plan_set_top_list(None, 1) == -1
    assert lib.rc_plan_get_top_list(None, None, None, None) == -1
    assert b"plan is NULL" in lib.rc_last_error()


def test_new_entry_points_reject_null_arguments(lib):
    """The pipelined host solve, its wait and the two halves of the statistical equilibrium
    return RC_ERR_ARG on NULL handles before any device work."""
    assert lib.rc_formal_solve_host_async(None, None, None, 4, None, None) == -1
    assert lib.rc_plan_wait(None) == -1
    assert lib.rc_line_integrals(None, None, None, None, 0, 1, 16, None, None) == -1
    assert lib.rc_stat_eq_integrals(None, None, None, None, None, 16, None, None, None) == -1
    assert b"NULL" in lib.rc_last_error() or b"plan" in lib.rc_last_error()
