"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/mrtfdlb.h declares, and rejects invalid arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import build as B
from paper_1004_5442_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrtfdlb.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Bd.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrt_[a-z_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert names, "no declarations parsed"
    assert sorted(Bd.EXPORTED) == names
    for n in names:
        assert hasattr(lib, n), n


def _params(**kw):
    w = W.uniform(16, 8)
    p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s)
    for k, v in kw.items():
        setattr(p, k, v)
    return p, w


@pytest.mark.parametrize("field,value", [("nx", 2), ("ny", 1), ("dx", 0.0), ("dt", -1.0),
                                         ("gamma", 1.0), ("precision", 7), ("bc_x", 3),
                                         ("kernel", 4), ("kernel", 9), ("tile", 8), ("tile", -1),
                                         ("Pr", float("nan")), ("advection", 2), ("advection", -1)])
def test_invalid_params_rejected(lib, field, value):
    p, w = _params(**{field: value})
    h = ctypes.c_void_p()
    arr = [np.ascontiguousarray(a) for a in (w.rho, w.ux, w.uy, w.T)]
    rc = lib.mrt_create(ctypes.byref(p), *(ctypes.c_void_p(a.ctypes.data) for a in arr), 0, None,
                        ctypes.byref(h))
    assert rc == Bd.MRT_EINVAL
    assert lib.mrt_last_error().decode()


def test_negative_rate_rejected(lib):
    p, w = _params()
    p.s[9] = -1.0
    h = ctypes.c_void_p()
    arr = [np.ascontiguousarray(a) for a in (w.rho, w.ux, w.uy, w.T)]
    rc = lib.mrt_create(ctypes.byref(p), *(ctypes.c_void_p(a.ctypes.data) for a in arr), 0, None,
                        ctypes.byref(h))
    assert rc == Bd.MRT_EINVAL and "s_10" in lib.mrt_last_error().decode()


def test_null_pointers_rejected(lib):
    p, w = _params()
    h = ctypes.c_void_p()
    assert lib.mrt_create(ctypes.byref(p), None, None, None, None, 0, None, ctypes.byref(h)) == Bd.MRT_EINVAL
    assert lib.mrt_create(None, None, None, None, None, 0, None, ctypes.byref(h)) == Bd.MRT_EINVAL
    assert lib.mrt_step(None, 1) == Bd.MRT_EINVAL
    assert lib.mrt_health(None) == Bd.MRT_EINVAL
    lib.mrt_destroy(None)


def test_unsplit_operator_tiles_rejected(lib):
    """The unsplit operator reads diagonal neighbours that tiles 2 and 3 do
    not keep; the check runs before anything touches the device."""
    for tile in (2, 3):
        p, w = _params(advection=Bd.ADV_LW2D, kernel=Bd.KERNEL_TMA, tile=tile)
        h = ctypes.c_void_p()
        arr = [np.ascontiguousarray(a) for a in (w.rho, w.ux, w.uy, w.T)]
        rc = lib.mrt_create(ctypes.byref(p), *(ctypes.c_void_p(a.ctypes.data) for a in arr), 0, None,
                            ctypes.byref(h))
        assert rc == Bd.MRT_EINVAL and "unsplit" in lib.mrt_last_error().decode()


def test_null_handles_of_later_entry_points_rejected(lib):
    t = ctypes.c_long()
    n = ctypes.c_long()
    assert lib.mrt_conserved_totals_async(None, None, ctypes.byref(t)) == Bd.MRT_EINVAL
    assert lib.mrt_totals_wait(None, 0) == Bd.MRT_EINVAL
    assert lib.mrt_save(None, b"/nonexistent/x") == Bd.MRT_EINVAL
    assert lib.mrt_load(None, b"/nonexistent/x") == Bd.MRT_EINVAL
    assert lib.mrt_debug_padding(None, ctypes.byref(n)) == Bd.MRT_EINVAL
    assert lib.mrt_debug_wait_timeout(None) == Bd.MRT_EINVAL
    r, r2 = ctypes.c_double(), ctypes.c_double()
    assert lib.mrt_debug_fma_rate(Bd.FP64, 100, 4, 256, 32, None, None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_fma_rate(7, 100, 4, 256, 32, ctypes.byref(r), None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_fma_rate(Bd.FP32, 0, 4, 256, 32, ctypes.byref(r), None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_fma_rate(Bd.FP32, 10, 9, 256, 32, ctypes.byref(r), None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_fma_rate(Bd.FP32, 10, 4, 100, 32, ctypes.byref(r), None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_fma_rate(Bd.FP32, 10, 4, 1024, 32, ctypes.byref(r), None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_fma_rate(Bd.FP32, 10, 4, 256, 0, ctypes.byref(r), None) == Bd.MRT_EINVAL
    assert lib.mrt_debug_launch_period(3, 1, 128, ctypes.byref(r), ctypes.byref(r2)) == Bd.MRT_EINVAL
    assert lib.mrt_debug_launch_period(10, 1, 2000, ctypes.byref(r), ctypes.byref(r2)) == Bd.MRT_EINVAL
    assert lib.mrt_debug_launch_period(10, 1, 128, None, ctypes.byref(r2)) == Bd.MRT_EINVAL


def test_status_strings(lib):
    for code, name in Bd._STATUS.items():
        assert lib.mrt_status_str(code).decode() == name
