"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/*.h, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import glob
import os
import re

import pytest

import oracle
import paper_2509_25347_gb300 as dx
from paper_2509_25347_gb300 import build as dxbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    dxbuild.build()
    return dx.load_library()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(drag_expm_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("drag_expm_apply", "drag_expm_backward", "drag_expm_select", "drag_expm_get_status", "drag_expm_theta",
                 "drag_expm_strerror", "drag_expm_version"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_strerror(lib):
    assert lib.drag_expm_version() >= 1
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert len(lib.drag_expm_strerror(code)) > 0
    assert b"unknown" in lib.drag_expm_strerror(-999)


def test_theta_matches_oracle_bitwise(lib):
    """The library computes theta_m (Eq. B8) by its own route (closed-form
    coefficients); it must agree with the oracle's Cauchy-product route."""
    th = oracle.theta_table()
    for k in range(1, 10):
        assert dx.theta(k) == th[k]
    out = ctypes.c_double()
    assert lib.drag_expm_theta(0, ctypes.byref(out)) == -1
    assert lib.drag_expm_theta(10, ctypes.byref(out)) == -1
    assert lib.drag_expm_theta(1, None) == -2


def test_host_argument_errors(lib):
    """Bad sizes, NULL and misaligned pointers are rejected before any CUDA call."""
    good = ctypes.c_void_p(4096)
    bad_align = ctypes.c_void_p(4097)
    null = ctypes.c_void_p(0)
    s = ctypes.c_void_p(0)
    apply = lib.drag_expm_apply
    assert apply(-1, 4, good, good, good, 1.0, good, good, s) == -1
    assert apply(10, 0, good, good, good, 1.0, good, good, s) == -1
    assert apply(10, 32, good, good, good, 1.0, good, good, s) == -1
    assert apply(10, 4, good, good, good, -1.0, good, good, s) == -1
    assert apply(10, 4, good, good, good, float("nan"), good, good, s) == -1
    assert apply(10, 4, good, good, good, float("inf"), good, good, s) == -1
    assert apply(10, 4, null, good, good, 1.0, good, good, s) == -2
    assert apply(10, 4, good, good, good, 1.0, null, good, s) == -2
    assert apply(10, 4, good, bad_align, good, 1.0, good, good, s) == -3
    assert apply(10, 4, good, good, good, 1.0, good, bad_align, s) == -3
    assert apply(0, 4, null, null, null, 1.0, null, null, s) == 0          # empty: no-op
    sel = lib.drag_expm_select
    assert sel(-5, 4, good, good, good, 1.0, good, good, s) == -1
    assert sel(10, 4, good, null, good, 1.0, good, good, s) == -2
    assert lib.drag_expm_get_status(s, None) == -2
    bwd = lib.drag_expm_backward
    assert bwd(-1, 4, good, good, good, 1.0, good, good, null, null, null, null, s) == -1
    assert bwd(10, 40, good, good, good, 1.0, good, good, null, null, null, null, s) == -1
    assert bwd(10, 4, good, good, good, 1.0, good, null, null, null, null, null, s) == -2
    assert bwd(10, 4, good, good, good, 1.0, good, good, bad_align, null, null, null, s) == -3
    assert bwd(0, 4, null, null, null, 1.0, null, null, null, null, null, null, s) == 0


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(dx.DragExpmError):
        dx.load_library(str(tmp_path / "missing.so"))
