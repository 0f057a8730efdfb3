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
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9):
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


def test_theta_targets_match_oracle(lib):
    """theta_{m_k} for the lower accuracy targets of Eq. B8 (u = 2^-24, 2^-11):
    the library's closed-form route against the oracle's Cauchy-product route
    (bisection on the same bound, so they agree to the last bits)."""
    for ubits in (53, 24, 11):
        th = oracle.theta_table(2.0 ** -ubits)
        for k in range(1, 10):
            got = dx.theta(k, ubits)
            assert abs(got - th[k]) <= 2 * 2.0 ** -52 * th[k], (ubits, k, got, th[k])
    out = ctypes.c_double()
    assert lib.drag_expm_theta_target(3, 20, ctypes.byref(out)) == -8
    assert lib.drag_expm_theta_target(3, 64, ctypes.byref(out)) == -8
    assert lib.drag_expm_theta_target(10, 24, ctypes.byref(out)) == -1
    # a lower target never needs a smaller theta
    for k in range(1, 10):
        assert dx.theta(k, 53) < dx.theta(k, 24) < dx.theta(k, 11)


def test_pade_theta_matches_oracle(lib):
    """theta_m of the Pade variant: the library's route (closed-form remainder
    e^x D - N times e^-x/D) against the oracle's (series division), both in
    double-double."""
    for ubits in (53, 24):
        for m in oracle.PADE_DEGREES:
            assert dx.pade_theta(m, ubits) == oracle.pade_theta(m, 2.0 ** -ubits)
    out = ctypes.c_double()
    assert lib.drag_expm_pade_theta(4, 53, ctypes.byref(out)) == -1
    assert lib.drag_expm_pade_theta(13, 11, ctypes.byref(out)) == -8


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
    at = lib.drag_expm_apply_target
    assert at(10, 4, good, good, good, 1.0, good, good, 20, s) == -8
    assert at(10, 4, good, good, good, 1.0, good, good, 0, s) == -8
    assert at(-1, 4, good, good, good, 1.0, good, good, 24, s) == -1
    assert at(10, 4, null, good, good, 1.0, good, good, 24, s) == -2
    ao = lib.drag_expm_apply_opts
    opts = dx.DragOptions(53, 1, 1, 0)                 # Pade with the bound test
    assert ao(ctypes.c_int64(10), 4, good, good, good, ctypes.c_double(1.0), good, good, ctypes.byref(opts), null,
              null, s) == -9
    opts = dx.DragOptions(11, 1, 0, 0)                 # Pade at 2^-11
    assert ao(ctypes.c_int64(10), 4, good, good, good, ctypes.c_double(1.0), good, good, ctypes.byref(opts), null,
              null, s) == -8
    opts = dx.DragOptions(53, 0, 1, 7)                 # arith outside {0, 1}
    assert ao(ctypes.c_int64(10), 4, good, good, good, ctypes.c_double(1.0), good, good, ctypes.byref(opts), null,
              null, s) == -9
    assert ao(ctypes.c_int64(10), 4, good, good, good, ctypes.c_double(1.0), good, good, None, null, null, s) == -2
    for bad in (dx.DragOptions(53, 0, 0, 1), dx.DragOptions(11, 0, 0, 1), dx.DragOptions(24, 1, 0, 1),
                dx.DragOptions(24, 0, 1, 1)):
        assert ao(ctypes.c_int64(10), 4, good, good, good, ctypes.c_double(1.0), good, good, ctypes.byref(bad),
                  null, null, s) == -9                   # FP32 arithmetic: Taylor, no bound test, ubits 24
    opts = dx.DragOptions(24, 0, 0, 1)
    assert ao(ctypes.c_int64(10), 4, good, good, good, ctypes.c_double(1.0), good, good, ctypes.byref(opts),
              good, null, s) == -9                       # no per-cell degrees on the FP32 path
    opts = dx.DragOptions(53, 0, 1, 0)
    assert ao(ctypes.c_int64(10), 4, good, bad_align, good, ctypes.c_double(1.0), good, good, ctypes.byref(opts),
              null, null, s) == -3
    ah = lib.drag_expm_apply_host
    assert ah(-1, 4, good, good, good, 1.0, good, good, 0, good, 1 << 30, s) == -1
    assert ah(10, 4, good, good, good, float("nan"), good, good, 0, good, 1 << 30, s) == -1
    assert ah(10, 4, good, null, good, 1.0, good, good, 0, good, 1 << 30, s) == -2
    assert ah(10, 4, good, good, good, 1.0, good, good, 0, null, 1 << 30, s) == -2
    assert ah(10, 4, good, good, good, 1.0, good, good, 64, good, 16, s) == -5
    assert ah(10, 4, good, good, good, 1.0, good, good, 64, ctypes.c_void_p(4104), 1 << 30, s) == -3
    st = lib.drag_expm_select_target
    assert st(10, 4, good, good, good, 1.0, 12, good, good, s) == -8
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
    assert lib.drag_expm_apply_launches(-1, 4) == 0 and lib.drag_expm_apply_launches(0, 4) == 0
    assert lib.drag_expm_apply_launches(10, 0) == 0 and lib.drag_expm_apply_launches(10, 32) == 0
    assert lib.drag_expm_backward_launches(-1, 4) == 0 and lib.drag_expm_backward_launches(0, 4) == 0
    assert lib.drag_expm_backward_launches(10, 0) == 0 and lib.drag_expm_backward_launches(10, 32) == 0
    # adjoint tape: geometry, then argument errors of the taped forward and adjoint
    tb = lib.drag_expm_tape_bytes
    assert tb(-1, 4, 3) == 0 and tb(10, 0, 3) == 0 and tb(10, 4, 0) == 0 and tb(10, 4, 2049) == 0
    assert tb(10, 16, 3) == 256 + 8 * 10 * 3 * 160          # 153 packed entries in 160-double slots
    assert tb(100, 1, 1) == 1024 + 8 * 100 * 16
    assert lib.drag_expm_tape_levels(-1) == 0
    assert [lib.drag_expm_tape_levels(k) for k in range(6)] == [1, 1, 1, 2, 3, 4]
    tape, big = ctypes.c_void_p(1 << 20), 1 << 40
    at = lib.drag_expm_apply_taped
    assert at(10, 4, good, good, good, 1.0, good, good, 0, tape, big, s) == -1
    assert at(10, 4, good, good, good, 1.0, good, good, 2049, tape, big, s) == -1
    assert at(10, 4, good, good, good, float("nan"), good, good, 3, tape, big, s) == -1
    assert at(10, 4, good, good, good, 1.0, good, good, 3, null, big, s) == -2
    assert at(10, 4, good, good, good, 1.0, null, good, 3, tape, big, s) == -2
    assert at(10, 4, good, good, good, 1.0, good, good, 3, ctypes.c_void_p((1 << 20) + 128), big, s) == -3
    assert at(10, 4, good, good, good, 1.0, good, bad_align, 3, tape, big, s) == -3
    assert at(10, 4, good, good, good, 1.0, good, good, 3, tape, tb(10, 4, 3) - 8, s) == -5
    assert at(0, 4, null, null, null, 1.0, null, null, 3, null, 0, s) == 0
    bt = lib.drag_expm_backward_taped
    assert bt(10, 4, good, good, good, 1.0, good, good, null, null, null, null, 0, tape, big, s) == -1
    assert bt(10, 4, good, good, good, 1.0, good, good, null, null, null, null, 3, null, big, s) == -2
    assert bt(10, 4, good, good, good, 1.0, good, good, null, null, null, null, 3, ctypes.c_void_p(4104), big,
              s) == -3
    assert bt(10, 4, good, good, good, 1.0, good, good, null, null, null, null, 3, tape, 64, s) == -5
    assert bt(0, 4, null, null, null, 1.0, null, null, null, null, null, null, 3, null, 0, s) == 0


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(dx.DragExpmError):
        dx.load_library(str(tmp_path / "missing.so"))
