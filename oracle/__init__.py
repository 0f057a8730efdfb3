"""CPU oracle for the exponential multi-fluid drag update (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
path (``paper_2509_25347_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``drag_oracle.c`` (plain FP64 C, no FMA contraction),
compiled by :func:`build` into ``liboracle_drag.so`` and called through ctypes.
``truth.py`` holds a second, independent check in extended precision.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drag_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_drag.so")
_lib = None

K_MAX = 9
NMAX = 64


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, portable flags)."""
    out = _LIB_PATH if not openmp else os.path.join(_HERE, "liboracle_drag_omp.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", out, _SRC, "-lm"]
        if openmp:
            cmd.insert(1, "-fopenmp")
            cmd.insert(1, "-DORC_OPENMP")
        subprocess.run(cmd, check=True)
    return out


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_theta_m.restype = ctypes.c_double
    lib.orc_theta_m.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.orc_theta_table.restype = None
    lib.orc_theta_table.argtypes = [dp]
    lib.orc_select_alg2.restype = ctypes.c_int
    lib.orc_select_alg2.argtypes = [ctypes.c_double, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    lib.orc_expm_dense.restype = ctypes.c_int
    lib.orc_expm_dense.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    lib.orc_assemble.restype = None
    lib.orc_assemble.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_double, ctypes.c_int, dp]
    lib.orc_theta_table_u.restype = None
    lib.orc_theta_table_u.argtypes = [ctypes.c_double, dp]
    lib.orc_select_alg2_u.restype = ctypes.c_int
    lib.orc_select_alg2_u.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double] + [ctypes.POINTER(ctypes.c_int)] * 3
    lib.orc_drag_apply_u.restype = ctypes.c_int
    lib.orc_drag_apply_u.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp, ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int16),
                                     ctypes.POINTER(ctypes.c_uint32)]
    lib.orc_pade_coeffs.restype = None
    lib.orc_pade_coeffs.argtypes = [ctypes.c_int, dp]
    lib.orc_pade_theta.restype = ctypes.c_double
    lib.orc_pade_theta.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.orc_select_pade.restype = ctypes.c_int
    lib.orc_select_pade.argtypes = [ctypes.c_double, ctypes.c_double] + [ctypes.POINTER(ctypes.c_int)] * 2
    lib.orc_drag_apply_opts.restype = ctypes.c_int
    lib.orc_drag_apply_opts.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int8),
                                        ctypes.POINTER(ctypes.c_int16), dp, ctypes.POINTER(ctypes.c_uint32)]
    lib.orc_drag_apply.restype = ctypes.c_int
    lib.orc_drag_apply.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int16),
                                   ctypes.POINTER(ctypes.c_uint32)]
    lib.orc_drag_backward.restype = ctypes.c_int
    lib.orc_drag_backward.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp, dp, dp, dp,
                                      dp, ctypes.POINTER(ctypes.c_uint32)]
    lib.orc_frechet_dense.restype = ctypes.c_int
    lib.orc_frechet_dense.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int]
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.orc_drag_apply_batched.restype = ctypes.c_int
    lib.orc_drag_apply_batched.argtypes = [ctypes.c_int64, i64p, i64p, i64p, i32p, i32p, dp, dp, dp, dp, dp, dp,
                                           ctypes.POINTER(ctypes.c_uint32)]
    lib.orc_drag_heat.restype = ctypes.c_int
    lib.orc_drag_heat.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, dp, dp]
    lib.orc_rk1_apply.restype = ctypes.c_int
    lib.orc_rk1_apply.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp,
                                  ctypes.POINTER(ctypes.c_uint32)]
    for name in ("orc_table_mk", "orc_table_qk", "orc_table_rk"):
        getattr(lib, name).restype = ctypes.c_int
        getattr(lib, name).argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


U_DOUBLE = 2.0 ** -53


def theta_table(u: float = U_DOUBLE) -> np.ndarray:
    """theta_{m_k} for k = 0..9 (index 0 unused), Eq. B8 with unit round-off u
    (2^-53 by default; Eq. B8 also names 2^-11, 2^-24, 2^-113, 2^-237)."""
    out = np.zeros(K_MAX + 1)
    if u == U_DOUBLE:
        _load().orc_theta_table(_dptr(out))
    else:
        _load().orc_theta_table_u(float(u), _dptr(out))
    return out


def theta_m(m: int, u: float = 2.0 ** -53) -> float:
    """theta_m of Eq. B8 for any order m and unit round-off u."""
    return _load().orc_theta_m(int(m), float(u))


def table_b1(k: int) -> tuple[int, int, int]:
    """(m_k, q_k, r_k) of Table B.1."""
    lib = _load()
    return lib.orc_table_mk(k), lib.orc_table_qk(k), lib.orc_table_rk(k)


def select(norm: float, u: float = U_DOUBLE) -> tuple[int, int, int]:
    """Algorithm 2 (K = 9) with the theta table of unit round-off u: returns
    (k*, m*, s*) for a given 1-norm."""
    k, m, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    if u == U_DOUBLE:
        _load().orc_select_alg2(float(norm), K_MAX, ctypes.byref(k), ctypes.byref(m), ctypes.byref(s))
    else:
        _load().orc_select_alg2_u(float(norm), K_MAX, float(u), ctypes.byref(k), ctypes.byref(m), ctypes.byref(s))
    return k.value, m.value, s.value


def expm(A: np.ndarray, structured: bool = True) -> tuple[np.ndarray, int, int, int]:
    """exp(A) by the oracle's Taylor scaling and squaring. Returns (P, k*, m*, s*)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    P = np.zeros_like(A)
    k, m, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = _load().orc_expm_dense(n, _dptr(A), _dptr(P), int(structured), ctypes.byref(k), ctypes.byref(m),
                                ctypes.byref(s))
    if rc == -2:
        raise ValueError("matrix too large for the oracle")
    return P, k.value, m.value, s.value


def assemble(rho_g: float, rho_d: np.ndarray, t_s: np.ndarray, dt: float, structured: bool = True) -> np.ndarray:
    """A = dt * Omega_v for one cell (velocity form of Eq. jacobian)."""
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    t_s = np.ascontiguousarray(t_s, dtype=np.float64)
    N = rho_d.shape[0]
    A = np.zeros((N + 1, N + 1))
    _load().orc_assemble(N, float(rho_g), _dptr(rho_d), _dptr(t_s), float(dt), int(structured), _dptr(A))
    return A


def drag_apply(rho_g, rho_d, t_s, dt, v_in, structured: bool = True, return_ks: bool = False,
               u: float = U_DOUBLE):
    """Forward drag update over SoA arrays (layout of the CUDA library).

    rho_g: (C,), rho_d: (N, C), t_s: (N, C), v_in: (3, N+1, C). Returns v_out of
    the same shape as v_in (and, with return_ks, k*, s* per cell and the status word).
    u: unit round-off whose theta table Algorithm 2 selects (k*, s*) from; the
    arithmetic is FP64 whatever u is.
    """
    rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    t_s = np.ascontiguousarray(t_s, dtype=np.float64)
    v_in = np.ascontiguousarray(v_in, dtype=np.float64)
    C = rho_g.shape[0]
    N = rho_d.shape[0]
    assert rho_d.shape == (N, C) and t_s.shape == (N, C) and v_in.shape == (3, N + 1, C)
    v_out = np.empty_like(v_in)
    k_out = np.zeros(C, dtype=np.int8)
    s_out = np.zeros(C, dtype=np.int16)
    st = ctypes.c_uint32(0)
    kp = k_out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    sp = s_out.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
    if u == U_DOUBLE:
        rc = _load().orc_drag_apply(C, N, _dptr(rho_g), _dptr(rho_d), _dptr(t_s), float(dt), _dptr(v_in),
                                    _dptr(v_out), int(structured), kp, sp, ctypes.byref(st))
    else:
        rc = _load().orc_drag_apply_u(C, N, _dptr(rho_g), _dptr(rho_d), _dptr(t_s), float(dt), _dptr(v_in),
                                      _dptr(v_out), int(structured), float(u), kp, sp, ctypes.byref(st))
    if rc != 0:
        raise ValueError(f"oracle rejected sizes (rc={rc})")
    if return_ks:
        return v_out, k_out, s_out, st.value
    return v_out


PADE_DEGREES = (3, 5, 7, 9, 13)


def pade_coeffs(m: int) -> np.ndarray:
    """c_0..c_m of N_mm (Eq. PadeEqu, p = q = m); D_mm(x) = N_mm(-x)."""
    out = np.zeros(32)
    _load().orc_pade_coeffs(int(m), _dptr(out))
    return out[:m + 1].copy()


def pade_theta(m: int, u: float = U_DOUBLE) -> float:
    """theta of the [m/m] Pade approximant: Eqs. B5-B8 with T_m replaced by R_mm."""
    return _load().orc_pade_theta(int(m), float(u))


def select_pade(norm: float, u: float = U_DOUBLE) -> tuple[int, int]:
    """(m, s) of the Pade variant for a given 1-norm."""
    m, s = ctypes.c_int(), ctypes.c_int()
    _load().orc_select_pade(float(norm), float(u), ctypes.byref(m), ctypes.byref(s))
    return m.value, s.value


def drag_apply_opts(rho_g, rho_d, t_s, dt, v_in, u: float = U_DOUBLE, method: str = "taylor",
                    bound_test: bool = False, structured: bool = True):
    """Forward update with the options of the CUDA library's drag_expm_apply_opts.

    method 'taylor' (Algorithm 2; bound_test adds the second modification,
    Eqs. Pat_Stk4-7) or 'pade' (Eq. PadeEqu). Returns (v_out, k, m, s, ratio,
    status): k* (Taylor) or the Pade degree, the degree actually evaluated,
    s*, and for the bound test its left side over u for the top block.
    """
    rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    t_s = np.ascontiguousarray(t_s, dtype=np.float64)
    v_in = np.ascontiguousarray(v_in, dtype=np.float64)
    C, N = rho_g.shape[0], rho_d.shape[0]
    assert rho_d.shape == (N, C) and t_s.shape == (N, C) and v_in.shape == (3, N + 1, C)
    v_out = np.empty_like(v_in)
    k = np.zeros(C, dtype=np.int8)
    m = np.zeros(C, dtype=np.int8)
    s = np.zeros(C, dtype=np.int16)
    ratio = np.zeros(C)
    st = ctypes.c_uint32(0)
    meth = {"taylor": 0, "pade": 1}[method]
    rc = _load().orc_drag_apply_opts(C, N, _dptr(rho_g), _dptr(rho_d), _dptr(t_s), float(dt), _dptr(v_in),
                                     _dptr(v_out), int(structured), float(u), meth, int(bound_test),
                                     k.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                     m.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                     s.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), _dptr(ratio),
                                     ctypes.byref(st))
    if rc != 0:
        raise ValueError(f"oracle rejected sizes (rc={rc})")
    return v_out, k, m, s, ratio, st.value


def frechet_T(A: np.ndarray, G: np.ndarray, structured: bool = False) -> np.ndarray:
    """Z = L(A^T, G): Frechet derivative of exp at A^T in direction G (block S&S).

    structured=True only for A with zero row sums (drag matrices)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    Z = np.zeros_like(A)
    rc = _load().orc_frechet_dense(A.shape[0], _dptr(A), _dptr(G), _dptr(Z), int(structured))
    if rc == -2:
        raise ValueError("matrix too large for the oracle")
    return Z


def drag_backward(rho_g, rho_d, t_s, dt, v_in, grad_v_out):
    """Gradients of <grad_v_out, v_out> through one drag step.

    Returns (grad_v_in (3,N+1,C), grad_rho_g (C,), grad_rho_d (N,C), grad_t_s (N,C), status).
    """
    rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    t_s = np.ascontiguousarray(t_s, dtype=np.float64)
    v_in = np.ascontiguousarray(v_in, dtype=np.float64)
    g = np.ascontiguousarray(grad_v_out, dtype=np.float64)
    C = rho_g.shape[0]
    N = rho_d.shape[0]
    assert g.shape == v_in.shape == (3, N + 1, C)
    gv = np.empty_like(v_in)
    grg = np.empty(C)
    grd = np.empty((N, C))
    gts = np.empty((N, C))
    st = ctypes.c_uint32(0)
    rc = _load().orc_drag_backward(C, N, _dptr(rho_g), _dptr(rho_d), _dptr(t_s), float(dt), _dptr(v_in), _dptr(g),
                                   _dptr(gv), _dptr(grg), _dptr(grd), _dptr(gts), ctypes.byref(st))
    if rc != 0:
        raise ValueError(f"oracle rejected sizes (rc={rc})")
    return gv, grg, grd, gts, st.value


def drag_apply_batched(desc, rho_g, rho_d, t_s, v_in):
    """Batched forward over packed block slabs.

    desc: structured array with fields cell_offset, dust_offset, vel_offset
    (int64), ncells, nspecies (int32), dt (float64). Returns (v_out, status).
    """
    f = lambda name, dt_: np.ascontiguousarray(desc[name], dtype=dt_)
    co, do, vo = f("cell_offset", np.int64), f("dust_offset", np.int64), f("vel_offset", np.int64)
    nc, ns, dts = f("ncells", np.int32), f("nspecies", np.int32), f("dt", np.float64)
    rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    t_s = np.ascontiguousarray(t_s, dtype=np.float64)
    v_in = np.ascontiguousarray(v_in, dtype=np.float64)
    v_out = v_in.copy()
    st = ctypes.c_uint32(0)
    p64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    p32 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    rc = _load().orc_drag_apply_batched(len(desc), p64(co), p64(do), p64(vo), p32(nc), p32(ns), _dptr(dts),
                                        _dptr(rho_g), _dptr(rho_d), _dptr(t_s), _dptr(v_in), _dptr(v_out),
                                        ctypes.byref(st))
    if rc != 0:
        raise ValueError(f"oracle rejected a block (rc={rc})")
    return v_out, st.value


def rk1_apply(rho_g, rho_d, t_s, dt, v_in):
    """Analytic implicit RK1 drag step (App. A.2) over SoA arrays; returns v_out."""
    rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    t_s = np.ascontiguousarray(t_s, dtype=np.float64)
    v_in = np.ascontiguousarray(v_in, dtype=np.float64)
    C, N = rho_g.shape[0], rho_d.shape[0]
    v_out = np.empty_like(v_in)
    st = ctypes.c_uint32(0)
    rc = _load().orc_rk1_apply(C, N, _dptr(rho_g), _dptr(rho_d), _dptr(t_s), float(dt), _dptr(v_in), _dptr(v_out),
                               ctypes.byref(st))
    if rc != 0:
        raise ValueError(f"oracle rejected sizes (rc={rc})")
    return v_out


def drag_heat(rho_g, rho_d, v_in, v_out):
    """Kinetic energy dissipated by a drag step, per cell (frictional heating)."""
    rho_g = np.ascontiguousarray(rho_g, dtype=np.float64)
    rho_d = np.ascontiguousarray(rho_d, dtype=np.float64)
    v_in = np.ascontiguousarray(v_in, dtype=np.float64)
    v_out = np.ascontiguousarray(v_out, dtype=np.float64)
    C, N = rho_g.shape[0], rho_d.shape[0]
    heat = np.empty(C)
    rc = _load().orc_drag_heat(C, N, _dptr(rho_g), _dptr(rho_d), _dptr(v_in), _dptr(v_out), _dptr(heat))
    if rc != 0:
        raise ValueError(f"oracle rejected sizes (rc={rc})")
    return heat
