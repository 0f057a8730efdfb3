"""Pins of the oracle's analytic implicit RK1 step (App. A.2, Eqs. analytic_1-4)."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W


@pytest.mark.parametrize("name,C", [("dustybox_n1_32k", 64), ("mrn_n4_128cube", 64), ("mrn_n16_128cube", 16)])
def test_rk1_solves_its_linear_system(name, C):
    """The step satisfies (I - dt Omega_v) v' = v (Eq. analytic_1 in velocity
    form) to rounding: residual <= 64 u (|I - A|_inf |v'| + |v|)."""
    cells = W.workload(name, ncells=C)
    w = oracle.rk1_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    u = 2.0 ** -53
    for c in range(C):
        A = oracle.assemble(cells.rho_g[c], cells.rho_d[:, c], cells.t_s[:, c], cells.dt)
        M = np.eye(A.shape[0]) - A
        res = M @ w[:, :, c].T - cells.v[:, :, c].T
        bound = 64 * u * (np.max(np.abs(M).sum(axis=1)) * np.max(np.abs(w[:, :, c])) + np.max(np.abs(cells.v[:, :, c])))
        assert np.max(np.abs(res)) <= bound


def test_rk1_dustybox_closed_form():
    """N = 1: backward Euler keeps V_CM and damps v_d - v_g by 1/(1 + (1+eps) dt/T_s)."""
    rng = np.random.default_rng(1)
    C = 200
    eps = rng.uniform(0.01, 5.0, C)
    ts = 10.0 ** rng.uniform(-5, 4, C)
    rho_g = np.exp(rng.standard_normal(C))
    v = rng.standard_normal((3, 2, C))
    w = oracle.rk1_apply(rho_g, (rho_g * eps)[None, :], ts[None, :], 1.0, v)
    vcm = (v[:, 0] + eps * v[:, 1]) / (1 + eps)
    dv = (v[:, 1] - v[:, 0]) / (1 + (1 + eps) / ts)
    sc = np.abs(v).max(axis=1)
    assert np.all(np.abs(w[:, 0] - (vcm - eps * dv / (1 + eps))) <= 4e-15 * sc)
    assert np.all(np.abs(w[:, 1] - (vcm + dv / (1 + eps))) <= 4e-15 * sc)


def test_rk1_is_first_order_consistent_with_exp():
    """|RK1 - EXP| = O(dt^2) per step for small dt: halving dt quarters the gap."""
    cells = W.workload("mrn_n4_128cube", ncells=32)
    ts = cells.t_s * 1e8                            # dt/t_s <= 1e-3 below: the non-stiff regime
    gaps = []
    for dt in (0.1, 0.05, 0.025):
        r = oracle.rk1_apply(cells.rho_g, cells.rho_d, ts, dt, cells.v)
        e = oracle.drag_apply(cells.rho_g, cells.rho_d, ts, dt, cells.v)
        gaps.append(np.max(np.abs(r - e)))
    assert 3.5 < gaps[0] / gaps[1] < 4.5 and 3.5 < gaps[1] / gaps[2] < 4.5


def test_rk1_conservation_limits_and_zero_density():
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=64)
    cells.rho_d[3, ::3] = 0.0
    w = oracle.rk1_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    rho = np.vstack([cells.rho_g[None, :], cells.rho_d])
    mi = np.einsum("fc,dfc->dc", rho, cells.v)
    mo = np.einsum("fc,dfc->dc", rho, w)
    assert np.all(np.abs(mo - mi) <= 8e-15 * np.einsum("fc,dfc->dc", rho, np.abs(cells.v)))
    zero = oracle.rk1_apply(cells.rho_g, cells.rho_d, cells.t_s, 0.0, cells.v)   # (rho v)/rho: within 1 ulp
    assert np.all(np.abs(zero - cells.v) <= 2.3e-16 * np.abs(cells.v))
    # infinitely stiff: every fluid at V_CM
    big = oracle.rk1_apply(cells.rho_g, cells.rho_d, cells.t_s * 1e-16, cells.dt, cells.v)   # dt/t_s >= 1e12
    vcm = mi / rho.sum(axis=0)
    assert np.max(np.abs(big - vcm[:, None, :]) / np.abs(cells.v).max(axis=1, keepdims=True)) < 1e-10
