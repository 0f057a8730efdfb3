"""Pins of the oracle's frictional heating (energy epilogue; Eqs. GenEq_3, CompVar4)."""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W


def test_heat_dustybox_closed_form():
    """N = 1: the relative velocity decays as exp(-lambda dt), lambda = (1+eps)/T_s,
    so the dissipated energy is 1/2 mu |dv|^2 (1 - exp(-2 lambda dt)) with the
    reduced mass mu = rho_g rho_d / (rho_g + rho_d)."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(2)
    C = 200
    rho_g = np.exp(rng.standard_normal(C))
    eps = rng.uniform(0.01, 3.0, C)
    ts = 10.0 ** rng.uniform(-3, 3, C)
    v = rng.standard_normal((3, 2, C)) + 5.0              # common offset: exercises the V_CM shift
    rho_d = (rho_g * eps)[None, :]
    out = oracle.drag_apply(rho_g, rho_d, ts[None, :], 1.0, v)
    h = oracle.drag_heat(rho_g, rho_d, v, out)
    for c in range(C):
        rg, rd = mp.mpf(float(rho_g[c])), mp.mpf(float(rho_d[0, c]))
        lam = (1 + rd / rg) / mp.mpf(float(ts[c]))
        dv2 = sum((mp.mpf(float(v[d, 1, c])) - mp.mpf(float(v[d, 0, c]))) ** 2 for d in range(3))
        ref = 0.5 * rg * rd / (rg + rd) * dv2 * (1 - mp.exp(-2 * lam))
        scale = 0.5 * float(rg * rd / (rg + rd) * dv2)
        assert abs(h[c] - float(ref)) <= 1e-14 * scale + 1e-300


@pytest.mark.parametrize("name", ["mrn_n4_128cube", "mrn_n16_128cube"])
def test_heat_is_dissipation(name):
    """heat >= 0 (drag only dissipates), heat -> all relative kinetic energy as
    dt/T_s -> infinity, and heat ~ dt * sum rho_d |v_d - v_g|^2 / T_s for small dt."""
    cells = W.workload(name, ncells=64)
    out = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    h = oracle.drag_heat(cells.rho_g, cells.rho_d, cells.v, out)
    rho = np.vstack([cells.rho_g[None, :], cells.rho_d])
    V = np.einsum("fc,dfc->dc", rho, cells.v) / rho.sum(axis=0)
    krel = 0.5 * np.einsum("fc,dfc->c", rho, (cells.v - V[:, None, :]) ** 2)
    assert np.all(h >= -1e-15 * krel) and np.all(h <= krel * (1 + 1e-14))
    big = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s * 1e-12, cells.dt, cells.v)
    hb = oracle.drag_heat(cells.rho_g, cells.rho_d, cells.v, big)
    assert np.all(np.abs(hb - krel) <= 1e-12 * krel)
    dt = 1e-12                                            # dt/T_s <= 1e-4 on these workloads
    small = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, dt, cells.v)
    hs = oracle.drag_heat(cells.rho_g, cells.rho_d, cells.v, small)
    rate = np.einsum("ic,dic->c", cells.rho_d / cells.t_s, (cells.v[:, 1:] - cells.v[:, :1]) ** 2)
    assert np.all(np.abs(hs - dt * rate) <= 1e-3 * dt * rate + 1e-13 * krel)
