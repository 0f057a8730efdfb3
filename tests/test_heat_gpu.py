"""GPU energy epilogue (drag_expm_apply_heat through the C ABI): v_out equals
drag_expm_apply's bit for bit and the dissipated kinetic energy matches the
oracle's to 1e-12 of the cell's kinetic energy about its centre of mass."""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    from paper_2509_25347_gb300 import build
    build.build()
    import paper_2509_25347_gb300 as m
    m.load_library()
    m.get_status()
    return m


def t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def krel(cells):
    rho = np.vstack([cells.rho_g[None, :], cells.rho_d])
    V = np.einsum("fc,dfc->dc", rho, cells.v) / rho.sum(axis=0)
    return 0.5 * np.einsum("fc,dfc->c", rho, (cells.v - V[:, None, :]) ** 2)


@pytest.mark.parametrize("N,mode", [(1, None), (4, None), (8, None), (16, None), (31, None),
                                    (4, 0), (4, 2), (8, 0), (8, 3), (10, 2), (10, 3), (11, 3)])
def test_heat_parity(dx, N, mode):
    cells = W.mrn(777, N, seed=40 + N, stiff_lo=-4.0, stiff_hi=8.0)
    cells.v += 3.0                                     # common motion must not matter
    old = dx.get_mode(N)
    try:
        if mode is not None:
            dx.set_mode(N, mode)
        plain = dx.apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v)).cpu().numpy()
        out, heat = dx.apply_heat(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v))
    finally:
        dx.set_mode(N, old)
    out, heat = out.cpu().numpy(), heat.cpu().numpy()
    assert np.array_equal(out, plain)
    ref_out = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    ref = oracle.drag_heat(cells.rho_g, cells.rho_d, cells.v, ref_out)
    k = krel(cells)
    assert np.all(np.abs(heat - ref) <= 1e-12 * k)
    assert np.all(heat >= -1e-13 * k)


def test_heat_invalid_and_in_place(dx):
    cells = W.workload("mrn_n4_128cube", ncells=50)
    cells.rho_g[7] = -1.0
    v = t(cells.v)
    _, heat = dx.apply_heat(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, v, v)
    heat = heat.cpu().numpy()
    assert np.isnan(heat[7]) and np.all(np.isfinite(np.delete(heat, 7)))
    assert dx.get_status() & dx.STATUS_BAD_CELL
