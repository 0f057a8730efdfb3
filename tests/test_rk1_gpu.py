"""GPU analytic RK1 (drag_rk1_apply through the C ABI) against the oracle's
RK1 (App. A.2), 1e-13 of max |v_in| per cell and component."""
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


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 31])
def test_rk1_parity(dx, N):
    cells = W.mrn(1000 + N, N, seed=900 + N, stiff_lo=-4.0, stiff_hi=8.0)
    cells.rho_d[0, ::7] = 0.0
    cells.t_s[-1, ::5] = np.inf
    out = dx.rk1_apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v)).cpu().numpy()
    ref = oracle.rk1_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    sc = np.abs(cells.v).max(axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / sc) <= 1e-13
    assert dx.get_status() == 0


def test_rk1_full_size_in_place_and_invalid(dx):
    import torch
    cells = W.workload("mrn_n16_128cube")
    v = t(cells.v)
    dx.rk1_apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, v, v)
    idx = np.random.default_rng(0).integers(0, cells.ncells, 128)
    sub = cells.subset(idx)
    ref = oracle.rk1_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    got = v[:, :, torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.max(np.abs(got - ref) / np.abs(sub.v).max(axis=1, keepdims=True)) <= 1e-13
    bad = W.workload("mrn_n4_128cube", ncells=10)
    bad.t_s[1, 4] = -2.0
    out = dx.rk1_apply(t(bad.rho_g), t(bad.rho_d), t(bad.t_s), bad.dt, t(bad.v)).cpu().numpy()
    assert np.all(np.isnan(out[:, :, 4])) and np.all(np.isfinite(out[:, :, 5]))
    assert dx.get_status() & dx.STATUS_BAD_CELL
