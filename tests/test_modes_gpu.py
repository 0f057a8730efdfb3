"""Every kernel family for every size it supports (lane per cell in registers,
lane per cell in shared memory, lane per cell hybrid, warp per cell) against the
oracle, and the autotuner: valid choices, cache round trip, parity after tuning."""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13


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


def valid_modes(N):
    n = N + 1
    modes = [0]
    if n <= 6:
        modes.append(1)
    if n <= 12:
        modes.append(2)
    if 7 <= n <= 12:
        modes.append(3)
    return modes


@pytest.mark.parametrize("N", list(range(1, 14)))
def test_every_mode_parity(dx, N):
    cells = W.mrn(161, N, seed=500 + N, stiff_lo=-4.0, stiff_hi=8.0)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    sc = np.abs(cells.v).max(axis=1, keepdims=True)
    old = dx.get_mode(N)
    outs = {}
    try:
        for mode in valid_modes(N):
            dx.set_mode(N, mode)
            assert dx.get_mode(N) == mode
            outs[mode] = dx.apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v))
            out = outs[mode].cpu().numpy()
            assert np.max(np.abs(out - ref) / sc) <= TOL, (N, mode)
        for bad in (4, -1) + ((3,) if not 7 <= N + 1 <= 12 else ()) + ((2,) if N + 1 > 12 else ()):
            with pytest.raises(dx.DragExpmError):
                dx.set_mode(N, bad)
    finally:
        dx.set_mode(N, old)
    if 3 in outs:
        # the hybrid and the all-shared storage agree to rounding
        d = (outs[2] - outs[3]).abs().max().item()
        assert d <= 4e-16 * float(np.abs(cells.v).max()), d
    assert dx.get_status() == 0


def test_default_modes(dx):
    """Built-in table (every test here restores what it changes): lane per cell in
    registers up to n = 6, hybrid up to n = 12, warp per cell above."""
    for N in range(1, dx.NMAX + 1):
        n = N + 1
        assert dx.get_mode(N) == (dx.MODE_LANE_REGISTERS if n <= 6 else
                                  dx.MODE_LANE_HYBRID if n <= 12 else dx.MODE_WARP_PER_CELL), N


def test_autotune_and_cache(dx, tmp_path):
    cache = str(tmp_path / "modes.txt")
    before = {N: dx.get_mode(N) for N in range(1, 9)}
    try:
        chosen = dx.autotune(8, cache)
        assert set(chosen) == set(range(1, 9))
        for N, m in chosen.items():
            assert m in valid_modes(N)
        text = open(cache).read().split()
        assert len(text) == 3 * 8
        for N in range(1, 9):          # scramble, then reload from the cache
            dx.set_mode(N, 0)
        assert dx.autotune(8, cache) == chosen
        for N in (1, 4, 8):
            cells = W.mrn(97, N, seed=700 + N, stiff_lo=-4.0, stiff_hi=8.0)
            ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
            out = dx.apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v)).cpu().numpy()
            assert np.max(np.abs(out - ref) / np.abs(cells.v).max(axis=1, keepdims=True)) <= TOL
    finally:
        for N, m in before.items():
            dx.set_mode(N, m)
