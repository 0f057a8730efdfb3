"""GPU parity of the mixed-precision path (drag_expm_apply_opts with
arith = FP32): FP64 set-up and Algorithm 2 on the theta table of u = 2^-24
(Eq. B8's single-precision target), FP32 Taylor step, squarings and
applications.

Reference: the oracle at the same target (same (k*, s*), FP64 arithmetic), so
the difference is FP32 rounding only. Tolerance per cell and component:
|v_gpu - v_oracle| <= 64 u32 max_f |v_in[d, f]|, u32 = 2^-24 (3.8e-6). The
matrices are entrywise non-negative (exp of a Metzler matrix), so each n-term
product carries a relative error of order n u32, and the restorations keep
the stationary mode exact; measured errors stay below 20 u32 on stiff and
non-stiff cells for N = 1..31, and 64 u32 leaves a 3x margin.
"""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W
from tests.test_forward_gpu import assert_parity, dev

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
TOL = 64 * U32


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    from paper_2509_25347_gb300 import build
    build.build()
    import paper_2509_25347_gb300 as m
    m.load_library()
    m.get_status()
    return m


def mixed(dx, cells, ubits, dt=None, out=None):
    rg, rd, ts, v = dev(cells)
    o = dx.apply_opts(rg, rd, ts, cells.dt if dt is None else dt, v, out, ubits=ubits, arith="fp32")
    return o.cpu().numpy()


CASES = [("dustybox_n1_32k", 3001), ("mrn_n4_128cube", 1501), ("mrn_n8_128cube_adjoint", 901),
         ("mrn_n16_128cube", 501)]


@pytest.mark.parametrize("name,C", CASES)
def test_mixed_parity(dx, name, C):
    cells = W.workload(name, ncells=C)
    out = mixed(dx, cells, 24)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
    assert_parity(out, ref, cells.v, tol=TOL)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9, 12, 16, 17, 24, 31])
def test_mixed_every_size(dx, N):
    for cells in (W.mrn(71 + N, N, seed=800 + N, stiff_lo=-4.0, stiff_hi=8.0),
                  W.mrn(71 + N, N, seed=850 + N, stiff_lo=-4.0, stiff_hi=2.0)):
        out = mixed(dx, cells, 24)
        ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
        assert_parity(out, ref, cells.v, tol=TOL)


def test_mixed_conserves_momentum_and_stays_convex(dx):
    """The restorations keep P row-stochastic in FP32 too: momentum is
    conserved and the outputs stay inside the inputs' range, to FP32 rounding."""
    cells = W.workload("mrn_n16_128cube", ncells=400)
    out = mixed(dx, cells, 24)
    rho = np.concatenate([cells.rho_g[None, :], cells.rho_d], axis=0)
    p_in = np.sum(rho[None] * cells.v, axis=1)
    p_out = np.sum(rho[None] * out, axis=1)
    scale = np.sum(rho[None] * np.abs(cells.v), axis=1)
    assert np.max(np.abs(p_out - p_in) / scale) <= TOL
    lo, hi = cells.v.min(axis=1), cells.v.max(axis=1)
    span = np.abs(cells.v).max(axis=1)
    assert np.all(out.min(axis=1) >= lo - TOL * span) and np.all(out.max(axis=1) <= hi + TOL * span)


def test_mixed_edge_cases(dx):
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=100)
    # dt = 0: the identity up to FP32 rounding. The FP32 apply forms
    # v_i' = tau_i sum_j E_ij sigma_j v_j, so v_i comes back through sigma_i, its
    # reciprocal and two products: at most a few FP32 roundings of v_i.
    out = mixed(dx, cells, 24, dt=0.0)
    assert np.all(np.abs(out - cells.v) <= 8 * U32 * np.abs(cells.v))
    # in place
    rg, rd, ts, v = dev(cells)
    dx.apply_opts(rg, rd, ts, cells.dt, v, v, ubits=24, arith="fp32")
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
    assert_parity(v.cpu().numpy(), ref, cells.v, tol=TOL)
    # zero dust density and a decoupled species
    z = W.workload("mrn_n4_128cube", ncells=64)
    z.rho_d[2, :] = 0.0
    z.t_s[3, :7] = np.inf
    out = mixed(dx, z, 24)
    ref = oracle.drag_apply(z.rho_g, z.rho_d, z.t_s, z.dt, z.v, u=2.0 ** -24)
    assert_parity(out, ref, z.v, tol=TOL)
    # invalid cells: NaN and the status bit
    bad = W.workload("mrn_n4_128cube", ncells=40)
    bad.rho_d[0, 5] = -1.0
    out = mixed(dx, bad, 24)
    assert np.all(np.isnan(out[:, :, 5])) and np.all(np.isfinite(np.delete(out, 5, axis=2)))
    assert dx.get_status() & dx.STATUS_BAD_CELL
    for ub in (53, 11):
        with pytest.raises(dx.DragExpmError):
            dx.apply_opts(*dev(bad)[:3], bad.dt, dev(bad)[3], ubits=ub, arith="fp32")


def test_mixed_full_size_sampled(dx):
    import torch
    cells = W.workload("mrn_n16_128cube")
    rg, rd, ts, v = dev(cells)
    out = dx.apply_opts(rg, rd, ts, cells.dt, v, ubits=24, arith="fp32")
    idx = np.random.default_rng(29).choice(cells.ncells, 400, replace=False)
    sub = cells.subset(idx)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, u=2.0 ** -24)
    got = out[:, :, torch.from_numpy(idx).cuda()].cpu().numpy()
    assert_parity(got, ref, sub.v, tol=TOL)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [1, 4, 8, 11])
def test_mixed_both_kernel_families(dx, N):
    """Up to N = 11 the mixed-precision path runs lane per cell under the
    default modes (FP32 registers, all s* squarings, one apply) and one warp
    per cell under the warp-per-cell mode (the last two squarings as four
    applications); both match the oracle at the 2^-24 target to 64 u32."""
    cells = W.mrn(333 + N, N, seed=880 + N, stiff_lo=-4.0, stiff_hi=8.0)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
    saved = dx.get_mode(N)
    assert saved != dx.MODE_WARP_PER_CELL
    assert_parity(mixed(dx, cells, 24), ref, cells.v, tol=TOL)
    dx.set_mode(N, dx.MODE_WARP_PER_CELL)
    try:
        out = mixed(dx, cells, 24)
    finally:
        dx.set_mode(N, saved)
    assert_parity(out, ref, cells.v, tol=TOL)
    assert dx.get_status() == 0


def test_mixed_sizes_past_the_fp64_lane_range(dx):
    """n = 13..17 run lane per cell on the mixed-precision path whatever the
    mode (F in FP32 registers, G in shared memory, tile-sorted), also under the
    warp-per-cell mode; ragged counts spanning several tiles."""
    for N in (12, 14, 16):
        cells = W.mrn(1111 + N, N, seed=890 + N, stiff_lo=-4.0, stiff_hi=8.0)
        ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
        assert dx.get_mode(N) == dx.MODE_WARP_PER_CELL
        assert_parity(mixed(dx, cells, 24), ref, cells.v, tol=TOL)
    assert dx.get_status() == 0


def test_mixed_full_size_lane_per_cell(dx):
    """The N = 4 workload at full size (2,097,152 cells) through the
    lane-per-cell mixed-precision kernel: 400 sampled cells against the oracle."""
    import torch
    cells = W.workload("mrn_n4_128cube")
    rg, rd, ts, v = dev(cells)
    out = dx.apply_opts(rg, rd, ts, cells.dt, v, ubits=24, arith="fp32")
    idx = np.random.default_rng(31).choice(cells.ncells, 400, replace=False)
    sub = cells.subset(idx)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, u=2.0 ** -24)
    got = out[:, :, torch.from_numpy(idx).cuda()].cpu().numpy()
    assert_parity(got, ref, sub.v, tol=TOL)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [4, 16, 24])
def test_mixed_extreme_norms(dx, N):
    """Norms up to 1.5e308 (s* ~ 1023) on the mixed-precision path, lane per
    cell in registers (N = 4) and hybrid (N = 16), and warp per cell (N = 24):
    every cell has relaxed to V_CM and matches the oracle at the 2^-24 target
    to 64 u32."""
    from tests.test_forward_gpu import extreme_cells
    cells = extreme_cells(N, [1e8, 1e14, 1e250, 1e300, 1.5e308])
    out = mixed(dx, cells, 24)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
    assert np.all(np.isfinite(out))
    assert_parity(out, ref, cells.v, tol=TOL)
    assert dx.get_status() == 0
