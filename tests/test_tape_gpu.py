"""Adjoint tape (drag_expm_apply_taped / drag_expm_backward_taped) through the C ABI.

The taped forward stores the restored iterates E_0 .. E_{s*-2} it forms; the
taped adjoint reads them instead of recomputing the Taylor step and those
squarings. From n = 13 (and for any n whose mode is warp per cell) the forward
runs warp per cell, and both sides form each E_t by the same FP64 operations in
the same order, so:
* the taped forward's v_out equals the warp-per-cell drag_expm_apply's bit for bit;
* the taped adjoint's four gradients equal drag_expm_backward's bit for bit,
  for recorded cells, for cells past the tape's capacity (recomputed) and for
  cells whose inputs no longer match the tape's fingerprint (recomputed).
For n <= 12 with the default modes the lane-per-cell forward writes the tape: its
v_out equals drag_expm_apply's bit for bit. Up to n = 9 the adjoint runs lane per
cell too and forms E_t by the same steps, so the taped gradients equal the
recomputed ones bit for bit; for n = 10..12 the warp-per-cell adjoint reads the
tape, whose E_t differ from its own recomputation by rounding (its Taylor step
sums G_00 in another order), so there the taped gradients are checked against
the oracle's adjoint at the 1e-13 tolerances of tests/test_backward_gpu.py.
"""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W
from tests.test_backward_gpu import assert_adjoint_parity
from tests.test_oracle_adjoint_pins import assert_fd_agreement, finite_difference_gradients

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


def spread_cells(N, C, seed):
    """Cells whose s* covers 0, 1, 2, 3 and up to ~20: an MRN population over
    ten decades of stiffness with its first cells at small dt/t_s."""
    cells = W.mrn(C, N, seed=seed, stiff_lo=-6.0, stiff_hi=7.0)
    ts = cells.t_s.copy()
    for c, scale in enumerate([1e-6] + list(np.geomspace(1e-2, 40.0, 60))):
        ts[:, c] = cells.dt / scale * np.linspace(1.0, 2.0, N)
    return W.Cells(cells.rho_g, cells.rho_d, ts, cells.v, cells.dt)


def dev_args(cells):
    return t(cells.rho_g), t(cells.rho_d), t(cells.t_s)


@pytest.fixture
def wpc_mode(dx):
    """Runs the plain forward warp per cell for every size, restoring the table after."""
    saved = {N: dx.get_mode(N) for N in range(1, dx.NMAX + 1)}
    for N in saved:
        dx.set_mode(N, dx.MODE_WARP_PER_CELL)
    yield
    for N, mode in saved.items():
        dx.set_mode(N, mode)


@pytest.mark.parametrize("N", [1, 4, 8, 11, 16, 31])
def test_taped_forward_is_the_forward(dx, wpc_mode, N):
    import torch
    cells = spread_cells(N, 203, seed=40 + N)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    plain = dx.apply(rg, rd, ts, cells.dt, v)
    taped, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    assert torch.equal(plain, taped)
    assert tape.levels == dx.tape_levels(int(dx.select(rg, rd, ts, cells.dt)[1].max()))
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [1, 2, 4, 8, 11, 16, 24, 31])
def test_taped_backward_is_the_backward(dx, wpc_mode, N):
    import torch
    cells = spread_cells(N, 211, seed=70 + N)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    s = dx.select(rg, rd, ts, cells.dt)[1].cpu().numpy()
    assert {0, 1, 2, 3} <= set(s.tolist()) and s.max() >= 10
    g = t(np.random.default_rng(N).standard_normal(cells.v.shape))
    _, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    plain = dx.backward(rg, rd, ts, cells.dt, v, g)
    taped = dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)
    for a, b in zip(plain, taped):
        assert torch.equal(a, b)
    assert dx.get_status() == 0


def test_taped_backward_oracle_parity(dx):
    cells = W.workload("mrn_n16_128cube", ncells=97)
    rg, rd, ts = dev_args(cells)
    g = np.random.default_rng(17).standard_normal(cells.v.shape)
    _, tape = dx.apply_taped(rg, rd, ts, cells.dt, t(cells.v))
    got = [o.cpu().numpy() for o in dx.backward(rg, rd, ts, cells.dt, t(cells.v), t(g), tape=tape)]
    rv, rrg, rrd, rts, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)
    assert_adjoint_parity(cells, g, got, (rv, rrg, rrd, rts))


@pytest.mark.parametrize("N", [16, 8])
def test_tape_capacity_short(dx, N):
    """Cells needing more levels than the capacity are not recorded; their
    adjoint recomputes and the gradients stay identical (N = 16 warp per cell;
    N = 8 lane per cell with the hybrid storage, tape written by the
    lane-per-cell forward)."""
    import torch
    cells = spread_cells(N, 150, seed=5)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    g = t(np.random.default_rng(3).standard_normal(cells.v.shape))
    s = dx.select(rg, rd, ts, cells.dt)[1].cpu().numpy()
    levels = 4
    assert (s - 1 > levels).any() and (s - 1 <= levels).any()
    _, tape = dx.apply_taped(rg, rd, ts, cells.dt, v, levels=levels)
    assert tape.nbytes == dx.tape_bytes(150, N, levels)
    plain = dx.backward(rg, rd, ts, cells.dt, v, g)
    taped = dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)
    for a, b in zip(plain, taped):
        assert torch.equal(a, b)


@pytest.mark.parametrize("N", [12, 8])
def test_stale_and_foreign_tapes(dx, N):
    """A tape is used only where the cell's inputs reproduce its fingerprint:
    changed inputs (by one ulp), another dt, or random bytes all give the
    recomputed gradients exactly (N = 8: lane per cell, hybrid storage)."""
    import torch
    cells = spread_cells(N, 180, seed=9)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    g = t(np.random.default_rng(4).standard_normal(cells.v.shape))
    _, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)

    rd2 = rd.clone()
    rd2[N // 2, ::2] = torch.nextafter(rd2[N // 2, ::2], torch.full_like(rd2[N // 2, ::2], np.inf))
    ts2 = ts.clone()
    ts2[0, 1::4] = torch.nextafter(ts2[0, 1::4], torch.zeros_like(ts2[0, 1::4]))
    for args, dt in (((rg, rd2, ts), cells.dt), ((rg, rd, ts2), cells.dt), ((rg, rd, ts), np.nextafter(cells.dt, 2.0))):
        plain = dx.backward(*args, dt, v, g)
        taped = dx.backward(*args, dt, v, g, tape=tape)
        for a, b in zip(plain, taped):
            assert torch.equal(a, b)

    junk = dx.Tape(torch.randint(0, 256, (tape.nbytes,), dtype=torch.uint8, device="cuda"), tape.ncells,
                   tape.nspecies, tape.levels)
    plain = dx.backward(rg, rd, ts, cells.dt, v, g)
    taped = dx.backward(rg, rd, ts, cells.dt, v, g, tape=junk)
    for a, b in zip(plain, taped):
        assert torch.equal(a, b)


def test_tape_on_host_is_refused(dx):
    """A Tape whose buffer is not a CUDA tensor never reaches the library."""
    import torch
    cells = spread_cells(4, 64, seed=3)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    _, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    host_tape = dx.Tape(tape.buf.cpu(), tape.ncells, tape.nspecies, tape.levels)
    with pytest.raises(dx.DragExpmError, match="CUDA tensor"):
        dx.backward(rg, rd, ts, cells.dt, v, torch.ones_like(v), tape=host_tape)
    with pytest.raises(dx.DragExpmError, match="CUDA tensor"):
        dx.apply_taped(rg, rd, ts, cells.dt, v, tape=host_tape)


@pytest.mark.parametrize("N", [4, 12])
def test_tape_invalid_cells(dx, N):
    """Invalid cells: NaN outputs and gradients and the status bit, as untaped;
    the valid cells' gradients as untaped (bit for bit warp per cell, to the
    adjoint tolerance when the lane-per-cell forward wrote the tape)."""
    import torch
    cells = spread_cells(N, 64, seed=11)
    rd_np = cells.rho_d.copy()
    rd_np[1, 7] = np.nan
    ts_np = cells.t_s.copy()
    ts_np[2, 20] = -1.0
    rg, rd, ts = t(cells.rho_g), t(rd_np), t(ts_np)
    v = t(cells.v)
    g = t(np.random.default_rng(5).standard_normal(cells.v.shape))
    out, tape = dx.apply_taped(rg, rd, ts, cells.dt, v, levels=32)
    assert dx.get_status() & dx.STATUS_BAD_CELL
    assert torch.isnan(out[:, :, 7]).all() and torch.isnan(out[:, :, 20]).all()
    ok = [c for c in range(64) if c not in (7, 20)]
    assert torch.isfinite(out[:, :, ok]).all()
    plain = dx.backward(rg, rd, ts, cells.dt, v, g)
    dx.get_status()
    taped = dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)
    assert dx.get_status() & dx.STATUS_BAD_CELL
    for a, b in zip(plain, taped):
        assert torch.isnan(b[..., 7]).all()
    if N + 1 > 12:
        for a, b in zip(plain, taped):
            assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    else:
        sub = cells.subset(np.array(ok))
        got = [x.cpu().numpy()[..., ok] for x in taped]
        ref = [x.cpu().numpy()[..., ok] for x in plain]
        assert_adjoint_parity(sub, g.cpu().numpy()[:, :, ok], got, ref)


def test_tape_full_size_sampled(dx):
    """The N = 16 configuration at full size (2,097,152 cells, the launch the
    benchmark times): taped and plain gradients identical on the whole array,
    the oracle's adjoint on 48 sampled cells."""
    import torch
    cells = W.workload("mrn_n16_128cube")
    C, N = cells.ncells, cells.nspecies
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    g_np = W.adjoint_target(C, N)
    g = t(g_np)
    out, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    assert torch.equal(out, dx.apply(rg, rd, ts, cells.dt, v))
    del out
    taped = dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)
    del tape
    plain = dx.backward(rg, rd, ts, cells.dt, v, g)
    for a, b in zip(plain, taped):
        assert torch.equal(a, b)
    idx = np.sort(np.random.default_rng(8).choice(C, 48, replace=False))
    sub = cells.subset(idx)
    gs = g_np[:, :, idx]
    rv, rrg, rrd, rts, _ = oracle.drag_backward(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, gs)
    got = [x.cpu().numpy()[..., idx] for x in taped]
    assert_adjoint_parity(sub, gs, got, (rv, rrg, rrd, rts))
    assert dx.get_status() == 0


def test_autograd_taped(dx):
    """DragExpmTaped gives DragExpm's values and gradients exactly."""
    import torch
    cells = W.workload("mrn_n16_128cube", ncells=500)
    target = t(W.adjoint_target(cells.ncells, cells.nspecies))
    grads = []
    outs = []
    for fn in (dx.DragExpm, dx.DragExpmTaped):
        rg = t(cells.rho_g).requires_grad_(True)
        rd = t(cells.rho_d).requires_grad_(True)
        ts = t(cells.t_s).requires_grad_(True)
        v = t(cells.v).requires_grad_(True)
        out = fn.apply(rg, rd, ts, cells.dt, v)
        loss = 0.5 * ((out - target) ** 2).sum()
        loss.backward()
        outs.append(out.detach())
        grads.append((rg.grad, rd.grad, ts.grad, v.grad))
    assert torch.equal(outs[0], outs[1])
    for a, b in zip(*grads):
        assert torch.equal(a, b)


@pytest.mark.parametrize("N", [1, 4, 5, 8, 9, 11])
def test_lane_per_cell_tape(dx, N):
    """n <= 12, default modes: the lane-per-cell forward writes the tape. Its v_out
    is drag_expm_apply's bit for bit; the taped gradients match the oracle's
    adjoint (and the recomputing adjoint) at the adjoint tolerances, bit for bit
    for n <= 9 where the adjoint runs lane per cell too; a tape whose
    fingerprints do not match (another dt) gives the recomputed gradients exactly
    (bit for bit up to n = 9, where the adjoint runs lane per cell too)."""
    import torch
    cells = spread_cells(N, 211, seed=170 + N)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    g_np = np.random.default_rng(N).standard_normal(cells.v.shape)
    g = t(g_np)
    out, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    assert torch.equal(out, dx.apply(rg, rd, ts, cells.dt, v))
    taped = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)]
    rv, rrg, rrd, rts, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g_np)
    assert_adjoint_parity(cells, g_np, taped, (rv, rrg, rrd, rts))
    plain = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g)]
    assert_adjoint_parity(cells, g_np, taped, plain)
    if N + 1 <= 9:
        # the lane-per-cell adjoint forms E as the lane-per-cell forward does: the
        # tape changes the work, not one bit of the gradients
        for a, b in zip(taped, plain):
            assert np.array_equal(a, b)
    dt2 = float(np.nextafter(cells.dt, 2.0))
    stale = dx.backward(rg, rd, ts, dt2, v, g, tape=tape)
    fresh = dx.backward(rg, rd, ts, dt2, v, g)
    for a, b in zip(stale, fresh):
        assert torch.equal(a, b)
    assert dx.get_status() == 0


def test_taped_finite_differences_64_cells(dx):
    """The N = 8 differentiation workload through the tape (written there by the
    lane-per-cell forward): loss 0.5 ||v_out - v_target||^2, gradients with
    respect to v_in, rho_d, t_s on 64 random cells against central differences
    of the GPU forward (1e-6 relative, as for the recomputing adjoint)."""
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=8192)
    target = W.adjoint_target(cells.ncells, cells.nspecies)
    idx = np.sort(np.random.default_rng(4321).choice(cells.ncells, 64, replace=False))
    sub = cells.subset(idx)
    vt = target[:, :, idx]

    def fwd(c):
        return dx.apply(t(c.rho_g), t(c.rho_d), t(c.t_s), c.dt, t(c.v)).cpu().numpy()

    rg, rd, ts = dev_args(sub)
    out, tape = dx.apply_taped(rg, rd, ts, sub.dt, t(sub.v))
    g = out.cpu().numpy() - vt
    gv, _, grd, gts = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, sub.dt, t(sub.v), t(g), tape=tape)]
    gv_fd, grd_fd, gts_fd = finite_difference_gradients(fwd, sub, vt)
    assert_fd_agreement(sub, g, gv, grd, gts, gv_fd, grd_fd, gts_fd)



@pytest.mark.parametrize("N", [4, 8, 10])
def test_binned_tape(dx, N):
    """Above its binning size the lane-per-cell taped forward runs the binned
    pipeline (6 launches), writing the same tape: v_out equals drag_expm_apply's
    bit for bit, and the taped gradients match the recomputing adjoint's to the
    adjoint tolerance on 1,500 sampled cells."""
    import torch
    C = 300001
    cells = W.mrn(C, N, seed=60 + N, stiff_lo=-4.0, stiff_hi=8.0)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    g_np = np.random.default_rng(N).standard_normal(cells.v.shape)
    g = t(g_np)
    assert dx.apply_launches(C, N) == 6
    out, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    assert torch.equal(out, dx.apply(rg, rd, ts, cells.dt, v))
    taped = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)]
    plain = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g)]
    idx = np.sort(np.random.default_rng(9).choice(C, 1500, replace=False))
    sub = cells.subset(idx)
    assert_adjoint_parity(sub, g_np[:, :, idx], [x[..., idx] for x in taped], [x[..., idx] for x in plain])
    if N + 1 <= 9:   # lane-per-cell adjoint (binned too): bit for bit
        for a, b in zip(taped, plain):
            assert np.array_equal(a, b)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [2, 5, 8])
def test_tape_across_kernel_families(dx, N):
    """One tape format for both kernel families: a tape the warp-per-cell
    forward wrote, read by the lane-per-cell adjoint, and one the lane-per-cell
    forward wrote, read by the warp-per-cell adjoint, both give the oracle's
    gradients at the adjoint tolerances."""
    cells = spread_cells(N, 223, seed=260 + N)
    rg, rd, ts = dev_args(cells)
    v = t(cells.v)
    g_np = np.random.default_rng(26 + N).standard_normal(cells.v.shape)
    g = t(g_np)
    ref = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g_np)[:4]
    saved = dx.get_mode(N)
    assert saved != dx.MODE_WARP_PER_CELL
    dx.set_mode(N, dx.MODE_WARP_PER_CELL)
    try:
        _, tape_w = dx.apply_taped(rg, rd, ts, cells.dt, v)
    finally:
        dx.set_mode(N, saved)
    got = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape_w)]
    assert_adjoint_parity(cells, g_np, got, ref)
    _, tape_l = dx.apply_taped(rg, rd, ts, cells.dt, v)
    dx.set_mode(N, dx.MODE_WARP_PER_CELL)
    try:
        got = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape_l)]
    finally:
        dx.set_mode(N, saved)
    assert_adjoint_parity(cells, g_np, got, ref)
    assert dx.get_status() == 0
