"""GPU adjoint (drag_expm_backward through the C ABI) against the oracle's
adjoint and against central finite differences of the GPU forward.

Tolerances:
* dL/dv_in = P^T g: per component, |gpu - oracle| <= 1e-13 * sum_f |g_{d,f}|
  (the 1-norm bounds |P^T g| since P is row-stochastic);
* parameter gradients, in log-derivative units x dL/dx, against the cell's
  loss scale S = sum_{d,f} |g_{d,f}| max_f' |v_{d,f'}|:
  |x (gpu - oracle)| <= 1e-13 S. Both implementations drop the stationary
  block of the Frechet direction (it cancels in every parameter gradient) and
  then sit within ~5e-15 S of a 50-digit truth even at dt/t_s = 1e8 (the
  oracle's pins), so 1e-13 S bounds their difference with margin;
* finite differences: 1e-6 relative (see
  tests/test_oracle_adjoint_pins.py for the exact criterion and its noise floor).
"""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W
from tests.dispatch_sizes import binned_threshold
from tests.test_oracle_adjoint_pins import assert_fd_agreement, finite_difference_gradients, loss_scale

pytestmark = pytest.mark.gpu
TOL_V = 1e-13
TOL_P = 1e-13


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


def gpu_backward(dx, cells, g):
    out = dx.backward(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v), t(g))
    return [o.cpu().numpy() for o in out]


def assert_adjoint_parity(cells, g, got, ref):
    gv, grg, grd, gts = got
    rv, rrg, rrd, rts = ref
    gsc = np.abs(g).sum(axis=1, keepdims=True)
    assert np.all(np.isfinite(gv)) and np.all(np.isfinite(grd)) and np.all(np.isfinite(gts))
    ev = np.max(np.abs(gv - rv) / gsc)
    assert ev <= TOL_V, ev
    S = np.array([loss_scale(g[:, :, c], cells.v[:, :, c]) for c in range(cells.ncells)])
    erd = np.max(np.abs(cells.rho_d * (grd - rrd)) / S[None, :])
    ets = np.max(np.abs(cells.t_s * (gts - rts)) / S[None, :])
    erg = np.max(np.abs(cells.rho_g * (grg - rrg)) / S)
    assert erd <= TOL_P and ets <= TOL_P and erg <= TOL_P, (erd, ets, erg)
    return ev, erd, ets, erg


CASES = [("dustybox_n1_32k", 1001), ("mrn_n4_128cube", 513), ("mrn_n8_128cube_adjoint", 385),
         ("mrn_n16_128cube", 97)]


@pytest.mark.parametrize("name,C", CASES)
def test_backward_parity_small(dx, name, C):
    cells = W.workload(name, ncells=C)
    g = np.random.default_rng(17).standard_normal(cells.v.shape)
    got = gpu_backward(dx, cells, g)
    rv, rrg, rrd, rts, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)
    assert_adjoint_parity(cells, g, got, (rv, rrg, rrd, rts))
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9, 12, 15, 20, 24, 31])
def test_backward_every_size(dx, N):
    cells = W.mrn(45 + N, N, seed=300 + N, stiff_lo=-4.0, stiff_hi=8.0)
    g = np.random.default_rng(N).standard_normal(cells.v.shape)
    got = gpu_backward(dx, cells, g)
    rv, rrg, rrd, rts, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)
    assert_adjoint_parity(cells, g, got, (rv, rrg, rrd, rts))


def test_backward_finite_differences_64_cells(dx):
    """The N=8 adjoint workload: loss 0.5 ||v_out - v_target||^2 with
    v_target ~ N(0,1); adjoint gradients with respect to v_in, rho_d, t_s on 64
    random cells against central differences of the GPU forward (1e-6 relative)."""
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=8192)
    target = W.adjoint_target(cells.ncells, cells.nspecies)
    idx = np.sort(np.random.default_rng(1234).choice(cells.ncells, 64, replace=False))
    sub = cells.subset(idx)
    vt = target[:, :, idx]

    def fwd(c):
        return dx.apply(t(c.rho_g), t(c.rho_d), t(c.t_s), c.dt, t(c.v)).cpu().numpy()

    g = fwd(sub) - vt
    gv, _, grd, gts = gpu_backward(dx, sub, g)
    gv_fd, grd_fd, gts_fd = finite_difference_gradients(fwd, sub, vt)
    assert_fd_agreement(sub, g, gv, grd, gts, gv_fd, grd_fd, gts_fd)


def test_autograd_function(dx):
    """torch.autograd through DragExpm gives the same gradients as the raw entry point."""
    import torch
    cells = W.workload("mrn_n4_128cube", ncells=300)
    target = t(W.adjoint_target(cells.ncells, cells.nspecies))
    rg = t(cells.rho_g).requires_grad_(True)
    rd = t(cells.rho_d).requires_grad_(True)
    ts = t(cells.t_s).requires_grad_(True)
    v = t(cells.v).requires_grad_(True)
    out = dx.DragExpm.apply(rg, rd, ts, cells.dt, v)
    loss = 0.5 * ((out - target) ** 2).sum()
    loss.backward()
    g = (out - target).detach()
    gv, grg, grd, gts = dx.backward(rg.detach(), rd.detach(), ts.detach(), cells.dt, v.detach(), g)
    assert torch.equal(v.grad, gv) and torch.equal(rd.grad, grd) and torch.equal(ts.grad, gts)
    assert torch.equal(rg.grad, grg)


def test_autograd_fit_stopping_times(dx):
    """Gradient descent on log t_s through the adjoint recovers stopping times
    from observed velocities (the fitting use of the adjoint)."""
    import torch
    rng = np.random.default_rng(5)
    C, N = 256, 3
    cells = W.mrn(C, N, seed=77, stiff_lo=-1.0, stiff_hi=4.0)
    true_ts = t(cells.t_s)
    obs = dx.apply(t(cells.rho_g), t(cells.rho_d), true_ts, cells.dt, t(cells.v))
    log_ts = (torch.log(true_ts) + torch.from_numpy(rng.uniform(-0.3, 0.3, (N, C))).cuda()).requires_grad_(True)
    opt = torch.optim.Adam([log_ts], lr=0.05)
    first = None
    for it in range(150):
        opt.zero_grad()
        out = dx.DragExpm.apply(t(cells.rho_g), t(cells.rho_d), torch.exp(log_ts), cells.dt, t(cells.v))
        loss = ((out - obs) ** 2).sum()
        loss.backward()
        opt.step()
        first = float(loss.detach()) if first is None else first
    assert float(loss.detach()) < 1e-3 * first


def test_backward_partial_outputs_and_invalid(dx):
    import torch
    cells = W.workload("mrn_n4_128cube", ncells=64)
    cells.t_s[2, 5] = -1.0
    g = np.random.default_rng(2).standard_normal(cells.v.shape)
    gv, grg, grd, gts = dx.backward(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v), t(g),
                                    need_v_in=False, need_rho_g=False)
    assert gv is None and grg is None
    grd, gts = grd.cpu().numpy(), gts.cpu().numpy()
    assert np.all(np.isnan(grd[:, 5])) and np.all(np.isnan(gts[:, 5]))
    assert dx.get_status() & dx.STATUS_BAD_CELL
    good = [c for c in range(64) if c != 5]
    sub = cells.subset(good)
    rv, rrg, rrd, rts, _ = oracle.drag_backward(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, g[:, :, good])
    S = np.array([loss_scale(g[:, :, c], cells.v[:, :, c]) for c in good])
    assert np.max(np.abs(sub.rho_d * (grd[:, good] - rrd)) / S) <= TOL_P


@pytest.mark.parametrize("name", ["mrn_n8_128cube_adjoint"])
def test_backward_full_size_sampled(dx, name):
    """Full-size adjoint workload in the benchmark's launch configuration;
    128 sampled cells against the oracle's adjoint."""
    import torch
    cells = W.workload(name)
    target = W.adjoint_target(cells.ncells, cells.nspecies)
    rg, rd, ts, v = t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v)
    out = dx.apply(rg, rd, ts, cells.dt, v)
    g = out - t(target)
    gv, grg, grd, gts = dx.backward(rg, rd, ts, cells.dt, v, g)
    torch.cuda.synchronize()
    assert dx.get_status() == 0
    idx = np.unique(np.concatenate([np.random.default_rng(3).integers(0, cells.ncells, 126), [0, cells.ncells - 1]]))
    sub = cells.subset(idx)
    ti = torch.from_numpy(idx).cuda()
    gs = g[:, :, ti].cpu().numpy()
    ref = oracle.drag_backward(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, gs)[:4]
    got = (gv[:, :, ti].cpu().numpy(), grg[ti].cpu().numpy(), grd[:, ti].cpu().numpy(), gts[:, ti].cpu().numpy())
    assert_adjoint_parity(sub, gs, got, ref)


def test_backward_extreme_norms(dx):
    """The adjoint at very large norms. dL/dv_in = P^T g must match the oracle
    up to norms of 1.5e308 (s* ~ 1023, every cell fully relaxed). The parameter
    gradients come from the chain rule alpha dt (Z_0i - Z_00) etc., in which
    alpha dt multiplies the rounding of Z: they are checked in full up to
    |A| ~ 1e14 (alpha dt u << 1); beyond ~1/u both implementations return
    rounding-dominated values, as the design notes state."""
    from tests.test_forward_gpu import extreme_cells
    cells = extreme_cells(8, [1e250, 1e300, 1.5e308])
    g = np.random.default_rng(8).standard_normal(cells.v.shape)
    gv = gpu_backward(dx, cells, g)[0]
    rv = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)[0]
    assert np.all(np.isfinite(gv))
    assert np.max(np.abs(gv - rv) / np.abs(g).sum(axis=1, keepdims=True)) <= TOL_V
    cells = extreme_cells(8, [1e8, 1e11, 1e14])
    g = np.random.default_rng(9).standard_normal(cells.v.shape)
    got = gpu_backward(dx, cells, g)
    ref = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)[:4]
    assert_adjoint_parity(cells, g, got, ref)
    assert dx.get_status() == 0


# ---- lane-per-cell adjoint (n = N + 1 <= 9 under a lane-per-cell mode, the default there;
# n = 7..9 keep L in registers and E in shared memory)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_backward_both_kernel_families(dx, N):
    """Under the default (lane-per-cell) mode the adjoint runs one lane per cell;
    under the warp-per-cell mode one warp per cell. Both match the oracle's
    adjoint on a ragged count of cells spread over ten decades of stiffness."""
    cells = W.mrn(677 + 3 * N, N, seed=500 + N, stiff_lo=-5.0, stiff_hi=8.0)
    g = np.random.default_rng(50 + N).standard_normal(cells.v.shape)
    ref = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)[:4]
    assert dx.get_mode(N) != dx.MODE_WARP_PER_CELL
    assert_adjoint_parity(cells, g, gpu_backward(dx, cells, g), ref)
    saved = dx.get_mode(N)
    dx.set_mode(N, dx.MODE_WARP_PER_CELL)
    try:
        wpc = gpu_backward(dx, cells, g)
    finally:
        dx.set_mode(N, saved)
    assert_adjoint_parity(cells, g, wpc, ref)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [1, 4, 6, 8])
def test_lane_per_cell_backward_extreme_norms(dx, N):
    """The lane-per-cell adjoint at norms up to 1.5e308 (s* ~ 1023; dL/dv_in
    checked) and up to 1e14 (all gradients), as for the warp-per-cell one."""
    from tests.test_forward_gpu import extreme_cells
    cells = extreme_cells(N, [1e250, 1e300, 1.5e308])
    g = np.random.default_rng(8).standard_normal(cells.v.shape)
    gv = gpu_backward(dx, cells, g)[0]
    rv = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)[0]
    assert np.all(np.isfinite(gv))
    assert np.max(np.abs(gv - rv) / np.abs(g).sum(axis=1, keepdims=True)) <= TOL_V
    cells = extreme_cells(N, [1e8, 1e11, 1e14])
    g = np.random.default_rng(9).standard_normal(cells.v.shape)
    ref = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)[:4]
    assert_adjoint_parity(cells, g, gpu_backward(dx, cells, g), ref)
    assert dx.get_status() == 0


def test_lane_per_cell_backward_finite_differences(dx):
    """The N = 4 workload through the lane-per-cell adjoint: 64 random cells
    against central differences of the GPU forward (1e-6 relative)."""
    cells = W.workload("mrn_n4_128cube", ncells=8192)
    target = W.adjoint_target(cells.ncells, cells.nspecies)
    idx = np.sort(np.random.default_rng(99).choice(cells.ncells, 64, replace=False))
    sub = cells.subset(idx)
    vt = target[:, :, idx]

    def fwd(c):
        return dx.apply(t(c.rho_g), t(c.rho_d), t(c.t_s), c.dt, t(c.v)).cpu().numpy()

    g = fwd(sub) - vt
    gv, _, grd, gts = gpu_backward(dx, sub, g)
    gv_fd, grd_fd, gts_fd = finite_difference_gradients(fwd, sub, vt)
    assert_fd_agreement(sub, g, gv, grd, gts, gv_fd, grd_fd, gts_fd)


def test_lane_per_cell_backward_full_size_sampled(dx):
    """The N = 4 workload at full size (2,097,152 cells: tiles of 512 sorted
    cells): 128 sampled cells against the oracle's adjoint."""
    test_backward_full_size_sampled(dx, "mrn_n4_128cube")


@pytest.mark.parametrize("N", [1, 4, 5, 6, 8])
def test_lane_per_cell_backward_binned(dx, N):
    """From its binning size on (per N, as the library reports it) the
    lane-per-cell adjoint bins the cells by (k*, s*) over the whole input
    before running them: its gradients equal, bit for bit, those of the
    tile-sorted kernel that runs on the cells below that size (the per-cell
    arithmetic does not depend on the grouping), and sampled cells match the
    oracle's adjoint; through the tape they are unchanged."""
    import torch
    C = 300007
    thr = binned_threshold(dx, N, adjoint=True)
    assert dx.backward_launches(C, N) == 6 and dx.backward_launches(thr - 1, N) == 1
    cells = W.mrn(C, N, seed=410 + N, stiff_lo=-5.0, stiff_hi=8.0)
    g_np = np.random.default_rng(41 + N).standard_normal(cells.v.shape)
    rg, rd, ts, v, g = t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v), t(g_np)
    binned = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g)]
    head = np.arange(thr - 1)
    sub = cells.subset(head)
    tiled = gpu_backward(dx, sub, g_np[:, :, head])
    for a, b in zip(binned, tiled):
        assert np.array_equal(a[..., head], b)
    idx = np.unique(np.concatenate([np.random.default_rng(N).integers(0, C, 160), [0, C - 1]]))
    sub = cells.subset(idx)
    ref = oracle.drag_backward(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, g_np[:, :, idx])[:4]
    assert_adjoint_parity(sub, g_np[:, :, idx], [x[..., idx] for x in binned], ref)
    _, tape = dx.apply_taped(rg, rd, ts, cells.dt, v)
    taped = [x.cpu().numpy() for x in dx.backward(rg, rd, ts, cells.dt, v, g, tape=tape)]
    for a, b in zip(binned, taped):
        assert np.array_equal(a, b)
    assert dx.get_status() == 0
    torch.cuda.synchronize()


def test_lane_per_cell_backward_in_cuda_graph(dx):
    """The binned adjoint (scratch from the library's stream-ordered pool) can
    be captured in a CUDA graph and replayed with the same results."""
    import torch
    C, N = 270001, 4
    cells = W.mrn(C, N, seed=77, stiff_lo=-4.0, stiff_hi=8.0)
    rg, rd, ts, v = t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v)
    g = t(np.random.default_rng(7).standard_normal(cells.v.shape))
    ref = dx.backward(rg, rd, ts, cells.dt, v, g)
    out = tuple(torch.empty_like(x) for x in ref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        dx.backward(rg, rd, ts, cells.dt, v, g, out=out)   # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        dx.backward(rg, rd, ts, cells.dt, v, g, out=out)
    for x in out:
        x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [4, 8])
def test_lane_per_cell_backward_binned_invalid_cells(dx, N):
    """Invalid cells inside a binned lane-per-cell adjoint (270,001 cells; N = 8
    with the hybrid storage): NaN gradients and the status bit there, oracle
    gradients elsewhere."""
    import torch
    C = 270001
    cells = W.mrn(C, N, seed=91, stiff_lo=-4.0, stiff_hi=8.0)
    bad = [5, 123456, C - 1]
    cells.t_s[1, bad[0]] = -1.0
    cells.rho_d[N - 1, bad[1]] = np.nan
    cells.t_s[0, bad[2]] = 0.0
    g_np = np.random.default_rng(91).standard_normal(cells.v.shape)
    out = [x.cpu().numpy() for x in dx.backward(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v),
                                                 t(g_np))]
    torch.cuda.synchronize()
    for x in out:
        assert np.all(np.isnan(x[..., bad]))
    assert dx.get_status() & dx.STATUS_BAD_CELL
    idx = np.setdiff1d(np.unique(np.random.default_rng(5).integers(0, C, 120)), bad)
    sub = cells.subset(idx)
    ref = oracle.drag_backward(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, g_np[:, :, idx])[:4]
    assert_adjoint_parity(sub, g_np[:, :, idx], [x[..., idx] for x in out], ref)
