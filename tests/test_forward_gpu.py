"""GPU forward parity: libdragexpm (through its C ABI) against the CPU oracle.

Tolerance: per cell and velocity component d, for every fluid f,
|v_gpu - v_oracle| <= 1e-13 * max_f |v_in[d, f]| (the update is a convex
combination of the inputs, so this is the natural scale of the result).
"""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W
from tests.dispatch_sizes import binned_threshold

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


def dev(cells):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v)


def gpu_apply(dx, cells, dt=None):
    rg, rd, ts, v = dev(cells)
    out = dx.apply(rg, rd, ts, cells.dt if dt is None else dt, v)
    return out.cpu().numpy()


def assert_parity(out, ref, vin, tol=TOL):
    sc = np.abs(vin).max(axis=1, keepdims=True)
    sc = np.where(sc > 0, sc, 1.0)
    err = np.abs(out - ref) / sc
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert np.all(np.isfinite(out))
    assert err.max() <= tol, f"max scaled error {err.max():.3e} at {worst}"
    return err.max()


CASES = [("dustybox_n1_32k", 3001), ("mrn_n4_128cube", 1537), ("mrn_n8_128cube_adjoint", 777),
         ("mrn_n16_128cube", 301)]


@pytest.mark.parametrize("name,C", CASES)
def test_forward_parity_small(dx, name, C):
    cells = W.workload(name, ncells=C)
    out = gpu_apply(dx, cells)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert_parity(out, ref, cells.v)
    assert dx.get_status() == 0


@pytest.mark.parametrize("name,C", CASES)
def test_select_bit_exact(dx, name, C):
    """(k*, s*) of Algorithm 2: integer decisions must match the oracle exactly."""
    cells = W.workload(name, ncells=C)
    rg, rd, ts, _ = dev(cells)
    k, s = dx.select(rg, rd, ts, cells.dt)
    _, ko, so, _ = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, return_ks=True)
    assert np.array_equal(k.cpu().numpy(), ko)
    assert np.array_equal(s.cpu().numpy(), so)


@pytest.mark.parametrize("N", list(range(1, 32)))
def test_forward_every_nspecies(dx, N):
    """Every supported species count, stiff MRN-like cells, ragged cell count."""
    cells = W.mrn(97 + N, N, seed=100 + N, stiff_lo=-4.0, stiff_hi=8.0)
    out = gpu_apply(dx, cells)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert_parity(out, ref, cells.v)


@pytest.mark.parametrize("dt", [0.0, 1e-12, 1e-3, 1.0, 1e3])
def test_forward_dt_range(dx, dt):
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=129)
    out = gpu_apply(dx, cells, dt=dt)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, dt, cells.v)
    assert_parity(out, ref, cells.v)
    if dt == 0.0:
        assert np.array_equal(out, cells.v)


def test_in_place(dx):
    import torch
    cells = W.workload("mrn_n4_128cube", ncells=1000)
    rg, rd, ts, v = dev(cells)
    ref = dx.apply(rg, rd, ts, cells.dt, v).clone()
    dx.apply(rg, rd, ts, cells.dt, v, v_out=v)
    assert torch.equal(ref, v)


def test_decoupled_and_zero_density(dx):
    rng = np.random.default_rng(1)
    N, C = 5, 64
    cells = W.mrn(C, N, seed=9, stiff_lo=-2.0, stiff_hi=6.0)
    cells.t_s[1] = np.inf
    cells.rho_d[2] = 0.0
    cells.rho_d[3, ::2] = 1e-250 * cells.rho_g[::2]
    out = gpu_apply(dx, cells)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert_parity(out, ref, cells.v)
    assert np.array_equal(out[:, 2], cells.v[:, 2])


def test_invalid_cells_flagged(dx):
    cells = W.workload("mrn_n4_128cube", ncells=40)
    cells.rho_g[3] = 0.0
    cells.rho_d[1, 7] = -1.0
    cells.t_s[2, 11] = 0.0
    cells.t_s[0, 13] = np.nan
    cells.rho_d[3, 17] = np.inf
    out = gpu_apply(dx, cells)
    bad = [3, 7, 11, 13, 17]
    good = [c for c in range(40) if c not in bad]
    assert np.all(np.isnan(out[:, :, bad]))
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert_parity(out[:, :, good], ref[:, :, good], cells.v[:, :, good])
    assert dx.get_status() & dx.STATUS_BAD_CELL
    assert dx.get_status() == 0          # cleared by the read


def test_empty_is_noop(dx):
    import torch
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    out = dx.apply(z, z.reshape(4, 0), z.reshape(4, 0), 1.0, z.reshape(3, 5, 0))
    assert out.shape == (3, 5, 0)


def test_matches_eigen_truth(dx):
    pytest.importorskip("mpmath")
    from oracle.truth import drag_truth
    cells = W.workload("mrn_n16_128cube", ncells=24)
    out = gpu_apply(dx, cells)
    ref = drag_truth(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert_parity(out, ref, cells.v, tol=4e-15)


@pytest.mark.parametrize("name", ["mrn_n16_128cube", "mrn_n4_128cube", "mrn_n8_128cube_adjoint", "dustybox_n1_32k"])
def test_full_size_sampled(dx, name):
    """Full-size workload in the benchmark's launch configuration: 256 sampled
    cells against the oracle, conservation and convexity on every cell."""
    import torch
    cells = W.workload(name)
    rg, rd, ts, v = dev(cells)
    out = dx.apply(rg, rd, ts, cells.dt, v)
    torch.cuda.synchronize()
    assert dx.get_status() == 0
    C = cells.ncells
    idx = np.unique(np.concatenate([np.random.default_rng(0).integers(0, C, 254), [0, C - 1]]))
    sub = cells.subset(idx)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    assert_parity(out[:, :, torch.from_numpy(idx).cuda()].cpu().numpy(), ref, sub.v)
    rho = torch.cat([rg[None, :], rd], 0)
    mom_in = torch.einsum("fc,dfc->dc", rho, v)
    mom_out = torch.einsum("fc,dfc->dc", rho, out)
    scale = torch.einsum("fc,dfc->dc", rho, v.abs())
    assert bool(((mom_out - mom_in).abs() <= 8e-15 * scale).all())
    vsc = v.abs().amax(dim=1)
    assert bool((out.amin(dim=1) >= v.amin(dim=1) - 4e-15 * vsc).all())
    assert bool((out.amax(dim=1) <= v.amax(dim=1) + 4e-15 * vsc).all())


@pytest.mark.parametrize("N", [1, 4, 7, 9])
def test_sorted_tiles_parity(dx, N):
    """320,077 cells, every cell against the oracle, through both lane-per-cell
    paths: the binned pipeline (the default at this size for N = 2..8) and the
    tile-sorted kernel (each tile of up to 512 cells sorted by a cost proxy,
    ragged last tile; forced here by the all-shared storage mode)."""
    cells = W.mrn(320077, N, seed=900 + N, stiff_lo=-4.0, stiff_hi=8.0)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    out = gpu_apply(dx, cells)
    assert_parity(out, ref, cells.v)
    old = dx.get_mode(N)
    try:
        dx.set_mode(N, dx.MODE_LANE_SHARED)
        assert dx.apply_launches(cells.ncells, N) == 1
        out = gpu_apply(dx, cells)
    finally:
        dx.set_mode(N, old)
    assert_parity(out, ref, cells.v)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [2, 4, 6, 8, 10])
def test_binned_forward(dx, N):
    """From its binning size on (per N, as the library reports it) a default
    lane-per-cell size runs the batched pipeline over one block (6 launches).
    The per-cell arithmetic is that of the tile-sorted kernel, which
    drag_expm_apply_heat always uses: identical v_out. In place, invalid cells
    (NaN and the status bit) and dt = 0 too."""
    import torch
    thr = binned_threshold(dx, N)
    C = max(300001, thr + 17)
    cells = W.mrn(C, N, seed=40 + N, stiff_lo=-4.0, stiff_hi=8.0)
    cells.rho_d[0, 11] = np.nan
    cells.t_s[-1, 222222] = 0.0
    rg, rd, ts, v = dev(cells)
    assert dx.apply_launches(C, N) == 6 and dx.apply_launches(thr - 1, N) == 1
    out = dx.apply(rg, rd, ts, cells.dt, v)
    assert dx.get_status() & dx.STATUS_BAD_CELL
    heat_out, _ = dx.apply_heat(rg, rd, ts, cells.dt, v)
    dx.get_status()
    assert torch.equal(torch.nan_to_num(out, nan=3.0), torch.nan_to_num(heat_out, nan=3.0))
    assert bool(torch.isnan(out[:, :, 11]).all()) and bool(torch.isnan(out[:, :, 222222]).all())
    ok = torch.ones(C, dtype=torch.bool, device=out.device)
    ok[[11, 222222]] = False
    assert bool(torch.isfinite(out[:, :, ok]).all())
    vin = v.clone()
    dx.apply(rg, rd, ts, cells.dt, vin, vin)                        # in place
    dx.get_status()
    assert torch.equal(torch.nan_to_num(vin, nan=3.0), torch.nan_to_num(out, nan=3.0))
    zero = dx.apply(rg, rd, ts, 0.0, v)
    dx.get_status()
    assert torch.equal(zero[:, :, ok], v[:, :, ok])


@pytest.mark.parametrize("N", [1, 3, 5])
def test_tile_sorted_forward_small_and_prefix(dx, N):
    """Below its binning size a register-storage size (n <= 6) runs one
    tile-sorted (or balanced-block) launch. Ragged sizes (part of a CTA, one
    cell) against the oracle; and, since the per-cell routine is the binned
    pipeline's, the cells below the binning size of an input ~100,000 cells
    above it give the binned run's v_out bit for bit."""
    import torch
    for C in (1, 100, 1025, 32785):
        cells = W.mrn(C, N, seed=70 + C % 97 + N, stiff_lo=-5.0, stiff_hi=8.0)
        ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
        assert dx.apply_launches(C, N) == 1
        assert_parity(gpu_apply(dx, cells), ref, cells.v)
    thr = binned_threshold(dx, N)
    if thr is None:   # N = 1 never bins: one launch at any size
        assert dx.apply_launches(2 * 10**6, N) == 1
        return
    C, head = thr + 99998, thr - 1
    cells = W.mrn(C, N, seed=80 + N, stiff_lo=-4.0, stiff_hi=8.0)
    rg, rd, ts, v = dev(cells)
    binned = dx.apply(rg, rd, ts, cells.dt, v)
    sub = cells.subset(np.arange(head))
    srg, srd, sts, sv = dev(sub)
    tiled = dx.apply(srg, srd, sts, cells.dt, sv)
    assert dx.apply_launches(head, N) == 1 and dx.apply_launches(C, N) == 6
    assert torch.equal(tiled, binned[:, :, :head])
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [1, 4, 5])
def test_balanced_blocks_forward_edges(dx, N):
    """Register-storage sizes with more than 128 cells per SM run blocks of up
    to 16 warps (8 at n = 6), a multiple of the SM count of them, each sorting
    a contiguous share and dealing its groups to the warp slots in snake order.
    Against the oracle (every cell): just past 128 cells per SM, the most one
    block per SM takes, and one cell more (two blocks per SM). The first 128 x SMs
    cells bit for bit against a one-block-per-SM tile-sorted launch on them;
    the energy epilogue through the same kernel."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    top = sms * (512 if N <= 4 else 256)
    low = 128 * sms
    for C in (low + 1, top, top + 1):
        cells = W.mrn(C, N, seed=900 + C % 89 + N, stiff_lo=-4.0, stiff_hi=8.0)
        rg, rd, ts, v = dev(cells)
        out = dx.apply(rg, rd, ts, cells.dt, v)
        assert dx.get_status() == 0
        ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
        assert_parity(out.cpu().numpy(), ref, cells.v)
        prg, prd, pts, pv = dev(cells.subset(np.arange(low)))
        tiled = dx.apply(prg, prd, pts, cells.dt, pv)
        assert torch.equal(tiled, out[:, :, :low])
        hout, heat = dx.apply_heat(rg, rd, ts, cells.dt, v)
        _, pheat = dx.apply_heat(prg, prd, pts, cells.dt, pv)
        assert torch.equal(hout, out) and torch.equal(pheat, heat[:low])
        assert bool(torch.isfinite(heat).all())
        assert dx.get_status() == 0


def test_binned_forward_wide_chunks(dx):
    """Above 64 chunks of 65,536 cells the binned forward widens its chunks
    (here 4,500,001 cells of N = 2: 64 chunks of 70,313 cells, the last one
    ragged). Sampled cells against the oracle, the first 196,607 cells (below
    the binning size) bit for bit against the tile-sorted kernel, and the
    status word clean."""
    import torch
    C, N = 4500001, 2
    cells = W.mrn(C, N, seed=4242, stiff_lo=-4.0, stiff_hi=8.0)
    rg, rd, ts, v = dev(cells)
    assert dx.apply_launches(C, N) == 6
    out = dx.apply(rg, rd, ts, cells.dt, v)
    assert dx.get_status() == 0
    idx = np.unique(np.concatenate([np.random.default_rng(1).integers(0, C, 400),
                                    [0, 70312, 70313, C - 2, C - 1]]))
    sub = cells.subset(idx)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    assert_parity(out[:, :, idx].cpu().numpy(), ref, sub.v)
    head = binned_threshold(dx, N) - 1
    hrg, hrd, hts, hv = dev(cells.subset(np.arange(head)))
    tiled = dx.apply(hrg, hrd, hts, cells.dt, hv)
    assert torch.equal(tiled, out[:, :, :head])
    assert dx.get_status() == 0


def extreme_cells(N, norms, seed=3):
    """Cells whose 1-norm |A|_1 is about `norms[c]` (rho_d = rho_g = 1, dt = 1,
    stopping times spread over a factor 2): s* up to ~1023."""
    rng = np.random.default_rng(seed)
    C = len(norms)
    t_s = np.empty((N, C))
    for c, nrm in enumerate(norms):
        t_s[:, c] = 2.0 * N / nrm * (1.0 + np.arange(N) / N)
    return W.Cells(np.ones(C), np.ones((N, C)), t_s, rng.standard_normal((3, N + 1, C)), 1.0)


@pytest.mark.parametrize("N", [4, 16])
def test_extreme_norms(dx, N):
    """Norms from 1e250 to 1.5e308: the scaling 2^-s* leaves the normal range
    past s* = 1022; every cell must still match the oracle. A norm that
    overflows (a stopping time below 1/DBL_MAX) is an invalid cell on both
    sides: NaN outputs and the status bit."""
    norms = [1e250, 1e300, 5e306, 1.5e308]
    cells = extreme_cells(N, norms)
    out = gpu_apply(dx, cells)
    ref, k, s, st = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, return_ks=True)
    assert st == 0 and s.max() >= 1022, s
    assert_parity(out, ref, cells.v)
    kg, sg = dx.select(*dev(cells)[:3], cells.dt)
    assert np.array_equal(kg.cpu().numpy(), k) and np.array_equal(sg.cpu().numpy(), s)
    assert dx.get_status() == 0
    bad = extreme_cells(N, [1e300, 1e300])
    bad.t_s[0, 1] = 1e-310
    out = gpu_apply(dx, bad)
    ref, _, _, st = oracle.drag_apply(bad.rho_g, bad.rho_d, bad.t_s, bad.dt, bad.v, return_ks=True)
    assert st == 1 and np.all(np.isnan(ref[:, :, 1]))
    assert np.all(np.isnan(out[:, :, 1])) and np.all(np.isfinite(out[:, :, 0]))
    assert dx.get_status() & dx.STATUS_BAD_CELL


def test_binned_forward_in_cuda_graph(dx):
    """The binned forward (scratch taken stream-ordered from the library's pool)
    is captured in a CUDA graph and replayed: same outputs as eager calls, also
    after the inputs change in place between replays."""
    import torch
    N, C = 4, 262147
    cells = W.mrn(C, N, seed=77, stiff_lo=-4.0, stiff_hi=8.0)
    rg, rd, ts, v = dev(cells)
    assert dx.apply_launches(C, N) == 6
    out = torch.empty_like(v)
    eager = dx.apply(rg, rd, ts, cells.dt, v)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        dx.apply(rg, rd, ts, cells.dt, v, out)          # warm-up outside capture (pool, attributes)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dx.apply(rg, rd, ts, cells.dt, v, out)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    v.mul_(-0.5)
    ts.mul_(3.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, dx.apply(rg, rd, ts, cells.dt, v))
    assert dx.get_status() == 0


@pytest.mark.parametrize("N", [12, 15, 16, 17])
def test_paired_setup_any_partner(dx, N):
    """For N <= 16 the warp-per-cell forward sets up two cells at a time (one
    half-warp each): consecutive cells in drag_expm_apply, consecutive cells
    of a (k*, s*) bin in the batched entry point, so a cell gets another
    partner in each. One block of 37 cells through both (the last pair of a
    16-cell block holds one cell), with invalid cells in the first and the
    second slot of a pair: v_out equal bit for bit (NaN where invalid), the
    valid cells against the oracle, the status bit set by both. N = 17 sets up
    one cell at a time in both. (That the paired set-up gives the one-cell
    set-up's bits is checked through the tape: the warp-per-cell adjoint
    re-forms E_t after a one-cell set-up and must reproduce the taped
    gradients bit for bit, tests/test_tape_gpu.py.)"""
    import torch
    C = 37
    cells = W.mrn(C, N, seed=600 + N, stiff_lo=-4.0, stiff_hi=8.0)
    cells.rho_d[N - 1, 5] = -1.0         # second cell of a pair
    cells.t_s[0, 8] = 0.0                # first cell of a pair
    cells.rho_g[36] = np.nan             # the lone cell of the last pair
    bad = [5, 8, 36]
    rg, rd, ts, v = dev(cells)
    dx.get_status()
    plain = dx.apply(rg, rd, ts, cells.dt, v)
    assert dx.get_status() & dx.STATUS_BAD_CELL
    desc, brg, brd, bts, bv = W.Batch([(N, cells.dt, cells)]).pack()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    batched = dx.apply_batched(desc, t(brg), t(brd), t(bts), t(bv)).reshape(plain.shape)
    assert dx.get_status() & dx.STATUS_BAD_CELL
    assert torch.equal(torch.nan_to_num(plain, nan=5.0), torch.nan_to_num(batched, nan=5.0))
    assert bool(torch.isnan(plain[:, :, bad]).all())
    ok = np.setdiff1d(np.arange(C), bad)
    sub = cells.subset(ok)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    assert_parity(plain[:, :, ok].cpu().numpy(), ref, sub.v)


@pytest.mark.parametrize("C", [1000, 40000])
def test_velocity_form_n1_special_cells(dx, C):
    """N = 1 runs in the velocity form (the pair (p, q) of P = I + W), through the
    tile-sorted kernel (1,000 cells) or the balanced blocks with the counting
    sort (40,000). Decoupled cells (t_s = inf) return v_in exactly; cells
    without dust keep the gas velocity exactly; a dust-to-gas ratio of 1e-250
    and the rest against the oracle; dt = 0 returns v_in exactly."""
    cells = W.mrn(C, 1, seed=77 + C % 13, stiff_lo=-4.0, stiff_hi=8.0)
    cells.t_s[0, ::7] = np.inf
    cells.rho_d[0, 3::7] = 0.0
    cells.rho_d[0, 5::7] = 1e-250 * cells.rho_g[5::7]
    out = gpu_apply(dx, cells)
    assert dx.get_status() == 0
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert_parity(out, ref, cells.v)
    assert np.array_equal(out[:, :, ::7], cells.v[:, :, ::7])
    assert np.array_equal(out[:, 0, 3::7], cells.v[:, 0, 3::7])
    assert np.array_equal(gpu_apply(dx, cells, dt=0.0), cells.v)
