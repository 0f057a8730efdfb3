"""GPU batched entry point (drag_expm_apply_batched through the C ABI) against
the oracle's batched update, block by block. Same 1e-13 forward tolerance."""
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


def mixed_batch(seed=0):
    """Ragged blocks: sizes 0, 1, 31, 32, 33, 200; N in 1..31; dt in {0, 2^-k}."""
    rng = np.random.default_rng(seed)
    blocks = []
    sizes = [0, 1, 31, 32, 33, 200, 5, 64]
    for b in range(48):
        N = int(rng.choice([1, 2, 3, 4, 5, 7, 8, 9, 10, 12, 13, 16, 20, 31]))
        C = sizes[b % len(sizes)]
        dt = 0.0 if b % 11 == 3 else 2.0 ** -int(rng.integers(0, 7))
        cells = W.mrn(C, N, seed=1000 + b, stiff_lo=-4.0, stiff_hi=8.0, dt=dt, t_ref=1.0) if C else \
            W.Cells(np.zeros(0), np.zeros((N, 0)), np.zeros((N, 0)), np.zeros((3, N + 1, 0)), dt)
        blocks.append((N, dt, cells))
    return W.Batch(blocks)


def assert_block_parity(desc, v_in, out, ref):
    for b in range(len(desc)):
        N, C, vo = int(desc[b]["nspecies"]), int(desc[b]["ncells"]), int(desc[b]["vel_offset"])
        if C == 0:
            continue
        sl = slice(vo, vo + 3 * (N + 1) * C)
        o = out[sl].reshape(3, N + 1, C)
        r = ref[sl].reshape(3, N + 1, C)
        vi = v_in[sl].reshape(3, N + 1, C)
        sc = np.abs(vi).max(axis=1, keepdims=True)
        sc = np.where(sc > 0, sc, 1.0)
        err = np.max(np.abs(o - r) / sc)
        assert np.all(np.isfinite(o)) and err <= TOL, (b, N, C, err)


def test_batched_parity_mixed(dx):
    batch = mixed_batch()
    desc, rg, rd, ts, v = batch.pack()
    out = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v)).cpu().numpy()
    ref, st = oracle.drag_apply_batched(desc, rg, rd, ts, v)
    assert dx.get_status() == 0 and st == 0
    assert_block_parity(desc, v, out, ref)


def test_batched_follows_mode_table(dx):
    """The batched path takes lane- or warp-per-cell per n from the mode table:
    with N = 4 and N = 8 set to warp per cell, those blocks run warp per cell
    and still match the oracle."""
    batch = mixed_batch(seed=3)
    desc, rg, rd, ts, v = batch.pack()
    ref, st = oracle.drag_apply_batched(desc, rg, rd, ts, v)
    old = {N: dx.get_mode(N) for N in (4, 8)}
    try:
        for N in old:
            dx.set_mode(N, dx.MODE_WARP_PER_CELL)
        out = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v)).cpu().numpy()
    finally:
        for N, m in old.items():
            dx.set_mode(N, m)
    assert dx.get_status() == 0 and st == 0
    assert_block_parity(desc, v, out, ref)


def test_batched_matches_plain_entry_point(dx):
    """Per block, the batched result equals drag_expm_apply on the same cells to 1e-13
    (bit-identical where both take the same kernel family)."""
    batch = mixed_batch(seed=1)
    desc, rg, rd, ts, v = batch.pack()
    out = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v)).cpu().numpy()
    for b, (N, dt, cells) in enumerate(batch.blocks):
        if cells.ncells == 0:
            continue
        plain = dx.apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), dt, t(cells.v)).cpu().numpy()
        vo = int(desc[b]["vel_offset"])
        o = out[vo:vo + plain.size].reshape(plain.shape)
        sc = np.abs(cells.v).max(axis=1, keepdims=True)
        assert np.max(np.abs(o - plain) / sc) <= TOL


def test_batched_in_place_and_graph_replay(dx):
    import torch
    batch = mixed_batch(seed=2)
    desc, rg, rd, ts, v = batch.pack()
    ref = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v)).cpu().numpy()
    dblocks = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
    nmax = int(desc["nspecies"].max())
    a_rg, a_rd, a_ts, a_v = t(rg), t(rd), t(ts), t(v)
    out = torch.empty_like(a_v)
    ws = torch.empty(dx.batched_workspace_bytes(len(desc), rg.size), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dx.apply_batched(dblocks, a_rg, a_rd, a_ts, a_v, out, nspecies_max=nmax, workspace=ws)   # warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dx.apply_batched(dblocks, a_rg, a_rd, a_ts, a_v, out, nspecies_max=nmax, workspace=ws)
    out.zero_()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    # in place
    inp = t(v)
    dx.apply_batched(desc, a_rg, a_rd, a_ts, inp, inp)
    assert np.array_equal(inp.cpu().numpy(), ref)


def test_batched_bad_blocks_and_cells(dx):
    import torch
    batch = mixed_batch(seed=3)
    desc, rg, rd, ts, v = batch.pack()
    bad = desc.copy()
    victims = [i for i in range(len(bad)) if bad[i]["ncells"] > 0][:5]
    bad[victims[0]]["nspecies"] = 0
    bad[victims[1]]["dt"] = -1.0
    bad[victims[2]]["vel_offset"] = v.size            # out of range
    bad[victims[3]]["dt"] = np.nan
    bad[victims[4]]["cell_offset"] = -1
    sentinel = np.full_like(v, 7.0)
    out = dx.apply_batched(bad, t(rg), t(rd), t(ts), t(v), t(sentinel)).cpu().numpy()
    assert dx.get_status() & dx.STATUS_BAD_BLOCK
    ref, _ = oracle.drag_apply_batched(desc, rg, rd, ts, v)
    for b in range(len(desc)):
        N, C, vo = int(desc[b]["nspecies"]), int(desc[b]["ncells"]), int(desc[b]["vel_offset"])
        if C == 0:
            continue
        sl = slice(vo, vo + 3 * (N + 1) * C)
        if b in victims:
            assert np.all(out[sl] == 7.0)           # skipped blocks are left untouched
        else:
            sc = np.abs(v[sl].reshape(3, N + 1, C)).max(axis=1, keepdims=True)
            assert np.max(np.abs(out[sl] - ref[sl]).reshape(3, N + 1, C) / sc) <= TOL
    # invalid cell data inside a valid block
    rg2 = rg.copy()
    b = [i for i in range(len(desc)) if desc[i]["ncells"] > 1][0]
    rg2[desc[b]["cell_offset"]] = -1.0
    out2 = dx.apply_batched(desc, t(rg2), t(rd), t(ts), t(v)).cpu().numpy()
    assert dx.get_status() & dx.STATUS_BAD_CELL
    N, C, vo = int(desc[b]["nspecies"]), int(desc[b]["ncells"]), int(desc[b]["vel_offset"])
    o = out2[vo:vo + 3 * (N + 1) * C].reshape(3, N + 1, C)
    assert np.all(np.isnan(o[:, :, 0])) and np.all(np.isfinite(o[:, :, 1:]))


@pytest.mark.parametrize("nmax", [8, 15])
def test_batched_rejects_blocks_above_nspecies_max(dx, nmax):
    """A block whose N exceeds the nspecies_max argument (which sizes the main
    kernels' shared memory) is a bad block: it sets DRAG_STATUS_BAD_BLOCK and
    its v_out slice is left untouched; every other block matches the oracle.
    nmax = 8: the N = 9 blocks are one species over (n = 10 would run lane per
    cell); nmax = 15: the warp-per-cell sizes N = 16, 20, 31 are over."""
    batch = mixed_batch(seed=5)
    desc, rg, rd, ts, v = batch.pack()
    over = [b for b in range(len(desc)) if desc[b]["nspecies"] > nmax and desc[b]["ncells"] > 0]
    assert any(desc[b]["nspecies"] == nmax + 1 for b in over)
    sentinel = np.full_like(v, 7.0)
    dx.get_status()
    out = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v), t(sentinel), nspecies_max=nmax).cpu().numpy()
    assert dx.get_status() & dx.STATUS_BAD_BLOCK
    ok = np.array([b not in over for b in range(len(desc))])
    ref, st = oracle.drag_apply_batched(desc[ok], rg, rd, ts, v)
    assert st == 0
    for b in over:
        N, C, vo = int(desc[b]["nspecies"]), int(desc[b]["ncells"]), int(desc[b]["vel_offset"])
        assert np.all(out[vo:vo + 3 * (N + 1) * C] == 7.0), (b, N)
    assert_block_parity(desc[ok], v, out, ref)


def test_batched_workspace_and_argument_errors(dx):
    import torch
    batch = mixed_batch(seed=4)
    desc, rg, rd, ts, v = batch.pack()
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(dx.DragExpmError, match="-5"):
        dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v), workspace=small)
    with pytest.raises(dx.DragExpmError):
        dx.apply_batched(desc, t(rg), t(rd), t(ts[:-1]), t(v))
    assert dx.batched_workspace_bytes(len(desc), rg.size) > 12 * rg.size


def test_batched_amr_workload_full_size(dx):
    """The 1M-cell AMR-like mix (2048 blocks of 8^3 cells, N in {1,4,8,16},
    dt = 2^-k): every block of a 96-block sample against the oracle."""
    batch = W.batched()
    desc, rg, rd, ts, v = batch.pack()
    out = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v)).cpu().numpy()
    assert dx.get_status() == 0
    pick = np.random.default_rng(0).choice(len(desc), 96, replace=False)
    sub = desc[pick]
    ref, _ = oracle.drag_apply_batched(sub, rg, rd, ts, v)
    assert_block_parity(sub, v, out, ref)
