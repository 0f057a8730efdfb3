"""Sharding of a drag workload over ranks (CPU; gloo, world size 2).

The drag step is cell local (Sec. 2.4), so a partitioned run must give, rank
by rank, exactly the cells' results of a single-rank run. Checked here with
the oracle as each rank's compute: contiguous cell ranges of a single-N
workload, and whole blocks of an AMR-like batch dealt by cost, both gathered
to rank 0 and compared bit for bit with one rank's result."""
import os
import socket

import numpy as np
import pytest

from paper_2509_25347_gb300 import shard
from paper_2509_25347_gb300 import workloads as W


def test_cell_ranges_cover_every_cell_once():
    for C in (0, 1, 7, 32768, 2097152, 2097153):
        for world in (1, 2, 3, 4, 8):
            seen = np.zeros(C, dtype=np.int64)
            sizes = []
            for r in range(world):
                a, b = shard.cell_range(C, r, world)
                seen[a:b] += 1
                sizes.append(b - a)
            assert np.all(seen == 1)
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.cell_range(10, 2, 2)


def test_balance_blocks_partition_and_bound():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        cost = 10.0 ** rng.uniform(2, 6, 501)          # costs spanning four decades, as (N, s*) do
        parts = shard.balance_blocks(cost, world)
        allb = np.sort(np.concatenate(parts))
        assert np.array_equal(allb, np.arange(cost.size))
        loads = np.array([cost[p].sum() for p in parts])
        assert loads.max() <= cost.sum() / world + cost.max()
        if world > 1:
            assert loads.max() <= 1.05 * cost.sum() / world   # many small blocks: near-perfect balance
    assert [p.size for p in shard.balance_blocks([5.0, 1.0, 1.0], 2)] == [1, 2]


def test_built_flops_structure():
    """The per-cell FLOP count of the kernels as built: the squarings dominate
    at n = 17 (a squaring is n^2 (n+1)); warp per cell trades the last two
    squarings for four applications; both forms grow by one squaring per s*."""
    k, s = np.array([6]), np.array([15])
    wpc = shard.built_flops(16, k, s, True)[0]
    lpc = shard.built_flops(16, k, s, False)[0]
    n = 17
    assert lpc - wpc == pytest.approx(2 * n * n * (n + 1) - (4 * 6 * n * n + 9 * n - (6 * n * n + 6 * n)))
    assert shard.built_flops(16, k, s + 1, True)[0] - wpc == pytest.approx(n * n * (n + 1))
    # k* picks m_k of Table B.1: one more Horner step per degree
    assert shard.built_flops(4, np.array([7]), s, False)[0] - shard.built_flops(4, np.array([6]), s, False)[0] == \
        pytest.approx((20 - 16) * (2 * 25 + 20 - 4))
    # s* < 2: the warp-per-cell form squares nothing and applies 2^s* times
    assert shard.built_flops(4, np.array([1]), np.array([0]), True)[0] == shard.built_flops(4, np.array([1]),
                                                                                           np.array([0]), False)[0]
    # n = 2 lane per cell: the velocity form, 2 FLOPs per degree and 4 per squaring
    one = shard.built_flops(1, np.array([6, 7]), np.array([3, 4]), False)
    assert one[1] - one[0] == pytest.approx(2 * (20 - 16) + 4)
    assert one[0] == pytest.approx(10 + 2 * 15 + 3 + 3 * 4 + 15)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    rng = np.random.default_rng(7)
    blocks = []
    for b in range(24):
        N = int(rng.choice([1, 4, 8, 16]))
        dt = 2.0 ** -int(rng.integers(0, 7))
        blocks.append((N, dt, W.mrn(8, N, seed=500 + b, stiff_lo=-4.0, stiff_hi=8.0, dt=dt, t_ref=1.0)))
    return W.Batch(blocks)


def _block_costs(desc, rg, rd, ts):
    import oracle
    k = np.zeros(rg.size, dtype=np.int64)
    s = np.zeros(rg.size, dtype=np.int64)
    for d in desc:
        C, N, c0, d0 = int(d["ncells"]), int(d["nspecies"]), int(d["cell_offset"]), int(d["dust_offset"])
        v = np.zeros((3, N + 1, C))
        _, kk, ss, _ = oracle.drag_apply(rg[c0:c0 + C], rd[d0:d0 + N * C].reshape(N, C),
                                         ts[d0:d0 + N * C].reshape(N, C), float(d["dt"]), v, return_ks=True)
        k[c0:c0 + C], s[c0:c0 + C] = kk, ss
    return shard.block_cost(desc, k, s, lambda N: N >= 12)


def _worker(rank, world, port, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    # single-N workload: this rank's contiguous range of 301 cells at N = 4
    cells = W.mrn(301, 4, seed=3, stiff_lo=-3.0, stiff_hi=2.0)
    a, b = shard.cell_range(cells.ncells, rank, world)
    sub = cells.subset(np.arange(a, b))
    part = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    # AMR-like batch: whole blocks dealt by cost; each rank packs its own blocks
    batch = _batch()
    desc, rg, rd, ts, v = batch.pack()
    mine = shard.balance_blocks(_block_costs(desc, rg, rd, ts), world)[rank]
    pb = W.Batch([batch.blocks[i] for i in mine])
    pdesc, prg, prd, pts, pv = pb.pack()
    pout, st = oracle.drag_apply_batched(pdesc, prg, prd, pts, pv)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, (a, b), part, mine, pout, st))
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        out_q.put(gathered)


def test_sharded_results_equal_single_rank_gloo():
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered.sort(key=lambda g: g[0])
    # single-N: the ranks' ranges tile the cells and their outputs concatenate to one rank's
    cells = W.mrn(301, 4, seed=3, stiff_lo=-3.0, stiff_hi=2.0)
    whole = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert [g[1] for g in gathered] == [(0, 151), (151, 301)]
    assert np.array_equal(np.concatenate([g[2] for g in gathered], axis=2), whole)
    # batch: every block on exactly one rank, each block's slab equal to one rank's run of the whole batch
    batch = _batch()
    desc, rg, rd, ts, v = batch.pack()
    ref, st = oracle.drag_apply_batched(desc, rg, rd, ts, v)
    assert st == 0
    owner = np.concatenate([g[3] for g in gathered])
    assert np.array_equal(np.sort(owner), np.arange(len(desc)))
    cost = _block_costs(desc, rg, rd, ts)
    loads = [cost[g[3]].sum() for g in gathered]
    assert max(loads) <= cost.sum() / 2 + cost.max()
    for rank, _, _, mine, pout, pst in gathered:
        assert pst == 0
        pdesc = W.Batch([batch.blocks[i] for i in mine]).pack()[0]
        for j, b in enumerate(mine):
            N, C = int(desc[b]["nspecies"]), int(desc[b]["ncells"])
            n_v = 3 * (N + 1) * C
            got = pout[int(pdesc[j]["vel_offset"]):int(pdesc[j]["vel_offset"]) + n_v]
            exp = ref[int(desc[b]["vel_offset"]):int(desc[b]["vel_offset"]) + n_v]
            assert np.array_equal(got, exp), (rank, b)


def test_bench_cell_loading_partition_and_replicas():
    """bench.py's per-rank cells: under --partition the ranks' contiguous shares of
    one workload concatenate to the single-rank draw; otherwise each rank gets an
    independent draw of the same size (rank 0's is the workload itself)."""
    import bench
    name, nc = "mrn_n4_128cube", 1001
    full, total = bench.load_cells(name, 0, 1, True, ncells=nc)
    assert total == nc
    parts = [bench.load_cells(name, r, 3, True, ncells=nc) for r in range(3)]
    assert all(t == nc for _, t in parts)
    assert np.array_equal(np.concatenate([p.v for p, _ in parts], axis=2), full.v)
    assert np.array_equal(np.concatenate([p.t_s for p, _ in parts], axis=1), full.t_s)
    r0, tot0 = bench.load_cells(name, 0, 2, False, ncells=nc)
    r1, tot1 = bench.load_cells(name, 1, 2, False, ncells=nc)
    assert tot0 == tot1 == 2 * nc
    assert np.array_equal(r0.v, full.v) and not np.array_equal(r1.v, full.v)
    assert r1.ncells == nc and r1.rho_d.shape == full.rho_d.shape
