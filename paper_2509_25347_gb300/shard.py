"""Partitions of a drag workload over ranks (one process per GPU).

The drag step is cell local (Sec. 2.4: it is one operator of the split
step, and every cell solves its own drag equation), so shards need no data
exchange; only the timing of a benchmark takes a barrier and a max-reduce.

- Single-N workloads: rank r takes one contiguous range of cells, sizes
  differing by at most one cell (`cell_range`).
- AMR-like block batches: whole blocks, so a block's slabs stay on one rank.
  Blocks differ in N and in (k*, s*), hence in cost by orders of magnitude;
  they are dealt by the longest-processing-time rule on a per-block cost
  estimate (`balance_blocks`), which bounds every rank's load by the mean
  load plus the largest single block.

`block_cost` gives that estimate: the FP64 FLOPs the kernels execute for each
cell's (k*, s*) (`built_flops`), summed over the block.
"""
from __future__ import annotations

import numpy as np

# m_k of Table B.1: the Taylor degree reached with k matrix products (K = 9).
M_K = (0, 2, 4, 6, 9, 12, 16, 20, 25, 30)

# The warp-per-cell forward replaces its last min(s*, APPLY_Q) squarings by
# 2^q applications of the propagator (P^(2^q) v = P(P(...P v))).
APPLY_Q = 2


def cell_range(ncells: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of rank's contiguous share of ncells cells."""
    if world < 1 or not 0 <= rank < world or ncells < 0:
        raise ValueError("need 0 <= rank < world and ncells >= 0")
    base, extra = divmod(ncells, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def built_flops(N, k, s, warp_per_cell: bool) -> np.ndarray:
    """FP64 FLOPs per cell of the update as the kernels compute it (an FMA is
    2; a division, square root or scaling 1), from the cell's (k*, s*):

    - set-up (A = dt Omega_v, its 1-norm, the scaled symmetric arrowhead X):
      13 N;
    - Taylor by Horner in the arrowhead X: F = b_m X + b_(m-1) I (3n), then
      m - 1 steps G = F X + b_j I over the upper triangle, 2 FMAs per entry
      and an n-term sum for G_00: 2n^2 + 4n - 4 each, m = m_(k*);
    - the row-sum restoration of the Taylor result: n FMAs per row, 2n^2;
    - a squaring in the symmetric form: n(n-1)/2 dot products of length n and
      n restorations of n FMAs, n^2 (n+1);
    - an application to the three velocity components:
      3 (n (2n + 1) + n) = 6n^2 + 6n.

    Lane per cell: s* squarings and one application. Warp per cell: s* - q
    squarings and 2^q applications, q = min(s*, 2); before the last one an
    application carries sigma o v alone, n FMAs per entry (6n^2), and the last
    one then forms v = tau o (sigma o v) first (6n^2 + 9n).

    Lane per cell at n = 2 (one dust species) the update runs in the velocity
    form on the off-diagonal pair (p, q) of P = I + W: set-up 10 (eps, alpha,
    the norm's products and sums, x and y); Taylor -(x + y), one FMA per degree
    and p = b x, q = b y, 2 (m - 1) + 3; a squaring (p, q) <- (2 - p - q)(p, q),
    4; the application v_1 - v_0 and two FMAs per component, 15."""
    n = N + 1
    k = np.asarray(k, dtype=np.int64)
    s = np.asarray(s, dtype=np.float64)
    m = np.asarray(M_K, dtype=np.float64)[k]
    fixed = 13.0 * N + 3.0 * n + (m - 1.0) * (2.0 * n * n + 4.0 * n - 4.0) + 2.0 * n * n
    sq = n * n * (n + 1.0)
    app = 6.0 * n * n + 6.0 * n
    if n == 2 and not warp_per_cell:
        return 10.0 + 2.0 * (m - 1.0) + 3.0 + s * 4.0 + 15.0
    if warp_per_cell:
        q = np.minimum(s, APPLY_Q)
        apps = np.where(q > 0, np.exp2(q) * 6.0 * n * n + 9.0 * n, app)
        return fixed + (s - q) * sq + apps
    return fixed + s * sq + app


def block_cost(desc, k, s, warp_per_cell) -> np.ndarray:
    """Estimated FP64 FLOPs of each block: the sum of built_flops over its
    cells. desc: block records (fields ncells, nspecies, cell_offset); k, s:
    (k*, s*) of every gas cell, indexed like rho_g; warp_per_cell(N) -> bool."""
    cost = np.zeros(len(desc))
    for b in range(len(desc)):
        C, N, c0 = int(desc[b]["ncells"]), int(desc[b]["nspecies"]), int(desc[b]["cell_offset"])
        if C > 0:
            cost[b] = float(built_flops(N, k[c0:c0 + C], s[c0:c0 + C], warp_per_cell(N)).sum())
    return cost


def balance_blocks(cost, world: int) -> list[np.ndarray]:
    """Deal blocks to `world` ranks by the longest-processing-time rule: the
    costliest remaining block goes to the least loaded rank (ties: lower
    rank, then lower block index). Returns each rank's block indices in
    ascending order. Every rank's load is at most mean + max(cost)."""
    cost = np.asarray(cost, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.lexsort((np.arange(cost.size), -cost))
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for b in order:
        r = int(np.argmin(load))
        parts[r].append(int(b))
        load[r] += cost[b]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]
