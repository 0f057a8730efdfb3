"""Seeded synthetic inputs for the drag update (host numpy, PCG64).

This module only draws inputs; it contains none of the drag method's
arithmetic. Both the CUDA path and the CPU oracle are fed from it.

The paper measures on its Dustywave runs (Sec. 3.5), whose densities and
stopping times come from an external table that is not reproduced here. These
generators stand in for them with the shapes and value ranges of the five
workloads this library is measured on:

* ``dustybox``: N = 1, rho_g = 1, dust-to-gas ratio U[0.01, 1], t_s = dt*10^U(-4,2).
* ``mrn``: N species on an MRN-like size grid. Relative grain sizes
  a_j = 10^(4 j/(N-1)) (four decades), dust mass per bin proportional to
  a_j^0.5, total dust-to-gas ratio U[0.01, 1], rho_g log-normal (sigma = 1),
  t_s,j proportional to a_j with dt/t_s spanning a chosen number of decades.
* ``batched``: blocks of 8^3 cells with N drawn from {1, 4, 8, 16} (equal cell
  share, shuffled order) and per-block dt = 2^-k, k uniform in 0..6.

Layout (structure of arrays, FP64, C-contiguous):
  rho_g (C,), rho_d (N, C), t_s (N, C), v (3, N+1, C)  with v[d, 0] the gas and
  v[d, i] dust species i, d = x, y, z.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Cells:
    rho_g: np.ndarray
    rho_d: np.ndarray
    t_s: np.ndarray
    v: np.ndarray
    dt: float

    @property
    def ncells(self) -> int:
        return int(self.rho_g.shape[0])

    @property
    def nspecies(self) -> int:
        return int(self.rho_d.shape[0])

    def subset(self, idx) -> "Cells":
        return Cells(np.ascontiguousarray(self.rho_g[idx]), np.ascontiguousarray(self.rho_d[:, idx]),
                     np.ascontiguousarray(self.t_s[:, idx]), np.ascontiguousarray(self.v[:, :, idx]), self.dt)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def dustybox(ncells: int, seed: int = 0, dt: float = 1.0) -> Cells:
    """One dust species: rho_g = 1, eps ~ U[0.01,1], t_s = dt*10^U(-4,2), v ~ N(0,1)."""
    rng = _rng(seed)
    rho_g = np.ones(ncells)
    eps = rng.uniform(0.01, 1.0, ncells)
    x = rng.uniform(-4.0, 2.0, ncells)
    v = rng.standard_normal((3, 2, ncells))
    rho_d = (rho_g * eps)[None, :].copy()
    t_s = (dt * 10.0 ** x)[None, :].copy()
    return Cells(rho_g, rho_d, t_s, v, dt)


def mrn(ncells: int, nspecies: int, seed: int, stiff_lo: float, stiff_hi: float, dt: float = 1.0,
        t_ref: float | None = None) -> Cells:
    """MRN-like multi-species cells.

    log10(t_ref/t_s) spans [stiff_lo, stiff_hi] over the whole population: each
    cell draws an offset and its N species cover four decades above it (one
    species with four decades when N = 1 is not possible, so N = 1 cells draw
    log10(t_ref/t_s) directly from [stiff_lo, stiff_hi]). ``t_ref`` defaults to dt.
    """
    rng = _rng(seed)
    N = int(nspecies)
    t_ref = dt if t_ref is None else t_ref
    rho_g = np.exp(rng.standard_normal(ncells))
    eps_tot = rng.uniform(0.01, 1.0, ncells)
    if N > 1:
        x0 = rng.uniform(stiff_lo, stiff_hi - 4.0, ncells)
        a = 10.0 ** (4.0 * np.arange(N) / (N - 1))
    else:
        x0 = rng.uniform(stiff_lo, stiff_hi, ncells)
        a = np.ones(1)
    v = rng.standard_normal((3, N + 1, ncells))
    w = np.sqrt(a) / np.sqrt(a).sum()
    rho_d = np.ascontiguousarray(w[:, None] * (rho_g * eps_tot)[None, :])
    # t_ref/t_s,j = 10^(x0 + 4) / a_j (N > 1): species 0 is the stiffest
    top = 4.0 if N > 1 else 0.0
    t_s = np.ascontiguousarray(t_ref * a[:, None] * 10.0 ** (-(x0 + top))[None, :])
    return Cells(rho_g, rho_d, t_s, v, dt)


# The five measured workloads -------------------------------------------------

WORKLOADS = {
    # name: (description, ncells, nspecies, seed)
    "dustybox_n1_32k": ("Dustybox-like, N=1, 32^3 cells, dt/t_s in [1e-2, 1e4]", 32768, 1, 0),
    "mrn_n4_128cube": ("MRN-like, N=4, 128^3 cells, dt/t_s in [1e-3, 1e6]", 2097152, 4, 1),
    "mrn_n16_128cube": ("MRN-like, N=16, 128^3 cells, dt/t_s in [1e-4, 1e8]", 2097152, 16, 2),
    "batched_amr_1m": ("AMR-like blocks of 8^3 cells, N in {1,4,8,16}, dt = 2^-k", 1048576, 0, 3),
    "mrn_n8_128cube_adjoint": ("MRN-like, N=8, 128^3 cells, dt/t_s in [1e-4, 1e8], fwd + adjoint", 2097152, 8, 4),
}


def replica_seed(seed: int, replica: int) -> int:
    """Seed of an independent copy of a workload (replica 0 is the workload itself)."""
    return seed if replica == 0 else seed + 1_000_003 * replica


def workload(name: str, ncells: int | None = None, replica: int = 0) -> Cells:
    """Cells of one plain (single-N) workload; ``ncells`` truncates the draw size;
    ``replica`` > 0 draws an independent copy with the same recipe."""
    desc, C, N, seed = WORKLOADS[name]
    seed = replica_seed(seed, replica)
    C = C if ncells is None else int(ncells)
    if name == "dustybox_n1_32k":
        return dustybox(C, seed=seed)
    if name == "mrn_n4_128cube":
        return mrn(C, 4, seed, -3.0, 6.0)
    if name == "mrn_n16_128cube":
        return mrn(C, 16, seed, -4.0, 8.0)
    if name == "mrn_n8_128cube_adjoint":
        return mrn(C, 8, seed, -4.0, 8.0)
    raise KeyError(name)


def adjoint_target(ncells: int, nspecies: int, seed: int = 4) -> np.ndarray:
    """v_target ~ N(0,1) for the loss 0.5 ||v_out - v_target||^2."""
    return _rng(seed + 1000).standard_normal((3, nspecies + 1, ncells))


BLOCK_DTYPE = np.dtype([("cell_offset", "<i8"), ("dust_offset", "<i8"), ("vel_offset", "<i8"),
                        ("ncells", "<i4"), ("nspecies", "<i4"), ("dt", "<f8")])


@dataclass
class Batch:
    """Blocks for the batched entry point: one SoA slab per block."""
    blocks: list          # list of (nspecies, dt, Cells)

    def pack(self):
        """Concatenate the blocks' slabs. Returns (desc, rho_g, rho_d, t_s, v)
        with desc a BLOCK_DTYPE array: block b's gas densities start at
        rho_g[cell_offset], its species-major dust slab (N x ncells) at
        rho_d[dust_offset] and t_s[dust_offset], its velocity slab
        (3 x (N+1) x ncells) at v[vel_offset]."""
        desc = np.zeros(len(self.blocks), dtype=BLOCK_DTYPE)
        rg, rd, ts, vv = [], [], [], []
        co = do = vo = 0
        for b, (N, dt, cells) in enumerate(self.blocks):
            C = cells.ncells
            desc[b] = (co, do, vo, C, N, dt)
            rg.append(cells.rho_g)
            rd.append(cells.rho_d.reshape(-1))
            ts.append(cells.t_s.reshape(-1))
            vv.append(cells.v.reshape(-1))
            co += C
            do += N * C
            vo += 3 * (N + 1) * C
        cat = lambda parts: np.ascontiguousarray(np.concatenate(parts)) if parts else np.zeros(0)
        return desc, cat(rg), cat(rd), cat(ts), cat(vv)

    @property
    def ncells(self) -> int:
        return int(sum(c.ncells for _, _, c in self.blocks))


def batched(nblocks: int = 2048, block_cells: int = 512, seed: int = 3, species=(1, 4, 8, 16), kmax: int = 6) -> Batch:
    """AMR-like mix: equal share of blocks per N, shuffled, dt = 2^-k, k ~ U{0..kmax}.

    Cells follow the N = 16 workload's recipe at their own N with t_ref = 1
    (log10(1/t_s) in [-4, 8]); the block's dt = 2^-k then scales the stiffness.
    """
    rng = _rng(seed)
    per = nblocks // len(species)
    ns = np.repeat(np.array(species), per)
    ns = np.concatenate([ns, rng.choice(np.array(species), nblocks - ns.size)])
    rng.shuffle(ns)
    ks = rng.integers(0, kmax + 1, nblocks)
    blocks = []
    for b in range(nblocks):
        dtb = 2.0 ** (-int(ks[b]))
        cells = mrn(block_cells, int(ns[b]), seed * 1_000_003 + b, -4.0, 8.0, dt=dtb, t_ref=1.0)
        blocks.append((int(ns[b]), dtb, cells))
    return Batch(blocks)
