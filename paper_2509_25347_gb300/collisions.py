"""Collisions time series (Sec. 3.1): the set-ups of tests B and C (Table 1)
and of the 20-species case, and a driver that steps them on the GPU.

The Collisions tests integrate the drag sub-system alone: gas plus dust fluids
with constant stopping times, initial velocities given, no transport. Each
time step is one call of the GPU drag update (EXP or the analytic RK1 of
App. A.2). The exact solution these trajectories are measured against, and
the Er1 metric (Eq. Error1_eq), belong to the checks, not to this package.

This is a driver around the drag kernels, not part of the drag path; it needs
a CUDA device.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CollisionSetup:
    rho_g: float
    rho_d: np.ndarray      # (N,)
    t_s: np.ndarray        # (N,)
    v0: np.ndarray         # (N+1,) initial velocities, gas first


def collisions_b() -> CollisionSetup:
    """Collisions test B (stiff, short stopping times), Table 1."""
    return CollisionSetup(1.0, np.array([1.0, 1.0]), np.array([0.01, 0.002]), np.array([1.0, 2.0, 0.5]))


def collisions_c() -> CollisionSetup:
    """Collisions test C (high dust-to-gas ratios), Table 1."""
    return CollisionSetup(1.0, np.array([10.0, 100.0]), np.array([2.0, 1.0]), np.array([1.0, 2.0, 0.5]))


def collisions_20_species(seed: int = 20, eps_total: float = 1.0, ts_min: float = 1e-3, ts_max: float = 10.0,
                    n: int = 20) -> CollisionSetup:
    """The 20-species collision test: stopping times log-spaced over
    [ts_min, ts_max] and dust-to-gas ratios from Eq. dust_to_gas_ratio,
    eps_i = eps (sqrt(T_{i+1}) - sqrt(T_i)) / (sqrt(T_max) - sqrt(T_min)),
    which needs n+1 nodes T_1..T_{n+1}; species i uses T_i. The paper does not
    give the initial velocities; they are drawn N(0,1) with a fixed seed."""
    nodes = np.logspace(np.log10(ts_min), np.log10(ts_max), n + 1)
    eps = eps_total * (np.sqrt(nodes[1:]) - np.sqrt(nodes[:-1])) / (np.sqrt(ts_max) - np.sqrt(ts_min))
    v0 = np.random.default_rng(seed).standard_normal(n + 1)
    return CollisionSetup(1.0, eps.copy(), nodes[:-1].copy(), v0)


def integrate(setup: CollisionSetup, dt: float, nsteps: int, method: str = "exp") -> np.ndarray:
    """Velocities after each of nsteps drag steps of length dt on the GPU
    (method 'exp' or 'rk1'); returns an (nsteps, N+1) array (x component)."""
    import torch

    import paper_2509_25347_gb300 as dx

    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    N = setup.rho_d.size
    rg = dev([setup.rho_g])
    rd = dev(setup.rho_d.reshape(N, 1))
    ts = dev(setup.t_s.reshape(N, 1))
    v = torch.zeros((3, N + 1, 1), dtype=torch.float64, device="cuda")
    v[0, :, 0] = dev(setup.v0)
    hist = torch.empty((nsteps, N + 1), dtype=torch.float64, device="cuda")
    step = dx.apply if method == "exp" else dx.rk1_apply
    for k in range(nsteps):
        step(rg, rd, ts, dt, v, v)
        hist[k] = v[0, :, 0]
    return hist.cpu().numpy()
