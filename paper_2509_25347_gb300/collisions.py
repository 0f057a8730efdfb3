"""Collisions time series and the Er1 convergence metric (Sec. 3.1).

The Collisions tests integrate the drag sub-system alone: gas plus dust fluids
with constant stopping times, initial velocities given, no transport. Each
time step is one call of the GPU drag update (EXP or the analytic RK1 of
App. A.2). The exact solution V(t) = V_CM + sum_j c_j exp(lambda_j t)
(Eq. V_analytic) is evaluated from the eigen-decomposition of the drag matrix
(Eq. eigen_problem), in its symmetric similarity form so that numpy's
symmetric eigensolver applies. Er1 (Eq. Error1_eq) averages the relative
error of every fluid over the time steps of a run.

This is a validation driver around the drag kernels, not part of the drag
path; it needs a CUDA device.
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


def exact_solution(setup: CollisionSetup, times: np.ndarray) -> np.ndarray:
    """V(t) for every time (rows) and fluid (columns), from the eigenpairs of the
    symmetric form S = D^(1/2) Omega_v D^(-1/2) of the drag matrix."""
    eps = setup.rho_d / setup.rho_g
    alpha = 1.0 / setup.t_s
    n = eps.size + 1
    sig = np.concatenate([[1.0], np.sqrt(eps)])
    S = np.zeros((n, n))
    S[0, 0] = -np.sum(eps * alpha)
    S[0, 1:] = S[1:, 0] = sig[1:] * alpha
    S[1:, 1:] = np.diag(-alpha)
    lam, Q = np.linalg.eigh(S)
    y0 = Q.T @ (sig * setup.v0)
    out = np.exp(np.outer(times, lam)) * y0[None, :] @ Q.T
    return out / sig[None, :]


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


def er1(setup: CollisionSetup, dt: float, t_final: float, method: str = "exp") -> float:
    """Er1 of Eq. Error1_eq: (1/M) sum over fluids and the M time steps of
    |v_num - v_exact| / |v_exact|."""
    M = int(round(t_final / dt))
    num = integrate(setup, dt, M, method)
    ref = exact_solution(setup, dt * np.arange(1, M + 1))
    return float(np.sum(np.abs(num - ref) / np.abs(ref)) / M)


def convergence(setup: CollisionSetup, dt0: float, t_final: float, method: str = "exp"):
    """Er1 for dt = dt0, 2 dt0, 4 dt0, ... up to t_final (the Fig. 2 sweep)."""
    out = []
    dt = dt0
    while dt <= t_final * (1 + 1e-12):
        out.append((dt, er1(setup, dt, t_final, method)))
        dt *= 2.0
    return out
