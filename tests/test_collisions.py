"""Collisions tests B, C and the 20-species case (Sec. 3.1) driven through the
GPU drag update, with Er1 (Eq. Error1_eq) against the exact solution."""
import math

import numpy as np
import pytest

from oracle.truth import collisions_exact
from paper_2509_25347_gb300 import collisions as CO
from tests.conftest import read_golden_table


def exact(setup, times):
    return collisions_exact(setup.rho_g, setup.rho_d, setup.t_s, setup.v0, times)


def er1(setup, dt, t_final, method="exp"):
    """Er1 of Eq. Error1_eq: (1/M) sum over fluids and the M time steps of
    |v_num - v_exact| / |v_exact|."""
    M = int(round(t_final / dt))
    num = CO.integrate(setup, dt, M, method)
    ref = exact(setup, dt * np.arange(1, M + 1))
    return float(np.sum(np.abs(num - ref) / np.abs(ref)) / M)


def convergence(setup, dt0, t_final, method="exp"):
    """Er1 for dt = dt0, 2 dt0, 4 dt0, ... up to t_final (the Fig. 2 sweep)."""
    out = []
    dt = dt0
    while dt <= t_final * (1 + 1e-12):
        out.append((dt, er1(setup, dt, t_final, method)))
        dt *= 2.0
    return out


def test_exact_solution_matches_table1():
    """V(t) from the eigenpairs reproduces Table 1's printed modes (CPU)."""
    T = {r[0]: (float(r[1]), float(r[2])) for r in read_golden_table("collisions_table1.txt")}
    for col, setup in ((0, CO.collisions_b()), (1, CO.collisions_c())):
        lam = [T["lambda1"][col], T["lambda2"][col]]
        coef = [(T["c_g1"][col], T["c_g2"][col]), (T["c_d11"][col], T["c_d12"][col]),
                (T["c_d21"][col], T["c_d22"][col])]
        times = np.linspace(0.0, 0.05 if col == 0 else 2.0, 9)
        got = exact(setup, times)
        for k, tt in enumerate(times):
            ref = [T["V_CM"][col] + sum(c * math.exp(l * tt) for c, l in zip(coef[f], lam)) for f in range(3)]
            assert np.allclose(got[k], ref, atol=2e-5, rtol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("which,dt0,t_final", [("b", 1e-4, 0.1), ("c", 1e-3, 2.0)])
def test_er1_exp_flat_and_rk1_first_order(which, dt0, t_final):
    """EXP stays at machine precision for every dt of the Fig. 2 sweep (the
    paper reports a flat ~1e-8); RK1's Er1 falls linearly with dt."""
    setup = CO.collisions_b() if which == "b" else CO.collisions_c()
    exp = convergence(setup, dt0, t_final, "exp")
    assert max(e for _, e in exp) < 1e-12                # M steps accumulate ~M u at worst
    rk1 = convergence(setup, dt0, t_final, "rk1")
    (d0, e0), (d1, e1) = rk1[0], rk1[1]
    assert 1.6 < e1 / e0 < 2.4                           # halving dt halves the error at small dt
    assert all(e_rk > 1e3 * e_exp for (_, e_rk), (_, e_exp) in zip(rk1, exp))


@pytest.mark.gpu
def test_20_species_collision():
    """20 dust species, stopping times 1e-3..10, eps by Eq. dust_to_gas_ratio:
    the EXP trajectory stays within 1e-13 of the exact solution (the paper
    reports errors ~1e-7)."""
    setup = CO.collisions_20_species()
    assert abs(setup.rho_d.sum() - 1.0) < 1e-14
    dt, steps = 0.01, 300
    num = CO.integrate(setup, dt, steps, "exp")
    ref = exact(setup, dt * np.arange(1, steps + 1))
    assert np.max(np.abs(num - ref)) <= 1e-13 * np.max(np.abs(setup.v0))
