"""Pins of the lower accuracy targets of Eq. B8 (u = 2^-24 and 2^-11).

Eq. B8 defines theta_m for any unit round-off u; the paper names 2^-11,
2^-24, 2^-113 and 2^-237 besides 2^-53. With a larger u, Algorithm 2 picks
fewer Taylor terms and squarings. The oracle's tables and the forward result
at these targets are pinned here against:

* the closed form of the bound's coefficients, solved in mpmath (an
  independent route to the same definition);
* the meaning of theta_m: for x < 0 (the side of the drag spectrum) every
  term c_j x^j of rho(x) = e^-x T_m(x) - 1 has the sign (-1)^m, so
  |rho(-theta)| = f_m(theta) and the backward error log(e^-x T_m(x)) of the
  scaled exponential at x = -theta_m equals u theta_m up to O(u theta_m)
  (evaluated directly from exp and the Taylor sum, no coefficients); for
  x > 0 the terms alternate and it stays below u x;
* the forward error bound of the truncation: T_m(X) = exp(X + h(X)) with h a
  power series, so after the squarings the computed propagator is
  exp(A + 2^s h(2^-s A)), a function of A that only moves each eigenvalue
  lambda of A by at most u |lambda| (|lambda| <= |A|_1 <= 2^s theta_m).
  In the symmetric form (eigenvalues <= 0) a mode changes by at most
  |lambda| e^lambda u <= u / e, so in the mass-weighted norm
  |sigma o (v - v_exact)|_2 <= (u / e) |sigma o v_in|_2, sigma_f^2 = rho_f / rho_g,
  whatever the stiffness.
"""
import numpy as np
import pytest

import oracle
from oracle import truth
from paper_2509_25347_gb300 import workloads as W

TARGETS = (24, 11)


@pytest.mark.parametrize("ubits", TARGETS)
def test_theta_targets_match_closed_form(ubits):
    mp = pytest.importorskip("mpmath")
    th = oracle.theta_table(2.0 ** -ubits)
    for k in range(1, 10):
        m = oracle.table_b1(k)[0]
        ref = truth.theta_closed_form(m, u=mp.mpf(2) ** -ubits)
        assert abs(th[k] - ref) <= 1e-13 * ref, (k, th[k], ref)


@pytest.mark.parametrize("ubits", (53,) + TARGETS)
def test_theta_is_where_backward_error_reaches_u(ubits):
    """|log(e^theta T_m(-theta))| = u theta (direct evaluation, 80 digits)."""
    mp = pytest.importorskip("mpmath")
    th = oracle.theta_table(2.0 ** -ubits)
    with mp.workdps(80):
        u = mp.mpf(2) ** -ubits
        for k in range(1, 10):
            m = oracle.table_b1(k)[0]
            x = mp.mpf(th[k])

            def h(y):
                T = mp.fsum(y ** j / mp.factorial(j) for j in range(m + 1))
                return mp.log(mp.exp(-y) * T)

            # rho(-theta) = (-1)^m f with -log(1 - f) = u theta: |h| = u theta
            # for odd m, log(1 + f) = log(2 - e^(-u theta)) for even m
            ratio = abs(h(-x)) / (u * x)
            expect = 1 if m % 2 else mp.log(2 - mp.exp(-u * x)) / (u * x)
            assert abs(ratio - expect) < 1e-11, (k, float(ratio), float(expect))
            assert abs(h(x)) <= u * x
            if m % 2:
                # attained exactly for odd m: just past theta the error exceeds u |x|
                assert abs(h(-x * (1 + mp.mpf(2) ** -20))) > u * x * (1 + mp.mpf(2) ** -20)


def test_targets_order_theta_and_cost():
    """A looser target never raises the cost k* + s* Algorithm 2 assigns."""
    rng = np.random.default_rng(7)
    norms = np.concatenate([10.0 ** rng.uniform(-9, 9, 400), [0.0, 1e-300, 1.0, 3.53966635, 1e12]])
    t53 = oracle.theta_table()
    for ubits in TARGETS:
        tt = oracle.theta_table(2.0 ** -ubits)
        assert np.all(tt[1:] > t53[1:])
        for a in norms:
            k0, _, s0 = oracle.select(a)
            k1, _, s1 = oracle.select(a, 2.0 ** -ubits)
            assert k1 + s1 <= k0 + s0, (a, ubits)
            # the chosen order covers the scaled norm: 2^-s |A| <= theta (or 2, 4 theta on Algorithm 2's branches)
            assert a * 2.0 ** -s1 <= 4 * tt[k1] * (1 + 1e-15)


def _weighted_error(cells, v, ref):
    sig = np.concatenate([np.ones((1, cells.ncells)), np.sqrt(cells.rho_d / cells.rho_g[None, :])], axis=0)
    num = np.sqrt(np.sum((sig[None] * (v - ref)) ** 2, axis=1))          # (3, C)
    den = np.sqrt(np.sum((sig[None] * cells.v) ** 2, axis=1))
    return num / den


@pytest.mark.parametrize("ubits", (53,) + TARGETS)
@pytest.mark.parametrize("name,N,lo,hi", [("mrn4", 4, -3.0, 6.0), ("mrn16", 16, -4.0, 8.0), ("mrn8", 8, -4.0, 8.0)])
def test_forward_error_within_target_bound(ubits, name, N, lo, hi):
    """Oracle at target u vs the 40-digit eigen truth, mass-weighted norm."""
    pytest.importorskip("mpmath")
    cells = W.mrn(12, N, seed=11 + N, stiff_lo=lo, stiff_hi=hi)
    v = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -ubits)
    ref = truth.drag_truth(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    err = _weighted_error(cells, v, ref)
    bound = 2.0 ** -ubits / np.e * (1 + 1e-6) + 5e-15      # truncation + FP64 rounding
    assert err.max() <= bound, (err.max(), bound)


def _nonstiff_cells(C=24, N=4, seed=3):
    """|A|_1 of order 1: the truncation of a loose target is visible there
    (stiff modes decay to nothing and slow modes sit far inside theta)."""
    rng = np.random.default_rng(seed)
    return W.Cells(np.ones(C), rng.uniform(0.1, 1.0, (N, C)), 10.0 ** rng.uniform(-0.7, 0.7, (N, C)),
                   rng.standard_normal((3, N + 1, C)), 1.0)


def test_looser_targets_truncate_more_within_bound():
    pytest.importorskip("mpmath")
    cells = _nonstiff_cells()
    ref = truth.drag_truth(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    errs, costs = {}, {}
    for ubits in (53,) + TARGETS:
        v, k, s, _ = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -ubits,
                                       return_ks=True)
        errs[ubits] = _weighted_error(cells, v, ref).max()
        costs[ubits] = int(k.sum() + s.sum())
        assert errs[ubits] <= 2.0 ** -ubits / np.e * (1 + 1e-6) + 5e-15
    assert errs[24] > 10 * errs[53] and errs[11] > 1e3 * errs[24], errs
    assert costs[11] < costs[24] < costs[53], costs


def test_dustybox_target_closed_form():
    """N = 1 (Dustybox, Sec. 3.1): the relative velocity decays as
    exp(-(1 + eps) dt / t_s); at target u the computed decay factor must stay
    within u/e of it in the mass-weighted norm (checked per cell)."""
    cells = W.dustybox(64, seed=5)
    for ubits in TARGETS:
        v = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -ubits)
        eps = cells.rho_d[0] / cells.rho_g
        lam = -(1 + eps) * cells.dt / cells.t_s[0]
        vg, vd = cells.v[:, 0, :], cells.v[:, 1, :]
        vcm = (vg + eps * vd) / (1 + eps)
        dv = (vd - vg) * np.exp(lam)
        ref = np.stack([vcm - eps / (1 + eps) * dv, vcm + dv / (1 + eps)], axis=1)
        err = _weighted_error(cells, v, ref)
        assert err.max() <= 2.0 ** -ubits / np.e * (1 + 1e-6) + 5e-15, (ubits, err.max())
