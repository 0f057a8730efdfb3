"""Pins of the oracle's Taylor bound test (the paper's second modification,
Eqs. Pat_Stk4-Pat_Stk7) and its Pade variant (Eq. PadeEqu).

* Pade coefficients against mpmath's own Pade routine (the [m/m] approximant
  is unique).
* theta of the Pade variant (Eqs. B5-B8 with T_m replaced by R_mm) against a
  60-digit computation of the same definition through mpmath's series.
* Both variants' results against the 40-digit eigen truth, within the u/e
  mass-weighted bound of any truncation that is a function of X (the Pade
  error log(e^-x R_mm(x)) is a power series too).
* The bound test's meaning (Eq. Pat_Stk4): every block it drops changes T_m by
  at most u |e^X| in the 1-norm, checked from the powers of X directly.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import truth
from paper_2509_25347_gb300 import workloads as W
from tests.test_oracle_precision_pins import _weighted_error

PADE_M = oracle.PADE_DEGREES


@pytest.mark.parametrize("m", PADE_M)
def test_pade_coefficients_match_mpmath_pade(m):
    mp = pytest.importorskip("mpmath")
    with mp.workdps(50):
        taylor = [mp.mpf(1) / mp.factorial(j) for j in range(2 * m + 1)]
        p, q = mp.pade(taylor, m, m)
        p = [x / q[0] for x in p]
        q = [x / q[0] for x in q]
    c = oracle.pade_coeffs(m)
    for j in range(m + 1):
        assert abs(c[j] - float(p[j])) <= 1e-15 * abs(float(p[j]))
        assert abs(c[j] * (-1) ** j - float(q[j])) <= 1e-15 * abs(float(q[j]))


def _pade_theta_mp(m, ubits, mp):
    with mp.workdps(60):
        c = [mp.factorial(2 * m - j) * mp.factorial(m) / (mp.factorial(2 * m) * mp.factorial(j) * mp.factorial(m - j))
             for j in range(m + 1)]
        L = 2 * m + 200
        rho = mp.taylor(lambda x: mp.exp(-x) * mp.polyval(c[::-1], x) / mp.polyval(c[::-1], -x) - 1, 0, L)
        u = mp.mpf(2) ** -ubits

        def ok(th):
            f = mp.fsum(abs(rho[j]) * th ** j for j in range(2 * m + 1, L + 1))
            return f < 1 and -mp.log(1 - f) / th <= u

        lo, hi = mp.mpf(0), mp.mpf(16)
        for _ in range(60):
            mid = (lo + hi) / 2
            lo, hi = (mid, hi) if ok(mid) else (lo, mid)
        return float(lo)


@pytest.mark.parametrize("ubits", (53, 24))
def test_pade_theta_matches_60_digit_series(ubits):
    """The Pade variant supports u = 2^-53 and 2^-24; at 2^-11, theta_13 would
    sit at 0.86 of the approximant's pole radius (17.9), where the bound's
    series converges too slowly to evaluate."""
    mp = pytest.importorskip("mpmath")
    for m in PADE_M:
        got = oracle.pade_theta(m, 2.0 ** -ubits)
        ref = _pade_theta_mp(m, ubits, mp)
        assert abs(got - ref) <= 1e-12 * ref, (m, got, ref)


def test_pade_selection_covers_scaled_norm():
    rng = np.random.default_rng(4)
    for a in np.concatenate([10.0 ** rng.uniform(-9, 9, 300), [0.0, 1.0, 5.36, 1e12]]):
        m, s = oracle.select_pade(a)
        assert m in PADE_M
        assert a * 2.0 ** -s <= oracle.pade_theta(m)
        if s > 0:                                  # minimal scaling
            assert m == 13 and a * 2.0 ** -(s - 1) > oracle.pade_theta(13)
        else:                                      # smallest degree that covers
            assert all(a > oracle.pade_theta(mm) for mm in PADE_M if mm < m)


@pytest.mark.parametrize("method,bt,ubits", [("pade", False, 53), ("pade", False, 24), ("taylor", True, 53),
                                             ("taylor", True, 24), ("taylor", True, 11)])
@pytest.mark.parametrize("N,lo,hi", [(4, -3.0, 6.0), (16, -4.0, 8.0)])
def test_variant_forward_within_bound(method, bt, ubits, N, lo, hi):
    pytest.importorskip("mpmath")
    cells = W.mrn(10, N, seed=31 + N, stiff_lo=lo, stiff_hi=hi)
    v = oracle.drag_apply_opts(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -ubits,
                               method=method, bound_test=bt)[0]
    ref = truth.drag_truth(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    err = _weighted_error(cells, v, ref)
    assert err.max() <= 2.0 ** -ubits / math.e * (1 + 1e-6) + 8e-15, err.max()


def _assemble(rg, rd, ts, dt):
    N = rd.size
    n = N + 1
    A = np.zeros((n, n))
    eps, al = rd / rg, 1.0 / ts
    A[0, 1:] = eps * al * dt
    A[1:, 0] = al * dt
    A[np.arange(1, n), np.arange(1, n)] = -al * dt
    A[0, 0] = -A[0, 1:].sum()
    return A


def test_bound_test_drops_only_negligible_blocks():
    """Eq. Pat_Stk4: |T_m(X) - T_m'(X)|_1 <= u |e^X|_1 for every cell where the
    test kept m' < m terms (powers and e^X formed here in numpy / mpmath)."""
    mp = pytest.importorskip("mpmath")
    cells = W.workload("mrn_n16_128cube", ncells=60)
    _, k, m_eff, s, ratio, st = oracle.drag_apply_opts(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v,
                                                       bound_test=True)
    assert st == 0
    _, k0, m0, s0, _, _ = oracle.drag_apply_opts(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    assert np.array_equal(k, k0) and np.array_equal(s, s0)
    dropped = 0
    for c in range(cells.ncells):
        m_full, q = oracle.table_b1(int(k[c]))[0], oracle.table_b1(int(k[c]))[1]
        assert m_eff[c] <= m_full and (m_full - m_eff[c]) % q == 0 and m_eff[c] >= q
        assert (ratio[c] <= 1.0) == (m_eff[c] < m_full)
        if m_eff[c] == m_full:
            continue
        dropped += 1
        X = _assemble(cells.rho_g[c], cells.rho_d[:, c], cells.t_s[:, c], cells.dt) * 2.0 ** -int(s[c])
        P = np.eye(X.shape[0])
        tail = np.zeros_like(X)
        for i in range(1, m_full + 1):
            P = P @ X / i
            if i > m_eff[c]:
                tail += P
        with mp.workdps(30):
            eX = np.array(mp.expm(mp.matrix(X.tolist())).tolist(), dtype=float)
        lhs = np.abs(tail).sum(axis=0).max()
        rhs = 2.0 ** -53 * np.abs(eX).sum(axis=0).max()
        assert lhs <= rhs * (1 + 1e-6), (c, lhs, rhs)
    assert dropped > 0.5 * cells.ncells            # N = 16: the test passes for most cells


def test_bound_test_off_is_the_plain_method():
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=40)
    a = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    b = oracle.drag_apply_opts(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)[0]
    assert np.array_equal(a, b)
