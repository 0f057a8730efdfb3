"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: numbers printed in
the paper (Table B.1, Table 1), closed forms, invariants, special cases and
an extended-precision eigendecomposition or brute-force Taylor series.
"""
import math

import numpy as np
import pytest

import oracle
from tests.conftest import read_golden_table
from paper_2509_25347_gb300 import workloads as W

U = 2.0 ** -53


# ---------------------------------------------------------------- Table B.1 ---

def test_table_b1_parameters_and_cost():
    """m_k, q_k, r_k as printed in Table B.1; m_k = q_k r_k and Pi_{m_k} = k."""
    for row in read_golden_table("table_b1.txt"):
        k, mk, qk, rk, _, _, pik = row
        k, mk, qk, rk, pik = int(k), int(mk), int(qk), int(rk), int(pik)
        assert oracle.table_b1(k) == (mk, qk, rk)
        assert mk == qk * rk
        # q-1 products for the powers X^2..X^q and r-1 Horner products
        assert (qk - 1) + (rk - 1) == pik == k


def test_theta_matches_table_b1_printed_digits():
    """theta_{m_k} from Eq. B8 rounds to every digit Table B.1 prints."""
    th = oracle.theta_table()
    for row in read_golden_table("table_b1.txt"):
        k, printed, digits = int(row[0]), float(row[4]), int(row[5])
        mant_exp = math.floor(math.log10(printed))
        scale = 10.0 ** (mant_exp - digits + 1)
        assert abs(th[k] - printed) <= 0.5 * scale * (1 + 1e-9), (k, th[k], printed)


def test_theta_matches_independent_closed_form():
    """Same theta from the closed form |c_j| = C(j-1,m)/j! in 50-digit mpmath."""
    pytest.importorskip("mpmath")
    from oracle.truth import theta_closed_form
    th = oracle.theta_table()
    for k in range(1, 10):
        m = oracle.table_b1(k)[0]
        ref = theta_closed_form(m)
        assert abs(th[k] - ref) <= 4e-15 * ref, (k, th[k], ref)


def test_theta_other_precisions_increase():
    """Eq. B8 with larger u (half, single precision) gives larger theta."""
    for m in (6, 16, 30):
        t53 = oracle.theta_m(m, 2.0 ** -53)
        t24 = oracle.theta_m(m, 2.0 ** -24)
        t11 = oracle.theta_m(m, 2.0 ** -11)
        assert t11 > t24 > t53 > 0


# -------------------------------------------------------------- Algorithm 2 ---

def _smin(x, th_k):
    s = 0
    while math.ldexp(x, -s) > th_k:
        s += 1
    return s


def test_alg2_bound_and_minimal_cost():
    """Alg 2 output satisfies 2^-s |A| <= theta_{m_k} (the premise of the
    backward-error theorem, App. B) and reaches the minimal cost k + s over all
    (k, s) of Table B.1 that satisfy it (App. B, "Numerical cost")."""
    th = oracle.theta_table()
    rng = np.random.default_rng(7)
    norms = list(10.0 ** rng.uniform(-10, 12, 4000))
    for k in range(1, 10):
        for f in (1.0, 1 + 2e-16, 2.0, 2 * (1 + 2e-16), 4.0, 4 * (1 + 2e-16), 0.5):
            norms.append(th[k] * f)
    norms += [0.0, 5e-324]
    for x in norms:
        k, m, s = oracle.select(x)
        assert m == oracle.table_b1(k)[0]
        assert math.ldexp(x, -s) <= th[k]
        best = min(kk + _smin(x, th[kk]) for kk in range(1, 10))
        assert k + s == best, (x, k, s, best)


@pytest.mark.parametrize("x,expect", [
    (0.0, (1, 2, 0)),          # first row: dt = 0 or decoupled species
    (1e-3, (3, 6, 0)),         # smallest k with |A| <= theta
    (0.5, (6, 16, 0)),
    (1.5, (6, 16, 1)),         # k^ = 8, |A| <= 2 theta_16: two fewer products, one squaring
    (2.0, (8, 25, 0)),         # k^ = 8 but |A| > 2 theta_16: no reduction
    (3.0, (6, 16, 2)),         # k^ = 9, |A| <= 4 theta_16 (v3 has priority)
    (3.3, (9, 30, 0)),         # k^ = 9, |A| > 4 theta_16: m = 30
    (10.0, (6, 16, 4)),        # s^ = 2, |A|/4 = 2.5 <= 4 theta_16
    (7.0, (9, 30, 1)),         # s^ = 1, |A|/2 = 3.5 > 4 theta_16
])
def test_alg2_worked_cases(x, expect):
    assert oracle.select(x) == expect


def test_alg2_nonfinite_norm_rejected():
    assert oracle.select(float("inf"))[2] == 0  # no endless scaling loop


# ---------------------------------------------------------- Table 1 (Sec 3.1) ---

def _table1():
    rows = read_golden_table("collisions_table1.txt")
    return {r[0]: (float(r[1]), float(r[2])) for r in rows}


def _cell_from_table(T, col):
    rho_g = T["rho_g"][col]
    rho_d = np.array([T["rho_d1"][col], T["rho_d2"][col]])
    t_s = np.array([T["Ts1"][col], T["Ts2"][col]])
    v0 = np.array([T["v_g"][col], T["v_d1"][col], T["v_d2"][col]])
    return rho_g, rho_d, t_s, v0


@pytest.mark.parametrize("col", [0, 1])
def test_collisions_table1_eigenvalues(col):
    """The nonzero eigenvalues of Omega (Eq. eigen_problem) are Table 1's
    lambda_1, lambda_2; V_CM of Eq. V_cm (with the sum over species) matches."""
    T = _table1()
    rho_g, rho_d, t_s, v0 = _cell_from_table(T, col)
    A = oracle.assemble(rho_g, rho_d, t_s, 1.0)
    lam = np.sort(np.linalg.eigvals(A).real)
    assert abs(lam[2]) < 1e-9
    np.testing.assert_allclose(lam[:2], sorted([T["lambda1"][col], T["lambda2"][col]]), rtol=0, atol=6e-5)
    eps = rho_d / rho_g
    vcm = (v0[0] + np.sum(eps * v0[1:])) / (1 + eps.sum())
    assert abs(vcm - T["V_CM"][col]) <= 5e-6


@pytest.mark.parametrize("col", [0, 1])
def test_collisions_table1_solution(col):
    """One drag step of length t reproduces V(t) = V_CM + sum c_j e^{lambda_j t}
    with Table 1's printed coefficients (to their printed precision), and many
    steps of the Fig. 1 time step reproduce it too (semigroup)."""
    T = _table1()
    rho_g, rho_d, t_s, v0 = _cell_from_table(T, col)
    lam = [T["lambda1"][col], T["lambda2"][col]]
    coef = {0: (T["c_g1"][col], T["c_g2"][col]), 1: (T["c_d11"][col], T["c_d12"][col]),
            2: (T["c_d21"][col], T["c_d22"][col])}
    dt = T["dt_fig1"][col]

    def analytic(t):
        return np.array([T["V_CM"][col] + sum(c * math.exp(l * t) for c, l in zip(coef[f], lam)) for f in range(3)])

    v = np.zeros((3, 3, 1))
    v[:, :, 0] = v0[None, :]
    cur = v.copy()
    for step in range(1, 41):
        cur = oracle.drag_apply(np.array([rho_g]), rho_d[:, None], t_s[:, None], dt, cur)
        one = oracle.drag_apply(np.array([rho_g]), rho_d[:, None], t_s[:, None], dt * step, v)
        ref = analytic(dt * step)
        # printed coefficients carry 5 decimals: 2 modes x 5e-6 + V_CM 5e-6
        np.testing.assert_allclose(one[0, :, 0], ref, atol=2e-5, rtol=0)
        np.testing.assert_allclose(cur[0, :, 0], one[0, :, 0], atol=5e-15, rtol=0)


@pytest.mark.parametrize("col", [0, 1])
def test_collisions_against_eigen_truth(col):
    pytest.importorskip("mpmath")
    from oracle.truth import drag_truth_cell
    T = _table1()
    rho_g, rho_d, t_s, v0 = _cell_from_table(T, col)
    for dt in (1e-4, 0.005, 0.05, 1.0, 100.0):
        v = np.tile(v0, (3, 1))
        out = oracle.drag_apply(np.array([rho_g]), rho_d[:, None], t_s[:, None], dt, v[:, :, None])[:, :, 0]
        ref = drag_truth_cell(rho_g, rho_d, t_s, dt, v)
        assert np.max(np.abs(out - ref)) <= 2e-15 * np.max(np.abs(v0)), dt


# ------------------------------------------------------ closed forms (N = 1) ---

def test_dustybox_closed_form():
    """N = 1 (Dustybox): V_CM = (v_g + eps v_d)/(1+eps) is constant and
    v_d - v_g decays as exp(-(1+eps) dt/T_s) (Sec. 3.1, Eqs. V_analytic, V_cm)."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(3)
    C = 300
    eps = rng.uniform(0.01, 5.0, C)
    x = rng.uniform(-6, 9, C)
    ts = 10.0 ** (-x)
    rho_g = np.exp(rng.standard_normal(C))
    v = rng.standard_normal((3, 2, C))
    out = oracle.drag_apply(rho_g, (rho_g * eps)[None, :], ts[None, :], 1.0, v)
    for c in range(C):
        e = mp.mpf(float(rho_g[c] * eps[c])) / mp.mpf(float(rho_g[c]))
        decay = mp.exp(-(1 + e) / mp.mpf(float(ts[c])))
        for d in range(3):
            vg, vd = mp.mpf(float(v[d, 0, c])), mp.mpf(float(v[d, 1, c]))
            vcm = (vg + e * vd) / (1 + e)
            dv = (vd - vg) * decay
            ref_g = vcm - e * dv / (1 + e)
            ref_d = vcm + dv / (1 + e)
            sc = max(abs(v[d, 0, c]), abs(v[d, 1, c]))
            assert abs(out[d, 0, c] - float(ref_g)) <= 2e-15 * sc
            assert abs(out[d, 1, c] - float(ref_d)) <= 2e-15 * sc


def test_equal_stopping_times_closed_form():
    """All species with the same alpha: eigenvalues 0, -alpha(1+E), -alpha
    (E = sum eps_i), and the closed form
      v_g(t) = V + (v_g0 - V) e^{-alpha(1+E)t},
      v_i(t) = V + (v_i0 - V) e^{-alpha t} + (v_g0 - V)(e^{-alpha t} - e^{-alpha(1+E)t})/E,
    derived from Eq. DragEq with alpha_i = alpha."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(11)
    for N in (2, 5, 16):
        for trial in range(6):
            rho_g = float(np.exp(rng.standard_normal()))
            eps = rng.uniform(0.001, 3.0, N)
            ts = float(10.0 ** rng.uniform(-6, 3))
            v = rng.standard_normal((3, N + 1, 1))
            out = oracle.drag_apply(np.array([rho_g]), (rho_g * eps)[:, None], np.full((N, 1), ts), 1.0, v)
            e = [mp.mpf(float(rho_g * x)) / mp.mpf(rho_g) for x in eps]
            E = sum(e)
            a = 1 / mp.mpf(ts)
            g1, g2 = mp.exp(-a), mp.exp(-a * (1 + E))
            for d in range(3):
                vv = [mp.mpf(float(x)) for x in v[d, :, 0]]
                V = (vv[0] + sum(ei * vi for ei, vi in zip(e, vv[1:]))) / (1 + E)
                sc = np.max(np.abs(v[d, :, 0]))
                assert abs(out[d, 0, 0] - float(V + (vv[0] - V) * g2)) <= 2e-15 * sc
                for i in range(N):
                    ref = V + (vv[i + 1] - V) * g1 + (vv[0] - V) * (g1 - g2) / E
                    assert abs(out[d, i + 1, 0] - float(ref)) <= 2e-15 * sc


# --------------------------------------------------------------- invariants ---

def _workload_sample(name, C):
    return W.workload(name, ncells=C)


@pytest.mark.parametrize("name,C", [("dustybox_n1_32k", 400), ("mrn_n4_128cube", 200),
                                    ("mrn_n8_128cube_adjoint", 100), ("mrn_n16_128cube", 60)])
def test_invariants_on_workloads(name, C):
    """Momentum conservation (Eq. DragEq sums to zero), convexity of the update
    (exp(dt Omega_v) is row-stochastic), and detailed balance rho_i P_ij = rho_j P_ji."""
    cells = _workload_sample(name, C)
    out = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    rho = np.vstack([cells.rho_g[None, :], cells.rho_d])          # (n, C)
    mom_in = np.einsum("fc,dfc->dc", rho, cells.v)
    mom_out = np.einsum("fc,dfc->dc", rho, out)
    scale = np.einsum("fc,dfc->dc", rho, np.abs(cells.v))
    assert np.all(np.abs(mom_out - mom_in) <= 4e-15 * scale)
    lo = cells.v.min(axis=1)
    hi = cells.v.max(axis=1)
    sc = np.abs(cells.v).max(axis=1)
    assert np.all(out.min(axis=1) >= lo - 2e-15 * sc)
    assert np.all(out.max(axis=1) <= hi + 2e-15 * sc)
    for c in range(min(C, 20)):
        A = oracle.assemble(cells.rho_g[c], cells.rho_d[:, c], cells.t_s[:, c], cells.dt)
        P, _, _, _ = oracle.expm(A)
        DP = rho[:, c][:, None] * P
        assert np.max(np.abs(DP - DP.T)) <= 1e-15 * np.max(np.abs(DP))
        assert np.all(P >= -1e-16)


def test_relaxation_to_center_of_mass():
    """dt/T_s -> infinity: every fluid moves with V_CM (Eq. V_cm)."""
    rng = np.random.default_rng(5)
    N, C = 6, 50
    rho_g = np.exp(rng.standard_normal(C))
    rho_d = rng.uniform(0.01, 1, (N, C)) * rho_g
    ts = 10.0 ** rng.uniform(-9, -7, (N, C))
    v = rng.standard_normal((3, N + 1, C))
    out = oracle.drag_apply(rho_g, rho_d, ts, 1.0, v)
    rho = np.vstack([rho_g[None, :], rho_d])
    vcm = np.einsum("fc,dfc->dc", rho, v) / rho.sum(axis=0)
    assert np.max(np.abs(out - vcm[:, None, :])) <= 2e-15 * np.abs(v).max()


def test_semigroup_and_identity():
    """P(dt1) P(dt2) = P(dt1 + dt2) and dt = 0 returns v_in exactly."""
    cells = _workload_sample("mrn_n8_128cube_adjoint", 40)
    zero = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, 0.0, cells.v)
    assert np.array_equal(zero, cells.v)
    for dt1, dt2 in ((0.3, 0.7), (1e-3, 2.5)):
        a = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, dt1, cells.v)
        b = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, dt2, a)
        c = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, dt1 + dt2, cells.v)
        sc = np.abs(cells.v).max(axis=1, keepdims=True)
        assert np.max(np.abs(b - c) / sc) <= 4e-15


def test_decoupled_species():
    """t_s = +inf (alpha = 0) leaves that species untouched; rho_d = 0 species
    relax to the gas without feeding back on it."""
    rng = np.random.default_rng(9)
    N, C = 3, 20
    rho_g = np.ones(C)
    rho_d = rng.uniform(0.1, 1, (N, C))
    ts = rng.uniform(0.1, 2, (N, C))
    ts[1] = np.inf
    rho_d[2] = 0.0
    v = rng.standard_normal((3, N + 1, C))
    out = oracle.drag_apply(rho_g, rho_d, ts, 1.0, v)
    assert np.array_equal(out[:, 2], v[:, 2])
    # the zero-density species 3 does not influence the others
    v2 = v.copy()
    v2[:, 3] += 10.0
    out2 = oracle.drag_apply(rho_g, rho_d, ts, 1.0, v2)
    assert np.array_equal(out2[:, :3], out[:, :3])


def test_invalid_cells_flagged():
    C, N = 6, 2
    rho_g = np.ones(C)
    rho_d = np.full((N, C), 0.5)
    ts = np.full((N, C), 0.5)
    rho_g[1] = 0.0
    rho_d[0, 2] = -1.0
    ts[1, 3] = 0.0
    ts[0, 4] = np.nan
    v = np.ones((3, N + 1, C))
    out, k, s, st = oracle.drag_apply(rho_g, rho_d, ts, 1.0, v, return_ks=True)
    assert st & 1
    bad = [1, 2, 3, 4]
    assert np.all(np.isnan(out[:, :, bad]))
    assert np.all(np.isfinite(out[:, :, [0, 5]]))


# ---------------------------------------------------------------- brute force ---

def test_small_dense_bruteforce_taylor():
    """2x2 and 3x3 (and a few larger) matrices of modest norm: the oracle's S&S
    agrees with an un-scaled 80-term Taylor series in 60-digit arithmetic."""
    pytest.importorskip("mpmath")
    from oracle.truth import expm_taylor_mp
    rng = np.random.default_rng(2)
    for n in (2, 3, 5):
        for trial in range(8):
            A = rng.standard_normal((n, n)) * rng.uniform(0.01, 3.0)
            P, k, m, s = oracle.expm(A, structured=False)
            ref = expm_taylor_mp(A)
            assert np.max(np.abs(P - ref)) <= 1e-14 * np.max(np.abs(ref)), (n, trial, k, s)


def test_drag_cells_bruteforce_taylor():
    """Drag matrices with N = 1, 2 and |A| up to ~8: structured oracle vs the
    un-scaled mpmath Taylor series of A itself."""
    pytest.importorskip("mpmath")
    from oracle.truth import expm_taylor_mp
    rng = np.random.default_rng(4)
    for N in (1, 2):
        for trial in range(10):
            rho_d = rng.uniform(0.05, 2, N)
            ts = rng.uniform(0.3, 4, N)
            A = oracle.assemble(1.0, rho_d, ts, rng.uniform(0.1, 2.0))
            P, k, m, s = oracle.expm(A)
            ref = expm_taylor_mp(A, terms=120, dps=80)
            assert np.max(np.abs(P - ref)) <= 2e-15


@pytest.mark.parametrize("name,C", [("dustybox_n1_32k", 120), ("mrn_n4_128cube", 60),
                                    ("mrn_n8_128cube_adjoint", 30), ("mrn_n16_128cube", 16)])
def test_oracle_vs_eigen_truth_on_workloads(name, C):
    """Structured oracle vs the extended-precision eigen truth on the stiff
    workloads (dt/t_s up to 1e8): forward error below 2e-15 of max |v_in|."""
    pytest.importorskip("mpmath")
    from oracle.truth import drag_truth
    cells = _workload_sample(name, C)
    out = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    ref = drag_truth(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    sc = np.abs(cells.v).max(axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / sc) <= 2e-15


def test_raw_mode_drifts_in_stiff_cells():
    """The literal reading (no row-sum restoration) loses accuracy when s is
    large; this is why both implementations restore row sums."""
    pytest.importorskip("mpmath")
    from oracle.truth import drag_truth
    cells = _workload_sample("mrn_n16_128cube", 16)
    raw = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, structured=False)
    ref = drag_truth(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v)
    sc = np.abs(cells.v).max(axis=1, keepdims=True)
    assert np.max(np.abs(raw - ref) / sc) > 1e-12
