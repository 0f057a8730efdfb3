"""Pins of the oracle's adjoint (Frechet derivative of the exponential).

Error measure for parameter gradients: log-derivative units x * dL/dx against
the cell's loss scale S = sum_{d,f} |g_{d,f}| max_f' |v_{d,f'}| (for the
linear functional L = <g, v_out>). A fully relaxed species has a true
dL/dt_s of ~1e-30, so a relative-to-itself measure is meaningless there.
"""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W


def loss_scale(g, v):
    return float(np.sum(np.abs(g) * np.abs(v).max(axis=0, keepdims=True)))


def test_frechet_dense_vs_directional_derivative():
    """Z = L(A^T, G) against its definition d/dh exp(A^T + h G) at h = 0,
    by central differences of mpmath's expm in 50-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(21)
    for n in (2, 3, 4):
        for trial in range(4):
            A = rng.standard_normal((n, n)) * rng.uniform(0.1, 6.0)
            G = rng.standard_normal((n, n))
            Z = oracle.frechet_T(A, G)
            with mp.workdps(50):
                At = mp.matrix(A.T.tolist())
                Gm = mp.matrix(G.tolist())
                h = mp.mpf("1e-20")
                D = (mp.expm(At + h * Gm) - mp.expm(At - h * Gm)) / (2 * h)
                ref = np.array([[float(D[i, j]) for j in range(n)] for i in range(n)])
            assert np.max(np.abs(Z - ref)) <= 1e-12 * np.max(np.abs(ref)), (n, trial)


def test_frechet_structured_drag_matrix():
    """Structured mode (column sums of exp(A^T) restored) on drag matrices
    against the same directional-derivative definition."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(22)
    for N in (1, 2, 3):
        for trial in range(3):
            A = oracle.assemble(1.0, rng.uniform(0.1, 2.0, N), 10.0 ** rng.uniform(-2, 1, N), 1.0)
            G = rng.standard_normal((N + 1, N + 1))
            Z = oracle.frechet_T(A, G, structured=True)
            with mp.workdps(50):
                At = mp.matrix(A.T.tolist())
                Gm = mp.matrix(G.tolist())
                h = mp.mpf("1e-20")
                D = (mp.expm(At + h * Gm) - mp.expm(At - h * Gm)) / (2 * h)
                ref = np.array([[float(D[i, j]) for j in range(N + 1)] for i in range(N + 1)])
            assert np.max(np.abs(Z - ref)) <= 1e-12 * np.max(np.abs(ref)), (N, trial)


STIFF_N1 = "stiff_n1"


@pytest.mark.parametrize("name,C", [("dustybox_n1_32k", 8), ("mrn_n4_128cube", 6), ("mrn_n8_128cube_adjoint", 4),
                                    (STIFF_N1, 12)])
def test_adjoint_vs_extended_truth(name, C):
    """Gradients of <g, v_out> against central differences of the 50-digit
    eigendecomposition truth (independent of the Frechet machinery),
    including fully relaxed cells (dt/t_s up to 1e8)."""
    pytest.importorskip("mpmath")
    from oracle.truth import drag_truth_grad_cell
    if name == STIFF_N1:
        cells = W.mrn(46, 1, seed=301, stiff_lo=-4.0, stiff_hi=8.0).subset([1, 13, 18, 27, 40, 44, 0, 2, 3, 5, 7, 9])
    else:
        cells = W.workload(name, ncells=C)
    g = np.random.default_rng(5).standard_normal(cells.v.shape)
    gv, grg, grd, gts, st = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)
    assert st == 0
    for c in range(C):
        tv, trg, trd, tts = drag_truth_grad_cell(cells.rho_g[c], cells.rho_d[:, c], cells.t_s[:, c], cells.dt,
                                                 cells.v[:, :, c], g[:, :, c])
        S = loss_scale(g[:, :, c], cells.v[:, :, c])
        gsc = np.abs(g[:, :, c]).sum(axis=1, keepdims=True)
        assert np.max(np.abs(gv[:, :, c] - tv) / gsc) <= 2e-15
        assert np.max(np.abs(cells.rho_d[:, c] * (grd[:, c] - trd))) <= 1e-14 * S
        assert np.max(np.abs(cells.t_s[:, c] * (gts[:, c] - tts))) <= 1e-14 * S
        assert abs(cells.rho_g[c] * (grg[c] - trg)) <= 1e-14 * S


def _perturbed_batch(sub, h_rel=1e-6):
    """All +/- perturbations of one parameter per copy, stacked as cells."""
    N, n, C = sub.nspecies, sub.nspecies + 1, sub.ncells
    params = [("v", d, f) for d in range(3) for f in range(n)] + [("rd", i, None) for i in range(N)] + \
             [("ts", i, None) for i in range(N)]
    P = len(params)
    rg = np.tile(sub.rho_g, 2 * P)
    rd = np.tile(sub.rho_d, (1, 2 * P))
    ts = np.tile(sub.t_s, (1, 2 * P))
    v = np.tile(sub.v, (1, 1, 2 * P))
    hs = np.zeros((P, C))
    for p, (kind, a, b) in enumerate(params):
        for sgn, blk in ((1.0, 2 * p), (-1.0, 2 * p + 1)):
            sl = slice(blk * C, (blk + 1) * C)
            if kind == "v":
                x = sub.v[a, b]
                h = h_rel * np.maximum(np.abs(x), 1e-3)
                v[a, b, sl] = x + sgn * h
            elif kind == "rd":
                x = sub.rho_d[a]
                h = h_rel * np.abs(x)
                rd[a, sl] = x + sgn * h
            else:
                x = sub.t_s[a]
                h = h_rel * np.abs(x)
                ts[a, sl] = x + sgn * h
            hs[p] = h
    return params, hs, W.Cells(rg, rd, ts, v, sub.dt)


def finite_difference_gradients(forward, sub, vt):
    """Per-cell loss L_c = 0.5 ||v_out - v_target||^2; returns FD gradients
    (gv (3,n,C), grd (N,C), gts (N,C))."""
    N, n, C = sub.nspecies, sub.nspecies + 1, sub.ncells
    params, hs, big = _perturbed_batch(sub)
    out = forward(big)
    vt_big = np.tile(vt, (1, 1, 2 * len(params)))
    Lc = 0.5 * np.sum((out - vt_big) ** 2, axis=(0, 1))
    gv = np.zeros((3, n, C))
    grd = np.zeros((N, C))
    gts = np.zeros((N, C))
    for p, (kind, a, b) in enumerate(params):
        lp = Lc[(2 * p) * C:(2 * p + 1) * C]
        lm = Lc[(2 * p + 1) * C:(2 * p + 2) * C]
        fd = (lp - lm) / (2 * hs[p])
        if kind == "v":
            gv[a, b] = fd
        elif kind == "rd":
            grd[a] = fd
        else:
            gts[a] = fd
    return gv, grd, gts


def assert_fd_agreement(sub, g, gv_ad, grd_ad, gts_ad, gv_fd, grd_fd, gts_fd, rel=1e-6):
    C = sub.ncells
    for c in range(C):
        S = loss_scale(g[:, :, c], sub.v[:, :, c]) + 1e-300
        for ad, fd, x in ((gv_ad[:, :, c], gv_fd[:, :, c], np.maximum(np.abs(sub.v[:, :, c]), 1e-3)),
                          (grd_ad[:, c], grd_fd[:, c], np.abs(sub.rho_d[:, c])),
                          (gts_ad[:, c], gts_fd[:, c], np.abs(sub.t_s[:, c]))):
            kind_scale = np.max(np.abs(fd))
            bound = rel * np.maximum(np.abs(fd), kind_scale) + 1e-9 * S / x
            assert np.all(np.abs(ad - fd) <= bound), (c, np.max(np.abs(ad - fd) / bound))


def test_adjoint_finite_differences_64_cells():
    """The N=8 adjoint workload: loss 0.5 ||v_out - v_target||^2, gradients with
    respect to v_in, rho_d, t_s on 64 random cells against central differences
    of the forward oracle (1e-6 relative)."""
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=4096)
    target = W.adjoint_target(cells.ncells, cells.nspecies)
    idx = np.sort(np.random.default_rng(64).choice(cells.ncells, 64, replace=False))
    sub = cells.subset(idx)
    vt = target[:, :, idx]
    fwd = lambda c: oracle.drag_apply(c.rho_g, c.rho_d, c.t_s, c.dt, c.v)
    g = fwd(sub) - vt
    gv, _, grd, gts, st = oracle.drag_backward(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, g)
    assert st == 0
    gv_fd, grd_fd, gts_fd = finite_difference_gradients(fwd, sub, vt)
    assert_fd_agreement(sub, g, gv, grd, gts, gv_fd, grd_fd, gts_fd)


def test_adjoint_v_in_identity_and_dt_zero():
    """dL/dv_in = P^T g = rho o P (g / rho) (detailed balance), and with dt = 0
    every parameter gradient vanishes and dL/dv_in = g."""
    cells = W.workload("mrn_n4_128cube", ncells=32)
    g = np.random.default_rng(3).standard_normal(cells.v.shape)
    gv, grg, grd, gts, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)
    rho = np.vstack([cells.rho_g[None, :], cells.rho_d])
    alt = rho[None] * oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, g / rho[None])
    sc = np.abs(g).sum(axis=1, keepdims=True)
    assert np.max(np.abs(gv - alt) / sc) <= 4e-15
    gv0, grg0, grd0, gts0, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, 0.0, cells.v, g)
    assert np.array_equal(gv0, g)
    assert np.all(grd0 == 0) and np.all(gts0 == 0) and np.all(grg0 == 0)


def test_adjoint_rho_g_scaling_invariance():
    """Scaling rho_g and every rho_d by the same factor leaves v_out unchanged
    (only eps_i = rho_d,i/rho_g enters), so rho_g dL/drho_g + sum_i rho_d,i dL/drho_d,i = 0."""
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=64)
    g = np.random.default_rng(8).standard_normal(cells.v.shape)
    gv, grg, grd, gts, _ = oracle.drag_backward(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, g)
    tot = cells.rho_g * grg + np.sum(cells.rho_d * grd, axis=0)
    S = np.array([loss_scale(g[:, :, c], cells.v[:, :, c]) for c in range(cells.ncells)])
    assert np.all(np.abs(tot) <= 1e-14 * S)
