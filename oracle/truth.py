"""Extended-precision truth for the drag update (test infrastructure only).

An independent route to exp(dt Omega_v) v (Eq. ExacSolEqu in velocity form):
the symmetric similarity S = D^(1/2) Omega_v D^(-1/2) (D = diag(rho)),
S_00 = -sum eps_i alpha_i, S_0i = S_i0 = sqrt(eps_i) alpha_i, S_ii = -alpha_i,
is built from the FP64 inputs in mpmath precision, diagonalised (mp.eigsy),
exponentiated through its eigenvalues and mapped back,
v_out = D^(-1/2) Q exp(dt Lambda) Q^T D^(1/2) v. The eigenvalues are those of
the eigenvalue problem of Eq. eigen_problem (Sec. 3.1). It shares nothing with
the FP64 Taylor scaling-and-squaring oracle in drag_oracle.c.

Requires mpmath (present where sympy is installed; tests importorskip it).
"""
from __future__ import annotations

import numpy as np


def _mp():
    import mpmath
    return mpmath


def drag_truth_cell(rho_g, rho_d, t_s, dt, v, dps: int = 40) -> np.ndarray:
    """exp(dt Omega_v) applied to v (shape (3, N+1)) for one cell, via eigsy."""
    mp = _mp()
    with mp.workdps(dps):
        N = len(rho_d)
        n = N + 1
        rg = mp.mpf(float(rho_g))
        eps = [mp.mpf(float(x)) / rg for x in rho_d]
        al = [mp.mpf(0) if np.isinf(x) else 1 / mp.mpf(float(x)) for x in t_s]
        dtm = mp.mpf(float(dt))
        S = mp.zeros(n, n)
        for i in range(1, n):
            S[0, i] = S[i, 0] = mp.sqrt(eps[i - 1]) * al[i - 1] * dtm
            S[i, i] = -al[i - 1] * dtm
            S[0, 0] -= eps[i - 1] * al[i - 1] * dtm
        lam, Q = mp.eigsy(S)
        sig = [mp.mpf(1)] + [mp.sqrt(e) for e in eps]
        out = np.zeros((3, n))
        for d in range(3):
            y = mp.matrix([sig[j] * mp.mpf(float(v[d][j])) for j in range(n)])
            z = Q.T * y
            z = mp.matrix([z[j] * mp.exp(lam[j]) for j in range(n)])
            z = Q * z
            for i in range(n):
                out[d, i] = float(z[i] / sig[i])
        return out


def drag_truth(rho_g, rho_d, t_s, dt, v, dps: int = 40) -> np.ndarray:
    """Truth over SoA arrays: rho_g (C,), rho_d (N, C), t_s (N, C), v (3, N+1, C)."""
    C = len(rho_g)
    out = np.zeros_like(np.asarray(v, dtype=np.float64))
    for c in range(C):
        out[:, :, c] = drag_truth_cell(rho_g[c], rho_d[:, c], t_s[:, c], dt, v[:, :, c], dps)
    return out


def propagator_truth(rho_g, rho_d, t_s, dt, dps: int = 40) -> np.ndarray:
    """P = exp(dt Omega_v) for one cell (rows: output fluid, columns: input fluid)."""
    N = len(rho_d)
    n = N + 1
    P = np.zeros((n, n))
    for j in range(n):
        e = np.zeros((3, n))
        e[:, j] = 1.0
        P[:, j] = drag_truth_cell(rho_g, rho_d, t_s, dt, e, dps)[0]
    return P


def expm_taylor_mp(A, terms: int = 80, dps: int = 60) -> np.ndarray:
    """exp(A) of a small dense matrix by an un-scaled Taylor series in mpmath.

    Only for tiny inputs with modest norm (brute force check of the S&S code).
    """
    mp = _mp()
    with mp.workdps(dps):
        n = len(A)
        M = mp.matrix([[mp.mpf(float(A[i][j])) for j in range(n)] for i in range(n)])
        term = mp.eye(n)
        acc = mp.eye(n)
        for k in range(1, terms + 1):
            term = term * M / k
            acc += term
        return np.array([[float(acc[i, j]) for j in range(n)] for i in range(n)])


def theta_closed_form(m: int, u=None, dps: int = 50) -> float:
    """theta_m of Eq. B8 by an independent route, in mpmath.

    The coefficients of rho(x) = e^-x T_m(x) - 1 have the closed form
    |c_j| = C(j-1, m) / j!  (j >= m+1): from c_j = -sum_{l=m+1}^{j}
    (-1)^{j-l} / ((j-l)! l!) = (-1)^(j+m) C(j-1, m) / j!, using
    sum_{l=0}^{m} (-1)^l C(j, l) = (-1)^m C(j-1, m). The root of
    -log(1 - f_m(theta))/theta = u is then found with mpmath's solver.
    """
    mp = _mp()
    with mp.workdps(dps):
        u = mp.mpf(2) ** -53 if u is None else mp.mpf(u)

        def f(th):
            s = mp.mpf(0)
            for j in range(m + 1, m + 140):
                s += mp.binomial(j - 1, m) / mp.factorial(j) * th ** j
            return s

        def g(th):
            ft = f(th)
            return mp.inf if ft >= 1 else -mp.log(1 - ft) / th - u

        lo, hi = mp.mpf("1e-12"), mp.mpf(10)
        for _ in range(130):
            mid = (lo + hi) / 2
            if g(mid) <= 0:
                lo = mid
            else:
                hi = mid
        return float(lo)


def drag_truth_grad_cell(rho_g, rho_d, t_s, dt, v, g, dps: int = 50, rel_h: float = 1e-14):
    """Gradients of <g, v_out> for one cell by central differences of the
    eigendecomposition truth carried out in ``dps``-digit arithmetic (the
    O(h^2) truncation and the rounding are both far below FP64 resolution).

    Returns (grad_v_in (3, n), grad_rho_g, grad_rho_d (N,), grad_t_s (N,)).
    Independent of the Frechet-derivative machinery of the FP64 oracle.
    """
    mp = _mp()
    N = len(rho_d)
    n = N + 1
    with mp.workdps(dps):
        def loss(rg, rd, ts):
            rg = mp.mpf(rg)
            eps = [mp.mpf(x) / rg for x in rd]
            al = [1 / mp.mpf(x) for x in ts]
            dtm = mp.mpf(float(dt))
            S = mp.zeros(n, n)
            for i in range(1, n):
                S[0, i] = S[i, 0] = mp.sqrt(eps[i - 1]) * al[i - 1] * dtm
                S[i, i] = -al[i - 1] * dtm
                S[0, 0] -= eps[i - 1] * al[i - 1] * dtm
            lam, Q = mp.eigsy(S)
            sig = [mp.mpf(1)] + [mp.sqrt(e) for e in eps]
            tot = mp.mpf(0)
            for d in range(3):
                y = mp.matrix([sig[j] * mp.mpf(float(v[d][j])) for j in range(n)])
                z = Q.T * y
                z = mp.matrix([z[j] * mp.exp(lam[j]) for j in range(n)])
                z = Q * z
                for i in range(n):
                    tot += mp.mpf(float(g[d][i])) * z[i] / sig[i]
            return tot

        rg0 = mp.mpf(float(rho_g))
        rd0 = [mp.mpf(float(x)) for x in rho_d]
        ts0 = [mp.mpf(float(x)) for x in t_s]

        def cd(f, x0):
            h = abs(x0) * mp.mpf(rel_h)
            return (f(x0 + h) - f(x0 - h)) / (2 * h)

        g_rg = cd(lambda x: loss(x, rd0, ts0), rg0)
        g_rd, g_ts = [], []
        for i in range(N):
            g_rd.append(cd(lambda x: loss(rg0, rd0[:i] + [x] + rd0[i + 1:], ts0), rd0[i]))
            g_ts.append(cd(lambda x: loss(rg0, rd0, ts0[:i] + [x] + ts0[i + 1:]), ts0[i]))
    P = propagator_truth(rho_g, rho_d, t_s, dt, dps=dps)
    gv = np.einsum("ji,dj->di", P, np.asarray(g, dtype=np.float64))
    return gv, float(g_rg), np.array([float(x) for x in g_rd]), np.array([float(x) for x in g_ts])


def collisions_exact(rho_g, rho_d, t_s, v0, times) -> np.ndarray:
    """Exact velocities of the Collisions tests (Sec. 3.1, Eq. V_analytic:
    V(t) = V_CM + sum_j c_j exp(lambda_j t)) for every time (rows) and fluid
    (columns, gas first), from the eigenpairs of the symmetric form
    S = D^(1/2) Omega_v D^(-1/2) of the drag matrix (Eq. eigen_problem), in FP64
    through numpy's symmetric eigensolver. rho_d, t_s: the N species; v0: the
    N+1 initial velocities. Pinned by Table 1's printed modes."""
    rho_d = np.asarray(rho_d, dtype=np.float64)
    t_s = np.asarray(t_s, dtype=np.float64)
    eps = rho_d / float(rho_g)
    alpha = 1.0 / t_s
    n = eps.size + 1
    sig = np.concatenate([[1.0], np.sqrt(eps)])
    S = np.zeros((n, n))
    S[0, 0] = -np.sum(eps * alpha)
    S[0, 1:] = S[1:, 0] = sig[1:] * alpha
    S[1:, 1:] = np.diag(-alpha)
    lam, Q = np.linalg.eigh(S)
    y0 = Q.T @ (sig * np.asarray(v0, dtype=np.float64))
    out = np.exp(np.outer(np.asarray(times, dtype=np.float64), lam)) * y0[None, :] @ Q.T
    return out / sig[None, :]
