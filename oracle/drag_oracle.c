/*
 * CPU oracle for the exponential ("EXP") multi-fluid drag update.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. The product path (the CUDA library
 * and its Python binding) never calls it, links it or shares code with it.
 *
 * Plain, slow, FP64 C that follows the paper step by step:
 *   Sec. 2.2, Eqs. DragEq..jacobian : the drag matrix Omega of gas + N dust species
 *   Sec. 2.3, Eq. ExacSolEqu        : U(t) = exp(t Omega) U(t0)
 *   App. B, Eqs. B1-B8              : backward-error bound, theta_m for u = 2^-53
 *   App. B, Table B.1               : m_k, q_k, r_k for k = 1..9
 *   App. B, Algorithm 2             : choice of (k*, m*, s*)
 *   App. B, Eqs. Pat_Stk..Pat_Stk3, Algorithm 3 : Paterson-Stockmeyer evaluation
 *   Sec. 2.3.2, Eq. ExpEq1/def_s, Algorithm 6   : scaling and squaring
 *
 * Velocity form. The drag step keeps densities fixed, so with U = D v and
 * D = diag(rho_g, rho_d,1..N) the velocities obey dv/dt = Omega_v v with
 * Omega_v = D^-1 Omega D = Omega^T (Eq. jacobian transposed):
 *   (Omega_v)_00 = -sum_i eps_i alpha_i, (Omega_v)_0i = eps_i alpha_i,
 *   (Omega_v)_i0 = alpha_i,              (Omega_v)_ii = -alpha_i.
 * Every row of Omega_v sums to zero (momentum conservation, Eq. DragEq).
 *
 * "Structured" mode (the default) keeps that property exactly in floating
 * point: the diagonal of A = dt Omega_v is assembled as minus the sum of its
 * row's off-diagonals, and after the Taylor step and after every squaring the
 * diagonal of P is reset to 1 - sum of the row's off-diagonals. "Raw" mode is
 * the literal reading (diagonal accumulated as in Eq. jacobian, no reset); it
 * is kept only to report how far the literal method drifts in stiff cells.
 *
 * Everything is plain IEEE double with no FMA contraction (built with
 * -ffp-contract=off), so results are identical on x86-64 and aarch64.
 * No long double is used anywhere.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_K 9          /* maximum number of products in the Taylor phase (all Table B.1 rows) */
#define ORC_NMAX 64      /* largest matrix the oracle accepts (n = N + 1) */

/* Table B.1: k, m_k, q_k, r_k (index 0 unused). m_k = q_k * r_k. */
static const int orc_mk[ORC_K + 1] = {0, 2, 4, 6, 9, 12, 16, 20, 25, 30};
static const int orc_qk[ORC_K + 1] = {0, 1, 2, 2, 3, 3, 4, 4, 5, 5};
static const int orc_rk[ORC_K + 1] = {0, 2, 2, 3, 3, 4, 4, 5, 5, 6};

/* ------------------------------------------------------------------------ */
/* Eqs. B4-B8: theta_m                                                       */
/* ------------------------------------------------------------------------ */

/* Coefficients c_j of rho(x) = e^{-x} T_m(x) - 1 = sum_{j>=m+1} c_j x^j
 * (Eq. B5): rho(x) = -(sum_i (-x)^i/i!) (sum_{l>=m+1} x^l/l!), so
 * c_j = -sum_{l=m+1}^{j} (-1)^{j-l} / ((j-l)! l!).  Returns c_{m+1..m+L}. */
static void orc_rho_coeffs(int m, int L, double *c)
{
    for (int t = 0; t < L; t++) {
        int j = m + 1 + t;
        double acc = 0.0;
        for (int l = m + 1; l <= j; l++) {
            double term = 1.0;
            for (int a = 2; a <= j - l; a++) term /= a;   /* 1/(j-l)! */
            for (int a = 2; a <= l; a++) term /= a;       /* 1/l! */
            if ((j - l) & 1) term = -term;
            acc += term;
        }
        c[t] = -acc;
    }
}

/* f_m(theta) = sum_{j>=m+1} |c_j| theta^j (Eq. B6), truncated after L terms. */
static double orc_fm(int m, int L, const double *c, double theta)
{
    double f = 0.0, p = pow(theta, (double)(m + 1));
    for (int t = 0; t < L; t++) {
        f += fabs(c[t]) * p;
        p *= theta;
    }
    return f;
}

/* theta_m = max{theta : -log(1 - f_m(theta))/theta <= u} (Eq. B8), found by
 * bisection; the bound is increasing in theta. */
double orc_theta_m(int m, double u)
{
    enum { L = 80 };
    double c[L];
    orc_rho_coeffs(m, L, c);
    double lo = 0.0, hi = 64.0;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = orc_fm(m, L, c, mid);
        double bound = (f < 1.0) ? -log1p(-f) / mid : INFINITY;
        if (bound <= u) lo = mid; else hi = mid;
    }
    return lo;
}

/* theta_{m_k}, k = 1..9, for u = 2^-53 (Table B.1, column theta_{m_k}). */
void orc_theta_table(double *theta /* [ORC_K + 1], index 0 unused */)
{
    theta[0] = 0.0;
    for (int k = 1; k <= ORC_K; k++) theta[k] = orc_theta_m(orc_mk[k], ldexp(1.0, -53));
}

static double g_theta[ORC_K + 1];
static int g_theta_ready = 0;

static const double *orc_thetas(void)
{
    if (!g_theta_ready) {
        orc_theta_table(g_theta);
        g_theta_ready = 1;
    }
    return g_theta;
}

/* theta_{m_k}, k = 1..9, for another unit round-off u (Eq. B8 names 2^-11,
 * 2^-24, 2^-113 and 2^-237 besides 2^-53). */
void orc_theta_table_u(double u, double *theta /* [ORC_K + 1] */)
{
    theta[0] = 0.0;
    for (int k = 1; k <= ORC_K; k++) theta[k] = orc_theta_m(orc_mk[k], u);
}

/* Tables for the last few distinct u asked for (computed once each). */
enum { ORC_U_SLOTS = 8 };
static double g_theta_u[ORC_U_SLOTS][ORC_K + 1];
static double g_theta_u_key[ORC_U_SLOTS];
static int g_theta_u_used = 0;

static const double *orc_thetas_u(double u)
{
    if (u == ldexp(1.0, -53)) return orc_thetas();
    for (int i = 0; i < g_theta_u_used; i++)
        if (g_theta_u_key[i] == u) return g_theta_u[i];
    int slot = g_theta_u_used < ORC_U_SLOTS ? g_theta_u_used++ : ORC_U_SLOTS - 1;
    orc_theta_table_u(u, g_theta_u[slot]);
    g_theta_u_key[slot] = u;
    return g_theta_u[slot];
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: polynomial order and scale factor                           */
/* ------------------------------------------------------------------------ */

/* Readings (the listing is ambiguous in places):
 *  - s^ = ceil(max(log2(|A|/theta_{m_K}), 0)) is taken as the smallest
 *    integer s >= 0 with 2^-s |A| <= theta_{m_K} (no log/ceil rounding).
 *  - s* starts at s^ (the listing writes s* = 0, which would leave large
 *    norms unscaled; Algorithm 1 sets s* = s^ in that case).
 *  - k^ is the k at which the search loop stopped (first k with
 *    |A| <= theta_{m_k}), or K if there is none.
 *  - The three reduction branches are taken only when v > 0; the listing's
 *    max() gives v3 priority over v2 over v1.
 *  - "m* = m_k*" means m* = m_{k*}.
 * Returns 0, or -1 if |A| is not finite (the caller marks the cell invalid). */
static int orc_select_alg2_th(const double *th, double normA, int K, int *kstar, int *mstar, int *sstar)
{
    if (!isfinite(normA) || normA < 0.0) {
        *kstar = K; *mstar = orc_mk[K]; *sstar = 0;
        return -1;
    }
    int ms = orc_mk[K];
    int ks = K;
    int shat = 0;
    while (ldexp(normA, -shat) > th[K]) shat++;
    int ss = shat;
    int cond = 0;
    int khat = K;
    for (int k = 1; k <= K && !cond; k++) {
        double lim = th[k] < th[K] ? th[k] : th[K];
        cond = normA <= lim;
        if (cond) {
            ms = orc_mk[k];
            ks = k;
            khat = k;
        }
    }
    double cmp = ldexp(normA, -shat);
    int v1 = (khat >= 7) && (cmp <= th[khat - 1]);
    int v2 = ((khat >= 8) && (cmp <= 2.0 * th[khat - 2])) * 2;
    int v3 = ((khat >= 9) && (cmp <= 4.0 * th[khat - 3])) * 3;
    int v = v1;
    if (v2 > v) v = v2;
    if (v3 > v) v = v3;
    if (v > 0) {
        if (v == v1) {
            ks = khat - 1; ms = orc_mk[ks];
        } else if (v == v2) {
            ks = khat - 2; ms = orc_mk[ks]; ss = (shat + 1 > 1) ? shat + 1 : 1;
        } else {
            ks = khat - 3; ms = orc_mk[ks]; ss = (shat + 2 > 2) ? shat + 2 : 2;
        }
    }
    *kstar = ks; *mstar = ms; *sstar = ss;
    return 0;
}

int orc_select_alg2(double normA, int K, int *kstar, int *mstar, int *sstar)
{
    return orc_select_alg2_th(orc_thetas(), normA, K, kstar, mstar, sstar);
}

/* Algorithm 2 with the theta table of unit round-off u. */
int orc_select_alg2_u(double normA, int K, double u, int *kstar, int *mstar, int *sstar)
{
    return orc_select_alg2_th(orc_thetas_u(u), normA, K, kstar, mstar, sstar);
}

/* ------------------------------------------------------------------------ */
/* Dense n x n helpers (row-major), plain loops, ascending index order       */
/* ------------------------------------------------------------------------ */

static void orc_matmul(int n, const double *A, const double *B, double *C)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0.0;
            for (int k = 0; k < n; k++) acc += A[i * n + k] * B[k * n + j];
            C[i * n + j] = acc;
        }
}

/* 1-norm: maximum absolute column sum. */
static double orc_norm1(int n, const double *A)
{
    double best = 0.0;
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += fabs(A[i * n + j]);
        if (s > best || isnan(s)) best = s;
    }
    return best;
}

/* Row-sum restoration: P_ii = 1 - sum_{j != i} P_ij. */
static void orc_restore(int n, double *P)
{
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int j = 0; j < n; j++)
            if (j != i) s += P[i * n + j];
        P[i * n + i] = 1.0 - s;
    }
}

/* ------------------------------------------------------------------------ */
/* Taylor scaling and squaring (Algorithm 6 with Algorithm 2 and the         */
/* Paterson-Stockmeyer evaluation of Eqs. Pat_Stk..Pat_Stk3 / Algorithm 3)   */
/* ------------------------------------------------------------------------ */

/* P = T_{m}(X) for X = 2^-s A, then s squarings.
 * T_m(X) = I + sum_{k=0}^{r-1} Bbar_k (X^q)^k with
 * Bbar_k = sum_{j=1}^{q} b_{qk+j} X^j, b_i = 1/i!  (Algorithm 3; m = q r),
 * evaluated by Horner in X^q with the stored powers X, X^2, ..., X^q.
 * With structured != 0 the diagonal is restored after the Taylor step and
 * after every squaring. Returns 0, or -1 when |A| is not finite. */
/* ------------------------------------------------------------------------ */
/* Second modification: the bound test (Eqs. Pat_Stk4-Pat_Stk7, Alg. 8/9)   */
/* ------------------------------------------------------------------------ */

/* Number of Paterson-Stockmeyer blocks to keep. pw[j] = X^j (j = 1..q, each
 * n x n), b[i] = 1/i!, T_m(X) = I + sum_{l<r} Bbar_l (X^q)^l with
 * Bbar_l = sum_{j=1}^{q} b_{ql+j} X^j.
 *   b_exp = |b_0 I + Bhat_0| + sum_{l=1}^{r-1} |Bhat_l| |X^q|^l     (Eq. Pat_Stk6)
 *   Bhat_l = sum_{j=1}^{q} (-1)^{ql+j} b_{ql+j} X^j                 (so b_exp >= |T_m(-X)|)
 * The highest block is dropped while
 *   b_exp |Bbar_{keep-1}| |X^q|^{keep-1} <= u                       (Eq. Pat_Stk5)
 * holds (reading of Algorithm 9's per-block condition; at least one block is
 * kept). ratio_out (optional) receives the left side for the top block / u. */
static int orc_bound_test_keep(int n, const double *pw, int q, int r, const double *b, double u, double *ratio_out)
{
    const size_t nn = (size_t)n * n;
    double *T = (double *)malloc(sizeof(double) * nn);
    const double xq = orc_norm1(n, pw + (size_t)q * nn);
    double bexp = 0.0, xql = 1.0;
    for (int l = 0; l < r; l++) {
        for (size_t e = 0; e < nn; e++) {
            double acc = 0.0;
            for (int j = 1; j <= q; j++) {
                const double c = ((q * l + j) & 1) ? -b[q * l + j] : b[q * l + j];
                acc += c * pw[(size_t)j * nn + e];
            }
            T[e] = acc;
        }
        if (l == 0)
            for (int i = 0; i < n; i++) T[(size_t)i * n + i] += b[0];
        bexp += orc_norm1(n, T) * xql;
        xql *= xq;
    }
    int keep = r;
    if (ratio_out) *ratio_out = 0.0;
    while (keep > 1) {
        const int l = keep - 1;
        for (size_t e = 0; e < nn; e++) {
            double acc = 0.0;
            for (int j = 1; j <= q; j++) acc += b[q * l + j] * pw[(size_t)j * nn + e];
            T[e] = acc;
        }
        double val = bexp * orc_norm1(n, T);
        for (int t = 0; t < l; t++) val *= xq;
        if (keep == r && ratio_out) *ratio_out = val / u;
        if (!(val <= u)) break;
        keep--;
    }
    free(T);
    return keep;
}

static int orc_expm_u(int n, const double *A, double *P, int structured, double u, int bound_test, int *k_out,
                      int *m_out, int *s_out, double *ratio_out)
{
    int k, m, s;
    int rc = orc_select_alg2_u(orc_norm1(n, A), ORC_K, u, &k, &m, &s);
    if (k_out) *k_out = k;
    if (m_out) *m_out = m;
    if (s_out) *s_out = s;
    if (rc != 0) {
        for (int i = 0; i < n * n; i++) P[i] = NAN;
        return -1;
    }
    const int q = orc_qk[k], r = orc_rk[k];
    const size_t nn = (size_t)n * n;
    double *pw = (double *)calloc((size_t)(q + 1) * nn, sizeof(double)); /* pw[j] = X^j */
    double *F = (double *)calloc(nn, sizeof(double));
    double *T = (double *)calloc(nn, sizeof(double));
    double *Bb = (double *)calloc(nn, sizeof(double));
    double b[64];
    b[0] = 1.0;
    for (int i = 1; i <= m; i++) b[i] = b[i - 1] / (double)i;

    for (size_t e = 0; e < nn; e++) pw[nn + e] = ldexp(A[e], -s);       /* X = 2^-s A */
    for (int j = 2; j <= q; j++) orc_matmul(n, pw + (size_t)(j - 1) * nn, pw + nn, pw + (size_t)j * nn);
    int rb = r;                                                          /* blocks kept */
    if (bound_test) {
        rb = orc_bound_test_keep(n, pw, q, r, b, u, ratio_out);
        if (m_out) *m_out = q * rb;
    }

    /* Horner in X^q: F = Bbar_{rb-1}; F = Bbar_k + F X^q for k = rb-2..0 */
    for (int kk = rb - 1; kk >= 0; kk--) {
        for (size_t e = 0; e < nn; e++) {
            double acc = 0.0;
            for (int j = 1; j <= q; j++) acc += b[q * kk + j] * pw[(size_t)j * nn + e];
            Bb[e] = acc;
        }
        if (kk == rb - 1) {
            memcpy(F, Bb, nn * sizeof(double));
        } else {
            orc_matmul(n, F, pw + (size_t)q * nn, T);
            for (size_t e = 0; e < nn; e++) F[e] = Bb[e] + T[e];
        }
    }
    for (size_t e = 0; e < nn; e++) P[e] = F[e];
    for (int i = 0; i < n; i++) P[i * n + i] += 1.0;                   /* + b_0 I */
    if (structured) orc_restore(n, P);

    for (int t = 0; t < s; t++) {                                       /* Eq. ExpEq1, n = 2^s */
        orc_matmul(n, P, P, T);
        memcpy(P, T, nn * sizeof(double));
        if (structured) orc_restore(n, P);
    }
    free(pw); free(F); free(T); free(Bb);
    return 0;
}

int orc_expm(int n, const double *A, double *P, int structured, int *k_out, int *m_out, int *s_out)
{
    return orc_expm_u(n, A, P, structured, ldexp(1.0, -53), 0, k_out, m_out, s_out, NULL);
}

/* ------------------------------------------------------------------------ */
/* Pade variant (Eq. PadeEqu): R_mm = D_mm^-1 N_mm, scaling and squaring      */
/* ------------------------------------------------------------------------ */

/* Coefficients of N_mm (Eq. PadeEqu with p = q = m):
 * c_j = (2m - j)! m! / ((2m)! j! (m - j)!), j = 0..m; D_mm(X) = N_mm(-X). */
void orc_pade_coeffs(int m, double *c)
{
    for (int j = 0; j <= m; j++) {
        double v = 1.0;
        for (int a = 2 * m - j + 1; a <= 2 * m; a++) v /= a;   /* (2m-j)!/(2m)! */
        for (int a = m - j + 1; a <= m; a++) v *= a;           /* m!/(m-j)! */
        for (int a = 2; a <= j; a++) v /= a;                   /* 1/j! */
        c[j] = v;
    }
}

/* Double-double numbers (hi + lo, |lo| <= ulp(hi)/2) for the Pade series:
 * error-free sum (Knuth) and product (explicit fma), so results are the same
 * on every IEEE platform. */
typedef struct { double hi, lo; } orc_dd;

static orc_dd orc_dd_add(orc_dd a, orc_dd b)
{
    double s = a.hi + b.hi, bb = s - a.hi;
    double e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
    orc_dd r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}

static orc_dd orc_dd_mul(orc_dd a, orc_dd b)
{
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    orc_dd r;
    r.hi = p + e;
    r.lo = e - (r.hi - p);
    return r;
}

static orc_dd orc_dd_div_int(orc_dd a, int k)   /* a / k, k > 0 */
{
    double q = a.hi / k;
    double e = fma(-q, (double)k, a.hi) + a.lo;    /* remainder a - q k */
    double q2 = e / k;
    orc_dd r;
    r.hi = q + q2;
    r.lo = q2 - (r.hi - q);
    return r;
}

static orc_dd orc_dd_neg(orc_dd a) { a.hi = -a.hi; a.lo = -a.lo; return a; }

/* Series of rho(x) = e^-x N_mm(x) / D_mm(x) - 1 up to x^(L-1): the inverse
 * series of D (D(0) = 1), times N, times e^-x, in double-double (the terms of
 * order <= 2m cancel, rho_j = 0 there, and the leading rho_j are ~10 orders
 * below the partial sums). */
static void orc_pade_rho(int m, int L, double *rho)
{
    orc_dd c[32], w[256], y[256], fac[256];
    for (int j = 0; j <= m; j++) {                 /* c_j = (2m-j)! m! / ((2m)! j! (m-j)!) */
        orc_dd v = {1.0, 0.0};
        for (int a = 2 * m - j + 1; a <= 2 * m; a++) v = orc_dd_div_int(v, a);
        for (int a = m - j + 1; a <= m; a++) v = orc_dd_mul(v, (orc_dd){(double)a, 0.0});
        for (int a = 2; a <= j; a++) v = orc_dd_div_int(v, a);
        c[j] = v;
    }
    fac[0] = (orc_dd){1.0, 0.0};                    /* 1/i! */
    for (int i = 1; i < L; i++) fac[i] = orc_dd_div_int(fac[i - 1], i);
    for (int k = 0; k < L; k++) {                 /* w = 1 / D, D_i = (-1)^i c_i */
        orc_dd acc = {k == 0 ? 1.0 : 0.0, 0.0};
        for (int i = 1; i <= m && i <= k; i++) {
            orc_dd t = orc_dd_mul(c[i], w[k - i]);
            acc = orc_dd_add(acc, (i & 1) ? t : orc_dd_neg(t));
        }
        w[k] = acc;
    }
    for (int k = 0; k < L; k++) {                 /* y = N w */
        orc_dd acc = {0.0, 0.0};
        for (int i = 0; i <= m && i <= k; i++) acc = orc_dd_add(acc, orc_dd_mul(c[i], w[k - i]));
        y[k] = acc;
    }
    for (int k = 0; k < L; k++) {                 /* rho = e^-x y - 1 */
        orc_dd acc = {k == 0 ? -1.0 : 0.0, 0.0};
        for (int i = 0; i <= k; i++) {
            orc_dd t = orc_dd_mul(fac[i], y[k - i]);
            acc = orc_dd_add(acc, (i & 1) ? orc_dd_neg(t) : t);
        }
        rho[k] = acc.hi + acc.lo;
    }
}

/* theta of the [m/m] Pade approximant: the construction of Eqs. B5-B8 with
 * T_m replaced by R_mm, i.e. the largest theta with
 * -log(1 - f(theta))/theta <= u, f(theta) = sum_{j>2m} |rho_j| theta^j. */
double orc_pade_theta(int m, double u)
{
    enum { L = 200 };
    double rho[L];
    orc_pade_rho(m, L, rho);
    double lo = 0.0, hi = 16.0;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = 0.0, p = pow(mid, 2.0 * m + 1.0);
        for (int j = 2 * m + 1; j < L; j++) {
            f += fabs(rho[j]) * p;
            p *= mid;
        }
        double bound = (f < 1.0) ? -log1p(-f) / mid : INFINITY;
        if (bound <= u) lo = mid; else hi = mid;
    }
    return lo;
}

static const int orc_pade_m[5] = {3, 5, 7, 9, 13};

/* Degree and scaling for the Pade variant: the smallest m in {3, 5, 7, 9}
 * with |A| <= theta_m and s = 0, else m = 13 and the smallest s with
 * 2^-s |A| <= theta_13 (the paper gives no selection for Pade; this is the
 * usual choice of the Pade scaling and squaring it cites). */
int orc_select_pade(double normA, double u, int *m_out, int *s_out)
{
    if (!isfinite(normA) || normA < 0.0) {
        *m_out = 13; *s_out = 0;
        return -1;
    }
    for (int i = 0; i < 4; i++)
        if (normA <= orc_pade_theta(orc_pade_m[i], u)) {
            *m_out = orc_pade_m[i]; *s_out = 0;
            return 0;
        }
    const double th = orc_pade_theta(13, u);
    int s = 0;
    while (ldexp(normA, -s) > th) s++;
    *m_out = 13; *s_out = s;
    return 0;
}

/* Solve D R = N for R (n x n), Gaussian elimination with partial pivoting
 * on copies of D and N. Returns -1 if a pivot is zero. */
static int orc_solve(int n, const double *Dm, const double *Nm, double *R)
{
    const size_t nn = (size_t)n * n;
    double *M = (double *)malloc(sizeof(double) * nn);
    memcpy(M, Dm, sizeof(double) * nn);
    memcpy(R, Nm, sizeof(double) * nn);
    int rc = 0;
    for (int j = 0; j < n && rc == 0; j++) {
        int p = j;
        for (int i = j + 1; i < n; i++)
            if (fabs(M[(size_t)i * n + j]) > fabs(M[(size_t)p * n + j])) p = i;
        if (M[(size_t)p * n + j] == 0.0) { rc = -1; break; }
        if (p != j)
            for (int c = 0; c < n; c++) {
                double t = M[(size_t)j * n + c]; M[(size_t)j * n + c] = M[(size_t)p * n + c]; M[(size_t)p * n + c] = t;
                t = R[(size_t)j * n + c]; R[(size_t)j * n + c] = R[(size_t)p * n + c]; R[(size_t)p * n + c] = t;
            }
        for (int i = j + 1; i < n; i++) {
            const double l = M[(size_t)i * n + j] / M[(size_t)j * n + j];
            for (int c = j; c < n; c++) M[(size_t)i * n + c] -= l * M[(size_t)j * n + c];
            for (int c = 0; c < n; c++) R[(size_t)i * n + c] -= l * R[(size_t)j * n + c];
        }
    }
    for (int j = n - 1; j >= 0 && rc == 0; j--)
        for (int c = 0; c < n; c++) {
            double acc = R[(size_t)j * n + c];
            for (int k = j + 1; k < n; k++) acc -= M[(size_t)j * n + k] * R[(size_t)k * n + c];
            R[(size_t)j * n + c] = acc / M[(size_t)j * n + j];
        }
    free(M);
    return rc;
}

/* P = R_mm(X)^(2^s), X = 2^-s A, with the structured restoration after the
 * Pade step and every squaring (as the Taylor path). */
static int orc_expm_pade(int n, const double *A, double *P, int structured, double u, int *m_out, int *s_out)
{
    int m, s;
    int rc = orc_select_pade(orc_norm1(n, A), u, &m, &s);
    if (m_out) *m_out = m;
    if (s_out) *s_out = s;
    const size_t nn = (size_t)n * n;
    if (rc != 0) {
        for (size_t e = 0; e < nn; e++) P[e] = NAN;
        return -1;
    }
    double c[32];
    orc_pade_coeffs(m, c);
    double *X = (double *)malloc(sizeof(double) * nn), *Xj = (double *)malloc(sizeof(double) * nn);
    double *T = (double *)malloc(sizeof(double) * nn), *Nm = (double *)calloc(nn, sizeof(double));
    double *Dm = (double *)calloc(nn, sizeof(double));
    for (size_t e = 0; e < nn; e++) X[e] = ldexp(A[e], -s);
    for (size_t e = 0; e < nn; e++) Xj[e] = 0.0;
    for (int i = 0; i < n; i++) Xj[(size_t)i * n + i] = 1.0;             /* X^0 */
    for (int j = 0; j <= m; j++) {
        if (j > 0) {
            orc_matmul(n, Xj, X, T);
            memcpy(Xj, T, sizeof(double) * nn);
        }
        for (size_t e = 0; e < nn; e++) {
            Nm[e] += c[j] * Xj[e];
            Dm[e] += ((j & 1) ? -c[j] : c[j]) * Xj[e];
        }
    }
    rc = orc_solve(n, Dm, Nm, P);
    if (rc == 0) {
        if (structured) orc_restore(n, P);
        for (int t = 0; t < s; t++) {
            orc_matmul(n, P, P, T);
            memcpy(P, T, sizeof(double) * nn);
            if (structured) orc_restore(n, P);
        }
    } else {
        for (size_t e = 0; e < nn; e++) P[e] = NAN;
    }
    free(X); free(Xj); free(T); free(Nm); free(Dm);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Drag matrix (Eqs. DragEqVar2, DragEqVar3, jacobian) in velocity form      */
/* ------------------------------------------------------------------------ */

/* Cell input check: rho_g > 0, rho_d >= 0, t_s > 0 (t_s = +inf allowed:
 * alpha = 0, a decoupled species), all finite except t_s = +inf. */
static int orc_cell_valid(int N, double rho_g, const double *rho_d, const double *t_s, double dt)
{
    if (!(rho_g > 0.0) || !isfinite(rho_g) || !(dt >= 0.0) || !isfinite(dt)) return 0;
    for (int i = 0; i < N; i++) {
        if (!(rho_d[i] >= 0.0) || !isfinite(rho_d[i])) return 0;
        if (!(t_s[i] > 0.0)) return 0;            /* also rejects NaN */
    }
    return 1;
}

/* A = dt * Omega_v, n = N + 1, row-major. */
void orc_assemble(int N, double rho_g, const double *rho_d, const double *t_s, double dt, int structured, double *A)
{
    const int n = N + 1;
    memset(A, 0, sizeof(double) * (size_t)n * n);
    double sum_ea = 0.0;
    for (int i = 1; i <= N; i++) {
        double eps = rho_d[i - 1] / rho_g;        /* Eq. DragEqVar2 */
        double alpha = 1.0 / t_s[i - 1];          /* Eq. DragEqVar3 */
        A[0 * n + i] = (eps * alpha) * dt;
        A[i * n + 0] = alpha * dt;
        A[i * n + i] = -(alpha * dt);
        sum_ea += eps * alpha;
    }
    if (structured) {
        double s = 0.0;
        for (int i = 1; i <= N; i++) s += A[0 * n + i];
        A[0] = -s;
    } else {
        A[0] = -sum_ea * dt;
    }
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */

/* Forward drag update for ncells cells, same SoA layout as the CUDA library:
 *   rho_g[c], rho_d[i*C + c], t_s[i*C + c]  (i = 0..N-1),
 *   v[(d*n + f)*C + c]  (d = x,y,z; f = 0 gas, f = i dust species i).
 * Invalid cells get NaN outputs and set bit 0 of *status.
 * k_out / s_out (optional) receive k* and s* per cell. */
int orc_drag_apply_u(int64_t C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt,
                     const double *v_in, double *v_out, int structured, double u, int8_t *k_out, int16_t *s_out,
                     uint32_t *status)
{
    if (C < 0 || N < 1 || N + 1 > ORC_NMAX) return -1;
    const int n = N + 1;
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *P = (double *)malloc(sizeof(double) * (size_t)n * n);
    double rd[ORC_NMAX], ts[ORC_NMAX], vin[ORC_NMAX];
    uint32_t st = 0;
    for (int64_t c = 0; c < C; c++) {
        for (int i = 0; i < N; i++) {
            rd[i] = rho_d[(int64_t)i * C + c];
            ts[i] = t_s[(int64_t)i * C + c];
        }
        int k = 0, m = 0, s = 0;
        int ok = orc_cell_valid(N, rho_g[c], rd, ts, dt);
        if (ok) {
            orc_assemble(N, rho_g[c], rd, ts, dt, structured, A);
            ok = orc_expm_u(n, A, P, structured, u, 0, &k, &m, &s, NULL) == 0;
        }
        if (k_out) k_out[c] = (int8_t)k;
        if (s_out) s_out[c] = (int16_t)s;
        for (int d = 0; d < 3; d++) {
            for (int f = 0; f < n; f++) vin[f] = v_in[((int64_t)d * n + f) * C + c];
            for (int i = 0; i < n; i++) {
                double acc = 0.0;
                for (int j = 0; j < n; j++) acc += P[i * n + j] * vin[j];
                v_out[((int64_t)d * n + i) * C + c] = ok ? acc : NAN;
            }
        }
        if (!ok) st |= 1u;
    }
    free(A); free(P);
    if (status) *status |= st;
    return 0;
}

/* Forward drag update with the options of the CUDA library: unit round-off
 * u of the theta tables, method 0 = Taylor (Algorithm 2; bound_test != 0
 * adds the second modification), 1 = Pade. k_out: k* (Taylor) or the Pade
 * degree; m_out: the polynomial degree actually evaluated; s_out: s*. */
int orc_drag_apply_opts(int64_t C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt,
                        const double *v_in, double *v_out, int structured, double u, int method, int bound_test,
                        int8_t *k_out, int8_t *m_out, int16_t *s_out, double *ratio_out, uint32_t *status)
{
    if (C < 0 || N < 1 || N + 1 > ORC_NMAX || method < 0 || method > 1) return -1;
    const int n = N + 1;
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *P = (double *)malloc(sizeof(double) * (size_t)n * n);
    double rd[ORC_NMAX], ts[ORC_NMAX], vin[ORC_NMAX];
    uint32_t st = 0;
    for (int64_t c = 0; c < C; c++) {
        for (int i = 0; i < N; i++) {
            rd[i] = rho_d[(int64_t)i * C + c];
            ts[i] = t_s[(int64_t)i * C + c];
        }
        int k = 0, m = 0, s = 0;
        double ratio = 0.0;
        int ok = orc_cell_valid(N, rho_g[c], rd, ts, dt);
        if (ok) {
            orc_assemble(N, rho_g[c], rd, ts, dt, structured, A);
            if (method == 0) {
                ok = orc_expm_u(n, A, P, structured, u, bound_test, &k, &m, &s, &ratio) == 0;
            } else {
                ok = orc_expm_pade(n, A, P, structured, u, &m, &s) == 0;
                k = m;
            }
        }
        if (k_out) k_out[c] = (int8_t)k;
        if (m_out) m_out[c] = (int8_t)m;
        if (s_out) s_out[c] = (int16_t)s;
        if (ratio_out) ratio_out[c] = ratio;
        for (int d = 0; d < 3; d++) {
            for (int f = 0; f < n; f++) vin[f] = v_in[((int64_t)d * n + f) * C + c];
            for (int i = 0; i < n; i++) {
                double acc = 0.0;
                for (int j = 0; j < n; j++) acc += P[i * n + j] * vin[j];
                v_out[((int64_t)d * n + i) * C + c] = ok ? acc : NAN;
            }
        }
        if (!ok) st |= 1u;
    }
    free(A); free(P);
    if (status) *status |= st;
    return 0;
}

int orc_drag_apply(int64_t C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt,
                   const double *v_in, double *v_out, int structured, int8_t *k_out, int16_t *s_out,
                   uint32_t *status)
{
    return orc_drag_apply_u(C, N, rho_g, rho_d, t_s, dt, v_in, v_out, structured, ldexp(1.0, -53), k_out, s_out,
                            status);
}

/* ------------------------------------------------------------------------ */
/* Adjoint: the Frechet derivative of the exponential                       */
/* ------------------------------------------------------------------------ */

/* Column-sum restoration of an n x n block stored inside a (ld x ld)
 * row-major matrix at (r0, r0): B_jj = 1 - sum_{i != j} B_ij. Used for the
 * diagonal blocks exp(A^T), whose columns sum to one. */
static void orc_restore_cols_block(int ld, int r0, int n, double *M)
{
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int i = 0; i < n; i++)
            if (i != j) s += M[(size_t)(r0 + i) * ld + r0 + j];
        M[(size_t)(r0 + j) * ld + r0 + j] = 1.0 - s;
    }
}

/* Z = L(A^T, G): the Frechet derivative of exp at A^T in direction G, read
 * off the top-right block of exp([[A^T, tau G], [0, A^T]]) (block-triangular
 * identity of the exponential), divided by tau. tau = 2^-e scales G so that
 * |tau G|_1 <= |A|_1 (exact). exp of the 2n x 2n matrix uses the same Taylor
 * scaling and squaring as the forward (Algorithm 2 on its 1-norm,
 * Paterson-Stockmeyer, squarings). For drag matrices (structured != 0) the
 * column sums of both diagonal blocks, exp(A^T), are restored to one after
 * the Taylor step and after every squaring, as in the forward. */
static int orc_frechet_T(int n, const double *A, const double *G, double *Z, int structured)
{
    const int n2 = 2 * n;
    double *M = (double *)calloc((size_t)n2 * n2, sizeof(double));
    double *E = (double *)calloc((size_t)n2 * n2, sizeof(double));
    double nA = orc_norm1(n, A), nG = orc_norm1(n, G);
    int e = 0;
    if (nA > 0.0)
        while (ldexp(nG, -e) > nA) e++;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            M[(size_t)i * n2 + j] = A[j * n + i];               /* A^T */
            M[(size_t)(n + i) * n2 + n + j] = A[j * n + i];     /* A^T */
            M[(size_t)i * n2 + n + j] = ldexp(G[i * n + j], -e);
        }
    int k, m, s;
    int rc = orc_select_alg2(orc_norm1(n2, M), ORC_K, &k, &m, &s);
    if (rc != 0) {
        for (int i = 0; i < n * n; i++) Z[i] = NAN;
        free(M); free(E);
        return -1;
    }
    /* Taylor (same Paterson-Stockmeyer evaluation as orc_expm) */
    const int q = orc_qk[k], r = orc_rk[k];
    const size_t nn = (size_t)n2 * n2;
    double *pw = (double *)calloc((size_t)(q + 1) * nn, sizeof(double));
    double *F = (double *)calloc(nn, sizeof(double));
    double *T = (double *)calloc(nn, sizeof(double));
    double *Bb = (double *)calloc(nn, sizeof(double));
    double b[64];
    b[0] = 1.0;
    for (int i = 1; i <= m; i++) b[i] = b[i - 1] / (double)i;
    for (size_t x = 0; x < nn; x++) pw[nn + x] = ldexp(M[x], -s);
    for (int j = 2; j <= q; j++) orc_matmul(n2, pw + (size_t)(j - 1) * nn, pw + nn, pw + (size_t)j * nn);
    for (int kk = r - 1; kk >= 0; kk--) {
        for (size_t x = 0; x < nn; x++) {
            double acc = 0.0;
            for (int j = 1; j <= q; j++) acc += b[q * kk + j] * pw[(size_t)j * nn + x];
            Bb[x] = acc;
        }
        if (kk == r - 1) {
            memcpy(F, Bb, nn * sizeof(double));
        } else {
            orc_matmul(n2, F, pw + (size_t)q * nn, T);
            for (size_t x = 0; x < nn; x++) F[x] = Bb[x] + T[x];
        }
    }
    memcpy(E, F, nn * sizeof(double));
    for (int i = 0; i < n2; i++) E[(size_t)i * n2 + i] += 1.0;
    if (structured) {
        orc_restore_cols_block(n2, 0, n, E);
        orc_restore_cols_block(n2, n, n, E);
    }
    for (int t = 0; t < s; t++) {
        orc_matmul(n2, E, E, T);
        memcpy(E, T, nn * sizeof(double));
        if (structured) {
            orc_restore_cols_block(n2, 0, n, E);
            orc_restore_cols_block(n2, n, n, E);
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Z[i * n + j] = ldexp(E[(size_t)i * n2 + n + j], e);
    free(pw); free(F); free(T); free(Bb); free(M); free(E);
    return 0;
}

/* Reverse-mode gradients of a loss L(v_out) through one drag step.
 * With g_d = dL/dv_out,d (d = x, y, z), P = exp(A), A = dt Omega_v:
 *   dL/dv_in,d = P^T g_d
 *   dL/dA = Z = L(A^T, G), G = sum_d g_d v_in,d^T
 * and, from A_0i = eps_i alpha_i dt, A_00 = -sum_i A_0i, A_i0 = -A_ii = alpha_i dt
 * (Eqs. DragEqVar2, DragEqVar3, jacobian):
 *   dL/deps_i   = alpha_i dt (Z_0i - Z_00)
 *   dL/dalpha_i = dt [eps_i (Z_0i - Z_00) + (Z_i0 - Z_ii)]
 *   dL/drho_d,i = dL/deps_i / rho_g,   dL/dt_s,i = -dL/dalpha_i / t_s,i^2
 *   dL/drho_g   = -sum_i eps_i dL/deps_i / rho_g.
 * Any output pointer may be NULL. Invalid cells get NaN gradients. */
int orc_drag_backward(int64_t C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt,
                      const double *v_in, const double *g_out, double *g_vin, double *g_rho_g, double *g_rho_d,
                      double *g_ts, uint32_t *status)
{
    if (C < 0 || N < 1 || N + 1 > ORC_NMAX) return -1;
    const int n = N + 1;
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *P = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *G = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * n);
    double rd[ORC_NMAX], ts[ORC_NMAX], vin[3][ORC_NMAX], gg[3][ORC_NMAX];
    uint32_t st = 0;
    for (int64_t c = 0; c < C; c++) {
        for (int i = 0; i < N; i++) {
            rd[i] = rho_d[(int64_t)i * C + c];
            ts[i] = t_s[(int64_t)i * C + c];
        }
        for (int d = 0; d < 3; d++)
            for (int f = 0; f < n; f++) {
                vin[d][f] = v_in[((int64_t)d * n + f) * C + c];
                gg[d][f] = g_out[((int64_t)d * n + f) * C + c];
            }
        int ok = orc_cell_valid(N, rho_g[c], rd, ts, dt);
        int k, m, s;
        if (ok) {
            orc_assemble(N, rho_g[c], rd, ts, dt, 1, A);
            ok = orc_expm(n, A, P, 1, &k, &m, &s) == 0;
        }
        if (ok) {
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    double acc = 0.0;
                    for (int d = 0; d < 3; d++) acc += gg[d][i] * vin[d][j];
                    G[i * n + j] = acc;
                }
            /* Remove the stationary block of G before differentiating.
             * rho^T A = 0 and A 1 = 0 (detailed balance and zero row sums of
             * Eq. jacobian in velocity form), so Pi = rho 1^T / (1^T rho) is
             * the spectral projector of A^T for eigenvalue 0 and
             * L(A^T, Pi G Pi) = Pi G Pi = kappa rho 1^T, kappa = 1^T G rho / (1^T rho)^2.
             * Its entries are constant along rows, so it adds nothing to
             * Z_0i - Z_00 or Z_i0 - Z_ii, the only combinations the gradients
             * use. Dropping it keeps the propagated derivative small in stiff
             * cells, where this block doubles at every squaring and its rounding
             * would otherwise be amplified by |A| in the chain rule. */
            double rho[ORC_NMAX], srho = 0.0, gr = 0.0;
            rho[0] = rho_g[c];
            for (int i = 1; i < n; i++) rho[i] = rd[i - 1];
            for (int i = 0; i < n; i++) srho += rho[i];
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) gr += G[i * n + j] * rho[j];
            const double kappa = gr / (srho * srho);
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) G[i * n + j] -= kappa * rho[i];
            ok = orc_frechet_T(n, A, G, Z, 1) == 0;
        }
        if (!ok) st |= 1u;
        if (g_vin)
            for (int d = 0; d < 3; d++)
                for (int i = 0; i < n; i++) {
                    double acc = 0.0;
                    for (int j = 0; j < n; j++) acc += P[j * n + i] * gg[d][j];
                    g_vin[((int64_t)d * n + i) * C + c] = ok ? acc : NAN;
                }
        double sum_eps_geps = 0.0;
        for (int i = 1; i <= N; i++) {
            double eps = ok ? rd[i - 1] / rho_g[c] : NAN;
            double alpha = ok ? 1.0 / ts[i - 1] : NAN;
            double d0 = ok ? Z[0 * n + i] - Z[0] : NAN;
            double geps = alpha * dt * d0;
            double galpha = dt * (eps * d0 + (Z[i * n + 0] - Z[i * n + i]));
            sum_eps_geps += eps * geps;
            if (g_rho_d) g_rho_d[(int64_t)(i - 1) * C + c] = ok ? geps / rho_g[c] : NAN;
            if (g_ts) g_ts[(int64_t)(i - 1) * C + c] = ok ? -galpha * (alpha * alpha) : NAN;
        }
        if (g_rho_g) g_rho_g[c] = ok ? -sum_eps_geps / rho_g[c] : NAN;
    }
    free(A); free(P); free(G); free(Z);
    if (status) *status |= st;
    return 0;
}

/* Batched forward: block b holds ncells[b] cells with nspecies[b] species and
 * time step dt[b]; its gas densities start at rho_g[cell_offset[b]], its dust
 * arrays at rho_d/t_s[dust_offset[b]] (species-major slab of N*ncells) and its
 * velocities at v[vel_offset[b]] (slab of 3*(N+1)*ncells). Each block is an
 * independent plain update (the drag step is cell local). */
int orc_drag_apply_batched(int64_t nblocks, const int64_t *cell_offset, const int64_t *dust_offset,
                           const int64_t *vel_offset, const int32_t *ncells, const int32_t *nspecies, const double *dt,
                           const double *rho_g, const double *rho_d, const double *t_s, const double *v_in,
                           double *v_out, uint32_t *status)
{
    for (int64_t b = 0; b < nblocks; b++) {
        int rc = orc_drag_apply(ncells[b], nspecies[b], rho_g + cell_offset[b], rho_d + dust_offset[b],
                                t_s + dust_offset[b], dt[b], v_in + vel_offset[b], v_out + vel_offset[b], 1, NULL,
                                NULL, status);
        if (rc != 0) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Frictional heating (energy epilogue)                                      */
/* ------------------------------------------------------------------------ */

/* Kinetic energy the drag step dissipates, per cell:
 *   heat = sum_f 1/2 rho_f (|v_in,f - V|^2 - |v_out,f - V|^2),
 *   V = sum_f rho_f v_in,f / sum_f rho_f  (centre-of-mass velocity, Eq. V_cm).
 * The drag terms of Eqs. GenEq_2/GenEq_5 change the mixture's kinetic energy at
 * the rate -sum_i rho_d,i |v_d,i - v_g|^2 / T_s,i, which Eq. GenEq_3 returns
 * to the gas as heat with weight w; over an exact step the integral is the
 * kinetic-energy drop, and since momentum is conserved it can be measured
 * about V (removing the common motion). The gas energy then changes by
 * 1/2 rho_g (|v_g,out|^2 - |v_g,in|^2) + w heat. */
int orc_drag_heat(int64_t C, int N, const double *rho_g, const double *rho_d, const double *v_in,
                  const double *v_out, double *heat)
{
    if (C < 0 || N < 1 || N + 1 > ORC_NMAX) return -1;
    const int n = N + 1;
    for (int64_t c = 0; c < C; c++) {
        double rho[ORC_NMAX], mass = 0.0;
        rho[0] = rho_g[c];
        for (int i = 1; i < n; i++) rho[i] = rho_d[(int64_t)(i - 1) * C + c];
        for (int f = 0; f < n; f++) mass += rho[f];
        double h = 0.0;
        for (int d = 0; d < 3; d++) {
            double mom = 0.0;
            for (int f = 0; f < n; f++) mom += rho[f] * v_in[((int64_t)d * n + f) * C + c];
            const double V = mom / mass;
            for (int f = 0; f < n; f++) {
                const double a = v_in[((int64_t)d * n + f) * C + c] - V;
                const double b = v_out[((int64_t)d * n + f) * C + c] - V;
                h += 0.5 * rho[f] * (a * a - b * b);
            }
        }
        heat[c] = h;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Implicit RK1 with the analytic solution (App. A.2, Eqs. analytic_1-4)     */
/* ------------------------------------------------------------------------ */

/* One backward-Euler drag step: (I - dt Omega) q = b with b the momenta
 * U^n = [rho_g v_g, rho_d,i v_d,i] (drag-only splitting, U^(n+1/2) = U^n in
 * Eq. eq_rk1_2), solved as in the paper:
 *   q_0 = (b_0 + dt B) / A,  A = 1 + sum_i (1 - 1/(1 + alpha_i dt)) eps_i,
 *                            B = sum_i alpha_i b_i / (1 + alpha_i dt)      (Eq. analytic_4)
 *   q_i = (b_i + eps_i alpha_i dt q_0) / (1 + alpha_i dt)                 (Eq. analytic_3)
 * then v = q / rho. For a species with rho_d,i = 0 the momentum q_i carries no
 * velocity; its velocity follows from row i of the same system in velocity
 * form, v_i' = (v_i + alpha_i dt v_g') / (1 + alpha_i dt). */
int orc_rk1_apply(int64_t C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt,
                  const double *v_in, double *v_out, uint32_t *status)
{
    if (C < 0 || N < 1 || N + 1 > ORC_NMAX) return -1;
    const int n = N + 1;
    double rd[ORC_NMAX], ts[ORC_NMAX], eps[ORC_NMAX], alpha[ORC_NMAX];
    uint32_t st = 0;
    for (int64_t c = 0; c < C; c++) {
        for (int i = 0; i < N; i++) {
            rd[i] = rho_d[(int64_t)i * C + c];
            ts[i] = t_s[(int64_t)i * C + c];
        }
        const int ok = orc_cell_valid(N, rho_g[c], rd, ts, dt);
        for (int i = 0; i < N; i++) {
            eps[i] = rd[i] / rho_g[c];
            alpha[i] = 1.0 / ts[i];
        }
        for (int d = 0; d < 3; d++) {
            double b[ORC_NMAX], q[ORC_NMAX];
            b[0] = rho_g[c] * v_in[((int64_t)d * n + 0) * C + c];
            for (int i = 1; i < n; i++) b[i] = rd[i - 1] * v_in[((int64_t)d * n + i) * C + c];
            double Acoef = 1.0, Bcoef = 0.0;
            for (int i = 1; i < n; i++) {
                const double den = 1.0 + alpha[i - 1] * dt;
                Acoef += (1.0 - 1.0 / den) * eps[i - 1];
                Bcoef += (alpha[i - 1] / den) * b[i];
            }
            q[0] = (b[0] + dt * Bcoef) / Acoef;
            const double vg = q[0] / rho_g[c];
            v_out[((int64_t)d * n + 0) * C + c] = ok ? vg : NAN;
            for (int i = 1; i < n; i++) {
                const double den = 1.0 + alpha[i - 1] * dt;
                double vi;
                if (rd[i - 1] > 0.0) {
                    q[i] = (b[i] + eps[i - 1] * alpha[i - 1] * dt * q[0]) / den;
                    vi = q[i] / rd[i - 1];
                } else {
                    vi = (v_in[((int64_t)d * n + i) * C + c] + alpha[i - 1] * dt * vg) / den;
                }
                v_out[((int64_t)d * n + i) * C + c] = ok ? vi : NAN;
            }
        }
        if (!ok) st |= 1u;
    }
    if (status) *status |= st;
    return 0;
}

/* Z = L(A^T, G) for one dense n x n pair (tests of the Frechet machinery).
 * structured != 0 only for A with zero row sums (column sums of exp(A^T) = 1). */
int orc_frechet_dense(int n, const double *A, const double *G, double *Z, int structured)
{
    if (n < 1 || n > ORC_NMAX) return -2;
    return orc_frechet_T(n, A, G, Z, structured);
}

/* exp(A) of one dense n x n matrix, for tests of the S&S machinery alone. */
int orc_expm_dense(int n, const double *A, double *P, int structured, int *k, int *m, int *s)
{
    if (n < 1 || n > 2 * ORC_NMAX) return -2;
    return orc_expm(n, A, P, structured, k, m, s);
}

int orc_table_mk(int k) { return (k >= 1 && k <= ORC_K) ? orc_mk[k] : -1; }
int orc_table_qk(int k) { return (k >= 1 && k <= ORC_K) ? orc_qk[k] : -1; }
int orc_table_rk(int k) { return (k >= 1 && k <= ORC_K) ? orc_rk[k] : -1; }
