// Forward variants of the drag update, warp per cell, selected through
// drag_expm_apply_opts:
//
//  * Taylor with the paper's second modification (App. B, Eqs. Pat_Stk4 to
//    Pat_Stk7, Algorithms 8 and 9): after Algorithm 2, the Paterson-Stockmeyer
//    blocks Bbar_l = sum_{j=1}^{q} b_{ql+j} X^j of T_m(X) are bounded, and the
//    highest ones are dropped while
//        b_exp |Bbar_{keep-1}| |X^q|^{keep-1} <= u,
//        b_exp = |b_0 I + Bhat_0| + sum_{l>=1} |Bhat_l| |X^q|^l  (|T_m(-X)| <= b_exp),
//        Bhat_l = sum_{j=1}^{q} (-1)^{ql+j} b_{ql+j} X^j,
//    so Horner runs q fewer terms per dropped block. The norms are 1-norms of
//    the velocity-form matrices, formed from the symmetric form as
//    |P_A|_1 = max_j sigma_j sum_i |P_S,ij| / sigma_i.
//  * Pade (Eq. PadeEqu): R_mm(X) = D_mm(X)^-1 N_mm(X), D_mm(X) = N_mm(-X), with
//    the degree m in {3, 5, 7, 9, 13} and the scaling chosen from theta_m
//    (Eqs. B5-B8 applied to R_mm). N and D are Horner chains in the arrowhead
//    X; D is symmetric positive definite here (X has a non-positive spectrum
//    and N has positive coefficients), so R comes from an LDL^T factorisation
//    without pivoting and two triangular solves.
//
// Both then take the row-sum restoration, the squaring chain and the apply of
// the plain forward (dx_wpc.cuh). For n = 2..6 under a lane-per-cell mode
// (the default there) both variants run one cell per lane instead
// (dx_forward_lpc_var): their matrices fit in registers, and a warp-per-cell
// round at these sizes keeps few lanes busy.
#include <cmath>

#include "dx_modes.h"
#include "dx_wpc.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kCellsPerBlock = 16;
constexpr int kVarMats = 5;       // n x n matrices per warp

__host__ __device__ __forceinline__ int var_warp_doubles(int n) { return kVarMats * n * dx_stride(n) + 19 * n; }

size_t var_smem_bytes(int n) {
    return sizeof(double) * (size_t)kWarpsPerBlock * var_warp_doubles(n) + 2 * kPairSlots * sizeof(unsigned short);
}

struct VarArgs {
    long long C;
    int N;
    const double *rho_g, *rho_d, *t_s, *v_in;
    double *v_out;
    double dt;
    uint32_t *status;
    int8_t *m_out;      // degree evaluated per cell (optional)
    int16_t *s_out;     // squarings per cell (optional)
    int method;         // 0 Taylor, 1 Pade
    int bound_test;     // Taylor only
};

// F = a X + c I (X the arrowhead), written into a zeroed n x n buffer.
__device__ __forceinline__ void var_init_lin(int lane, int n, int ns, const DxVecs &V, double a, double c, double *F) {
    for (int t = lane; t < n * ns; t += 32) F[t] = 0.0;
    __syncwarp();
    if (lane < n) {
        if (lane == 0) {
            F[0] = fma(a, V.xs[0], c);
        } else {
            F[lane] = F[lane * ns] = a * V.xs[lane];
            F[lane * ns + lane] = fma(a, V.ds[lane], c);
        }
    }
    __syncwarp();
}

// 1-norm of the velocity-form matrix D_sigma^-1 P D_sigma for a symmetric-form P:
// max_j sigma_j sum_i |P_ij| tau_i (non-negative, so the lane maximum is an
// integer maximum of bit patterns).
__device__ __forceinline__ double var_norm1(int lane, int n, int ns, const DxVecs &V, const double *P) {
    double col = 0.0;
    if (lane < n) {
        for (int i = 0; i < n; i++) col = fma(fabs(P[i * ns + lane]), V.tau[i], col);
        col *= V.sig[lane];
    }
    return __longlong_as_double(dx_warp_max_ll(dx_bits(col)));
}

// B = c0 I + sum_{j=1}^{q} cj[j] X^j with X^1 the arrowhead and X^j (j >= 2) in
// pw[j - 2]; upper triangle computed, mirrored.
__device__ __forceinline__ void var_block(int lane, int n, int ns, int n_hp, const unsigned short *hp, const DxVecs &V,
                                          double *const *pw, int q, const double *cj, double c0, double *B) {
    for (int t = lane; t <= n_hp; t += 32) {
        int i = 0, k = 0;
        if (t < n_hp) {
            const int p = hp[t];
            i = p >> 8;
            k = p & 255;
        }
        const double x1 = i == 0 ? V.xs[k] : (i == k ? V.ds[i] : 0.0);
        double acc = fma(cj[1], x1, i == k ? c0 : 0.0);
        for (int j = 2; j <= q; j++) acc = fma(cj[j], pw[j - 2][i * ns + k], acc);
        B[i * ns + k] = acc;
        B[k * ns + i] = acc;
    }
    __syncwarp();
}

// The second modification: number of Paterson-Stockmeyer blocks to keep (>= 1).
__device__ __forceinline__ int var_bound_test(int lane, int n, int ns, int n_hp, const unsigned short *hp,
                                              const DxVecs &V, const DxConsts &K, int q, int r, double u,
                                              double *const *M) {
    // powers X^2..X^q in M[0..q-2] (X^2 from a dense copy of X in M[4])
    double *pw[4] = {M[0], M[1], M[2], M[3]};
    if (q >= 2) {
        var_init_lin(lane, n, ns, V, 1.0, 0.0, M[4]);
        dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, 0.0, M[4], pw[0]);
        __syncwarp();
        for (int j = 3; j <= q; j++) {
            dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, 0.0, pw[j - 3], pw[j - 2]);
            __syncwarp();
        }
    }
    double *Bm = M[4];
    // |X^q|
    double xq;
    if (q == 1) {
        const double one[2] = {0.0, 1.0};
        var_block(lane, n, ns, n_hp, hp, V, pw, 1, one, 0.0, Bm);
        xq = var_norm1(lane, n, ns, V, Bm);
    } else {
        xq = var_norm1(lane, n, ns, V, pw[q - 2]);
    }
    __syncwarp();
    double cj[6];
    double bexp = 0.0, xql = 1.0;
    for (int l = 0; l < r; l++) {
        for (int j = 1; j <= q; j++) cj[j] = ((q * l + j) & 1) ? -K.b[q * l + j] : K.b[q * l + j];
        var_block(lane, n, ns, n_hp, hp, V, pw, q, cj, l == 0 ? K.b[0] : 0.0, Bm);
        bexp = fma(var_norm1(lane, n, ns, V, Bm), xql, bexp);
        __syncwarp();
        xql *= xq;
    }
    int keep = r;
    while (keep > 1) {
        const int l = keep - 1;
        for (int j = 1; j <= q; j++) cj[j] = K.b[q * l + j];
        var_block(lane, n, ns, n_hp, hp, V, pw, q, cj, 0.0, Bm);
        double val = bexp * var_norm1(lane, n, ns, V, Bm);
        __syncwarp();
        for (int t = 0; t < l; t++) val *= xq;
        if (!(val <= u)) break;
        keep--;
    }
    return keep;
}

// R = D^-1 N for symmetric positive definite D (LDL^T, unit lower L stored
// below D's diagonal, d_j on it; rcp[j] = 1/d_j), N overwritten by R.
__device__ __forceinline__ void var_solve_spd(int lane, int n, int ns, double *D, double *Nm, double *rcp) {
    for (int j = 0; j < n; j++) {
        const double r = __ddiv_rn(1.0, D[j * ns + j]);
        const int m = n - 1 - j;                        // trailing size
        // trailing update D_ik -= (D_ij / d_j) D_jk, then column j of L
        for (int t = lane; t < m * m; t += 32) {
            const int i = j + 1 + t / m, k = j + 1 + t % m;
            D[i * ns + k] = fma(-D[i * ns + j] * r, D[j * ns + k], D[i * ns + k]);
        }
        __syncwarp();
        for (int i = j + 1 + lane; i < n; i += 32) D[i * ns + j] *= r;
        if (lane == 0) rcp[j] = r;
        __syncwarp();
    }
    // forward substitution L Y = N (column-oriented, all right-hand sides at once)
    for (int k = 0; k < n - 1; k++) {
        const int rows = n - 1 - k;
        for (int t = lane; t < rows * n; t += 32) {
            const int i = k + 1 + t / n, c = t % n;
            Nm[i * ns + c] = fma(-D[i * ns + k], Nm[k * ns + c], Nm[i * ns + c]);
        }
        __syncwarp();
    }
    // Z = Delta^-1 Y, then back substitution L^T R = Z
    for (int t = lane; t < n * n; t += 32) {
        const int i = t / n, c = t % n;
        Nm[i * ns + c] *= rcp[i];
    }
    __syncwarp();
    for (int k = n - 1; k > 0; k--) {
        for (int t = lane; t < k * n; t += 32) {
            const int i = t / n, c = t % n;
            Nm[i * ns + c] = fma(-D[k * ns + i], Nm[k * ns + c], Nm[i * ns + c]);
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
dx_forward_wpc_var(VarArgs a, DxConsts K, DxPade P) {
    extern __shared__ double smem[];
    const int N = a.N, n = N + 1, ns = dx_stride(n);
    const int n_hp = n * (n + 1) / 2 - 1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wd = var_warp_doubles(n);
    unsigned short *od = reinterpret_cast<unsigned short *>(smem + kWarpsPerBlock * wd);
    unsigned short *hp = od + kPairSlots;
    dx_build_pairs(n, od, hp);
    __syncthreads();
    double *wsm = smem + wib * wd;
    double *M[kVarMats];
    for (int i = 0; i < kVarMats; i++) M[i] = wsm + i * n * ns;
    DxVecs V;
    DxFwdBufs B;
    dx_wpc_fwd_layout(wsm + kVarMats * n * ns, n, V, B);

    __shared__ int next;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kCellsPerBlock;
    for (int it = 0; it < kCellsPerBlock; it++) {
        int kc = 0;
        if (lane == 0) kc = atomicAdd(&next, 1);
        kc = __shfl_sync(DX_FULL, kc, 0);
        const long long c = base + kc;
        if (kc >= kCellsPerBlock || c >= a.C) break;
        double *vop = a.v_out + c;
        DxCellIn ci;
        dx_wpc_load_cell(lane, N, a.rho_g + c, a.rho_d + c, a.t_s + c, a.v_in + c, a.C, ci);
        DxLane L;
        if (!dx_wpc_setup(lane, N, ci.rg, ci.rd, ci.ts, a.dt, K, V, L, a.method == 1 ? &P : nullptr)) {
            dx_wpc_fail_cell(lane, n, vop, a.C, a.status, nullptr);
            if (lane == 0 && a.m_out) a.m_out[c] = 0;
            if (lane == 0 && a.s_out) a.s_out[c] = -1;
            continue;
        }
        double *F;
        int deg;
        if (a.method == 0) {
            int m = K.mk[L.k];
            if (a.bound_test)
                m = K.qk[L.k] * var_bound_test(lane, n, ns, n_hp, hp, V, K, K.qk[L.k], K.rk[L.k], K.u, M);
            deg = m;
            double *G = M[1];
            F = M[0];
            var_init_lin(lane, n, ns, V, K.b[m], K.b[m - 1], F);
            for (int j = m - 2; j >= 0; j--) {
                dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, K.b[j], F, G);
                __syncwarp();
                double *t = F; F = G; G = t;
            }
        } else {
            const int m = P.m[L.k];
            const double *cc = P.c[L.k];
            deg = m;
            // N in M[0]/M[1], D = N(-X) in M[2]/M[3]
            double *Fn = M[0], *Gn = M[1], *Fd = M[2], *Gd = M[3];
            const double sm = (m & 1) ? -1.0 : 1.0;      // (-1)^m
            var_init_lin(lane, n, ns, V, cc[m], cc[m - 1], Fn);
            var_init_lin(lane, n, ns, V, sm * cc[m], -sm * cc[m - 1], Fd);
            for (int j = m - 2; j >= 0; j--) {
                dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, cc[j], Fn, Gn);
                dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, (j & 1) ? -cc[j] : cc[j], Fd, Gd);
                __syncwarp();
                double *t = Fn; Fn = Gn; Gn = t;
                t = Fd; Fd = Gd; Gd = t;
            }
            var_solve_spd(lane, n, ns, Fd, Fn, B.wv0);
            F = Fn;
        }
        // restoration, s - q squarings on (F, a free buffer), then the applications
        double *other = (F == M[0]) ? M[1] : M[0];
        const int q = L.s < DX_APPLY_Q ? L.s : DX_APPLY_Q;
        F = dx_wpc_square_chain(lane, n, ns, L.s - q, F, other, 0, V) ? other : F;
        dx_wpc_apply_tail(lane, n, ns, V, B, F, q, ci, L.sg, vop, a.C, nullptr);
        if (lane == 0 && a.m_out) a.m_out[c] = (int8_t)deg;
        if (lane == 0 && a.s_out) a.s_out[c] = (int16_t)L.s;
    }
}

// ---- Both variants, lane per cell (n = 2..6): the same steps as the
// warp-per-cell kernel, each on one lane's packed symmetric matrices in
// registers. The 1-norm and the selection are the plain forward's
// (dx_lpc_norm_cell), so (k*, s*) and the Pade (m, s) match the warp-per-cell
// kernel's and the oracle's bit for bit.
constexpr int kVarLpcThreads = 128;
constexpr int kVarLpcTile = 512;   // cells a block orders by the cost proxy and runs

// R = D^-1 N for packed symmetric D (positive definite) and N: LDL^T of D in
// place (L_ij, i > j, in the slot of (i, j); d_j on the diagonal), then the
// two triangular solves for all n columns of N at once. R is symmetric (D and
// N are polynomials in X); its upper triangle is taken from the solves.
template <int NF, class MA>
__device__ __forceinline__ void pade_lpc_solve(MA &D, MA &Nm) {
    using Pk = DxPacked<NF>;
    double rcp[NF];
#pragma unroll
    for (int j = 0; j < NF; j++) {
        const double r = __ddiv_rn(1.0, D[Pk::at(j, j)]);
        rcp[j] = r;
#pragma unroll
        for (int i = j + 1; i < NF; i++) {
            const double lij = -D[Pk::at(i, j)] * r;
#pragma unroll
            for (int k = i; k < NF; k++) D[Pk::at(i, k)] = fma(lij, D[Pk::at(j, k)], D[Pk::at(i, k)]);
        }
#pragma unroll
        for (int i = j + 1; i < NF; i++) D[Pk::at(i, j)] *= r;
    }
    double R[NF][NF];
#pragma unroll
    for (int i = 0; i < NF; i++) {
#pragma unroll
        for (int c = 0; c < NF; c++) R[i][c] = Nm[Pk::at(i, c)];
    }
    // L Y = N, then Z = Delta^-1 Y, then L^T R = Z
#pragma unroll
    for (int k = 0; k < NF - 1; k++) {
#pragma unroll
        for (int i = k + 1; i < NF; i++) {
#pragma unroll
            for (int c = 0; c < NF; c++) R[i][c] = fma(-D[Pk::at(i, k)], R[k][c], R[i][c]);
        }
    }
#pragma unroll
    for (int i = 0; i < NF; i++) {
#pragma unroll
        for (int c = 0; c < NF; c++) R[i][c] *= rcp[i];
    }
#pragma unroll
    for (int k = NF - 1; k > 0; k--) {
#pragma unroll
        for (int i = 0; i < k; i++) {
#pragma unroll
            for (int c = 0; c < NF; c++) R[i][c] = fma(-D[Pk::at(k, i)], R[k][c], R[i][c]);
        }
    }
#pragma unroll
    for (int i = 0; i < NF; i++) {
#pragma unroll
        for (int c = i; c < NF; c++) Nm[Pk::at(i, c)] = R[i][c];
    }
}

template <int NF>
__device__ __forceinline__ void pade_lpc_cell(long long c, const VarArgs &a, const DxPade &P) {
    constexpr int N = NF - 1;
    constexpr int NT = DxPacked<NF>::NT;
    using Pk = DxPacked<NF>;
    const long long C = a.C;
    const double dt = a.dt;
    double *vop = a.v_out + c;
    double rg, eps[N], alpha[N], s1;
    unsigned long long fph;
    long long nb;
    if (!dx_lpc_norm_cell<NF>(a.rho_g + c, a.rho_d + c, a.t_s + c, C, dt, false, rg, eps, alpha, fph, s1, nb)) {
        dx_lpc_fail_cell<NF>(vop, C, nullptr, a.status);
        if (a.m_out) a.m_out[c] = 0;
        if (a.s_out) a.s_out[c] = -1;
        return;
    }
    int idx, s;
    dx_select_pade(__longlong_as_double(nb), P, idx, s);
    DxLaneArr<NF, false> sig, tau, xs, ds;
    dx_lpc_arrowhead<NF>(eps, alpha, dt, s, s1, sig, tau, xs, ds, DX_EPS_FLOOR);
    // N(X) and D(X) = N(-X) by Horner in the arrowhead X (coefficients c_j and (-1)^j c_j)
    const int m = P.m[idx];
    const double *cc = P.c[idx];
    const double sm = (m & 1) ? -1.0 : 1.0;
    DxLaneArr<NT, false> Fn, Gn, Fd, Gd;
    dx_lpc_taylor_init<NF>(Fn, xs, ds, cc[m], cc[m - 1]);
    dx_lpc_taylor_init<NF>(Fd, xs, ds, sm * cc[m], -sm * cc[m - 1]);
    for (int j = m - 2; j >= 0; j--) {
        dx_lpc_horner_step<NF>(Fn, Gn, xs, ds, cc[j]);
        dx_lpc_horner_step<NF>(Fd, Gd, xs, ds, (j & 1) ? -cc[j] : cc[j]);
        dx_lane_take(Fn, Gn);
        dx_lane_take(Fd, Gd);
    }
    pade_lpc_solve<NF>(Fd, Fn);
    // restoration, s squarings each restored, then the apply of the plain forward
    dx_lpc_restore<NF>(Fn, sig, tau);
    for (int it = 0; it < s; it++) {
        dx_lpc_square_offdiag<NF>(Fn, Gn);
        dx_lpc_restore<NF>(Gn, sig, tau);
        dx_lane_take(Fn, Gn);
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double v[NF], y[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) {
            v[f] = a.v_in[(d * NF + f) * C + c];
            y[f] = sig[f] * v[f];
        }
#pragma unroll
        for (int i = 0; i < NF; i++) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NF; k++)
                if (k != i) acc = fma(Fn[Pk::at(i, k)], y[k], acc);
            vop[(d * NF + i) * C] = fma(tau[i], acc, Fn[Pk::at(i, i)] * v[i]);
        }
    }
    if (a.m_out) a.m_out[c] = (int8_t)m;
    if (a.s_out) a.s_out[c] = (int16_t)s;
}

// Velocity-form 1-norm of a packed symmetric-form matrix, max_j sigma_j sum_i
// |M_ij| tau_i (the lane-per-cell counterpart of var_norm1: the same sums in
// the same order, the maximum taken on bit patterns).
template <int NF, class MA, class VA>
__device__ __forceinline__ double bound_lpc_norm1(MA &M, VA &sig, VA &tau) {
    using Pk = DxPacked<NF>;
    long long best = 0;
#pragma unroll
    for (int j = 0; j < NF; j++) {
        double col = 0.0;
#pragma unroll
        for (int i = 0; i < NF; i++) col = fma(fabs(M[Pk::at(i, j)]), tau[i], col);
        col *= sig[j];
        const long long b = dx_bits(col);
        best = b > best ? b : best;
    }
    return __longlong_as_double(best);
}

// B = c[0] I + sum_{j=1}^{q} c[j] X^j by Horner in the arrowhead X (the
// warp-per-cell variant forms the powers first; the sums differ in rounding
// only).
template <int NF, class MA, class VA>
__device__ __forceinline__ void bound_lpc_block(MA &F, MA &G, VA &xs, VA &ds, int q, const double *c) {
    dx_lpc_taylor_init<NF>(F, xs, ds, c[q], c[q - 1]);
    for (int j = q - 2; j >= 0; j--) {
        dx_lpc_horner_step<NF>(F, G, xs, ds, c[j]);
        dx_lane_take(F, G);
    }
}

// The second modification (Algorithms 8 and 9) on one lane: blocks of the
// Taylor sum to keep (>= 1), as var_bound_test decides it.
template <int NF, class MA, class VA>
__device__ __forceinline__ int bound_lpc_keep(MA &F, MA &G, VA &sig, VA &tau, VA &xs, VA &ds, const double *bsh,
                                              double u, int q, int r) {
    double c[6];
    // |X^q|
#pragma unroll
    for (int j = 0; j < 6; j++) c[j] = 0.0;
    c[q] = 1.0;
    bound_lpc_block<NF>(F, G, xs, ds, q, c);
    const double xq = bound_lpc_norm1<NF>(F, sig, tau);
    double bexp = 0.0, xql = 1.0;
    for (int l = 0; l < r; l++) {
        c[0] = l == 0 ? bsh[0] : 0.0;
        for (int j = 1; j <= q; j++) c[j] = ((q * l + j) & 1) ? -bsh[q * l + j] : bsh[q * l + j];
        bound_lpc_block<NF>(F, G, xs, ds, q, c);
        bexp = fma(bound_lpc_norm1<NF>(F, sig, tau), xql, bexp);
        xql *= xq;
    }
    int keep = r;
    while (keep > 1) {
        const int l = keep - 1;
        c[0] = 0.0;
        for (int j = 1; j <= q; j++) c[j] = bsh[q * l + j];
        bound_lpc_block<NF>(F, G, xs, ds, q, c);
        double val = bexp * bound_lpc_norm1<NF>(F, sig, tau);
        for (int t = 0; t < l; t++) val *= xq;
        if (!(val <= u)) break;
        keep--;
    }
    return keep;
}

template <int NF>
__device__ __forceinline__ void bound_lpc_cell(long long c, const VarArgs &a, const DxConsts &K, const double *bsh) {
    constexpr int N = NF - 1;
    constexpr int NT = DxPacked<NF>::NT;
    using Pk = DxPacked<NF>;
    const long long C = a.C;
    const double dt = a.dt;
    double *vop = a.v_out + c;
    DxLaneArr<NF, false> sig, tau, xs, ds;
    double rg, eps[N], alpha[N];
    int kk, s;
    unsigned long long fph;
    if (!dx_lpc_setup<NF>(a.rho_g + c, a.rho_d + c, a.t_s + c, C, dt, K, false, rg, eps, alpha, kk, s, fph, sig, tau,
                          xs, ds)) {
        dx_lpc_fail_cell<NF>(vop, C, nullptr, a.status);
        if (a.m_out) a.m_out[c] = 0;
        if (a.s_out) a.s_out[c] = -1;
        return;
    }
    DxLaneArr<NT, false> Fm, Gm;
    // Taylor of degree m_{k*}, or q_{k*} times the blocks the bound test keeps
    const int q = K.qk[kk];
    const int m = a.bound_test ? q * bound_lpc_keep<NF>(Fm, Gm, sig, tau, xs, ds, bsh, K.u, q, K.rk[kk]) : K.mk[kk];
    dx_lpc_chain<NF>(Fm, Gm, sig, tau, xs, ds, m, s, bsh, nullptr, 0, 0);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double v[NF], y[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) {
            v[f] = a.v_in[(d * NF + f) * C + c];
            y[f] = sig[f] * v[f];
        }
#pragma unroll
        for (int i = 0; i < NF; i++) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NF; k++)
                if (k != i) acc = fma(Fm[Pk::at(i, k)], y[k], acc);
            vop[(d * NF + i) * C] = fma(tau[i], acc, Fm[Pk::at(i, i)] * v[i]);
        }
    }
    if (a.m_out) a.m_out[c] = (int8_t)m;
    if (a.s_out) a.s_out[c] = (int16_t)s;
}

// n = 2 (one dust species) in the velocity form of the plain forward
// (dx_lpc2_forward_cell): every polynomial in X is c_0 I + beta X, since
// X^2 = tr(X) X with tr(X) = -(x + y). Pade: N(X) = c_0 I + b_N X and
// D(X) = N(-X) = c_0 I + b_D X give R = D^-1 N = I + (b_N - b_D) / (c_0 + b_D tr) X
// (c_0 + b_D tr = N(-tr) >= c_0 > 0). Bound test: a block c_0 I + beta X has the
// velocity-form 1-norm max(|c_0 - beta x| + |beta y|, |beta x| + |c_0 - beta y|),
// and |X^q| = |tr|^(q-1) (x + y).
__device__ __forceinline__ double var2_block_norm(double c0, const double *c, int q, double tr, double x, double y) {
    double beta = c[q];
    for (int j = q - 1; j >= 1; j--) beta = fma(tr, beta, c[j]);
    const double bx = beta * x, by = beta * y;
    const double n0 = fabs(c0 - bx) + fabs(by), n1 = fabs(bx) + fabs(c0 - by);
    const long long b0 = dx_bits(n0), b1 = dx_bits(n1);
    return __longlong_as_double(b0 > b1 ? b0 : b1);
}

__device__ __forceinline__ int var2_bound_keep(double tr, double x, double y, const double *bsh, double u, int q,
                                               int r) {
    double xq = x + y;
    for (int j = 1; j < q; j++) xq *= -tr;
    double c[6];
    double bexp = 0.0, xql = 1.0;
    for (int l = 0; l < r; l++) {
        for (int j = 1; j <= q; j++) c[j] = ((q * l + j) & 1) ? -bsh[q * l + j] : bsh[q * l + j];
        bexp = fma(var2_block_norm(l == 0 ? bsh[0] : 0.0, c, q, tr, x, y), xql, bexp);
        xql *= xq;
    }
    int keep = r;
    while (keep > 1) {
        const int l = keep - 1;
        for (int j = 1; j <= q; j++) c[j] = bsh[q * l + j];
        double val = bexp * var2_block_norm(0.0, c, q, tr, x, y);
        for (int t = 0; t < l; t++) val *= xq;
        if (!(val <= u)) break;
        keep--;
    }
    return keep;
}

__device__ __forceinline__ void var2_lpc_cell(long long c, const VarArgs &a, const DxConsts &K, const DxPade &P,
                                              const double *bsh) {
    const long long C = a.C;
    const double dt = a.dt;
    double *vop = a.v_out + c;
    double rg, eps[1], alpha[1], s1;
    unsigned long long fph;
    long long nb;
    if (!dx_lpc_norm_cell<2>(a.rho_g + c, a.rho_d + c, a.t_s + c, C, dt, false, rg, eps, alpha, fph, s1, nb)) {
        dx_lpc_fail_cell<2>(vop, C, nullptr, a.status);
        if (a.m_out) a.m_out[c] = 0;
        if (a.s_out) a.s_out[c] = -1;
        return;
    }
    int s, deg;
    double b;
    double x, y;
    if (a.method == DRAG_METHOD_PADE) {
        int idx;
        dx_select_pade(__longlong_as_double(nb), P, idx, s);
        x = dx_scale2(s1, s);
        y = dx_scale2(__dmul_rn(alpha[0], dt), s);
        const double tr = -(x + y);
        deg = P.m[idx];
        const double *cc = P.c[idx];
        double bn = cc[deg], bd = (deg & 1) ? -cc[deg] : cc[deg];
        for (int j = deg - 1; j >= 1; j--) {
            bn = fma(tr, bn, cc[j]);
            bd = fma(tr, bd, (j & 1) ? -cc[j] : cc[j]);
        }
        b = __ddiv_rn(bn - bd, fma(bd, tr, cc[0]));
    } else {
        int kk;
        dx_select(__longlong_as_double(nb), K, kk, s);
        x = dx_scale2(s1, s);
        y = dx_scale2(__dmul_rn(alpha[0], dt), s);
        const double tr = -(x + y);
        deg = a.bound_test ? K.qk[kk] * var2_bound_keep(tr, x, y, bsh, K.u, K.qk[kk], K.rk[kk]) : K.mk[kk];
        b = bsh[deg];
        for (int k = deg - 1; k >= 1; k--) b = fma(tr, b, bsh[k]);
    }
    // P = I + b X as the pair (p, q); squarings and the apply of the plain forward
    double p = b * x, q = b * y;
    for (int it = 0; it < s; it++) {
        const double w = 2.0 - (p + q);
        p *= w;
        q *= w;
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double v0 = a.v_in[(2 * d) * C + c], v1 = a.v_in[(2 * d + 1) * C + c];
        const double dv = v1 - v0;
        vop[(2 * d) * C] = fma(p, dv, v0);
        vop[(2 * d + 1) * C] = fma(-q, dv, v1);
    }
    if (a.m_out) a.m_out[c] = (int8_t)deg;
    if (a.s_out) a.s_out[c] = (int16_t)s;
}

// Each block orders a tile of rounds x threads consecutive cells by the cost
// proxy first, so that a warp's 32 cells share their degree and scaling.
template <int NF>
__global__ void __launch_bounds__(kVarLpcThreads) dx_forward_lpc_var(VarArgs a, DxConsts K, DxPade P, int rounds) {
    __shared__ unsigned long long key[kVarLpcTile];
    __shared__ unsigned short order[kVarLpcTile];
    __shared__ double bsh[32];
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    const long long base = (long long)blockIdx.x * rounds * kVarLpcThreads;
    dx_lpc_tile_order<NF - 1>(base, rounds, kVarLpcThreads, a.C, a.C, a.rho_g, a.rho_d, a.t_s, a.dt, key, order);
    for (int r = 0; r < rounds; r++) {
        const long long c = base + order[dx_lpc_round_pos(r, kVarLpcThreads)];
        if (c >= a.C) continue;
        if constexpr (NF == 2)
            var2_lpc_cell(c, a, K, P, bsh);
        else if (a.method == DRAG_METHOD_PADE)
            pade_lpc_cell<NF>(c, a, P);
        else
            bound_lpc_cell<NF>(c, a, K, bsh);
    }
}

template <int NF>
int launch_var_lpc(const VarArgs &a, const DxConsts &K, const DxPade &P, cudaStream_t stream) {
    int rounds = kVarLpcTile / kVarLpcThreads;
    while (rounds > 1 && (a.C + rounds * kVarLpcThreads - 1) / (rounds * kVarLpcThreads) < 4LL * dx_sm_count())
        rounds >>= 1;
    const long long blocks = (a.C + rounds * kVarLpcThreads - 1) / (rounds * kVarLpcThreads);
    dx_forward_lpc_var<NF><<<(unsigned)blocks, kVarLpcThreads, 0, stream>>>(a, K, P, rounds);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

// Matrix sizes the lane-per-cell variant kernel takes.
constexpr int kVarLpcNMin = 2, kVarLpcNMax = DX_LPC_REG_NMAX;

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

}  // namespace

extern "C" int drag_expm_apply_opts(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                    const double *t_s, double dt, const double *v_in, double *v_out,
                                    const drag_expm_options_t *opts, int8_t *m_out, int16_t *s_out,
                                    cudaStream_t stream) {
    if (!opts) return DRAG_ENULL;
    if (opts->arith < DRAG_ARITH_FP64 || opts->arith > DRAG_ARITH_FP32 || opts->method < DRAG_METHOD_TAYLOR ||
        opts->method > DRAG_METHOD_PADE || (opts->method == DRAG_METHOD_PADE && opts->bound_test))
        return DRAG_EINVAL_OPTION;
    const DxConsts *K = dx_consts_for(opts->ubits);
    if (!K) return DRAG_EINVAL_TARGET;
    if (opts->arith == DRAG_ARITH_FP32) {
        // mixed precision: plain Taylor at the single-precision target (Eq. B8 pairs u = 2^-24 with single
        // precision; at 2^-11, theta reaches ~8 and the Taylor sum's cancellation costs up to e^theta FP32 ulps)
        if (opts->method != DRAG_METHOD_TAYLOR || opts->bound_test || opts->ubits != 24 || m_out || s_out)
            return DRAG_EINVAL_OPTION;
        const int n = nspecies + 1;
        if (nspecies >= 1 && ((n <= DX_LPC_NMAX && dx_mode_for(n) != DX_MODE_WPC) ||
                              (n > DX_LPC_NMAX && n <= DX_LPC_F32_NMAX))) {
            // lane per cell: as the FP64 forward runs these sizes up to n = 12, and up to n = 17
            // whatever the mode (FP32 work in registers beats the warp-per-cell rounds there)
            if (ncells < 0 || !(dt >= 0.0) || !std::isfinite(dt)) return DRAG_EINVAL_SIZE;
            if (ncells == 0) return DRAG_OK;
            if (!rho_g || !rho_d || !t_s || !v_in || !v_out) return DRAG_ENULL;
            const void *ptrs[] = {rho_g, rho_d, t_s, v_in, v_out};
            for (const void *p : ptrs)
                if (!aligned8(p)) return DRAG_EALIGN;
            uint32_t *st = dx_status_ptr();
            if (!st) return DRAG_ECUDA;
            return dx_launch_forward_lpc_f32(*K, n, ncells, rho_g, rho_d, t_s, v_in, v_out, dt, st, stream);
        }
        return dx_launch_forward_f32(*K, ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, stream);
    }
    const DxPade *P = opts->method == DRAG_METHOD_PADE ? dx_pade_for(opts->ubits) : dx_pade_for(53);
    if (!P) return DRAG_EINVAL_TARGET;
    if (opts->method == DRAG_METHOD_TAYLOR && !opts->bound_test && !m_out && !s_out)
        return drag_expm_apply_target(ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, opts->ubits, stream);
    if (ncells < 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX || !(dt >= 0.0) || !std::isfinite(dt))
        return DRAG_EINVAL_SIZE;
    if (ncells == 0) return DRAG_OK;
    if (!rho_g || !rho_d || !t_s || !v_in || !v_out) return DRAG_ENULL;
    const void *ptrs[] = {rho_g, rho_d, t_s, v_in, v_out};
    for (const void *p : ptrs)
        if (p && !aligned8(p)) return DRAG_EALIGN;
    if (s_out && (reinterpret_cast<uintptr_t>(s_out) & 1)) return DRAG_EALIGN;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    if (!dx_once_per_device(3, [] {
            return cudaFuncSetAttribute(dx_forward_wpc_var, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)var_smem_bytes(DX_NMAXF)) == cudaSuccess;
        }))
        return DRAG_ECUDA;
    const int n = nspecies + 1;
    VarArgs a{ncells, nspecies, rho_g, rho_d, t_s, v_in, v_out, dt, st, m_out, s_out, opts->method,
              opts->bound_test ? 1 : 0};
    if (n >= kVarLpcNMin && n <= kVarLpcNMax && dx_mode_for(n) != DX_MODE_WPC) {
        switch (n) {
            case 2: return launch_var_lpc<2>(a, *K, *P, stream);
            case 3: return launch_var_lpc<3>(a, *K, *P, stream);
            case 4: return launch_var_lpc<4>(a, *K, *P, stream);
            case 5: return launch_var_lpc<5>(a, *K, *P, stream);
            case 6: return launch_var_lpc<6>(a, *K, *P, stream);
            default: break;
        }
    }
    const long long grid = (ncells + kCellsPerBlock - 1) / kCellsPerBlock;
    dx_forward_wpc_var<<<(unsigned)grid, kWarpsPerBlock * 32, var_smem_bytes(n), stream>>>(a, *K, *P);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}
