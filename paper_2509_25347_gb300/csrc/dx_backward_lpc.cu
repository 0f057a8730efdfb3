// Adjoint of the EXP drag update, lane-per-cell kernels for small matrices
// (n = N + 1 <= DX_BWD_LPC_NMAX).
//
// Same mathematics as the warp-per-cell adjoint (dx_backward.cu): with g_d =
// dL/dv_out,d, the forward-mode Frechet derivative L(S, H) of the symmetric
// similarity form is carried through the scaling and squaring beside E,
//   Taylor:   F <- F X + b_j I,   dF <- dF X + F H   (F H = sum_d (F a_d) b_d^T),
//   squaring: (E, L) <- (E^2, E L + L E),
// with the rank-4 direction H = 2^-s (sum_d a_d b_d^T - kappa sigma sigma^T),
// a_d = g_d / sigma, b_d = sigma o v_in,d, and the gradients read from row 0,
// column 0 and the diagonal of the last L (Eqs. DragEqVar2/3, jacobian).
//
// Here one lane owns one cell and runs all of it serially, so every FP64
// instruction of a warp works on 32 cells, where a warp-per-cell round keeps
// only part of its lanes busy (n(n-1)/2 upper-triangle entries, n-term
// reductions through shuffles, set-up and Taylor phases on n lanes). E is
// formed with the lane-per-cell forward's own steps (dx_lpc.cuh), so the taped
// variant, which reads E_0 .. E_{s-2} from the forward's tape instead, gives
// bit-identical gradients.
//
// Storage. Up to n = 6 E and L live in registers, double-buffered. For
// n = 7..9 (the hybrid storage) the per-lane state no longer fits: L (n^2
// doubles) stays in registers, E in shared memory, and the squaring's new L
// goes to shared memory before it is copied back (it needs all of the old L).
// E^2 forms in registers once the old L is dead. The derivative chain runs
// first (it carries y_d = F a_d by its own recurrence and never reads F); L
// then waits in shared memory while the Horner chain of F runs in registers.
// The Taylor derivative updates L in place (its row i needs only the old row
// i), so the n^2 slice of the new L can share its shared memory with the
// Taylor phase's vectors a_d, b_d, y_d (9n >= n^2 for n <= 9), and E with X
// and a_3, dead once F is done; a_d is formed again for the outputs, and eps,
// alpha are divided again there (the same roundings) instead of holding
// registers through the cell.
#include <cmath>

#include "dx_lpc.cuh"
#include "dx_modes.h"

namespace {

// Threads per block: 2 warps, or one for the hybrid storage, whose 27-37 KB of
// shared memory per warp would otherwise strand part of an SM; and the largest
// tile of cells a block sorts.
template <int NF>
__host__ __device__ constexpr int bwd_threads() { return NF >= 7 ? 32 : 64; }
template <int NF>
__host__ __device__ constexpr int bwd_tile() { return NF >= 7 ? 128 : 512; }

struct BwdLpcArgs {
    long long C;
    const double *rho_g, *rho_d, *t_s, *v_in, *g_out;
    double *g_vin, *g_rho_g, *g_rho_d, *g_ts;
    double dt;
    uint32_t *status;
    const long long *thdr;   // tape (TAPE kernels): fingerprints, then levels
    const double *tm;
    int levels, P;
};

// Storage per n: E (packed, double-buffered) and L (full, double-buffered) in
// registers; the n-vectors (sigma, tau, X_0f, X_ff, a_d, -kappa sigma, b_d, y_d:
// 14 n doubles) in registers up to n = 3 and in shared memory above. Hybrid
// (n >= 7): L in registers, E and the squaring's new L in shared memory; the
// Horner chain and E^2 form in registers while L is not live. Per lane the
// hybrid slice is sigma, tau (2n), then X_0f, X_ff, a_3 (3n) under E (n(n+1)/2),
// then a_d, b_d, y_d (9n) under the new L (n^2): 144 doubles at n = 9, six
// one-warp CTAs per SM (seven at n = 8, eight at n = 7).
template <int NF>
struct BwdLpcStore {
    static constexpr bool kVecShared = NF >= 4;
    static constexpr bool kHybrid = NF >= 7;
    static constexpr int kVec = 14 * NF;
    static constexpr int kNT = NF * (NF + 1) / 2;
    static constexpr int kE = 2 * NF;                           // hybrid: E over X_0f, X_ff, a_3
    static constexpr int kAv = kHybrid ? kE + kNT : 5 * NF;     // a_d, b_d, y_d (hybrid: under the new L)
    static constexpr int kWarpDoubles = kHybrid ? 32 * (kAv + 9 * NF) : kVecShared ? 32 * kVec : 0;
    static_assert(!kHybrid || NF * NF <= 9 * NF, "the new L overlays a_d, b_d, y_d");
    static_assert(!kHybrid || 3 * NF <= kNT, "E overlays X_0f, X_ff, a_3");
};

template <int NF>
__device__ __forceinline__ void bwd_lpc_fail(long long c, const BwdLpcArgs &a) {
    const long long C = a.C;
    if (a.g_vin)
        for (int e = 0; e < 3 * NF; e++) a.g_vin[e * C + c] = NAN;
    for (int i = 0; i < NF - 1; i++) {
        if (a.g_rho_d) a.g_rho_d[i * C + c] = NAN;
        if (a.g_ts) a.g_ts[i * C + c] = NAN;
    }
    if (a.g_rho_g) a.g_rho_g[c] = NAN;
    atomicOr(a.status, DRAG_STATUS_BAD_CELL);
}

// dF = b_m H for the rank-4 direction H = sum_d a_d b_d^T + a_3 sigma^T.
template <int NF, class LA, class VA, class WA>
__device__ __forceinline__ void bwd_lpc_dinit(LA &L, WA &av, WA &bv, VA &a3, VA &sig, double bm) {
#pragma unroll
    for (int i = 0; i < NF; i++) {
#pragma unroll
        for (int j = 0; j < NF; j++) {
            double acc = av[i] * bv[j];
            acc = fma(av[NF + i], bv[NF + j], acc);
            acc = fma(av[2 * NF + i], bv[2 * NF + j], acc);
            acc = fma(a3[i], sig[j], acc);
            L[i * NF + j] = bm * acc;
        }
    }
}

// y_d = F a_d for F = b_m X + b_{m-1} I.
template <int NF, class VA, class WA>
__device__ __forceinline__ void bwd_lpc_yinit(WA &yv, VA &xs, VA &ds, WA &av, double bm, double bm1) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < NF; k++) acc = fma(xs[k], av[d * NF + k], acc);
        yv[d * NF] = fma(bm, acc, bm1 * av[d * NF]);
#pragma unroll
        for (int f = 1; f < NF; f++)
            yv[d * NF + f] = fma(bm, fma(xs[f], av[d * NF], ds[f] * av[d * NF + f]), bm1 * av[d * NF + f]);
    }
}

// Row i of dF' = dF X + F H, with F H = sum_d y_d b_d^T + b_{j+1} a_3 sigma^T
// (X the arrowhead): column 0 is a dot product over the row, the other
// entries take two FMAs of dF X each. Reads row i of Lsrc before writing row
// i of Ldst, so Lsrc and Ldst may be the same array.
template <int NF, class LS, class LD, class VA, class WA>
__device__ __forceinline__ void bwd_lpc_drow(LS &Lsrc, LD &Ldst, int i, WA &yv, WA &bv, VA &a3, VA &sig, VA &xs,
                                             VA &ds, double bj1) {
    double r[NF];
#pragma unroll
    for (int k = 0; k < NF; k++) r[k] = Lsrc[i * NF + k];
    const double y0 = yv[i], y1 = yv[NF + i], y2 = yv[2 * NF + i], w = bj1 * a3[i];
    double acc = y0 * bv[0];
    acc = fma(y1, bv[NF], acc);
    acc = fma(y2, bv[2 * NF], acc);
    acc = fma(w, sig[0], acc);
#pragma unroll
    for (int k = 0; k < NF; k++) acc = fma(r[k], xs[k], acc);
#pragma unroll
    for (int j = 1; j < NF; j++) {
        double t = y0 * bv[j];
        t = fma(y1, bv[NF + j], t);
        t = fma(y2, bv[2 * NF + j], t);
        t = fma(w, sig[j], t);
        t = fma(r[0], xs[j], t);
        Ldst[i * NF + j] = fma(r[j], ds[j], t);
    }
    Ldst[i * NF] = acc;
}

// y_d <- X y_d + b_j a_d.
template <int NF, class VA, class WA>
__device__ __forceinline__ void bwd_lpc_ystep(WA &yv, VA &xs, VA &ds, WA &av, double bj) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double y0 = yv[d * NF];
        double acc = bj * av[d * NF];
#pragma unroll
        for (int k = 0; k < NF; k++) acc = fma(xs[k], yv[d * NF + k], acc);
#pragma unroll
        for (int f = 1; f < NF; f++)
            yv[d * NF + f] = fma(xs[f], y0, fma(ds[f], yv[d * NF + f], bj * av[d * NF + f]));
        yv[d * NF] = acc;
    }
}

// L' = E L + L E (E symmetric, packed; L full), each entry's two sums in
// ascending k. TRIM forms only row 0, column 0 and the diagonal (all the
// gradients read, in the last squaring). The entries are chosen at compile
// time, so the whole product is one straight block whose independent entries
// the compiler interleaves.
template <int NF, bool TRIM, class FA, class LA, class NA>
__device__ __forceinline__ void bwd_lpc_el_le(FA &Fm, LA &Lm, NA &Ln) {
    using P = DxPacked<NF>;
    if constexpr (!TRIM && BwdLpcStore<NF>::kHybrid) {
        // Hybrid storage (E in shared memory): a whole row of the new L at a
        // time, its n sums side by side, so E_ik is loaded once for the row and
        // row k of E once per k, and every step issues n independent FMAs.
        // Each entry still sums E_ik L_kj, then L_ik E_kj, in ascending k: the
        // same roundings as entry by entry (forward + adjoint on 262,144 cells of
        // N = 8: 24.7 against 25.3 ms, 21.8 against 22.2 through the tape).
#pragma unroll
        for (int i = 0; i < NF; i++) {
            double acc[NF];
#pragma unroll
            for (int j = 0; j < NF; j++) acc[j] = 0.0;
#pragma unroll
            for (int k = 0; k < NF; k++) {
                const double e = dx_lane_ld(Fm, P::at(i, k));
#pragma unroll
                for (int j = 0; j < NF; j++) acc[j] = fma(e, Lm[k * NF + j], acc[j]);
            }
#pragma unroll
            for (int k = 0; k < NF; k++) {
                const double l = Lm[i * NF + k];
#pragma unroll
                for (int j = 0; j < NF; j++) acc[j] = fma(l, dx_lane_ld(Fm, P::at(k, j)), acc[j]);
            }
#pragma unroll
            for (int j = 0; j < NF; j++) Ln[i * NF + j] = acc[j];
        }
    } else {
#pragma unroll
        for (int i = 0; i < NF; i++) {
#pragma unroll
            for (int j = 0; j < NF; j++) {
                if (TRIM && i != 0 && j != 0 && i != j) continue;
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < NF; k++) acc = fma(dx_lane_ld(Fm, P::at(i, k)), Lm[k * NF + j], acc);
#pragma unroll
                for (int k = 0; k < NF; k++) acc = fma(Lm[i * NF + k], dx_lane_ld(Fm, P::at(j, k)), acc);
                Ln[i * NF + j] = acc;
            }
        }
    }
}

template <int NF, bool TAPE>
__device__ __forceinline__ void bwd_lpc_cell(int lane, long long c, const BwdLpcArgs &a, const DxConsts &K,
                                             const double *bsh, double *wsm) {
    constexpr int N = NF - 1;
    constexpr int NT = DxPacked<NF>::NT;
    constexpr bool SV = BwdLpcStore<NF>::kVecShared;
    constexpr bool HY = BwdLpcStore<NF>::kHybrid;
    using P = DxPacked<NF>;
    const long long C = a.C;
    const double dt = a.dt;

    // ---------------- set-up, Algorithm 2 and X, as the lane-per-cell forward (dx_lpc_setup)
    DxLaneArr<NF, SV> sig, tau, xs, ds, a3;
    DxLaneArr<3 * NF, SV> av, bv, yv;
    if constexpr (SV) {
        sig.bind(wsm, lane);
        tau.bind(wsm + 32 * NF, lane);
        xs.bind(wsm + 64 * NF, lane);
        ds.bind(wsm + 96 * NF, lane);
        a3.bind(wsm + 128 * NF, lane);
        constexpr int kAv = BwdLpcStore<NF>::kAv;
        av.bind(wsm + 32 * kAv, lane);
        bv.bind(wsm + 32 * (kAv + 3 * NF), lane);
        yv.bind(wsm + 32 * (kAv + 6 * NF), lane);
    }
    double rg, eps[N], alpha[N];
    int kk, s;
    unsigned long long fph;
    if (!dx_lpc_setup<NF>(a.rho_g + c, a.rho_d + c, a.t_s + c, C, dt, K, TAPE, rg, eps, alpha, kk, s, fph, sig, tau,
                          xs, ds)) {
        bwd_lpc_fail<NF>(c, a);
        return;
    }
    const int m = K.mk[kk];
    const int tlev = dx_tape_levels(s);
    bool taped = false;
    const double *tcell = nullptr;
    if (TAPE) {
        const long long h = dx_fingerprint_final(fph, rg, dt, dx_tape_salt(a.levels, NF));
        taped = a.thdr[c] == h && tlev <= a.levels;
        tcell = a.tm + (size_t)c * a.levels * a.P;
    }
    {
        // a_d = g_d / sigma, b_d = 2^-s sigma o v_d, and the stationary block kappa
        double sa[3] = {0.0, 0.0, 0.0}, sb[3] = {0.0, 0.0, 0.0}, ss = 0.0;
#pragma unroll
        for (int f = 0; f < NF; f++) {
            const double sg = sig[f], tu = tau[f];
            ss = fma(sg, sg, ss);
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const double ad = a.g_out[(d * NF + f) * C + c] * tu;
                const double bd = dx_scale2(sg * a.v_in[(d * NF + f) * C + c], s);
                av[d * NF + f] = ad;
                bv[d * NF + f] = bd;
                sa[d] = fma(sg, ad, sa[d]);
                sb[d] = fma(sg, bd, sb[d]);
            }
        }
        const double kappa = __ddiv_rn(fma(sa[2], sb[2], fma(sa[1], sb[1], sa[0] * sb[0])), ss * ss);
#pragma unroll
        for (int f = 0; f < NF; f++) a3[f] = -kappa * sig[f];
    }

    // ---------------- Taylor and its derivative: F = b_m X + b_{m-1} I, dF = b_m H, y_d = F a_d
    DxLaneArr<NT, HY> Fm;                 // E (hybrid: shared memory)
    DxLaneArr<NT, false> Gm;              // the next E, or the Horner step's next F
    DxLaneArr<NF * NF, false> Lm, Lt;     // L, and the Taylor step's new L (in place for the compiler)
    DxLaneArr<NF * NF, HY> Ln;            // the squaring's new L
    if constexpr (HY) {
        Fm.bind(wsm + 32 * BwdLpcStore<NF>::kE, lane);    // over X_0f, X_ff, a_3, dead once F is done
        Ln.bind(wsm + 32 * BwdLpcStore<NF>::kAv, lane);   // over a_d, b_d, y_d, dead in the squarings
    }
    const double bm = bsh[m], bm1 = bsh[m - 1];
    if constexpr (HY) {
        // The derivative chain shares only X with the Horner chain of F (it
        // carries y_d = F a_d by its own recurrence): it runs first, with L in
        // registers; L then goes to the new L's slice (a_d, b_d, y_d are dead)
        // while the Horner chain runs in registers and leaves E_0 over X and
        // a_3, and comes back for the squarings.
        bwd_lpc_dinit<NF>(Lm, av, bv, a3, sig, bm);
        bwd_lpc_yinit<NF>(yv, xs, ds, av, bm, bm1);
        for (int jb = m - 2; jb >= 0; jb--) {
#pragma unroll
            for (int i = 0; i < NF; i++) {
                bwd_lpc_drow<NF>(Lm, Lt, i, yv, bv, a3, sig, xs, ds, bsh[jb + 1]);
                // one row at a time: overlapped, the rows' vector loads would
                // outgrow the registers L leaves free
                asm volatile("" ::: "memory");
            }
            bwd_lpc_ystep<NF>(yv, xs, ds, av, bsh[jb]);
            dx_lane_take(Lm, Lt);
        }
#pragma unroll
        for (int e = 0; e < NF * NF; e++) Ln[e] = Lm[e];
        asm volatile("" ::: "memory");   // L stored before the Horner chain takes its registers
        if (taped) {
#pragma unroll
            for (int e = 0; e < NT; e++) Fm[e] = tcell[e];
        } else {
            DxLaneArr<NT, false> Fr;
            dx_lpc_taylor_init<NF>(Fr, xs, ds, bm, bm1);
            for (int jb = m - 2; jb >= 0; jb--) {
                dx_lpc_horner_step<NF>(Fr, Gm, xs, ds, bsh[jb]);
                dx_lane_take(Fr, Gm);
            }
            dx_lpc_taylor_finish<NF>(Fr, xs);
            dx_lpc_restore<NF>(Fr, sig, tau);
#pragma unroll
            for (int e = 0; e < NT; e++) Fm[e] = Fr[e];
        }
        asm volatile("" ::: "memory");   // E_0 stored before L takes the registers back
#pragma unroll
        for (int e = 0; e < NF * NF; e++) Lm[e] = Ln[e];
    } else {
        if (!taped) dx_lpc_taylor_init<NF>(Fm, xs, ds, bm, bm1);
        bwd_lpc_dinit<NF>(Lm, av, bv, a3, sig, bm);
        bwd_lpc_yinit<NF>(yv, xs, ds, av, bm, bm1);
        for (int jb = m - 2; jb >= 0; jb--) {
            // F_jb = F X + b_jb I; dF_jb = dF X + F H, where F a_d = y_d (d < 3) and
            // F a_3 = b_{jb+1} a_3 (X sigma = 0); then y_d <- X y_d + b_jb a_d.
            if (!taped) {
                dx_lpc_horner_step<NF>(Fm, Gm, xs, ds, bsh[jb]);
                dx_lane_take(Fm, Gm);
            }
#pragma unroll
            for (int i = 0; i < NF; i++) bwd_lpc_drow<NF>(Lm, Lt, i, yv, bv, a3, sig, xs, ds, bsh[jb + 1]);
            bwd_lpc_ystep<NF>(yv, xs, ds, av, bsh[jb]);
            dx_lane_take(Lm, Lt);
        }
        if (taped) {
#pragma unroll
            for (int e = 0; e < NT; e++) Fm[e] = tcell[e];
        } else {
            dx_lpc_taylor_finish<NF>(Fm, xs);
            dx_lpc_restore<NF>(Fm, sig, tau);
        }
    }

    // ---------------- squarings: (E, L) <- (E^2, E L + L E); the last one forms only
    // row 0, column 0 and the diagonal of L (all the gradients read) and leaves E at E_{s-1}
    for (int sq = 0; sq < s; sq++) {
        const bool last = sq == s - 1;
        if (last)
            bwd_lpc_el_le<NF, true>(Fm, Lm, Ln);
        else
            bwd_lpc_el_le<NF, false>(Fm, Lm, Ln);

        if (!last) {
            // hybrid: the old L is dead once the new one is stored, so E^2 forms
            // in the registers it held and goes back over E
            if (taped && sq + 1 < tlev) {
                const double *lv = tcell + (size_t)(sq + 1) * a.P;
#pragma unroll
                for (int e = 0; e < NT; e++) Gm[e] = lv[e];
            } else {
                dx_lpc_square_offdiag<NF>(Fm, Gm);
                dx_lpc_restore<NF>(Gm, sig, tau);
            }
            dx_lane_take(Fm, Gm);
            if constexpr (HY) asm volatile("" ::: "memory");   // the new L loads after E^2 is stored
        }
        dx_lane_take(Lm, Ln);   // after the trimmed last squaring only the slots the gradients read are fresh
    }

    // ---------------- outputs
    if constexpr (HY) {
        // a_d = g_d / sigma again (its slice held the new L), and eps, alpha
        // divided again exactly as the set-up divided them
#pragma unroll
        for (int f = 0; f < NF; f++) {
#pragma unroll
            for (int d = 0; d < 3; d++) av[d * NF + f] = a.g_out[(d * NF + f) * C + c] * tau[f];
        }
#pragma unroll
        for (int i = 0; i < N; i++) {
            eps[i] = __ddiv_rn(a.rho_d[i * C + c], rg);
            alpha[i] = __drcp_rn(a.t_s[i * C + c]);
        }
    }
    if (a.g_vin) {
        // P^T g with P^T = D_sigma E D_sigma^-1: (P^T g)_i = E_ii g_i + sigma_i
        // sum_{k != i} E_ik a_k, a = g / sigma. After s >= 1 squarings E holds
        // E_{s-1} and P^T = (D_sigma E D_sigma^-1)^2: two applications, the first
        // into (y_d, a_d) = (g', g' / sigma).
        if (s >= 1) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
#pragma unroll
                for (int i = 0; i < NF; i++) {
                    double acc = 0.0;
#pragma unroll
                    for (int k = 0; k < NF; k++)
                        if (k != i) acc = fma(Fm[P::at(i, k)], av[d * NF + k], acc);
                    yv[d * NF + i] = fma(sig[i], acc, Fm[P::at(i, i)] * a.g_out[(d * NF + i) * C + c]);
                }
#pragma unroll
                for (int i = 0; i < NF; i++) av[d * NF + i] = tau[i] * yv[d * NF + i];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
            for (int i = 0; i < NF; i++) {
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < NF; k++)
                    if (k != i) acc = fma(Fm[P::at(i, k)], av[d * NF + k], acc);
                const double gi = s >= 1 ? yv[d * NF + i] : a.g_out[(d * NF + i) * C + c];
                a.g_vin[(d * NF + i) * C + c] = fma(sig[i], acc, Fm[P::at(i, i)] * gi);
            }
        }
    }
    double part = 0.0;
#pragma unroll
    for (int i = 1; i < NF; i++) {
        // explicit roundings (no contraction), so every instantiation gives the same bits
        const double z00 = Lm[0], zii = Lm[i * NF + i];
        const double z0i = __dmul_rn(Lm[i], tau[i]), zi0 = __dmul_rn(sig[i], Lm[i * NF]);
        const double d0 = __dsub_rn(z0i, z00);
        const double geps = __dmul_rn(__dmul_rn(alpha[i - 1], dt), d0);
        const double galpha = __dmul_rn(dt, fma(eps[i - 1], d0, __dsub_rn(zi0, zii)));
        if (a.g_rho_d) a.g_rho_d[(i - 1) * C + c] = __ddiv_rn(geps, rg);
        if (a.g_ts) a.g_ts[(i - 1) * C + c] = -galpha * (alpha[i - 1] * alpha[i - 1]);
        part = fma(eps[i - 1], geps, part);
    }
    if (a.g_rho_g) a.g_rho_g[c] = -__ddiv_rn(part, rg);
}

template <int NF, bool TAPE>
__global__ void __launch_bounds__(bwd_threads<NF>()) dx_backward_lpc(BwdLpcArgs a, DxConsts K, int rounds) {
    constexpr int kThreads = bwd_threads<NF>(), kTile = bwd_tile<NF>();
    constexpr bool HY = BwdLpcStore<NF>::kHybrid;
    extern __shared__ double smem[];
    // the hybrid storage sorts in the slices of the first cell's matrices and
    // keeps its own positions in registers before any cell starts
    __shared__ unsigned long long key_static[HY ? 1 : kTile];
    __shared__ unsigned short order_static[HY ? 1 : kTile];
    double *bsh = smem;
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    double *wsm = smem + 32 + (threadIdx.x >> 5) * BwdLpcStore<NF>::kWarpDoubles;
    unsigned long long *key = HY ? reinterpret_cast<unsigned long long *>(smem + 32 + 32 * BwdLpcStore<NF>::kE)
                                 : key_static;
    unsigned short *order = HY ? reinterpret_cast<unsigned short *>(key + kTile) : order_static;
    const long long C = a.C;
    const long long base = (long long)blockIdx.x * rounds * kThreads;
    // order the tile's cells by the cost proxy so that a warp's 32 cells share (k*, s*)
    dx_lpc_tile_order<NF - 1>(base, rounds, kThreads, C, C, a.rho_g, a.rho_d, a.t_s, a.dt, key, order);
    const int lane = threadIdx.x & 31;
    if constexpr (HY) {
        // at most 4 rounds of 32 cells: the 7-bit tile positions packed in one word
        static_assert(kTile / kThreads <= 4 && kTile <= 256, "positions packed 8 bits each");
        unsigned int mine = 0;
        for (int r = 0; r < rounds; r++) mine |= (unsigned int)order[r * kThreads + threadIdx.x] << (8 * r);
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < rounds; r++) {
            const long long c = base + ((mine >> (8 * r)) & 0xffu);
            if (c < C) bwd_lpc_cell<NF, TAPE>(lane, c, a, K, bsh, wsm);
        }
    } else {
        for (int r = 0; r < rounds; r++) {
            const long long c = base + order[dx_lpc_round_pos(r, kThreads)];
            if (c < C) bwd_lpc_cell<NF, TAPE>(lane, c, a, K, bsh, wsm);
        }
    }
}

// The same adjoint over the cells of the whole input binned by (k*, s*)
// (perm: cell indices bin by bin), so that a warp's 32 cells share their
// Taylor order and squaring count except where a warp straddles two bins.
// Blocks take the permutation from its end, so the costliest bins start first
// and the cheap ones fill the tail.
template <int NF, bool TAPE>
__global__ void __launch_bounds__(bwd_threads<NF>())
dx_backward_lpc_binned(BwdLpcArgs a, DxConsts K, const unsigned long long *perm) {
    constexpr int kThreads = bwd_threads<NF>();
    extern __shared__ double smem[];
    double *bsh = smem;
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    __syncthreads();
    const long long pos = a.C - 1 - ((long long)blockIdx.x * kThreads + threadIdx.x);
    double *wsm = smem + 32 + (threadIdx.x >> 5) * BwdLpcStore<NF>::kWarpDoubles;
    if (pos >= 0) bwd_lpc_cell<NF, TAPE>(threadIdx.x & 31, (long long)(perm[pos] & 0xffffffffull), a, K, bsh, wsm);
}

template <int NF, bool TAPE>
int launch(const BwdLpcArgs &a, cudaStream_t stream) {
    constexpr int kThreads = bwd_threads<NF>(), kTile = bwd_tile<NF>();
    static_assert(!BwdLpcStore<NF>::kHybrid ||
                      kTile * (sizeof(unsigned long long) + sizeof(unsigned short)) <= 32 * sizeof(double) *
                          BwdLpcStore<NF>::kNT,
                  "the sort keys fit the first warp's matrix slices");
    const size_t smem = sizeof(double) * (32 + (size_t)(kThreads / 32) * BwdLpcStore<NF>::kWarpDoubles);
    constexpr size_t kStatic =
        BwdLpcStore<NF>::kHybrid ? 16 : kTile * (sizeof(unsigned long long) + sizeof(unsigned short));
    if (a.C >= dx_binned_min_cells(NF, true) && a.C <= 0x7fffffffLL) {
        const unsigned long long *perm = nullptr;
        void *scratch = dx_binned_perm(dx_consts(), a.C, NF - 1, a.rho_g, a.rho_d, a.t_s, a.dt, a.status, stream, &perm);
        if (scratch) {
            int rc = DRAG_OK;
            if (smem > 48 * 1024 && cudaFuncSetAttribute(dx_backward_lpc_binned<NF, TAPE>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem) != cudaSuccess)
                rc = DRAG_ECUDA;
            if (rc == DRAG_OK) {
                const long long blocks = (a.C + kThreads - 1) / kThreads;
                dx_backward_lpc_binned<NF, TAPE><<<(unsigned)blocks, kThreads, smem, stream>>>(a, dx_consts(), perm);
                if (cudaGetLastError() != cudaSuccess) rc = DRAG_ECUDA;
            }
            const int rr = dx_binned_release(scratch, stream);
            return rc != DRAG_OK ? rc : rr;
        }
        // no scratch: the tile-sorted kernel below
    }
    // the opt-in covers dynamic + static shared memory (the sort keys and order) above 48 KB
    if (smem + kStatic > 48 * 1024 &&
        cudaFuncSetAttribute(dx_backward_lpc<NF, TAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return DRAG_ECUDA;
    int rounds = kTile / kThreads;
    while (rounds > 1 && (a.C + rounds * kThreads - 1) / (rounds * kThreads) < 4LL * dx_sm_count()) rounds >>= 1;
    const long long blocks = (a.C + rounds * kThreads - 1) / (rounds * kThreads);
    dx_backward_lpc<NF, TAPE><<<(unsigned)blocks, kThreads, smem, stream>>>(a, dx_consts(), rounds);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

}  // namespace

int dx_launch_backward_lpc(int n, long long C, const double *rho_g, const double *rho_d, const double *t_s,
                           double dt, const double *v_in, const double *grad_v_out, double *grad_v_in,
                           double *grad_rho_g, double *grad_rho_d, double *grad_t_s, uint32_t *status,
                           const long long *thdr, const double *tm, int levels, int P, cudaStream_t stream) {
    const BwdLpcArgs a{C,         rho_g,      rho_d,     t_s,    v_in, grad_v_out, grad_v_in, grad_rho_g,
                       grad_rho_d, grad_t_s, dt,         status, thdr, tm,         levels,    P};
    const bool tape = thdr != nullptr;
    switch (n) {
#define DX_CASE(NF) \
    case NF: return tape ? launch<NF, true>(a, stream) : launch<NF, false>(a, stream);
        DX_CASE(2)
        DX_CASE(3)
        DX_CASE(4)
        DX_CASE(5)
        DX_CASE(6)
        DX_CASE(7)
        DX_CASE(8)
        DX_CASE(9)
#undef DX_CASE
        default: return DRAG_EINVAL_SIZE;
    }
}
