// Adjoint of the EXP drag update: gradients of a loss through
// v_out = exp(dt Omega_v) v_in with respect to v_in, rho_d, t_s and rho_g.
//
// With g_d = dL/dv_out,d, P = exp(A), A = dt Omega_v:
//   dL/dv_in,d = P^T g_d,   dL/dA = Z = L(A^T, G),   G = sum_d g_d v_in,d^T,
// where L(., .) is the Frechet derivative of the exponential. In the symmetric
// similarity form (A = D_sigma^-1 S D_sigma, S symmetric):
//   Z = D_sigma L(S, G_S) D_sigma^-1,   G_S = D_sigma^-1 G D_sigma = sum_d a_d b_d^T,
//   a_d = g_d / sigma, b_d = sigma o v_in,d   (rank 3).
// The stationary block of the direction is removed first: sigma spans the null
// space of S, so with P = sigma sigma^T / |sigma|^2, L(S, P G_S P) = P G_S P,
// whose image under D_sigma . D_sigma^-1 has constant rows and therefore adds
// nothing to Z_0i - Z_00 or Z_i0 - Z_ii. Carrying G_S - P G_S P instead keeps
// the propagated derivative at the size of the answer in stiff cells (the
// stationary block doubles at every squaring, and its rounding would otherwise
// be amplified by |A| in the chain rule below). H is then rank 4:
//   H = 2^-s (sum_d a_d b_d^T - kappa sigma sigma^T), kappa = sum_d (sigma.a_d)(sigma.b_d)/|sigma|^4.
// L(S, G_S) is carried through the same scaling and squaring as the forward:
//   Taylor: the Horner recurrence F <- F X + b_j I is differentiated,
//           dF <- dF X + F H (F H = sum_d (F a_d) b_d^T over the 4 rank terms);
//   squaring: (E, L) <- (E^2, E L + L E)  (block-triangular identity
//           exp([[S, H], [0, S]]) = [[e^S, L(S, H)], [0, e^S]]).
// The parameter gradients follow from A_0i = eps_i alpha_i dt,
// A_00 = -sum_i A_0i, A_i0 = -A_ii = alpha_i dt (Eqs. DragEqVar2/3, jacobian):
//   dL/deps_i = alpha_i dt (Z_0i - Z_00),
//   dL/dalpha_i = dt [eps_i (Z_0i - Z_00) + (Z_i0 - Z_ii)],
//   dL/drho_d,i = dL/deps_i / rho_g,  dL/dt_s,i = -alpha_i^2 dL/dalpha_i,
//   dL/drho_g = -sum_i eps_i dL/deps_i / rho_g.
// The taped kernel reads E_0 .. E_{s-2} from the adjoint tape the forward wrote
// (dx_tape.cuh) wherever the cell's fingerprint matches, so it forms neither F
// nor those E^2; its squarings before the last two carry only E L + L E.
#include <cmath>

#include "dx_modes.h"
#include "dx_wpc.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kCellsPerBlock = 16;

struct BwdArgs {
    long long C;
    int N;
    const double *rho_g, *rho_d, *t_s, *v_in, *g_out;
    double *g_vin, *g_rho_g, *g_rho_d, *g_ts;
    double dt;
    uint32_t *status;
    // adjoint tape written by the forward (taped kernel only): cell c's
    // fingerprint at thdr[c], its level t at tm + (c * levels + t) * P
    const long long *thdr;
    const double *tm;
    int levels, P;
};

// 8-byte asynchronous copy global -> shared (no register staging), and the
// wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async8(double *sdst, const double *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Starts copying one tape level (packed upper triangle) into the full
// symmetric n x n matrix E; complete after cp_async_wait_all() + __syncwarp().
// hp[p - 1] is entry p of the packing (p = 0 is (0, 0)).
__device__ __forceinline__ void tape_load(int lane, int n, int ns, const unsigned short *hp, const double *src,
                                          double *E) {
    const int np = n * (n + 1) / 2;
    for (int p = lane; p < np; p += 32) {
        int i = 0, j = 0;
        if (p > 0) {
            const int c = hp[p - 1];
            i = c >> 8;
            j = c & 255;
        }
        cp_async8(E + i * ns + j, src + p);
        if (i != j) cp_async8(E + j * ns + i, src + p);
    }
    cp_async_commit();
}

// Per-warp shared memory (doubles): E0, E1, L0, L1, then n-vectors: sigma,
// tau, X_0f, X_ff, a_d and b_d (4 each), two buffers of y_d (3 each), g_d (3)
// and w = b_{j+1} a_3 of the current Taylor step.
__host__ __device__ __forceinline__ int bwd_warp_smem_doubles(int n) { return 4 * n * dx_stride(n) + 22 * n; }

constexpr int kRank = 4;   // rank of the Frechet direction H

// yo_d = c1 X y_d + c0 a_d for d = 0, 1, 2 (X the arrowhead; vectors at stride n).
// Entries f >= 1 take two FMAs each; entry 0 is a dot product over the row
// X_0k, split over three groups of eight lanes (one per d) and reduced.
__device__ __forceinline__ void bwd_xvec(int lane, int n, const DxVecs &V, double c1, double c0, const double *a,
                                         const double *y, double *yo) {
    const int m1 = n - 1;
    for (int t = lane; t < 3 * m1; t += 32) {
        const int d = t >= m1 ? (t >= 2 * m1 ? 2 : 1) : 0;
        const int f = t - d * m1 + 1;
        const double *yd = y + d * n;
        yo[d * n + f] = fma(c1, fma(V.xs[f], yd[0], V.ds[f] * yd[f]), c0 * a[d * n + f]);
    }
    const int d = lane >> 3, phi = lane & 7;
    const bool on = d < 3;
    const double *yd = y + (on ? d : 0) * n;
    double acc = 0.0;
    const int cnt = (n + 7) >> 3;
    for (int u = 0; u < cnt; u++) {
        const int k = phi + 8 * u;
        const bool ok = on && k < n;
        acc = fma(ok ? V.xs[ok ? k : 0] : 0.0, ok ? yd[ok ? k : 0] : 0.0, acc);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(DX_FULL, acc, o);
    if (on && phi == 0) yo[d * n] = fma(c1, acc, c0 * a[d * n]);
}

// Smallest n whose Taylor steps use the fused round below. Below it the
// round's per-step role selection costs more than the rounds it saves
// (measured: n = 4, 5, 6 slower by 5-7 %; n = 7, 8, 9, 17 faster by 1-3 %).
#ifndef DX_BWD_FOLD_NMIN
#define DX_BWD_FOLD_NMIN 7
#endif

// Lanes of the fused round below: n for column 0, 3 for y'_d[0], nx for the
// entries f >= 1 of the three y'_d, q entries each (3 FMAs per entry), all
// within the round's n + 4 FMA steps. False when n is too large for that.
__host__ __device__ __forceinline__ bool bwd_fold_fits(int n, int &nx, int &q) {
    nx = 32 - n - 3;
    if (nx < 1) return false;
    q = (3 * (n - 1) + nx - 1) / nx;
    return 3 * q <= n + 4;
}

// One Taylor step's column 0 of dF' = dF X + F H and the next y'_d = X y_d +
// c0 a_d (d = 0, 1, 2), as one round of n + 4 FMA steps issued uniformly by all
// lanes (each lane's operands depend on its role; absent terms are 0 * 0):
//   lane i < n       : dF'_i0 = sum_{d<3} y_d,i b_d,0 + w_i b_3,0 + sum_k dF_ik X_k0;
//   lane n + d (d<3) : y'_d,0 = c0 a_d,0 + sum_k X_0k y_d,k;
//   lanes n + 3 + r  : y'_d,f = c0 a_d,f + X_ff y_d,f + X_f0 y_d,0 for the entries
//                      (d, f) = r, r + nx, ... of the 3(n - 1) with f >= 1.
// Requires bwd_fold_fits(n).
__device__ __forceinline__ void bwd_col0_and_y(int lane, int n, int ns, int nx, int q, const DxVecs &V, double c0,
                                               const double *a, const double *b, const double *w, const double *y,
                                               const double *dF, double *dFn, double *yn) {
    const int K = n + 4;
    const int role = lane < n ? 0 : (lane < n + 3 ? 1 : (lane < n + 3 + nx ? 2 : 3));
    const int d1 = lane - n;          // role 1: component d
    const int r = lane - n - 3;       // role 2: first entry index
    double acc = 0.0;
    for (int st = 0; st < K; st++) {
        double x = 0.0, z = 0.0;
        double *dst = nullptr;
        if (role == 0) {
            if (st < 3) {
                x = y[st * n + lane];
                z = b[st * n];
            } else if (st == 3) {
                x = w[lane];
                z = b[3 * n];
            } else {
                x = dF[lane * ns + st - 4];
                z = V.xs[st - 4];
            }
            if (st == K - 1) dst = dFn + lane * ns;
        } else if (role == 1) {
            if (st == 0) {
                x = c0;
                z = a[d1 * n];
            } else if (st <= n) {
                x = V.xs[st - 1];
                z = y[d1 * n + st - 1];
            }
            if (st == n) dst = yn + d1 * n;
        } else if (role == 2) {
            const int e = st / 3, ph = st - 3 * e;
            const int t = r + nx * e;
            if (e < q && t < 3 * (n - 1)) {
                const int d = t / (n - 1), f = t - d * (n - 1) + 1;
                if (ph == 0) {
                    x = c0;
                    z = a[d * n + f];
                } else if (ph == 1) {
                    x = V.ds[f];
                    z = y[d * n + f];
                } else {
                    x = V.xs[f];
                    z = y[d * n];
                    dst = yn + d * n + f;
                }
            }
        }
        acc = fma(x, z, acc);
        if (dst) {
            *dst = acc;
            acc = 0.0;
        }
    }
}

// One squaring of (E, L): (E, L) <- (E^2, E L + L E), E^2 restored, as tasks
// of n FP64 operations dealt 32 per round:
//   O (i < j): En_ij = En_ji = sum_k E_ik E_jk;
//   A (i, j) : Ln_ij = sum_k E_ik L_kj;
//   B (i, j) : Ln_ij = Ln_ij + sum_k L_ik E_jk  (at least one round after its A);
//   R (i)    : En_ii = 1 - tau_i sum_{k != i} En_ik sigma_k  (after every O).
// mode kSqFull: all of the above. kSqTrimmed: only the entries of E L + L E in
// row 0, column 0 and on the diagonal, and no E^2 (the gradients read only
// those entries of the last L).
constexpr int kSqFull = 0, kSqTrimmed = 1;
__device__ __forceinline__ void bwd_square(int lane, int n, int ns, const unsigned short *od, const DxVecs &V,
                                           const double *E, const double *L, double *En, double *Ln, int mode) {
    const bool trimmed = mode == kSqTrimmed;
    const int nO = trimmed ? 0 : n * (n - 1) / 2;
    const int nL = trimmed ? 3 * n - 2 : n * n;
    const int nR = trimmed ? 0 : n;
    const int a0 = nO;
    const int b0 = nL >= 32 ? nO + nL : ((nO + nL + 31) & ~31);
    const int r0 = b0 + nL;
    const int ntask = r0 + nR;
    const int inv = (65536 + n - 1) / n;   // (e * inv) >> 16 == e / n for e < n^2 + 64, n <= 32
    for (int base = 0; base < ntask; base += 32) {
        const int t = base + lane;
        const double *pa = E, *pb = E;
        int sb = 1, skip = 32, kind = 0, i = 0, j = 0;
        double acc = 0.0;
        if (t < nO) {
            const int p = od[t];
            i = p >> 8;
            j = p & 255;
            pa = E + i * ns;
            pb = E + j * ns;
            kind = 1;
        } else if ((t >= a0 && t < a0 + nL) || (t >= b0 && t < r0)) {
            const bool isB = t >= b0;
            const int e = isB ? t - b0 : t - a0;
            if (!trimmed) {
                i = (e * inv) >> 16;
                j = e - i * n;
            } else if (e < n) {
                j = e;
            } else if (e < 2 * n - 1) {
                i = e - n + 1;
            } else {
                i = j = e - 2 * n + 2;
            }
            if (isB) {
                pa = L + i * ns;
                pb = E + j * ns;
                acc = Ln[i * ns + j];
            } else {
                pa = E + i * ns;
                pb = L + j;
                sb = ns;
            }
            kind = 2;
        } else if (t >= r0 && t < ntask) {
            i = t - r0;
            pa = En + i * ns;
            pb = V.sig;
            skip = i;
            kind = 3;
        }
        double res;
        if (base + 32 <= r0) {
            // no restoration in this round (warp uniform): plain n-term dot products
            for (int q = 0; q < n - 1; q++) acc = fma(pa[q], pb[q * sb], acc);
            res = fma(pa[n - 1], pb[(n - 1) * sb], acc);
        } else {
            for (int q = 0; q < n - 1; q++) {
                const int k = q + (q >= skip);
                acc = fma(pa[k], pb[k * sb], acc);
            }
            const bool isR = kind == 3;
            res = fma(isR ? -V.tau[i] : pa[n - 1], isR ? acc : pb[(n - 1) * sb], isR ? 1.0 : acc);
        }
        if (kind == 1) {
            En[i * ns + j] = res;
            En[j * ns + i] = res;
        } else if (kind == 2) {
            Ln[i * ns + j] = res;
        } else if (kind == 3) {
            En[i * ns + i] = res;
        }
        __syncwarp();
    }
}

// A-task order of an L-only squaring whose first tasks ran in the previous
// squaring's last round next to r of that squaring's B tasks (entries of row
// n - 1, columns n - r .. n - 1, when 0 < r < n): first the entries with
// i <= n - 2 and j <= n - 1 - r (safe to run in that round: their column of
// L is complete and their slot of the old L is read by no pending B task),
// then i <= n - 2 with j >= n - r, then row n - 1. r = 0: row major.
__device__ __forceinline__ void lonly_a_entry(int n, int r, int e, int &i, int &j) {
    if (r == 0) {
        i = e / n;
        j = e - i * n;
    } else if (e < (n - 1) * (n - r)) {
        i = e / (n - r);
        j = e - i * (n - r);
    } else if (e < (n - 1) * n) {
        const int e2 = e - (n - 1) * (n - r);
        i = e2 / r;
        j = n - r + (e2 - i * r);
    } else {
        i = n - 1;
        j = e - (n - 1) * n;
    }
}

// One squaring L' = E L + L E without E^2 (E and the next E from the tape), as
// A tasks (Ln_ij = sum_k E_ik L_kj) then B tasks (Ln_ij += sum_k L_ik E_jk),
// n-FMA tasks dealt 32 per round. kin of its A tasks (order lonly_a_entry with
// rin) already ran in the previous squaring's last round. When carry is set and
// the last round holds r < n B tasks, its other lanes run the first 32 - r A
// tasks of the next squaring (reading En, the next E, and Ln, whose columns
// they need are complete; writing L, whose slots they overwrite are no longer
// read); kout / rout describe them (0 / 0 otherwise). The tape copies into En
// are waited for before the last round. Per entry the arithmetic is that of
// bwd_square (same two n-FMA chains, in order), so results match it bit for bit.
__device__ __forceinline__ void bwd_square_lonly(int lane, int n, int ns, const double *E, double *L, const double *En,
                                                 double *Ln, int kin, int rin, bool carry, int &kout, int &rout) {
    const int nn = n * n;
    const int nA = nn - kin;
    const int b0 = nA;                                 // B tasks follow the A tasks directly (nn >= 32) ...
    const int b0p = nn >= 32 ? b0 : ((b0 + 31) & ~31); // ... or from the next round (B after its A)
    const int ntask = b0p + nn;
    const int rounds = (ntask + 31) >> 5;
    const int rem = ntask & 31;
    const int inv = (65536 + n - 1) / n;
    // fill: enough safe A tasks for the idle lanes, and in the next squaring every
    // B task at least a round after its A task (for the entries reordered behind
    // the safe ones the two lie nn - (n - rem)(n - 2) tasks apart)
    const bool fill = carry && nn >= 32 && rem > 0 && rem < n && (n - 1) * (n - rem) >= 32 - rem &&
                      nn - (n - rem) * (n - 2) >= 32;
    kout = fill ? 32 - rem : 0;
    rout = fill ? rem : 0;
    for (int rd = 0; rd < rounds; rd++) {
        if (rd == rounds - 1) {
            cp_async_wait_all();   // the next E (tape) before the round that may read it
            __syncwarp();
        }
        const int t = rd * 32 + lane;
        const double *pa = E, *pb = E;
        int sb = 1, i = 0, j = 0;
        double acc = 0.0;
        double *dst = nullptr;
        if (t < nA) {
            lonly_a_entry(n, rin, kin + t, i, j);
            pa = E + i * ns;
            pb = L + j;
            sb = ns;
            dst = Ln + i * ns + j;
        } else if (t >= b0p && t < ntask) {
            const int e = t - b0p;
            i = (e * inv) >> 16;
            j = e - i * n;
            pa = L + i * ns;
            pb = E + j * ns;
            acc = Ln[i * ns + j];
            dst = Ln + i * ns + j;
        } else if (fill && t >= ntask) {
            lonly_a_entry(n, rem, t - ntask, i, j);    // next squaring's A task
            pa = En + i * ns;
            pb = Ln + j;
            sb = ns;
            dst = L + i * ns + j;
        }
        for (int q = 0; q < n - 1; q++) acc = fma(pa[q], pb[q * sb], acc);
        const double res = fma(pa[n - 1], pb[(n - 1) * sb], acc);
        if (dst) *dst = res;
        __syncwarp();
    }
}

template <bool TAPE>
__device__ __forceinline__ void bwd_wpc_body(const BwdArgs &a, const DxConsts &K) {
    extern __shared__ double smem[];
    const int n = a.N + 1, N = a.N, ns = dx_stride(n);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n_hp = n * (n + 1) / 2 - 1;
    const int nn = n * n;

    unsigned short *od = reinterpret_cast<unsigned short *>(smem + kWarpsPerBlock * bwd_warp_smem_doubles(n));
    unsigned short *hp = od + kPairSlots;
    dx_build_pairs(n, od, hp);
    __syncthreads();

    double *E0 = smem + wib * bwd_warp_smem_doubles(n);
    double *E1 = E0 + n * ns;
    double *L0 = E1 + n * ns;
    double *L1 = L0 + n * ns;
    DxVecs V;
    V.sig = L1 + n * ns;
    V.tau = V.sig + n;
    V.xs = V.tau + n;
    V.ds = V.xs + n;
    double *av = V.ds + n;       // a_d = g_d / sigma, a_3 = -kappa sigma     [4][n]
    double *bv = av + 4 * n;     // 2^-s sigma o v_d, b_3 = sigma             [4][n]
    double *yv0 = bv + 4 * n;    // y_d = F a_d (d < 3), two buffers          [3][n] x 2
    double *yv1 = yv0 + 3 * n;
    double *gg = yv1 + 3 * n;    // g_d                                       [3][n]
    double *wv = gg + 3 * n;     // b_{j+1} a_3 of the current Taylor step    [n]
    int fold_nx = 0, fold_q = 0;
    const bool fold = n >= DX_BWD_FOLD_NMIN && bwd_fold_fits(n, fold_nx, fold_q);

    const long long C = a.C;
    // Each block owns kCellsPerBlock consecutive cells, taken one at a time by
    // its warps from a shared counter (balances cells of different s*).
    __shared__ int next;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    for (int it = 0; it < kCellsPerBlock; it++) {
        int kc = 0;
        if (lane == 0) kc = atomicAdd(&next, 1);
        kc = __shfl_sync(DX_FULL, kc, 0);
        const long long c = (long long)blockIdx.x * kCellsPerBlock + kc;
        if (kc >= kCellsPerBlock || c >= C) break;
        const double rg = a.rho_g[c];
        double rd = 0.0, ts = INFINITY;
        if (lane >= 1 && lane <= N) {
            rd = a.rho_d[(long long)(lane - 1) * C + c];
            ts = a.t_s[(long long)(lane - 1) * C + c];
        }
        double vin[3] = {0.0, 0.0, 0.0}, gin[3] = {0.0, 0.0, 0.0};
        if (lane < n) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                vin[d] = a.v_in[((long long)d * n + lane) * C + c];
                gin[d] = a.g_out[((long long)d * n + lane) * C + c];
            }
        }
        DxLane L;
        if (!dx_wpc_setup(lane, N, rg, rd, ts, a.dt, K, V, L)) {
            if (a.g_vin && lane < n)
                for (int d = 0; d < 3; d++) a.g_vin[((long long)d * n + lane) * C + c] = NAN;
            if (lane >= 1 && lane <= N) {
                if (a.g_rho_d) a.g_rho_d[(long long)(lane - 1) * C + c] = NAN;
                if (a.g_ts) a.g_ts[(long long)(lane - 1) * C + c] = NAN;
            }
            if (lane == 0) {
                if (a.g_rho_g) a.g_rho_g[c] = NAN;
                atomicOr(a.status, DRAG_STATUS_BAD_CELL);
            }
            continue;
        }
        const int m = K.mk[L.k];
        // Taped cell: E_0 .. E_{s-2} come from the forward's tape, so neither
        // the Taylor polynomial F nor the products E^2 before the last two
        // squarings are formed here (E_0 streams in during the Taylor step).
        bool taped = false;
        const double *tcell = nullptr;
        if (TAPE) {
            const long long h = dx_cell_fingerprint(lane, N, rg, rd, ts, a.dt, dx_tape_salt(a.levels, n));
            long long stored = 0;
            if (lane == 0) stored = a.thdr[c];
            stored = __shfl_sync(DX_FULL, stored, 0);
            taped = stored == h && dx_tape_levels(L.s) <= a.levels;
            tcell = a.tm + (size_t)c * a.levels * a.P;
            if (taped) tape_load(lane, n, ns, hp, tcell, E0);
        }
        {
            // rank-3 direction and its stationary block (kappa)
            double ad[3], bd[3], sa[3], sb[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                ad[d] = lane < n ? gin[d] * L.tu : 0.0;
                bd[d] = lane < n ? dx_scale2(L.sg * vin[d], L.s) : 0.0;
                sa[d] = L.sg * ad[d];
                sb[d] = L.sg * bd[d];
            }
            double ss = lane < n ? L.sg * L.sg : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ss += __shfl_xor_sync(DX_FULL, ss, o);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    sa[d] += __shfl_xor_sync(DX_FULL, sa[d], o);
                    sb[d] += __shfl_xor_sync(DX_FULL, sb[d], o);
                }
            }
            const double kappa = __ddiv_rn(fma(sa[2], sb[2], fma(sa[1], sb[1], sa[0] * sb[0])), ss * ss);
            if (lane < n) {
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    av[d * n + lane] = ad[d];
                    bv[d * n + lane] = bd[d];
                    gg[d * n + lane] = gin[d];
                }
                av[3 * n + lane] = -kappa * L.sg;
                bv[3 * n + lane] = L.sg;
            }
        }

        // ---- Taylor and its derivative: F = b_m X + b_{m-1} I, dF = b_m H,
        // y_d = F a_d
        double *F = E0, *Fn = E1, *dF = L0, *dFn = L1, *y = yv0, *yn = yv1;
        if (!taped) dx_wpc_taylor_init(lane, n, ns, m, K, V, F);
        for (int t = lane; t < nn; t += 32) {
            const int i = t / n, j = t - i * n;
            double acc = av[i] * bv[j];
#pragma unroll
            for (int d = 1; d < kRank; d++) acc = fma(av[d * n + i], bv[d * n + j], acc);
            dF[i * ns + j] = K.b[m] * acc;
        }
        bwd_xvec(lane, n, V, K.b[m], K.b[m - 1], av, av, y);
        __syncwarp();
        for (int jb = m - 2; jb >= 0; jb--) {
            // F_jb = F X + b_jb I (Horner), dF_jb = dF X + F H with
            // F H = sum_d (F a_d) b_d^T: F a_d = y_d for d < 3 and, as F is a
            // polynomial in X with constant term b_{jb+1} and X sigma = 0,
            // F a_3 = b_{jb+1} a_3. Finally y_d <- F_jb a_d = X y_d + b_jb a_d
            // (F_jb = X F + b_jb I: polynomials in X commute with X).
            if (!taped) dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, K.b[jb], F, Fn);
            if (lane < n) wv[lane] = K.b[jb + 1] * av[3 * n + lane];   // F a_3 = b_{jb+1} a_3
            __syncwarp();
            // columns j >= 1 (6 FMAs each: X has two nonzeros per column there),
            // then column 0 (n + 4 FMAs) together with y' = X y + b_jb a
            for (int t = lane; t < n * (n - 1); t += 32) {
                const int i = t / (n - 1), j = t - i * (n - 1) + 1;
                double acc = y[i] * bv[j];
                acc = fma(y[n + i], bv[n + j], acc);
                acc = fma(y[2 * n + i], bv[2 * n + j], acc);
                acc = fma(wv[i], bv[3 * n + j], acc);
                acc = fma(dF[i * ns], V.xs[j], acc);
                acc = fma(dF[i * ns + j], V.ds[j], acc);
                dFn[i * ns + j] = acc;
            }
            if (fold) {
                bwd_col0_and_y(lane, n, ns, fold_nx, fold_q, V, K.b[jb], av, bv, wv, y, dF, dFn, yn);
            } else {
                for (int i = lane; i < n; i += 32) {
                    double acc = y[i] * bv[0];
                    acc = fma(y[n + i], bv[n], acc);
                    acc = fma(y[2 * n + i], bv[2 * n], acc);
                    acc = fma(wv[i], bv[3 * n], acc);
                    const double *ri = dF + i * ns;
                    for (int k = 0; k < n; k++) acc = fma(ri[k], V.xs[k], acc);
                    dFn[i * ns] = acc;
                }
                bwd_xvec(lane, n, V, 1.0, K.b[jb], av, y, yn);
            }
            __syncwarp();
            double *t1 = F; F = Fn; Fn = t1;
            double *t2 = dF; dF = dFn; dFn = t2;
            double *t3 = y; y = yn; yn = t3;
        }
        if (taped) {
            F = E0;
            Fn = E1;
            cp_async_wait_all();
        } else {
            dx_wpc_restore(lane, n, ns, V, F);
        }
        __syncwarp();

        // ---- squarings: (E, L) <- (E^2, E L + L E); the last one only forms
        // the entries of L the gradients read and leaves E at E_{s-1}. Taped,
        // E_{sq+1} is loaded while the squaring forms L whenever the tape holds it.
        int ka = 0, ra = 0;   // A tasks of the next L-only squaring already run, and their order
        for (int sq = 0; sq < L.s; sq++) {
            const bool trimmed = sq == L.s - 1;
            const bool lonly = taped && sq + 1 < dx_tape_levels(L.s);
            if (lonly) {
                tape_load(lane, n, ns, hp, tcell + (size_t)(sq + 1) * a.P, Fn);
                const bool carry = sq + 2 < dx_tape_levels(L.s);   // the next squaring is L-only too
                bwd_square_lonly(lane, n, ns, F, dF, Fn, dFn, ka, ra, carry, ka, ra);
            } else {
                bwd_square(lane, n, ns, od, V, F, dF, Fn, dFn, trimmed ? kSqTrimmed : kSqFull);
                ka = ra = 0;
            }
            if (!trimmed) {
                double *t1 = F; F = Fn; Fn = t1;
            }
            double *t2 = dF; dF = dFn; dFn = t2;
        }

        // ---- outputs
        if (a.g_vin) {
            // P^T g with P^T = D_sigma E D_sigma^-1: (P^T g)_i = E_ii g_i +
            // sigma_i sum_{j != i} E_ij a_j, a = g / sigma. After s >= 1
            // squarings E holds E_{s-1} and P^T = (D_sigma E D_sigma^-1)^2:
            // two applications, the first into (yv0, yv1) = (g', g' / sigma).
            const int napply = L.s >= 1 ? 2 : 1;
            for (int ap = 0; ap < napply; ap++) {
                const bool last = ap == napply - 1;
                const double *cg = ap == 0 ? gg : yv0, *ca = ap == 0 ? av : yv1;
                for (int t = lane; t < 3 * n; t += 32) {
                    const int d = t >= n ? (t >= 2 * n ? 2 : 1) : 0;
                    const int i = t - d * n;
                    const double *adv = ca + d * n;
                    double acc = 0.0;
                    for (int q = 0; q < n - 1; q++) {
                        const int k = q + (q >= i);
                        acc = fma(F[i * ns + k], adv[k], acc);
                    }
                    const double out = fma(V.sig[i], acc, F[i * ns + i] * cg[d * n + i]);
                    if (last) {
                        a.g_vin[((long long)d * n + i) * C + c] = out;
                    } else {
                        yv0[d * n + i] = out;
                        yv1[d * n + i] = V.tau[i] * out;
                    }
                }
                __syncwarp();
            }
        }
        double geps = 0.0;
        if (lane >= 1 && lane <= N) {
            const int i = lane;
            const double z00 = dF[0], z0i = dF[i] * L.tu, zi0 = L.sg * dF[i * ns], zii = dF[i * ns + i];
            const double d0 = z0i - z00;
            geps = L.alpha * a.dt * d0;
            const double galpha = a.dt * fma(L.eps, d0, zi0 - zii);
            if (a.g_rho_d) a.g_rho_d[(long long)(i - 1) * C + c] = __ddiv_rn(geps, rg);
            if (a.g_ts) a.g_ts[(long long)(i - 1) * C + c] = -galpha * (L.alpha * L.alpha);
        }
        if (a.g_rho_g) {
            double part = L.eps * geps;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(DX_FULL, part, o);
            if (lane == 0) a.g_rho_g[c] = -__ddiv_rn(part, rg);
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4)
dx_backward_wpc(BwdArgs a, DxConsts K) {
    bwd_wpc_body<false>(a, K);
}

// The same adjoint, reading E_0 .. E_{s-2} from the forward's tape where the
// cell's fingerprint matches.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4)
dx_backward_wpc_taped(BwdArgs a, DxConsts K) {
    bwd_wpc_body<true>(a, K);
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

size_t bwd_smem_bytes(int n) {
    return sizeof(double) * (size_t)kWarpsPerBlock * bwd_warp_smem_doubles(n) + 2 * kPairSlots * sizeof(unsigned short);
}

}  // namespace

static int backward_impl(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                         const double *t_s, double dt, const double *v_in, const double *grad_v_out,
                         double *grad_v_in, double *grad_rho_g, double *grad_rho_d, double *grad_t_s, int32_t levels,
                         const void *tape, size_t tape_bytes, bool taped, cudaStream_t stream) {
    if (ncells < 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX || !(dt >= 0.0) || !std::isfinite(dt))
        return DRAG_EINVAL_SIZE;
    if (taped && (levels < 1 || levels > DRAG_TAPE_MAX_LEVELS)) return DRAG_EINVAL_SIZE;
    if (ncells == 0) return DRAG_OK;
    if (!rho_g || !rho_d || !t_s || !v_in || !grad_v_out) return DRAG_ENULL;
    if (taped && !tape) return DRAG_ENULL;
    const void *ptrs[] = {rho_g, rho_d, t_s, v_in, grad_v_out, grad_v_in, grad_rho_g, grad_rho_d, grad_t_s};
    for (const void *p : ptrs)
        if (p && !aligned8(p)) return DRAG_EALIGN;
    if (taped && (reinterpret_cast<uintptr_t>(tape) & 255) != 0) return DRAG_EALIGN;
    if (taped && tape_bytes < drag_expm_tape_bytes(ncells, nspecies, levels)) return DRAG_EWORKSPACE;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    if (!dx_once_per_device(1, [] {
            return cudaFuncSetAttribute(dx_backward_wpc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bwd_smem_bytes(DX_NMAXF)) == cudaSuccess &&
                   cudaFuncSetAttribute(dx_backward_wpc_taped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bwd_smem_bytes(DX_NMAXF)) == cudaSuccess;
        }))
        return DRAG_ECUDA;
    const int n = nspecies + 1;
    BwdArgs a{ncells, nspecies, rho_g, rho_d, t_s, v_in, grad_v_out, grad_v_in, grad_rho_g, grad_rho_d, grad_t_s,
              dt, st, nullptr, nullptr, 0, 0};
    if (taped) {
        a.thdr = static_cast<const long long *>(tape);
        a.tm = reinterpret_cast<const double *>(static_cast<const char *>(tape) + dx_tape_hdr_bytes(ncells));
        a.levels = levels;
        a.P = dx_tape_slot(n);
    }
    if (n <= DX_BWD_LPC_NMAX && dx_mode_for(n) != DX_MODE_WPC)
        return dx_launch_backward_lpc(n, ncells, rho_g, rho_d, t_s, dt, v_in, grad_v_out, grad_v_in, grad_rho_g,
                                      grad_rho_d, grad_t_s, st, a.thdr, a.tm, a.levels, a.P, stream);
    const long long grid = (ncells + kCellsPerBlock - 1) / kCellsPerBlock;
    if (taped)
        dx_backward_wpc_taped<<<(unsigned)grid, kWarpsPerBlock * 32, bwd_smem_bytes(n), stream>>>(a, dx_consts());
    else
        dx_backward_wpc<<<(unsigned)grid, kWarpsPerBlock * 32, bwd_smem_bytes(n), stream>>>(a, dx_consts());
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" int drag_expm_backward(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                  const double *t_s, double dt, const double *v_in, const double *grad_v_out,
                                  double *grad_v_in, double *grad_rho_g, double *grad_rho_d, double *grad_t_s,
                                  cudaStream_t stream) {
    return backward_impl(ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, grad_v_out, grad_v_in, grad_rho_g, grad_rho_d,
                         grad_t_s, 0, nullptr, 0, false, stream);
}

extern "C" int32_t drag_expm_backward_launches(int64_t ncells, int32_t nspecies) {
    if (ncells <= 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX) return 0;
    const int n = nspecies + 1;
    const bool binned = n <= DX_BWD_LPC_NMAX && dx_mode_for(n) != DX_MODE_WPC &&
                        ncells >= dx_binned_min_cells(n, true) && ncells <= 0x7fffffffLL;
    return binned ? 6 : 1;
}

extern "C" int drag_expm_backward_taped(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                        const double *t_s, double dt, const double *v_in, const double *grad_v_out,
                                        double *grad_v_in, double *grad_rho_g, double *grad_rho_d, double *grad_t_s,
                                        int32_t levels, const void *tape, size_t tape_bytes, cudaStream_t stream) {
    return backward_impl(ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, grad_v_out, grad_v_in, grad_rho_g, grad_rho_d,
                         grad_t_s, levels, tape, tape_bytes, true, stream);
}
