// Warp-per-cell building blocks shared by the forward and adjoint kernels.
//
// One warp owns one cell. Matrices are n x n (n = N + 1 <= 32), stored row
// major in shared memory with an odd row stride. Work inside a phase is split
// into independent "tasks" (one output entry each) dealt round-robin to the
// 32 lanes; __syncwarp() separates dependent phases.
//
// Symmetric similarity form. With D = diag(rho) and sigma_f = sqrt(rho_f/rho_g)
// (sigma_0 = 1, sigma_i = sqrt(eps_i)), S = D_sigma A D_sigma^-1 is a symmetric
// arrowhead for A = dt Omega_v (velocity form of Eq. jacobian):
//   S_00 = A_00 = -sum_i eps_i alpha_i dt, S_0i = S_i0 = sigma_i alpha_i dt,
//   S_ii = -alpha_i dt,
// S sigma = 0, and E = exp(S) = D_sigma exp(A) D_sigma^-1 is symmetric with
// E sigma = sigma.
#pragma once

#include "dx_common.cuh"
#include "dx_sched_tables.inc"   // generated at build time by sched.py
#include "dx_tape.cuh"

constexpr int kPairSlots = 544;   // >= n(n+1)/2 for n <= 32

// Row stride of the shared-memory matrices: odd, to spread banks.
__host__ __device__ __forceinline__ int dx_stride(int n) { return n | 1; }

// Block-wide pair tables: od[t] = (i<<8)|j, i<j (t < n(n-1)/2);
// hp[t] = (i<<8)|j, i<=j, (i,j) != (0,0) (t < n(n+1)/2 - 1).
__device__ __forceinline__ void dx_build_pairs(int n, unsigned short *od, unsigned short *hp) {
    const int n_od = n * (n - 1) / 2, n_hp = n * (n + 1) / 2 - 1;
    for (int t = threadIdx.x; t < n_od; t += blockDim.x) {
        int i = 0, r = t;
        while (r >= n - 1 - i) { r -= n - 1 - i; i++; }
        od[t] = (unsigned short)((i << 8) | (i + 1 + r));
    }
    for (int t = threadIdx.x; t < n_hp; t += blockDim.x) {
        int i = 0, r = t + 1;
        while (r >= n - i) { r -= n - i; i++; }
        hp[t] = (unsigned short)((i << 8) | (i + r));
    }
}

// Per-cell vectors of the symmetric form, kept in shared memory. T is the
// arithmetic type of the matrix work: double, or float on the mixed-precision
// path (set-up and selection stay FP64 there).
template <typename T>
struct DxVecsT {
    T *sig;   // sigma_f
    T *tau;   // 1 / sigma_f
    T *xs;    // xs[0] = X_00, xs[f] = X_0f (f >= 1)
    T *ds;    // ds[f] = X_ff (f >= 1)
};
using DxVecs = DxVecsT<double>;

// Lane-resident cell quantities after set-up (lane f = fluid f; species i on lane i).
struct DxLane {
    double eps, alpha;   // eps_i, alpha_i on species lanes, 0 elsewhere
    double sg, tu;       // sigma_f, 1/sigma_f on lanes f < n
    int k, s;            // k*, s* (warp uniform)
};

// Set-up of one cell: A = dt Omega_v entries, the 1-norm (summed in ascending
// species order, as the oracle does, so (k*, s*) are reproducible), Algorithm 2
// (or, with a Pade table, the Pade degree and scaling), and the scaled
// symmetric arrowhead X = 2^-s* S. Returns false (warp uniform) when the cell's
// data are invalid.
template <typename T>
__device__ __forceinline__ bool dx_wpc_setup(int lane, int N, double rg, double rd, double ts, double dt,
                                             const DxConsts &K, const DxVecsT<T> &V, DxLane &L,
                                             const DxPade *pade = nullptr) {
    const int n = N + 1;
    const bool okl = (lane == 0 || lane > N) || (dx_nonneg_finite(rd) && dx_pos_or_inf(ts));
    const bool ok = __all_sync(DX_FULL, okl) && dx_pos_finite(rg);
    if (!ok) return false;
    const bool sp = lane >= 1 && lane <= N;
    const double eps = sp ? __ddiv_rn(rd, rg) : 0.0;          // Eq. DragEqVar2
    const double alpha = sp ? __ddiv_rn(1.0, ts) : 0.0;       // Eq. DragEqVar3
    const double a0i = __dmul_rn(__dmul_rn(eps, alpha), dt);  // A_0i
    const double ai0 = __dmul_rn(alpha, dt);                  // A_i0 = -A_ii
    double s1 = 0.0;
    for (int i = 1; i <= N; i++) s1 = __dadd_rn(s1, dx_shfl(a0i, i));
    double col0 = s1;
    for (int i = 1; i <= N; i++) col0 = __dadd_rn(col0, dx_shfl(ai0, i));
    const double colj = sp ? __dadd_rn(a0i, ai0) : 0.0;
    long long nb = dx_warp_max_ll(dx_bits(colj));
    nb = nb > dx_bits(col0) ? nb : dx_bits(col0);
    if (!dx_norm_ok(nb)) return false;                          // warp uniform
    if (pade)
        dx_select_pade(__longlong_as_double(nb), *pade, L.k, L.s);   // L.k: index of the Pade degree
    else
        dx_select(__longlong_as_double(nb), K, L.k, L.s);
    double sg = 1.0, tu = 1.0;
    if (sp) {
        // FP32 work keeps sigma and 1/sigma inside its range: 1e-30 instead of 1e-200
        const double floor_eps = sizeof(T) == sizeof(double) ? DX_EPS_FLOOR : 1e-30;
        const double e = dx_bits(eps) < dx_bits(floor_eps) ? floor_eps : eps;
        sg = __dsqrt_rn(e);
        tu = __ddiv_rn(1.0, sg);
    }
    if (lane < n) {
        V.sig[lane] = (T)sg;
        V.tau[lane] = (T)tu;
        V.xs[lane] = (T)(lane == 0 ? dx_scale2(-s1, L.s) : __dmul_rn(__dmul_rn(sg, alpha), dx_scale2(dt, L.s)));
        V.ds[lane] = (T)(-dx_scale2(ai0, L.s));
    }
    L.eps = eps;
    L.alpha = alpha;
    L.sg = sg;
    L.tu = tu;
    __syncwarp();
    return true;
}

// Sizes whose warp-per-cell forward sets up two cells at a time (two half-warps of species lanes).
__host__ __device__ constexpr bool dx_wpc_pairs(int N) { return N <= 16; }

// Set-up of two cells at once, for N <= 16 in FP64: half-warp h (lanes
// 16 h .. 16 h + 15) takes cell h, and its lane 16 h + i - 1 species i. The
// species' divisions and square roots, and the norm's two ascending sums, then
// run for both cells in the same instructions (a warp-wide FP64 instruction
// costs the same with 16 or 32 lanes working). Every value is formed by the
// operations dx_wpc_setup uses, in the same order, so the results are the same
// bits. rg, dt: this half's cell; rd, ts: this lane's species (anything past N).
// Writes cell h's vectors (sigma, tau, X_0f, X_ff; fluid f at index f) to V0
// or V1, and (k*, s*) of both cells to (k0, s0), (k1, s1c) on every lane.
// Returns bit h set for a valid cell h.
__device__ __forceinline__ unsigned dx_wpc_setup_pair(int lane, int N, double rg, double rd, double ts, double dt,
                                                      const DxConsts &K, const DxVecs &V0, const DxVecs &V1, int &k0,
                                                      int &s0, int &k1, int &s1c) {
    const int h = lane >> 4, l = lane & 15, base = lane & 16;
    const bool sp = l < N;
    const bool okl = !sp || (dx_nonneg_finite(rd) && dx_pos_or_inf(ts));
    const unsigned bad = __ballot_sync(DX_FULL, !okl);
    bool ok = ((bad >> base) & 0xffffu) == 0 && dx_pos_finite(rg);
    const double eps = sp ? __ddiv_rn(rd, rg) : 0.0;          // Eq. DragEqVar2
    const double alpha = sp ? __ddiv_rn(1.0, ts) : 0.0;       // Eq. DragEqVar3
    const double a0i = __dmul_rn(__dmul_rn(eps, alpha), dt);  // A_0i
    const double ai0 = __dmul_rn(alpha, dt);                  // A_i0 = -A_ii
    double s1 = 0.0;
    for (int i = 0; i < N; i++) s1 = __dadd_rn(s1, dx_shfl(a0i, base + i));
    double col0 = s1;
    for (int i = 0; i < N; i++) col0 = __dadd_rn(col0, dx_shfl(ai0, base + i));
    const double colj = sp ? __dadd_rn(a0i, ai0) : 0.0;
    long long nb = dx_bits(colj);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(DX_FULL, nb, o);
        nb = w > nb ? w : nb;
    }
    nb = nb > dx_bits(col0) ? nb : dx_bits(col0);
    ok = ok && dx_norm_ok(nb);
    int k = 0, s = 0;
    if (ok) dx_select(__longlong_as_double(nb), K, k, s);
    k0 = __shfl_sync(DX_FULL, k, 0);
    s0 = __shfl_sync(DX_FULL, s, 0);
    k1 = __shfl_sync(DX_FULL, k, 16);
    s1c = __shfl_sync(DX_FULL, s, 16);
    const DxVecs V = h ? V1 : V0;
    if (ok) {
        if (sp) {
            const double e = dx_bits(eps) < dx_bits(DX_EPS_FLOOR) ? DX_EPS_FLOOR : eps;
            const double sg = __dsqrt_rn(e);
            V.sig[l + 1] = sg;
            V.tau[l + 1] = __ddiv_rn(1.0, sg);
            V.xs[l + 1] = __dmul_rn(__dmul_rn(sg, alpha), dx_scale2(dt, s));
            V.ds[l + 1] = -dx_scale2(ai0, s);
        }
        if (l == 0) {
            V.sig[0] = 1.0;
            V.tau[0] = 1.0;
            V.xs[0] = dx_scale2(-s1, s);
            V.ds[0] = -dx_scale2(0.0, s);
        }
    }
    const unsigned valid = __ballot_sync(DX_FULL, ok);
    __syncwarp();
    return (valid & 1u) | ((valid >> 16) & 1u) << 1;
}

// F = b_m X + b_{m-1} I (arrowhead), written into a zeroed n x n buffer.
template <typename T>
__device__ __forceinline__ void dx_wpc_taylor_init(int lane, int n, int ns, int m, const DxConsts &K,
                                                   const DxVecsT<T> &V, T *F) {
    for (int t = lane; t < n * ns; t += 32) F[t] = T(0);
    __syncwarp();
    const T bm = (T)K.b[m], bm1 = (T)K.b[m - 1];
    if (lane < n) {
        const T x = V.xs[lane];
        if (lane == 0) {
            F[0] = fma(bm, x, bm1);
        } else {
            F[lane] = F[lane * ns] = bm * x;
            F[lane * ns + lane] = fma(bm, V.ds[lane], bm1);
        }
    }
    __syncwarp();
}

// Lanes given to the dot product G_00 = sum_k F_0k X_k0 + bj in a Horner
// step: a power-of-two group g at the top of the warp, idle in the step's last
// round (32 rounds - n_hp >= g), each lane summing every g-th term, followed
// by log2 g shuffle levels. The group is chosen to minimise the FP64
// instructions the step adds beyond the two of its last round; 0 means the
// plain full-warp reduction (7 instructions) is cheaper.
__host__ __device__ __forceinline__ int dx_horner_g00_group(int n) {
    const int n_hp = n * (n + 1) / 2 - 1;
    const int idle = 32 * ((n_hp + 31) / 32) - n_hp;
    int best = 7, group = 0;
    for (int g = 1, lg = 0; g <= idle; g *= 2, lg++) {
        const int per = (n + g - 1) / g;
        const int cost = (per > 2 ? per - 2 : 0) + lg;
        if (cost < best) {
            best = cost;
            group = g;
        }
    }
    return group;
}

// One Horner step G = F X + bj I (F, G symmetric; X the arrowhead):
//   G_ij = F_i0 X_0j + F_ij X_jj (+ bj if i == j) for i <= j, (i,j) != (0,0),
//   G_00 = sum_k F_0k X_k0 + bj.
template <typename T>
__device__ __forceinline__ void dx_wpc_horner_step(int lane, int n, int ns, int n_hp, const unsigned short *hp,
                                                   const DxVecsT<T> &V, T bj, const T *F, T *G) {
    const int g = dx_horner_g00_group(n);
    if (g == 0) {
        for (int t = lane; t < n_hp; t += 32) {
            const int p = hp[t], i = p >> 8, jj = p & 255;
            T acc = fma(F[i * ns], V.xs[jj], i == jj ? bj : T(0));
            acc = fma(F[i * ns + jj], V.ds[jj], acc);
            G[i * ns + jj] = acc;
            G[jj * ns + i] = acc;
        }
        T part = lane < n ? F[lane] * V.xs[lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(DX_FULL, part, o);
        if (lane == 0) G[0] = part + bj;
        return;
    }
    // Rounds before the last: two FMAs per entry on every lane.
    const int last = (n_hp - 1) >> 5;
    for (int r = 0; r < last; r++) {
        const int p = hp[r * 32 + lane], i = p >> 8, jj = p & 255;
        T acc = fma(F[i * ns], V.xs[jj], i == jj ? bj : T(0));
        acc = fma(F[i * ns + jj], V.ds[jj], acc);
        G[i * ns + jj] = acc;
        G[jj * ns + i] = acc;
    }
    // Last round: the remaining entries, and on the g lanes at the top of the
    // warp the partial sums of G_00 (lane 32 - g + phi takes the terms
    // k = phi, phi + g, ...). Every lane issues the same, warp-uniform number
    // of FMAs, absent terms being 0 * 0.
    const int t = last * 32 + lane;
    const bool task = t < n_hp;
    const int phi = lane - (32 - g);
    const bool grp = !task && phi >= 0;
    const int cmax = (n + g - 1) / g;
    T a0 = T(0), b0 = T(0), a1 = T(0), b1 = T(0), c = T(0);
    int dst = 0, dstT = 0;
    if (task) {
        const int p = hp[t], i = p >> 8, jj = p & 255;
        a0 = F[i * ns];
        b0 = V.xs[jj];
        a1 = F[i * ns + jj];
        b1 = V.ds[jj];
        c = i == jj ? bj : T(0);
        dst = i * ns + jj;
        dstT = jj * ns + i;
    } else if (grp) {
        if (phi < n) {
            a0 = F[phi];
            b0 = V.xs[phi];
        }
        if (phi + g < n) {
            a1 = F[phi + g];
            b1 = V.xs[phi + g];
        }
        c = phi == 0 ? bj : T(0);
    }
    T acc = fma(a0, b0, c);
    acc = fma(a1, b1, acc);
    for (int u = 2; u < cmax; u++) {
        const int k = phi + u * g;
        const bool on = grp && k < n;
        acc = fma(on ? F[on ? k : 0] : T(0), on ? V.xs[on ? k : 0] : T(0), acc);
    }
    if (task) {
        G[dst] = acc;
        G[dstT] = acc;
    }
    for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(DX_FULL, acc, o);
    if (lane == 32 - g) G[0] = acc;
}

// Row-sum restoration in symmetric form: E_ii = 1 - tau_i sum_{k != i} E_ik sigma_k.
template <typename T>
__device__ __forceinline__ void dx_wpc_restore(int lane, int n, int ns, const DxVecsT<T> &V, T *E) {
    if (lane < n) {
        T acc = T(0);
        for (int q = 0; q < n - 1; q++) {
            const int k = q + (q >= lane);
            acc = fma(E[lane * ns + k], V.sig[k], acc);
        }
        E[lane * ns + lane] = fma(-V.tau[lane], acc, T(1));
    }
}

// Row-sum restoration of the starting matrix (t = 0) and s squarings with
// restoration (t = 1..s), run on the round schedule generated by sched.py:
// each round gives every lane one task of n FP64 operations, either an
// off-diagonal dot product of squaring t (i < j, reads E_{t-1}, writes E_t)
// or the restoration of row i of E_t (i == j). Restorations of squaring t
// share rounds with the first products of squaring t + 1 whenever the rows
// those need are complete. Chunks of at most DX_SCHED_H squarings each start
// with a restoration (a no-op on an already restored matrix). The matrix
// starts in B[p0]; returns the index of the buffer holding the result.
// wz (FP32 work only, may be null): an n x ns table whose row i is sigma with
// a zero at i. With it a restoration runs the same plain n-term loop as a
// product (the stale diagonal of the destination is multiplied by an exact 0),
// which costs one more FMA per round but drops the per-term index select that
// dominates instruction issue once the arithmetic is FP32.
// tape (FP64 only, may be null): the lane that computes an entry of E_t also
// stores it at tape[t * tP + dx_tape_index(n, i, j)] (entries of E_0 other than
// its diagonal are the caller's to store).
template <typename T>
__device__ __forceinline__ int dx_wpc_square_chain(int lane, int n, int ns, int s, T *B0, T *B1, int p0,
                                                   const DxVecsT<T> &V, const T *wz = nullptr,
                                                   double *tape = nullptr, int tP = 0) {
    const unsigned short *tab = dx_sched_task + (size_t)dx_sched_off[n] * 32;
    const unsigned short *endr = dx_sched_end + n * (DX_SCHED_H + 1);
    int remaining = s, parity = p0;
    do {
        const int h = remaining < DX_SCHED_H ? remaining : DX_SCHED_H;
        const int lvl0 = s - remaining;   // level of this chunk's starting matrix
        const int nr = endr[h];
        for (int r = 0; r < nr; r++) {
            const unsigned int code = tab[r * 32 + lane];
            const int t = (int)(code >> 10);
            if (code != 0xFFFFu && t <= h) {
                const int i = code & 31, j = (code >> 5) & 31;
                const bool isR = i == j;
                T *dst = (parity ^ (t & 1)) ? B1 : B0;
                const T *src = isR ? dst : ((parity ^ ((t - 1) & 1)) ? B1 : B0);
                const T *pa = src + i * ns;
                T res;
                if (sizeof(T) == sizeof(float) && wz) {
                    const T *pb = isR ? wz + i * ns : src + j * ns;
                    T acc = T(0);
#pragma unroll 4
                    for (int k = 0; k < n; k++) acc = fma(pa[k], pb[k], acc);
                    res = isR ? fma(-V.tau[i], acc, T(1)) : acc;
                } else {
                    const T *pb = isR ? V.sig : src + j * ns;
                    T acc = T(0);
                    for (int q = 0; q < n - 1; q++) {
                        const int k = (isR && q >= i) ? q + 1 : q;
                        acc = fma(pa[k], pb[k], acc);
                    }
                    const T x = isR ? -V.tau[i] : pa[n - 1];
                    const T y = isR ? acc : pb[n - 1];
                    const T z = isR ? T(1) : acc;
                    res = fma(x, y, z);
                }
                if (isR) {
                    dst[i * ns + i] = res;
                } else {
                    dst[i * ns + j] = res;
                    dst[j * ns + i] = res;
                }
                if (sizeof(T) == sizeof(double) && tape)
                    tape[(size_t)(lvl0 + t) * tP + dx_tape_index(n, i, j)] = (double)res;
            }
            __syncwarp();
        }
        parity ^= h & 1;
        remaining -= h;
    } while (remaining > 0);
    return parity;
}

// Warp-cooperative pair tables (one warp builds its own; used when n varies per item).
__device__ __forceinline__ void dx_build_pairs_warp(int lane, int n, unsigned short *od, unsigned short *hp) {
    const int n_od = n * (n - 1) / 2, n_hp = n * (n + 1) / 2 - 1;
    for (int t = lane; t < n_od; t += 32) {
        int i = 0, r = t;
        while (r >= n - 1 - i) { r -= n - 1 - i; i++; }
        od[t] = (unsigned short)((i << 8) | (i + 1 + r));
    }
    for (int t = lane; t < n_hp; t += 32) {
        int i = 0, r = t + 1;
        while (r >= n - i) { r -= n - i; i++; }
        hp[t] = (unsigned short)((i << 8) | (i + r));
    }
    __syncwarp();
}

// Per-warp shared-memory footprint of the forward cell routine (doubles):
// E0, E1, then n-vectors: sigma, tau, X_0f, X_ff, the input velocities (3 of
// them) and two buffers of (v, sigma o v) for the repeated apply (2 x 2 x 3).
__host__ __device__ __forceinline__ int dx_wpc_fwd_warp_doubles(int n) { return 2 * n * dx_stride(n) + 19 * n; }


// Per-cell vectors of the forward routines, laid out from vbase: sigma, tau,
// X_0f, X_ff (4 n), the input velocities (3 n) and two buffers of
// (v, sigma o v) for the repeated applications (12 n): 19 n doubles.
template <typename T>
struct DxFwdBufsT {
    T *v0;          // input velocities v_f, three components
    T *wv0, *wv1;   // current v, two buffers
    T *wy0, *wy1;   // sigma o current v
};
using DxFwdBufs = DxFwdBufsT<double>;

template <typename T>
__device__ __forceinline__ void dx_wpc_fwd_layout(T *vbase, int n, DxVecsT<T> &V, DxFwdBufsT<T> &B) {
    V.sig = vbase;
    V.tau = V.sig + n;
    V.xs = V.tau + n;
    V.ds = V.xs + n;
    B.v0 = V.ds + n;
    B.wv0 = B.v0 + 3 * n;
    B.wy0 = B.v0 + 6 * n;
    B.wv1 = B.v0 + 9 * n;
    B.wy1 = B.v0 + 12 * n;
}

// One cell's inputs on the lanes: lane f holds fluid f (species i on lane i).
struct DxCellIn {
    double rg, rd, ts, vin[3];
};

__device__ __forceinline__ void dx_wpc_load_cell(int lane, int N, const double *rgp, const double *rdp,
                                                 const double *tsp, const double *vip, long long stride,
                                                 DxCellIn &c) {
    const int n = N + 1;
    c.rg = *rgp;
    c.rd = 0.0;
    c.ts = INFINITY;
    if (lane >= 1 && lane <= N) {
        c.rd = rdp[(long long)(lane - 1) * stride];
        c.ts = tsp[(long long)(lane - 1) * stride];
    }
#pragma unroll
    for (int d = 0; d < 3; d++) c.vin[d] = lane < n ? vip[((long long)d * n + lane) * stride] : 0.0;
}

// Invalid cell: NaN outputs and the status bit.
__device__ __forceinline__ void dx_wpc_fail_cell(int lane, int n, double *vop, long long stride, uint32_t *status,
                                                 double *heat) {
    if (lane < n) {
#pragma unroll
        for (int d = 0; d < 3; d++) vop[((long long)d * n + lane) * stride] = NAN;
    }
    if (lane == 0) {
        atomicOr(status, DRAG_STATUS_BAD_CELL);
        if (heat) *heat = NAN;
    }
    __syncwarp();
}

// Apply P^(2^q) (P = D_sigma^-1 F D_sigma, F the restored symmetric form after
// s - q squarings) to the three velocity components and store v_out. heat
// (may be null, warp uniform): the kinetic energy the step dissipates,
// sum_f 1/2 rho_f (|v_in,f - V|^2 - |v_out,f - V|^2) with V the centre-of-mass
// velocity (frictional heating of Eq. GenEq_3, weight w = 1).
template <typename T>
__device__ __forceinline__ void dx_wpc_apply_tail(int lane, int n, int ns, const DxVecsT<T> &V,
                                                  const DxFwdBufsT<T> &B, const T *F, int q, const DxCellIn &c,
                                                  double sg, double *vop, long long stride, double *heat) {
    T *const v0 = B.v0;
    T *const wv0 = B.wv0, *const wv1 = B.wv1, *const wy0 = B.wy0, *const wy1 = B.wy1;
    const double rg = c.rg, rd = c.rd;
    const double *vin = c.vin;
    // v <- P v, 2^q times, P_ii = E_ii, P_ij = E_ij sigma_j / sigma_i (P = D_sigma^-1 E D_sigma):
    // v_i' = E_ii v_i + tau_i sum_{j != i} E_ij sigma_j v_j
    if (lane < n) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            v0[d * n + lane] = (T)vin[d];
            wv0[d * n + lane] = (T)vin[d];
            wy0[d * n + lane] = (T)(sg * vin[d]);
        }
    }
    __syncwarp();
    double vcm[3] = {0.0, 0.0, 0.0};
    if (heat) {
        // centre-of-mass velocity: masses rho_f (lane f), momenta rho_f v_f
        double mass = lane == 0 ? rg : (lane < n ? rd : 0.0);
        double mom[3];
#pragma unroll
        for (int d = 0; d < 3; d++) mom[d] = mass * vin[d];
        if (lane < n) V.ds[lane] = (T)mass;       // X_ff is no longer needed: reuse as the mass table
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mass += __shfl_xor_sync(DX_FULL, mass, o);
#pragma unroll
            for (int d = 0; d < 3; d++) mom[d] += __shfl_xor_sync(DX_FULL, mom[d], o);
        }
        const double inv = __ddiv_rn(1.0, mass);
#pragma unroll
        for (int d = 0; d < 3; d++) vcm[d] = mom[d] * inv;
        __syncwarp();
    }
    const int napply = 1 << q;
    double hsum = 0.0;
    for (int ap = 0; ap < napply; ap++) {
        const bool last = ap == napply - 1;
        const bool odd = ap & 1;
        const T *cv = odd ? wv1 : wv0, *cy = odd ? wy1 : wy0;
        T *nv = odd ? wv0 : wv1, *ny = odd ? wy0 : wy1;
        for (int t = lane; t < 3 * n; t += 32) {
            const int d = t / n, i = t - d * n;
            const T *y = cy + d * n;
            T acc = T(0);
            T out;
            if (sizeof(T) == sizeof(float)) {
                // FP32: the plain form tau_i sum_j E_ij sigma_j v_j (its j = i term is E_ii v_i) as
                // one unmasked loop; FP64 keeps E_ii v_i apart so that dt = 0 returns v_in exactly
#pragma unroll 4
                for (int k = 0; k < n; k++) acc = fma(F[i * ns + k], y[k], acc);
                out = V.tau[i] * acc;
            } else if (!last) {
                // before the last application only sigma o v is carried: (sigma o P v)_i =
                // sum_k E_ik (sigma o v)_k, one n-term sum (v itself is not formed)
                for (int k = 0; k < n; k++) acc = fma(F[i * ns + k], y[k], acc);
                ny[d * n + i] = acc;
                continue;
            } else {
                for (int qq = 0; qq < n - 1; qq++) {
                    const int k = qq + (qq >= i);
                    acc = fma(F[i * ns + k], y[k], acc);
                }
                // v_i: the input itself for a single application (dt = 0 returns v_in exactly),
                // else tau_i (sigma o v)_i of the previous one
                const T vi = ap == 0 ? cv[d * n + i] : V.tau[i] * y[i];
                out = fma(V.tau[i], acc, F[i * ns + i] * vi);
            }
            if (!last) {
                nv[d * n + i] = out;
                ny[d * n + i] = V.sig[i] * out;
                continue;
            }
            vop[((long long)d * n + i) * stride] = (double)out;
            if (heat) {
                const double vc = d == 0 ? vcm[0] : (d == 1 ? vcm[1] : vcm[2]);
                const double a = v0[d * n + i] - vc, b = out - vc;
                hsum = fma(0.5 * V.ds[i], (a - b) * (a + b), hsum);
            }
        }
        __syncwarp();
    }
    if (heat) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(DX_FULL, hsum, o);
        if (lane == 0) *heat = hsum;
    }
    __syncwarp();
}

// The forward of one cell after its set-up (dx_wpc_setup or
// dx_wpc_setup_pair): the Taylor step, s* - q squarings and 2^q applications.
// V: the cell's vectors; E0, E1: the two matrix buffers; B: the apply buffers;
// kk, s: (k*, s*); sg: sigma of this lane's fluid (1 past n); c: the cell's
// inputs on the lanes. tp: see dx_wpc_forward_cell.
template <typename T>
__device__ __forceinline__ void dx_wpc_forward_run(int lane, int N, const DxVecsT<T> &V, T *E0, T *E1,
                                                   const DxFwdBufsT<T> &B, int kk, int s, double sg,
                                                   const DxCellIn &c, double *vop, long long stride, double dt,
                                                   const DxConsts &K, const unsigned short *od,
                                                   const unsigned short *hp, double *heat, T *wz, DxTapeCell tp) {
    const int n = N + 1, ns = dx_stride(n);
    const int n_hp = n * (n + 1) / 2 - 1;
    const int m = K.mk[kk];
    double *tape = nullptr;
    if (sizeof(T) == sizeof(double) && tp.hdr) {
        const long long h = dx_cell_fingerprint(lane, N, c.rg, c.rd, c.ts, dt, dx_tape_salt(tp.levels, n));
        const bool fits = dx_tape_levels(s) <= tp.levels;
        if (lane == 0) *tp.hdr = fits ? h : ~h;
        if (fits) tape = tp.m;
    }

    // Taylor polynomial T_m(X) by Horner's rule in X
    T *F = E0, *G = E1;
    dx_wpc_taylor_init(lane, n, ns, m, K, V, F);
    for (int j = m - 2; j >= 0; j--) {
        dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, (T)K.b[j], F, G);
        __syncwarp();
        T *tmp = F; F = G; G = tmp;
    }

    if (tape) {
        // level 0 off the diagonal (the chain's first restoration stores the diagonal)
        for (int t = lane; t < n * (n - 1) / 2; t += 32) {
            const int p = od[t], i = p >> 8, j = p & 255;
            tape[dx_tape_index(n, i, j)] = (double)F[i * ns + j];
        }
    }

    // row-sum restoration, then s - q squarings (Eq. ExpEq1 with n = 2^s), each
    // restored; the remaining q squarings become 2^q applications
    const int q = s < DX_APPLY_Q ? s : DX_APPLY_Q;
    if (wz) {
        // row i of wz: sigma with a zero at i (restorations as plain n-term loops)
        for (int t = lane; t < n * n; t += 32) {
            const int i = t / n, k = t - i * n;
            wz[i * ns + k] = i == k ? T(0) : V.sig[k];
        }
        __syncwarp();
    }
    F = dx_wpc_square_chain(lane, n, ns, s - q, E0, E1, F == E1 ? 1 : 0, V, wz, tape, tp.P) ? E1 : E0;
    dx_wpc_apply_tail(lane, n, ns, V, B, F, q, c, sg, vop, stride, heat);
}

// Forward update of one cell by one warp (warp-uniform arguments). Element i
// of a per-species array is at p[i * stride]; velocity (d, f) at
// p[(d * n + f) * stride]. od/hp: pair tables for this n. v_out may alias v_in.
// heat: see dx_wpc_apply_tail. tp (FP64 only; tp.hdr null: none): the cell's
// adjoint tape, written when its levels fit (the fingerprint word always).
template <typename T>
__device__ __forceinline__ void dx_wpc_forward_cell(int lane, int N, const double *rgp, const double *rdp,
                                                    const double *tsp, const double *vip, double *vop,
                                                    long long stride, double dt, const DxConsts &K, T *wsm,
                                                    const unsigned short *od, const unsigned short *hp,
                                                    uint32_t *status, double *heat = nullptr, T *wz = nullptr,
                                                    DxTapeCell tp = DxTapeCell{nullptr, nullptr, 0, 0}) {
    const int n = N + 1, ns = dx_stride(n);
    T *E0 = wsm;
    T *E1 = E0 + n * ns;
    DxVecsT<T> V;
    DxFwdBufsT<T> B;
    dx_wpc_fwd_layout(E1 + n * ns, n, V, B);

    DxCellIn c;
    dx_wpc_load_cell(lane, N, rgp, rdp, tsp, vip, stride, c);
    DxLane L;
    if (!dx_wpc_setup(lane, N, c.rg, c.rd, c.ts, dt, K, V, L)) {
        dx_wpc_fail_cell(lane, n, vop, stride, status, heat);
        return;
    }
    dx_wpc_forward_run(lane, N, V, E0, E1, B, L.k, L.s, L.sg, c, vop, stride, dt, K, od, hp, heat, wz, tp);
}
