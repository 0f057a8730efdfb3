// Lane-per-cell building block for small matrices (n = N + 1 <= 12).
//
// Each lane owns one cell and runs the whole update serially: set-up and
// Algorithm 2, Horner Taylor in the symmetric arrowhead X, row-sum
// restoration, squarings and the apply (same arithmetic as the warp-per-cell
// path, see dx_wpc.cuh). Every FP64 instruction of a warp then does useful
// work on 32 cells, instead of the n(n-1)/2 or n lanes a warp-per-cell round
// keeps busy. Lanes of one warp run max(m*) Horner steps and max(s*)
// squarings; the batched entry point bins cells by (N, k*, s*) so that the
// lanes of a warp agree.
//
// The symmetric matrix is stored packed (upper triangle, NT = n(n+1)/2
// doubles), double-buffered as F (the current matrix) and G (the next one):
//   DX_LPC_REGS   : F, G and the n-vectors in registers (fully unrolled, n <= 6);
//   DX_LPC_SHARED : all in shared memory, a stride of 32 doubles between
//                   entries so that the 32 lanes of a warp hit 32 banks;
//   DX_LPC_HYBRID : F in registers, G and the n-vectors in shared memory. Half
//                   the shared memory of DX_LPC_SHARED (more warps per SM to
//                   cover FP64 latency) and register operands for every product;
//                   each step ends by copying G back into F.
#pragma once

#include <type_traits>
#include <utility>

#include "dx_common.cuh"
#include "dx_tape.cuh"

enum : int { DX_LPC_REGS = 0, DX_LPC_SHARED = 1, DX_LPC_HYBRID = 2 };

template <int NF>
struct DxPacked {
    static constexpr int NT = NF * (NF + 1) / 2;
    __host__ __device__ static constexpr int at(int i, int j) {
        return i <= j ? i * NF - i * (i - 1) / 2 + (j - i) : j * NF - j * (j - 1) / 2 + (i - j);
    }
};

// Storage of NT values (double, or float on the mixed-precision path) per
// lane: registers or a strided shared-memory slice.
template <int NT, bool SMEM, typename V = double>
struct DxLaneArr;

template <int NT, typename V>
struct DxLaneArr<NT, false, V> {
    V v[NT];
    __device__ __forceinline__ void bind(V *, int) {}
    __device__ __forceinline__ V &operator[](int e) { return v[e]; }
};

template <int NT, typename V>
struct DxLaneArr<NT, true, V> {
    V *p;
    __device__ __forceinline__ void bind(V *base, int lane) { p = base + lane; }
    __device__ __forceinline__ V &operator[](int e) { return p[e * 32]; }
};

// Entry e of a lane array read at its point of use: a register, or for a
// shared-memory slice a load the compiler may not merge with another read of
// the same entry (so it cannot hold a whole matrix in registers to reuse it).
template <int NT, typename V>
__device__ __forceinline__ V dx_lane_ld(DxLaneArr<NT, false, V> &a, int e) { return a.v[e]; }
template <int NT>
__device__ __forceinline__ double dx_lane_ld(DxLaneArr<NT, true, double> &a, int e) {
    double v;
    const unsigned addr = (unsigned)__cvta_generic_to_shared(a.p + e * 32);
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}

// F <- G after a step: copied into registers, or shared-memory slices swapped.
template <int NT, bool GS, typename V>
__device__ __forceinline__ void dx_lane_take(DxLaneArr<NT, false, V> &F, DxLaneArr<NT, GS, V> &G) {
#pragma unroll
    for (int e = 0; e < NT; e++) F.v[e] = G[e];
}
template <int NT, typename V>
__device__ __forceinline__ void dx_lane_take(DxLaneArr<NT, true, V> &F, DxLaneArr<NT, false, V> &G) {
#pragma unroll
    for (int e = 0; e < NT; e++) F[e] = G.v[e];
}
template <int NT, typename V>
__device__ __forceinline__ void dx_lane_take(DxLaneArr<NT, true, V> &F, DxLaneArr<NT, true, V> &G) {
    V *t = F.p;
    F.p = G.p;
    G.p = t;
}

// Element type of a DxLaneArr.
template <class A>
using DxElem = typename std::remove_reference<decltype(std::declval<A &>()[0])>::type;

// ---- per-lane steps shared by the forward and the adjoint (one cell, packed
// symmetric n x n matrices; FA, GA, VA are DxLaneArr types, all of one element
// type T, in which the arithmetic runs). Both sides form the iterates E_t with
// exactly these operations, so a lane-per-cell adjoint that recomputes them
// gets the values the forward's tape holds.

// n = 2 (one dust species), FP64. The symmetric form X of a 2 x 2 generator
// with zero row sums is singular (det X = 0), so Cayley-Hamilton gives
// X^2 = tr(X) X and every polynomial in X is a I + b X. The Horner chain then
// runs on the two coefficients, F X + b_j I = b_j I + (a + tr(X) b) X: one FMA
// a step where the packed product takes six. While the chain runs, the packed
// slots (0,0), (0,1), (1,1) hold a, b and tr(X); dx_lpc_taylor_finish turns
// them into the matrix. The mixed-precision path keeps the matrix Horner.
template <int NF, class FA>
__host__ __device__ constexpr bool dx_lpc_coef_chain() {
    return NF == 2 && std::is_same<DxElem<FA>, double>::value;
}

// F = b_m X + b_{m-1} I for the arrowhead X (xs: row 0, ds: diagonal).
template <int NF, class FA, class VA>
__device__ __forceinline__ void dx_lpc_taylor_init(FA &Fm, VA &xs, VA &ds, double bm_, double bm1_) {
    using P = DxPacked<NF>;
    using T = DxElem<FA>;
    const T bm = (T)bm_, bm1 = (T)bm1_;
    if constexpr (dx_lpc_coef_chain<NF, FA>()) {
        Fm[0] = bm1;
        Fm[1] = bm;
        Fm[2] = xs[0] + ds[1];
    } else {
#pragma unroll
        for (int e = 0; e < P::NT; e++) Fm[e] = T(0);
        Fm[0] = fma(bm, xs[0], bm1);
#pragma unroll
        for (int i = 1; i < NF; i++) {
            Fm[P::at(0, i)] = bm * xs[i];
            Fm[P::at(i, i)] = fma(bm, ds[i], bm1);
        }
    }
}

// One Horner step in X: G = F X + b_j I (F is a polynomial in X, so F X is
// symmetric; entry (i, j), j >= 1, needs F_i0 X_0j + F_ij X_jj).
template <int NF, class FA, class GA, class VA>
__device__ __forceinline__ void dx_lpc_horner_step(FA &Fm, GA &Gm, VA &xs, VA &ds, double bj_) {
    using P = DxPacked<NF>;
    using T = DxElem<FA>;
    const T bj = (T)bj_;
    if constexpr (dx_lpc_coef_chain<NF, FA>()) {
        Gm[0] = bj;
        Gm[1] = fma(Fm[2], Fm[1], Fm[0]);
        Gm[2] = Fm[2];
    } else {
        T g00 = fma(Fm[0], xs[0], bj);
#pragma unroll
        for (int k = 1; k < NF; k++) g00 = fma(Fm[P::at(0, k)], xs[k], g00);
#pragma unroll
        for (int jj = 1; jj < NF; jj++) {
#pragma unroll
            for (int i = 0; i <= jj; i++) {
                T acc = fma(Fm[P::at(i, 0)], xs[jj], i == jj ? bj : T(0));
                Gm[P::at(i, jj)] = fma(Fm[P::at(i, jj)], ds[jj], acc);
            }
        }
        Gm[0] = g00;
    }
}

// Ends the Horner chain: nothing to do for the arrowhead chain; for the n = 2
// coefficient chain, the off-diagonal entry b X_01 (the diagonal, which holds a
// and tr(X) until then, is left to dx_lpc_restore, which every caller runs next).
template <int NF, class FA, class VA>
__device__ __forceinline__ void dx_lpc_taylor_finish(FA &Fm, VA &xs) {
    if constexpr (dx_lpc_coef_chain<NF, FA>()) Fm[1] = Fm[1] * xs[1];
}

// Row-sum restoration E_ii = 1 - tau_i sum_{k != i} E_ik sigma_k (for n = 2
// in FP64, with sigma_0 = tau_0 = 1, the two entries as single FMAs).
template <int NF, class MA, class VA>
__device__ __forceinline__ void dx_lpc_restore(MA &M, VA &sig, VA &tau) {
    using P = DxPacked<NF>;
    using T = DxElem<MA>;
    if constexpr (dx_lpc_coef_chain<NF, MA>()) {
        const T e01 = M[1];
        M[0] = fma(-e01, sig[1], T(1));
        M[2] = fma(-tau[1], e01, T(1));
    } else {
#pragma unroll
        for (int i = 0; i < NF; i++) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < NF; k++)
                if (k != i) acc = fma(M[P::at(i, k)], sig[k], acc);
            M[P::at(i, i)] = fma(-tau[i], acc, T(1));
        }
    }
}

// Off-diagonal entries of G = F^2 (F symmetric); the diagonal comes from dx_lpc_restore.
template <int NF, class FA, class GA>
__device__ __forceinline__ void dx_lpc_square_offdiag(FA &Fm, GA &Gm) {
    using P = DxPacked<NF>;
#pragma unroll
    for (int i = 0; i < NF; i++) {
#pragma unroll
        for (int jj = i + 1; jj < NF; jj++) {
            DxElem<FA> acc = 0;
#pragma unroll
            for (int k = 0; k < NF; k++) acc = fma(Fm[P::at(i, k)], Fm[P::at(jj, k)], acc);
            Gm[P::at(i, jj)] = acc;
        }
    }
}

// FP32 cost proxy of a cell for grouping cells of similar (k*, s*) into warps:
// the 1-norm of A = dt Omega_v in FP32 (its binary exponent tracks s*), as an
// order-preserving bit pattern; non-finite and NaN norms sort last among valid cells.
template <int N>
__device__ __forceinline__ unsigned int dx_lpc_cost_proxy(const double *rgp, const double *rdp, const double *tsp,
                                                          long long stride, double dt) {
    const float rg = (float)*rgp, fdt = (float)dt;
    float col0 = 0.0f, cmax = 0.0f;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const float a = fdt / (float)tsp[i * stride];
        const float ea = a * ((float)rdp[i * stride] / rg);
        col0 += ea + a;
        cmax = fmaxf(cmax, ea + a);
    }
    const float nrm = fmaxf(col0, cmax);
    const unsigned int b = __float_as_uint(nrm);
    return (nrm >= 0.0f && b < 0x7f800000u) ? b : 0x7f800000u;
}

// Orders a tile of rounds x threads consecutive cells starting at base by the
// cost proxy (ties by position): order[rank] = tile index, key: the tile's
// scratch. Cells at or past `end` are padding and sort last; C is the SoA
// stride. Block-wide; ends with a barrier.
template <int N>
__device__ __forceinline__ void dx_lpc_tile_order(long long base, int rounds, int threads, long long end, long long C,
                                                  const double *rho_g, const double *rho_d, const double *t_s,
                                                  double dt, unsigned long long *key, unsigned short *order) {
    const int tile = rounds * threads;
    for (int r = 0; r < rounds; r++) {
        const int e = r * threads + threadIdx.x;
        const long long c = base + e;
        const unsigned int p = c < end ? dx_lpc_cost_proxy<N>(rho_g + c, rho_d + c, t_s + c, C, dt) : 0xffffffffu;
        key[e] = ((unsigned long long)p << 32) | (unsigned int)e;
    }
    __syncthreads();
    // rank sort: position of each key among the tile's distinct keys
    for (int r = 0; r < rounds; r++) {
        const int e = r * threads + threadIdx.x;
        const unsigned long long me = key[e];
        int rank = 0;
        for (int j = 0; j < tile; j++) rank += key[j] < me;
        order[rank] = (unsigned short)e;
    }
    __syncthreads();
}

// Orders the cells [c0, c1) of a block (c1 - c0 <= blockDim.x) by the
// half-octave of the cost proxy: a counting sort over 128 buckets (norms from
// 2^-31 to 2^32; the rest clamped to the end buckets), order[rank] = tile
// index. One shared-memory atomic per cell instead of dx_lpc_tile_order's pass
// over the whole tile; a warp's cells then share s* to within one. The order
// within a bucket follows the atomics' timing, which changes no output (a
// cell's arithmetic does not depend on its lane). hist: 128 words of shared
// memory. Block-wide; ends with a barrier.
template <int N>
__device__ __forceinline__ void dx_lpc_bucket_order(long long c0, long long c1, long long C, const double *rho_g,
                                                    const double *rho_d, const double *t_s, double dt,
                                                    unsigned int *hist, unsigned short *order) {
    constexpr int kBuckets = 128;
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const long long c = c0 + threadIdx.x;
    int bucket = 0;
    unsigned int slot = 0;
    if (c < c1) {
        const int h = (int)(dx_lpc_cost_proxy<N>(rho_g + c, rho_d + c, t_s + c, C, dt) >> 22) - 192;
        bucket = h < 0 ? 0 : (h > kBuckets - 1 ? kBuckets - 1 : h);
        slot = atomicAdd(&hist[bucket], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of the counts, four buckets per lane
        const int l = threadIdx.x;
        const unsigned int v0 = hist[4 * l], v1 = hist[4 * l + 1], v2 = hist[4 * l + 2], v3 = hist[4 * l + 3];
        const unsigned int tot = v0 + v1 + v2 + v3;
        unsigned int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(DX_FULL, incl, o);
            if (l >= o) incl += t;
        }
        const unsigned int ex = incl - tot;
        hist[4 * l] = ex;
        hist[4 * l + 1] = ex + v0;
        hist[4 * l + 2] = ex + v0 + v1;
        hist[4 * l + 3] = ex + v0 + v1 + v2;
    }
    __syncthreads();
    if (c < c1) order[hist[bucket] + slot] = (unsigned short)threadIdx.x;
    __syncthreads();
}

// Tile position of this thread's cell in round r of a multi-round tile. The
// rounds' groups of 32 sorted cells are dealt to the block's warps in snake
// order, warp w taking group w of even rounds and group nw - 1 - w of odd
// ones, so that no warp (and so no SM sub-partition) holds the costliest group
// of every round.
__device__ __forceinline__ int dx_lpc_round_pos(int r, int threads) {
    const int nw = threads >> 5, w = threadIdx.x >> 5;
    return r * threads + 32 * ((r & 1) ? nw - 1 - w : w) + (threadIdx.x & 31);
}

// Per-lane norm of one cell. Loads and validates rho_g, rho_d, t_s (integer
// checks on bit patterns); forms eps_i = rho_d,i / rho_g and alpha_i =
// 1 / t_s,i (Eqs. DragEqVar2, DragEqVar3) and the 1-norm of A = dt Omega_v
// summed in ascending species order (as the oracle sums it, so the selection
// is reproducible), returned as its bit pattern nb. s1 = -A_00 = sum_i eps_i
// alpha_i dt. With want_fp, fph is the XOR of the species' fingerprint terms
// over the raw inputs. Returns false for an invalid cell.
template <int NF>
__device__ __forceinline__ bool dx_lpc_norm_cell(const double *rgp, const double *rdp, const double *tsp,
                                                 long long stride, double dt, bool want_fp, double &rg,
                                                 double (&eps)[NF - 1], double (&alpha)[NF - 1],
                                                 unsigned long long &fph, double &s1, long long &nb) {
    constexpr int N = NF - 1;
    rg = *rgp;
    bool ok = dx_pos_finite(rg);
    fph = 0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const double rd = rdp[i * stride], ts = tsp[i * stride];
        ok = ok && dx_nonneg_finite(rd) && dx_pos_or_inf(ts);
        if (want_fp) fph ^= dx_fingerprint_term(i + 1, rd, ts);
        eps[i] = rd;
        alpha[i] = ts;
    }
    if (!ok) return false;
    s1 = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        eps[i] = __ddiv_rn(eps[i], rg);      // Eq. DragEqVar2
        alpha[i] = __drcp_rn(alpha[i]);       // Eq. DragEqVar3
        s1 = __dadd_rn(s1, __dmul_rn(__dmul_rn(eps[i], alpha[i]), dt));
    }
    double col0 = s1;
    long long cmax = 0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const double ai0 = __dmul_rn(alpha[i], dt);
        col0 = __dadd_rn(col0, ai0);
        const long long cb = dx_bits(__dadd_rn(__dmul_rn(__dmul_rn(eps[i], alpha[i]), dt), ai0));
        cmax = cb > cmax ? cb : cmax;
    }
    nb = dx_bits(col0) > cmax ? dx_bits(col0) : cmax;
    return dx_norm_ok(nb);
}

// dx_lpc_norm_cell, then Algorithm 2 on the norm: (k*, s*).
template <int NF>
__device__ __forceinline__ bool dx_lpc_select_cell(const double *rgp, const double *rdp, const double *tsp,
                                                   long long stride, double dt, const DxConsts &K, bool want_fp,
                                                   double &rg, double (&eps)[NF - 1], double (&alpha)[NF - 1],
                                                   int &kk, int &s, unsigned long long &fph, double &s1) {
    long long nb;
    if (!dx_lpc_norm_cell<NF>(rgp, rdp, tsp, stride, dt, want_fp, rg, eps, alpha, fph, s1, nb)) return false;
    dx_select(__longlong_as_double(nb), K, kk, s);
    return true;
}

// The scaled symmetric arrowhead X = 2^-s* D_sigma A D_sigma^-1 of a selected
// cell (sig, tau: sigma and 1 / sigma; xs: row 0; ds: the diagonal).
// Dust-to-gas ratios below eps_floor are raised to it in the symmetric form.
template <int NF, class VA>
__device__ __forceinline__ void dx_lpc_arrowhead(const double (&eps)[NF - 1], const double (&alpha)[NF - 1],
                                                 double dt, int s, double s1, VA &sig, VA &tau, VA &xs, VA &ds,
                                                 double eps_floor) {
    sig[0] = 1.0;
    tau[0] = 1.0;
    xs[0] = dx_scale2(-s1, s);
    ds[0] = 0.0;
#pragma unroll
    for (int i = 1; i < NF; i++) {
        const double e = dx_bits(eps[i - 1]) < dx_bits(eps_floor) ? eps_floor : eps[i - 1];
        // 1/sigma to within an ulp and sigma = eps / sqrt(eps) from it: the
        // similarity only needs sigma and 1/sigma used consistently, and the
        // adjoint forms them by this same routine
        const double tu = rsqrt(e);
        const double sg = __dmul_rn(e, tu);
        sig[i] = sg;
        tau[i] = tu;
        xs[i] = __dmul_rn(__dmul_rn(sg, alpha[i - 1]), dx_scale2(dt, s));
        ds[i] = -dx_scale2(__dmul_rn(alpha[i - 1], dt), s);
    }
}

// Per-lane set-up of one cell: dx_lpc_select_cell, then the symmetric
// arrowhead X (dx_lpc_arrowhead). Returns false for an invalid cell, before
// writing the vectors.
template <int NF, class VA>
__device__ __forceinline__ bool dx_lpc_setup(const double *rgp, const double *rdp, const double *tsp, long long stride,
                                             double dt, const DxConsts &K, bool want_fp, double &rg,
                                             double (&eps)[NF - 1], double (&alpha)[NF - 1], int &kk, int &s,
                                             unsigned long long &fph, VA &sig, VA &tau, VA &xs, VA &ds,
                                             double eps_floor = DX_EPS_FLOOR) {
    double s1;
    if (!dx_lpc_select_cell<NF>(rgp, rdp, tsp, stride, dt, K, want_fp, rg, eps, alpha, kk, s, fph, s1)) return false;
    dx_lpc_arrowhead<NF>(eps, alpha, dt, s, s1, sig, tau, xs, ds, eps_floor);
    return true;
}

// Shared-memory doubles one warp needs for storage mode ST.
template <int NF, int ST>
__host__ __device__ constexpr int dx_lpc_warp_smem_doubles() {
    return ST == DX_LPC_SHARED ? 32 * (2 * DxPacked<NF>::NT + 4 * NF)
                               : (ST == DX_LPC_HYBRID ? 32 * (DxPacked<NF>::NT + 4 * NF) : 0);
}

// Invalid cell: NaN outputs and the status bit.
template <int NF>
__device__ __forceinline__ void dx_lpc_fail_cell(double *vop, long long stride, double *heat, uint32_t *status) {
#pragma unroll
    for (int e = 0; e < 3 * NF; e++) vop[e * stride] = NAN;
    if (heat) *heat = NAN;
    atomicOr(status, DRAG_STATUS_BAD_CELL);
}

// Writes the cell's tape fingerprint (complemented when its s* - 1 levels do
// not fit) and returns where its levels go, or null.
template <int NF>
__device__ __forceinline__ double *dx_lpc_tape_begin(const DxTapeCell &tp, unsigned long long fph, double rg,
                                                     double dt, int s) {
    if (!tp.hdr) return nullptr;
    const long long h = dx_fingerprint_final(fph, rg, dt, dx_tape_salt(tp.levels, NF));
    const bool fits = dx_tape_levels(s) <= tp.levels;
    *tp.hdr = fits ? h : ~h;
    return fits ? tp.m : nullptr;
}

// The restored iterates of one cell in the symmetric form: the Taylor step
// F = b_m X + b_{m-1} I, F <- F X + b_j I (Horner in X), the restoration
// E_ii = 1 - tau_i sum_{k != i} E_ik sigma_k, then s squarings, each restored.
// Leaves E_s in Fm. tape (may be null): E_0 .. E_{tlev-1} stored at tape + t P.
template <int NF, class FA, class GA, class VA>
__device__ __forceinline__ void dx_lpc_chain(FA &Fm, GA &Gm, VA &sig, VA &tau, VA &xs, VA &ds, int m, int s,
                                             const double *bsh, double *tape, int tlev, int P) {
    constexpr int NT = DxPacked<NF>::NT;
    dx_lpc_taylor_init<NF>(Fm, xs, ds, bsh[m], bsh[m - 1]);
    for (int j = m - 2; j >= 0; j--) {
        dx_lpc_horner_step<NF>(Fm, Gm, xs, ds, bsh[j]);
        dx_lane_take(Fm, Gm);
    }
    dx_lpc_taylor_finish<NF>(Fm, xs);
    dx_lpc_restore<NF>(Fm, sig, tau);
    if (tape) {
#pragma unroll
        for (int e = 0; e < NT; e++) tape[e] = Fm[e];
    }
    for (int it = 0; it < s; it++) {
        dx_lpc_square_offdiag<NF>(Fm, Gm);
        dx_lpc_restore<NF>(Gm, sig, tau);
        if (tape && it + 1 < tlev) {
            double *lv = tape + (size_t)(it + 1) * P;
#pragma unroll
            for (int e = 0; e < NT; e++) lv[e] = Gm[e];
        }
        dx_lane_take(Fm, Gm);
    }
}

// One cell of n = 2 (one dust species) in the velocity form. The propagator
// of a 2 x 2 generator with zero row sums is P = I + W, W = [[-p, p], [q, -q]],
// so the pair (p, q) carries the whole update. For X = 2^-s* A, with
// x = X_01 and y = X_10, X^2 = -(x + y) X, so the Taylor polynomial is I + b X
// with b = sum_{k=1..m} b_k (-(x + y))^(k-1) (Horner, one FMA a degree), and a
// squaring maps W to 2 W + W^2 = (2 - p - q) W. Rows sum to one by
// construction, and no square root is needed: the symmetric form is formed
// only when the adjoint tape is written, by the symmetric steps the
// lane-per-cell adjoint recomputes (dx_lpc_chain), so that taped and recomputed
// gradients stay bit-identical. The outputs are v_0 + p (v_1 - v_0) and
// v_1 - q (v_1 - v_0).
__device__ __forceinline__ void dx_lpc2_forward_cell(const double *rgp, const double *rdp, const double *tsp,
                                                     const double *vip, double *vop, long long stride, double dt,
                                                     const DxConsts &K, const double *bsh, uint32_t *status,
                                                     double *heat, const DxTapeCell &tp) {
    double rg, eps[1], alpha[1], s1;
    int kk, s;
    unsigned long long fph;
    if (!dx_lpc_select_cell<2>(rgp, rdp, tsp, stride, dt, K, tp.hdr != nullptr, rg, eps, alpha, kk, s, fph, s1)) {
        dx_lpc_fail_cell<2>(vop, stride, heat, status);
        return;
    }
    const int m = K.mk[kk];
    double *tape = dx_lpc_tape_begin<2>(tp, fph, rg, dt, s);
    if (tape) {
        DxLaneArr<2, false> sig, tau, xs, ds;
        DxLaneArr<3, false> Fm, Gm;
        dx_lpc_arrowhead<2>(eps, alpha, dt, s, s1, sig, tau, xs, ds, DX_EPS_FLOOR);
        dx_lpc_chain<2>(Fm, Gm, sig, tau, xs, ds, m, s, bsh, tape, dx_tape_levels(s), tp.P);
    }
    const double x = dx_scale2(s1, s), y = dx_scale2(__dmul_rn(alpha[0], dt), s);
    const double tr = -(x + y);
    double b = bsh[m];
    for (int k = m - 1; k >= 1; k--) b = fma(tr, b, bsh[k]);
    double p = b * x, q = b * y;
    for (int it = 0; it < s; it++) {
        const double u = 2.0 - (p + q);
        p *= u;
        q *= u;
    }
    double rd = 0.0, mass = 0.0, hsum = 0.0;
    if (heat) {
        rd = *rdp;
        mass = rg + rd;
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double v0 = vip[(2 * d) * stride], v1 = vip[(2 * d + 1) * stride];
        const double dv = v1 - v0;
        const double o0 = fma(p, dv, v0), o1 = fma(-q, dv, v1);
        vop[(2 * d) * stride] = o0;
        vop[(2 * d + 1) * stride] = o1;
        if (heat) {
            const double vc = __ddiv_rn(fma(rd, v1, rg * v0), mass);
            const double a0 = v0 - vc, b0 = o0 - vc, a1 = v1 - vc, b1 = o1 - vc;
            hsum = fma(0.5 * rg, (a0 - b0) * (a0 + b0), hsum);
            hsum = fma(0.5 * rd, (a1 - b1) * (a1 + b1), hsum);
        }
    }
    if (heat) *heat = hsum;
}

// One cell per lane. Pointers address this cell; element (i) of a per-species
// array is at p[i * stride]; velocity (d, f) at p[(d * NF + f) * stride].
// smem_warp: this warp's slice (ST != DX_LPC_REGS); bsh: b_i = 1/i! in shared memory.
// tp (tp.hdr null: none): the cell's adjoint tape, written as by the warp-per-cell
// forward (the packed order here is the tape's): E_0 .. E_{s-2} when they fit,
// the fingerprint word always. n = 2 takes the velocity form (dx_lpc2_forward_cell).
template <int NF, int ST>
__device__ __forceinline__ void dx_lpc_forward_cell(int lane, const double *rgp, const double *rdp, const double *tsp,
                                                    const double *vip, double *vop, long long stride, double dt,
                                                    const DxConsts &K, const double *bsh, double *smem_warp,
                                                    uint32_t *status, double *heat = nullptr,
                                                    DxTapeCell tp = DxTapeCell{nullptr, nullptr, 0, 0}) {
    if constexpr (NF == 2) {
        dx_lpc2_forward_cell(rgp, rdp, tsp, vip, vop, stride, dt, K, bsh, status, heat, tp);
        return;
    }
    constexpr int N = NF - 1;
    constexpr int NT = DxPacked<NF>::NT;
    using P = DxPacked<NF>;

    // ---------------- set-up, Algorithm 2 and the scaled symmetric arrowhead X
    constexpr bool kSharedF = ST == DX_LPC_SHARED, kSharedG = ST != DX_LPC_REGS;
    DxLaneArr<NF, kSharedG> sig, tau, xs, ds;
    DxLaneArr<NT, kSharedF> Fm;
    DxLaneArr<NT, kSharedG> Gm;
    if constexpr (kSharedG) {
        constexpr int f = kSharedF ? 32 * NT : 0;   // F's slice, then G's, then the vectors
        if constexpr (kSharedF) Fm.bind(smem_warp, lane);
        Gm.bind(smem_warp + f, lane);
        sig.bind(smem_warp + f + 32 * NT, lane);
        tau.bind(smem_warp + f + 32 * NT + 32 * NF, lane);
        xs.bind(smem_warp + f + 32 * NT + 64 * NF, lane);
        ds.bind(smem_warp + f + 32 * NT + 96 * NF, lane);
    }
    double rg, eps[N], alpha[N];
    int kk, s;
    unsigned long long fph;   // fingerprint of the raw inputs (tape)
    if (!dx_lpc_setup<NF>(rgp, rdp, tsp, stride, dt, K, tp.hdr != nullptr, rg, eps, alpha, kk, s, fph, sig, tau, xs,
                          ds)) {
        dx_lpc_fail_cell<NF>(vop, stride, heat, status);
        return;
    }
    const int m = K.mk[kk];
    double *tape = dx_lpc_tape_begin<NF>(tp, fph, rg, dt, s);

    // ---------------- Taylor, restoration and s squarings
    dx_lpc_chain<NF>(Fm, Gm, sig, tau, xs, ds, m, s, bsh, tape, dx_tape_levels(s), tp.P);

    // ---------------- apply: v_out_i = E_ii v_i + tau_i sum_{k != i} E_ik sigma_k v_k
    double rho[NF];
    double mass = 0.0;
    if (heat) {
        rho[0] = rg;
#pragma unroll
        for (int i = 1; i < NF; i++) rho[i] = rdp[(i - 1) * stride];
#pragma unroll
        for (int f = 0; f < NF; f++) mass += rho[f];
    }
    double hsum = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double v[NF], y[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) {
            v[f] = vip[(d * NF + f) * stride];
            y[f] = sig[f] * v[f];
        }
        double vc = 0.0;
        if (heat) {
#pragma unroll
            for (int f = 0; f < NF; f++) vc = fma(rho[f], v[f], vc);
            vc = __ddiv_rn(vc, mass);
        }
#pragma unroll
        for (int i = 0; i < NF; i++) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NF; k++)
                if (k != i) acc = fma(Fm[P::at(i, k)], y[k], acc);
            const double out = fma(tau[i], acc, Fm[P::at(i, i)] * v[i]);
            vop[(d * NF + i) * stride] = out;
            if (heat) {
                const double a = v[i] - vc, b = out - vc;
                hsum = fma(0.5 * rho[i], (a - b) * (a + b), hsum);
            }
        }
    }
    if (heat) *heat = hsum;
}
