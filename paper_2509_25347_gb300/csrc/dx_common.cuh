// Shared device helpers of libdragexpm (GB300, sm_103a, FP64).
//
// Cost model that shapes every kernel here: on GB300 one warp-wide FP64
// instruction (DFMA/DADD/DMUL/DSETP) occupies an SM sub-partition's FP64 pipe
// for 64 cycles whatever the number of active lanes, while loads, shuffles,
// integer and FP32 instructions issue at one per cycle. So the kernels
//   * count warp-level FP64 instructions, not flops, and keep lanes busy;
//   * do every comparison, scaling decision and bookkeeping with integer ops
//     on the IEEE bit patterns instead of FP64 compares;
//   * exploit the structure of the drag matrix (arrowhead, symmetrisable,
//     zero row sums) to cut FP64 work.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/drag_expm.h"

#define DX_K 9            // Table B.1 rows (K = 9, m_k up to 30)
#define DX_NMAXF 32       // largest matrix (fluids) handled: n = N + 1 <= 32
#define DX_FULL 0xffffffffu

// Constants passed by value to every kernel (kernel-parameter space).
struct DxConsts {
    long long th[DX_K + 1];    // bit patterns of theta_{m_k} (Eq. B8), k = 1..9
    long long th2[DX_K + 1];   // 2 theta_{m_k}
    long long th4[DX_K + 1];   // 4 theta_{m_k}
    double b[32];              // Taylor coefficients b_i = 1/i!, i = 0..31
    int mk[DX_K + 1];          // m_k of Table B.1
    int qk[DX_K + 1];          // q_k, r_k of Table B.1 (m_k = q_k r_k; the bound test's blocks)
    int rk[DX_K + 1];
    double u;                  // unit round-off the theta tables were made for
};

// Pade variant (Eq. PadeEqu, diagonal [m/m] approximants).
#define DX_PADE_NM 5
struct DxPade {
    long long th[DX_PADE_NM];      // bit patterns of theta_m, m = 3, 5, 7, 9, 13
    int m[DX_PADE_NM];
    double c[DX_PADE_NM][14];      // N_mm(x) = sum_j c_j x^j, D_mm(x) = N_mm(-x)
};

// Host side (dx_host.cu)
const DxConsts &dx_consts();
// Tables for unit round-off u = 2^-ubits, ubits in {53, 24, 11}; nullptr otherwise.
const DxConsts *dx_consts_for(int ubits);
// Pade tables for u = 2^-ubits, ubits in {53, 24}; nullptr otherwise.
const DxPade *dx_pade_for(int ubits);
uint32_t *dx_status_ptr();     // device address of the sticky status word (current device)
int dx_sm_count();
// Runs fn() once per (device, slot); returns false if it failed (it is retried next time).
bool dx_once_per_device(int slot, bool (*fn)());

#define DX_EPS_FLOOR 1e-200    // dust-to-gas ratios below this are raised to it in the symmetric form

// ---------------------------------------------------------------- bit helpers
__device__ __forceinline__ long long dx_bits(double x) { return __double_as_longlong(x); }

// Non-negative, finite (also accepts -0.0).
__device__ __forceinline__ bool dx_nonneg_finite(double x) {
    long long b = dx_bits(x);
    return (b & 0x7fffffffffffffffLL) == 0 || (b > 0 && b < 0x7ff0000000000000LL);
}
// Strictly positive and finite.
__device__ __forceinline__ bool dx_pos_finite(double x) {
    long long b = dx_bits(x);
    return b > 0 && b < 0x7ff0000000000000LL;
}
// Strictly positive, +inf allowed (stopping times).
__device__ __forceinline__ bool dx_pos_or_inf(double x) {
    long long b = dx_bits(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}

// Algorithm 2 (K = 9) on the 1-norm of A = dt Omega_v, with integer compares of
// bit patterns (valid for non-negative finite doubles). Readings of the
// listing: s^ is the smallest s >= 0 with 2^-s |A| <= theta_{m_K}; s* starts at
// s^; k^ is the first k with |A| <= theta_{m_k} (K if none); the reductions
// apply only when v > 0, with v3 before v2 before v1 (the listing's max()).
__device__ __forceinline__ void dx_select(double norm, const DxConsts &K, int &kstar, int &sstar) {
    const long long nb = dx_bits(norm);
    const long long thK = K.th[DX_K];
    int shat = 0;
    long long cb = nb;
    if (nb > thK) {
        const int en = (int)(nb >> 52), et = (int)(thK >> 52);
        const long long mask = (1LL << 52) - 1;
        shat = en - et + (((nb & mask) > (thK & mask)) ? 1 : 0);
        cb = nb - ((long long)shat << 52);          // |A| 2^-s^ (exact, normal)
    }
    int khat = DX_K;
#pragma unroll
    for (int k = DX_K; k >= 1; k--)
        if (nb <= K.th[k]) khat = k;                // first k with |A| <= theta_{m_k}
    int ks = khat, ss = shat;
    const bool v1 = (khat >= 7) && (cb <= K.th[khat >= 7 ? khat - 1 : 1]);
    const bool v2 = (khat >= 8) && (cb <= K.th2[khat >= 8 ? khat - 2 : 1]);
    const bool v3 = (khat >= 9) && (cb <= K.th4[khat >= 9 ? khat - 3 : 1]);
    if (v3) {
        ks = khat - 3; ss = shat + 2;
    } else if (v2) {
        ks = khat - 2; ss = shat + 1;
    } else if (v1) {
        ks = khat - 1;
    }
    kstar = ks;
    sstar = ss;
}

// Pade degree and scaling: the smallest m in {3, 5, 7, 9} with |A| <= theta_m
// (s = 0), else m = 13 with the smallest s >= 0 such that 2^-s |A| <= theta_13.
// Integer compares of bit patterns; returns the index of m in DxPade::m.
__device__ __forceinline__ void dx_select_pade(double norm, const DxPade &P, int &idx, int &sstar) {
    const long long nb = dx_bits(norm);
    idx = DX_PADE_NM - 1;
#pragma unroll
    for (int i = DX_PADE_NM - 2; i >= 0; i--)
        if (nb <= P.th[i]) idx = i;
    sstar = 0;
    const long long th = P.th[DX_PADE_NM - 1];
    if (idx == DX_PADE_NM - 1 && nb > th) {
        const long long mask = (1LL << 52) - 1;
        sstar = (int)(nb >> 52) - (int)(th >> 52) + (((nb & mask) > (th & mask)) ? 1 : 0);
    }
}

// 2^e as a double for -1022 <= e <= 1023 (exact).
__device__ __forceinline__ double dx_pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// x 2^-s for 0 <= s <= 1100 (Algorithm 2 returns up to ~1025 for norms near the
// top of the double range): through two factors once 2^-s leaves the normal range.
__device__ __forceinline__ double dx_scale2(double x, int s) {
    return s <= 1022 ? x * dx_pow2(-s) : (x * dx_pow2(-1022)) * dx_pow2(-(s - 1022));
}

// A usable 1-norm (finite; the bit pattern of a non-negative double). An
// overflowing norm, e.g. alpha = 1/t_s beyond the double range, makes the
// cell invalid, as in the oracle.
__device__ __forceinline__ bool dx_norm_ok(long long nb) { return nb >= 0 && nb < 0x7ff0000000000000LL; }

__device__ __forceinline__ double dx_shfl(double x, int src) { return __shfl_sync(DX_FULL, x, src); }

__device__ __forceinline__ long long dx_warp_max_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long w = __shfl_xor_sync(DX_FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}
