// Mixed-precision (FP32 matrix work) forward, lane per cell, for n <= 17
// (drag_expm_apply_opts with arith = FP32). Its own translation unit so that
// the build compiles it beside the FP64 lane-per-cell kernels.
#include "dx_lpc.cuh"
#include "dx_modes.h"

namespace {

// Mixed-precision lane-per-cell forward: FP64 loads, set-up and Algorithm 2
// (dx_lpc_setup on the caller's theta table, dust-to-gas ratios floored at
// 1e-30 so that sigma and 1/sigma stay inside the FP32 range), then the Taylor
// step, the restorations, all s* squarings and the apply in FP32. The FP32
// pipe issues 64x faster than the FP64 one on this part. The apply uses the
// plain form v_i' = tau_i sum_j E_ij sigma_j v_j (its j = i term is E_ii v_i).
// Storage: n <= 12 all in registers, one cell per thread, no sorting (the
// FP64 set-up is most of the cost there); n = 13..17 F in registers, G and the
// n-vectors in shared memory (a 32-float stride between entries), one-warp
// blocks that first sort a tile of cells by the cost proxy, since the FP32
// squarings then dominate and a warp runs the largest s* of its 32 cells.
template <int NF>
struct F32Store {
    static constexpr int NT = DxPacked<NF>::NT;
    static constexpr bool kHyb = NF >= 13;
    static constexpr int kThreads = kHyb ? 32 : 128;
    static constexpr int kTile = 256;                              // cells a hybrid block sorts at most
    static constexpr int kWarpFloats = kHyb ? 32 * (NT + 4 * NF) : 0;
};

template <int NF>
__device__ __forceinline__ void f32_cell(int lane, long long c, long long C, const double *rho_g, const double *rho_d,
                                         const double *t_s, const double *v_in, double *v_out, double dt,
                                         uint32_t *status, const DxConsts &K, float *wsm) {
    constexpr int N = NF - 1;
    constexpr int NT = DxPacked<NF>::NT;
    constexpr bool kHyb = F32Store<NF>::kHyb;
    using P = DxPacked<NF>;
    DxLaneArr<NF, false> sgd, tud, xsd, dsd;
    double rg, eps[N], alpha[N];
    int kk, s;
    unsigned long long fph;
    if (!dx_lpc_setup<NF>(rho_g + c, rho_d + c, t_s + c, C, dt, K, false, rg, eps, alpha, kk, s, fph, sgd, tud, xsd,
                          dsd, 1e-30)) {
#pragma unroll
        for (int e = 0; e < 3 * NF; e++) v_out[e * C + c] = NAN;
        atomicOr(status, DRAG_STATUS_BAD_CELL);
        return;
    }
    DxLaneArr<NF, kHyb, float> sig, tau, xs, ds;
    DxLaneArr<NT, kHyb, float> Gm;
    if constexpr (kHyb) {
        Gm.bind(wsm, lane);
        sig.bind(wsm + 32 * NT, lane);
        tau.bind(wsm + 32 * NT + 32 * NF, lane);
        xs.bind(wsm + 32 * NT + 64 * NF, lane);
        ds.bind(wsm + 32 * NT + 96 * NF, lane);
    }
#pragma unroll
    for (int i = 0; i < NF; i++) {
        sig[i] = (float)sgd[i];
        tau[i] = (float)tud[i];
        xs[i] = (float)xsd[i];
        ds[i] = (float)dsd[i];
    }
    const int m = K.mk[kk];
    DxLaneArr<NT, false, float> Fm;
    dx_lpc_taylor_init<NF>(Fm, xs, ds, K.b[m], K.b[m - 1]);
    for (int j = m - 2; j >= 0; j--) {
        dx_lpc_horner_step<NF>(Fm, Gm, xs, ds, K.b[j]);
        dx_lane_take(Fm, Gm);
    }
    dx_lpc_taylor_finish<NF>(Fm, xs);
    dx_lpc_restore<NF>(Fm, sig, tau);
    for (int it = 0; it < s; it++) {
        dx_lpc_square_offdiag<NF>(Fm, Gm);
        dx_lpc_restore<NF>(Gm, sig, tau);
        dx_lane_take(Fm, Gm);
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
        float y[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) y[f] = sig[f] * (float)v_in[(d * NF + f) * C + c];
#pragma unroll
        for (int i = 0; i < NF; i++) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < NF; k++) acc = fmaf(Fm[P::at(i, k)], y[k], acc);
            v_out[(d * NF + i) * C + c] = (double)(tau[i] * acc);
        }
    }
}

template <int NF>
__global__ void __launch_bounds__(F32Store<NF>::kThreads)
dx_forward_lpc_f32(long long C, const double *rho_g, const double *rho_d, const double *t_s, const double *v_in,
                   double *v_out, double dt, uint32_t *status, DxConsts K, int rounds) {
    using S = F32Store<NF>;
    if constexpr (!S::kHyb) {
        const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (c < C) f32_cell<NF>(0, c, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, K, nullptr);
    } else {
        // sort keys overlay the warp's slices, which are first written after the sort
        extern __shared__ float smf[];
        static_assert(S::kTile * sizeof(unsigned long long) <= S::kWarpFloats * sizeof(float), "key overlay");
        __shared__ unsigned short order[S::kTile];
        unsigned long long *key = reinterpret_cast<unsigned long long *>(smf);
        const long long base = (long long)blockIdx.x * rounds * S::kThreads;
        dx_lpc_tile_order<NF - 1>(base, rounds, S::kThreads, C, C, rho_g, rho_d, t_s, dt, key, order);
        for (int r = 0; r < rounds; r++) {
            const long long c = base + order[r * S::kThreads + threadIdx.x];
            if (c < C) f32_cell<NF>(threadIdx.x, c, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, K, smf);
        }
    }
}

template <int NF>
int launch_f32(const DxConsts &K, long long C, const double *rho_g, const double *rho_d, const double *t_s,
               const double *v_in, double *v_out, double dt, uint32_t *status, cudaStream_t stream) {
    using S = F32Store<NF>;
    if constexpr (!S::kHyb) {
        const long long blocks = (C + S::kThreads - 1) / S::kThreads;
        dx_forward_lpc_f32<NF><<<(unsigned)blocks, S::kThreads, 0, stream>>>(C, rho_g, rho_d, t_s, v_in, v_out, dt,
                                                                            status, K, 1);
    } else {
        const size_t smem = sizeof(float) * (size_t)S::kWarpFloats;
        constexpr size_t kStatic = S::kTile * sizeof(unsigned short);
        if (smem + kStatic > 48 * 1024 &&
            cudaFuncSetAttribute(dx_forward_lpc_f32<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
            return DRAG_ECUDA;
        cudaFuncSetAttribute(dx_forward_lpc_f32<NF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int rounds = S::kTile / S::kThreads;
        while (rounds > 1 && (C + rounds * S::kThreads - 1) / (rounds * S::kThreads) < 8LL * dx_sm_count())
            rounds >>= 1;
        const long long blocks = (C + rounds * S::kThreads - 1) / (rounds * S::kThreads);
        dx_forward_lpc_f32<NF><<<(unsigned)blocks, S::kThreads, smem, stream>>>(C, rho_g, rho_d, t_s, v_in, v_out,
                                                                               dt, status, K, rounds);
    }
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

}  // namespace

int dx_launch_forward_lpc_f32(const DxConsts &K, int n, long long C, const double *rho_g, const double *rho_d,
                              const double *t_s, const double *v_in, double *v_out, double dt, uint32_t *status,
                              cudaStream_t stream) {
    switch (n) {
#define DX_CASE(NF) \
    case NF: return launch_f32<NF>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, stream);
        DX_CASE(2)
        DX_CASE(3)
        DX_CASE(4)
        DX_CASE(5)
        DX_CASE(6)
        DX_CASE(7)
        DX_CASE(8)
        DX_CASE(9)
        DX_CASE(10)
        DX_CASE(11)
        DX_CASE(12)
        DX_CASE(13)
        DX_CASE(14)
        DX_CASE(15)
        DX_CASE(16)
        DX_CASE(17)
#undef DX_CASE
        default: return DRAG_EINVAL_SIZE;
    }
}

