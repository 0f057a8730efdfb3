// Forward drag update, lane-per-cell kernels for n = N + 1 <= 12 (one thread
// per cell, consecutive threads on consecutive cells so every SoA load is
// coalesced). Templated on n; the matrix lives in registers (n <= 6) or in
// shared memory. See dx_lpc.cuh for the per-cell arithmetic.
#include "dx_lpc.cuh"
#include "dx_modes.h"

namespace {

constexpr int kThreads = 128;

template <int NF, bool SMEM>
__global__ void __launch_bounds__(kThreads)
dx_forward_lpc(long long C, const double *rho_g, const double *rho_d, const double *t_s, const double *v_in,
               double *v_out, double dt, uint32_t *status, double *heat, DxConsts K) {
    extern __shared__ double smem[];
    double *bsh = smem;
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    __syncthreads();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int lane = threadIdx.x & 31;
    double *wsm = SMEM ? smem + 32 + (threadIdx.x >> 5) * dx_lpc_warp_smem_doubles<NF>() : nullptr;
    dx_lpc_forward_cell<NF, SMEM>(lane, rho_g + c, rho_d + c, t_s + c, v_in + c, v_out + c, C, dt, K, bsh, wsm,
                                  status, heat ? heat + c : nullptr);
}

template <int NF, bool SMEM>
int launch_one(const DxConsts &K, long long C, const double *rho_g, const double *rho_d, const double *t_s, const double *v_in,
               double *v_out, double dt, uint32_t *status, double *heat, cudaStream_t stream) {
    const size_t smem = sizeof(double) * (32 + (SMEM ? (kThreads / 32) * dx_lpc_warp_smem_doubles<NF>() : 0));
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(dx_forward_lpc<NF, SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return DRAG_ECUDA;
    const long long blocks = (C + kThreads - 1) / kThreads;
    dx_forward_lpc<NF, SMEM><<<(unsigned)blocks, kThreads, smem, stream>>>(C, rho_g, rho_d, t_s, v_in, v_out, dt,
                                                                          status, heat, K);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

}  // namespace

int dx_launch_forward_lpc(const DxConsts &K, int n, bool smem, long long C, const double *rho_g, const double *rho_d, const double *t_s,
                          const double *v_in, double *v_out, double dt, uint32_t *status, double *heat,
                          cudaStream_t stream) {
#define DX_CASE_REG(NF) \
    case NF: return smem ? launch_one<NF, true>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream) \
                         : launch_one<NF, false>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream);
#define DX_CASE_SMEM(NF) \
    case NF: return launch_one<NF, true>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream);
    switch (n) {
        DX_CASE_REG(2)
        DX_CASE_REG(3)
        DX_CASE_REG(4)
        DX_CASE_REG(5)
        DX_CASE_REG(6)
        DX_CASE_SMEM(7)
        DX_CASE_SMEM(8)
        DX_CASE_SMEM(9)
        DX_CASE_SMEM(10)
        DX_CASE_SMEM(11)
        DX_CASE_SMEM(12)
        default: return DRAG_EINVAL_SIZE;
    }
#undef DX_CASE_REG
#undef DX_CASE_SMEM
}
