// Forward drag update, lane-per-cell kernels for n = N + 1 <= 12 (one thread
// per cell, consecutive threads on consecutive cells so every SoA load is
// coalesced). Templated on n; the matrix lives in registers (n <= 6) or in
// shared memory. See dx_lpc.cuh for the per-cell arithmetic.
#include "dx_lpc.cuh"
#include "dx_modes.h"

namespace {

constexpr int kTile = 512;   // largest tile of cells a block sorts and runs
// Tiles of fewer rounds than this run unsorted (the launcher uses one round,
// tiles of one block's threads, on inputs too small to fill the GPU otherwise).
#ifndef DX_LPC_SORT_MIN_ROUNDS
#define DX_LPC_SORT_MIN_ROUNDS 1
#endif

// Threads per block: 4 warps, or 2 warps when shared memory holds part of the
// matrices and n >= 9: there the slices (32 doubles per packed entry, 32 KB per
// warp at n = 9 with both buffers shared) set the residency and smaller blocks
// pack more warps onto an SM (measured: 1.3x at n = 9; 4-warp blocks stay
// faster up to n = 8).
template <int NF, int ST>
__host__ __device__ constexpr int lpc_threads() { return (ST != DX_LPC_REGS && NF >= 9) ? 64 : 128; }

// A warp runs the largest Taylor order and squaring count of its 32 cells, so
// each block first orders a tile of rounds x threads consecutive cells (the
// launcher shrinks the tile when the grid would leave SMs idle) by a cost proxy
// (dx_lpc_cost_proxy) and hands every warp 32 cells of similar cost. The proxy
// only groups cells; the cell routine still selects (k*, s*) from the FP64 norm.

// Register ceiling per thread. The register file is split among the four SM
// sub-partitions (16K registers each): at 168 registers a sub-partition can
// hold three warps instead of two, which at n = 9 (hybrid storage) paid for the
// spills it causes (5.31 against 5.57 ms on 240,000 cells; other n gained
// nothing from a ceiling).
template <int NF, int ST>
__host__ __device__ constexpr int lpc_max_regs() { return (ST == DX_LPC_HYBRID && NF == 9) ? 168 : 255; }

// Adjoint tape of a launch (TAPE kernels): cell c's fingerprint at hdr[c], its
// level t at m + (c * levels + t) * P.
struct LpcTape {
    long long *hdr;
    double *m;
    int levels, P;
};

template <int NF, int ST, bool TAPE>
__global__ void __launch_bounds__(lpc_threads<NF, ST>()) __maxnreg__((lpc_max_regs<NF, ST>()))
dx_forward_lpc(long long C, int rounds, const double *rho_g, const double *rho_d, const double *t_s,
               const double *v_in, double *v_out, double dt, uint32_t *status, double *heat, DxConsts K,
               LpcTape tp) {
    extern __shared__ double smem[];
    // Sort keys ((proxy << 32) | tile index, unique) live only until the tile is
    // sorted: with shared-memory storage they overlay the warps' matrix slices,
    // which are first written after that (5 KB less per CTA, one more CTA per SM
    // at n = 9).
    constexpr bool kOverlay = ST != DX_LPC_REGS && (kTile / lpc_threads<NF, ST>()) * lpc_threads<NF, ST>() *
                                                       sizeof(unsigned long long) <=
                                                   sizeof(double) * (lpc_threads<NF, ST>() / 32) *
                                                       dx_lpc_warp_smem_doubles<NF, ST>();
    __shared__ unsigned long long key_static[kOverlay ? 1 : kTile];
    unsigned long long *key = kOverlay ? reinterpret_cast<unsigned long long *>(smem + 32) : key_static;
    __shared__ unsigned short order[kTile];       // sorted position -> tile index
    double *bsh = smem;
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    constexpr int kThreads = lpc_threads<NF, ST>();
    const long long base = (long long)blockIdx.x * rounds * kThreads;
    if (rounds >= DX_LPC_SORT_MIN_ROUNDS) {
        dx_lpc_tile_order<NF - 1>(base, rounds, kThreads, C, C, rho_g, rho_d, t_s, dt, key, order);
    } else {
        order[threadIdx.x] = (unsigned short)threadIdx.x;   // unsorted
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    double *wsm = ST != DX_LPC_REGS ? smem + 32 + (threadIdx.x >> 5) * dx_lpc_warp_smem_doubles<NF, ST>() : nullptr;
    for (int r = 0; r < rounds; r++) {
        const long long c = base + order[dx_lpc_round_pos(r, kThreads)];
        if (c < C) {
            DxTapeCell tc{nullptr, nullptr, 0, 0};
            if (TAPE) tc = DxTapeCell{tp.hdr + c, tp.m + (size_t)c * tp.levels * tp.P, tp.levels, tp.P};
            dx_lpc_forward_cell<NF, ST>(lane, rho_g + c, rho_d + c, t_s + c, v_in + c, v_out + c, C, dt, K, bsh,
                                        wsm, status, heat ? heat + c : nullptr, tc);
        }
    }
}

// Balanced blocks (register storage). With one round of 4-warp blocks, the
// blocks that share an SM all hand their costliest 32 cells to the same warp
// slot, so one SM sub-partition (warp w runs on sub-partition w % 4) gets the
// costliest group of every block. Instead: blocks of up to 16 warps, as many
// as a multiple of the SM count, each on a contiguous share of C / gridDim.x
// cells ordered by the cost proxy's half-octave (a counting sort, cheaper than
// the rank sort: 15.7 against 17.1 us per launch at 32,768 cells of N = 1, the
// same at N = 4), with the sorted groups of 32 dealt to the
// warp slots in snake order over the four sub-partitions (costliest to 0, 1,
// 2, 3, then 3, 2, 1, 0, ...), which pairs costly groups with cheap ones.
// Groups are cut from the costly end, so the ragged one holds the cheapest
// cells.
template <int NF>
__host__ __device__ constexpr int lpc_wave_warps() { return NF <= 5 ? 16 : 8; }   // 128 / 255 registers

template <int NF>
__global__ void __launch_bounds__(32 * lpc_wave_warps<NF>())
dx_forward_lpc_wave(long long C, const double *rho_g, const double *rho_d, const double *t_s, const double *v_in,
                    double *v_out, double dt, uint32_t *status, double *heat, DxConsts K) {
    constexpr int kMax = 32 * lpc_wave_warps<NF>();
    __shared__ double bsh[32];
    __shared__ unsigned int hist[128];
    __shared__ unsigned short order[kMax];
    const long long c0 = (long long)blockIdx.x * C / gridDim.x;
    const long long c1 = ((long long)blockIdx.x + 1) * C / gridDim.x;
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    dx_lpc_bucket_order<NF - 1>(c0, c1, C, rho_g, rho_d, t_s, dt, hist, order);
    const int T = (int)(c1 - c0);
    const int q = threadIdx.x >> 5, row = q >> 2, sp = q & 3;
    const int k = 4 * row + ((row & 1) ? 3 - sp : sp);   // this slot's rank, costliest group first
    const int pos = T - 32 * (k + 1) + (threadIdx.x & 31);
    if (pos >= 0) {
        const long long c = c0 + order[pos];
        dx_lpc_forward_cell<NF, DX_LPC_REGS>(threadIdx.x & 31, rho_g + c, rho_d + c, t_s + c, v_in + c, v_out + c, C,
                                             dt, K, bsh, nullptr, status, heat ? heat + c : nullptr,
                                             DxTapeCell{nullptr, nullptr, 0, 0});
    }
}

template <int NF, int ST, bool TAPE = false>
int launch_one(const DxConsts &K, long long C, const double *rho_g, const double *rho_d, const double *t_s,
               const double *v_in, double *v_out, double dt, uint32_t *status, double *heat, cudaStream_t stream,
               LpcTape tp = LpcTape{nullptr, nullptr, 0, 0}) {
    constexpr int kThreads = lpc_threads<NF, ST>();
    if constexpr (ST == DX_LPC_REGS && !TAPE) {
        const long long sms = dx_sm_count();
        if (sms > 0 && C > (long long)kThreads * sms) {
            const long long cap = 32LL * lpc_wave_warps<NF>();
            const long long G = sms * ((C + sms * cap - 1) / (sms * cap));
            const long long per = (C + G - 1) / G;
            const int warps = (int)(((per + 31) / 32 + 3) / 4 * 4);
            dx_forward_lpc_wave<NF><<<(unsigned)G, 32 * warps, 0, stream>>>(C, rho_g, rho_d, t_s, v_in, v_out, dt,
                                                                           status, heat, K);
            return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
        }
    }
    const size_t smem = sizeof(double) * (32 + (size_t)(kThreads / 32) * dx_lpc_warp_smem_doubles<NF, ST>());
    // the opt-in covers dynamic + static shared memory (the sort order and, unless they
    // overlay the dynamic region, the keys) above 48 KB
    constexpr size_t kStatic = kTile * (sizeof(unsigned long long) + sizeof(unsigned short));
    if (smem + kStatic > 48 * 1024 &&
        cudaFuncSetAttribute(dx_forward_lpc<NF, ST, TAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return DRAG_ECUDA;
    // shared memory sets the residency of these kernels: ask for the largest carveout (a hint)
    if (ST != DX_LPC_REGS)
        cudaFuncSetAttribute(dx_forward_lpc<NF, ST, TAPE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    int rounds = kTile / kThreads;
    while (rounds > 1 && (C + rounds * kThreads - 1) / (rounds * kThreads) < 4LL * dx_sm_count()) rounds >>= 1;
    const long long blocks = (C + rounds * kThreads - 1) / (rounds * kThreads);
    dx_forward_lpc<NF, ST, TAPE><<<(unsigned)blocks, kThreads, smem, stream>>>(C, rounds, rho_g, rho_d, t_s, v_in,
                                                                                v_out, dt, status, heat, K, tp);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

// Storage modes built per n: registers or shared memory up to DX_LPC_REG_NMAX,
// shared memory or hybrid above.
template <int NF>
int launch_store(int store, const DxConsts &K, long long C, const double *rho_g, const double *rho_d,
                 const double *t_s, const double *v_in, double *v_out, double dt, uint32_t *status, double *heat,
                 cudaStream_t stream) {
    if constexpr (NF <= DX_LPC_REG_NMAX) {
        if (store == DX_LPC_REGS)
            return launch_one<NF, DX_LPC_REGS>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream);
    } else {
        if (store == DX_LPC_HYBRID)
            return launch_one<NF, DX_LPC_HYBRID>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream);
    }
    if (store == DX_LPC_SHARED)
        return launch_one<NF, DX_LPC_SHARED>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream);
    return DRAG_EINVAL_SIZE;
}

}  // namespace

int dx_launch_forward_lpc(const DxConsts &K, int n, int store, long long C, const double *rho_g,
                          const double *rho_d, const double *t_s, const double *v_in, double *v_out, double dt,
                          uint32_t *status, double *heat, cudaStream_t stream) {
    switch (n) {
#define DX_CASE(NF) \
    case NF: return launch_store<NF>(store, K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, heat, stream);
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
#undef DX_CASE
        default: return DRAG_EINVAL_SIZE;
    }
}

int dx_launch_forward_lpc_taped(const DxConsts &K, int n, long long C, const double *rho_g, const double *rho_d,
                                const double *t_s, const double *v_in, double *v_out, double dt, uint32_t *status,
                                long long *hdr, double *m, int levels, int P, cudaStream_t stream) {
    const LpcTape tp{hdr, m, levels, P};
    switch (n) {
#define DX_CASE(NF, ST) \
    case NF: return launch_one<NF, ST, true>(K, C, rho_g, rho_d, t_s, v_in, v_out, dt, status, nullptr, stream, tp);
        DX_CASE(2, DX_LPC_REGS)
        DX_CASE(3, DX_LPC_REGS)
        DX_CASE(4, DX_LPC_REGS)
        DX_CASE(5, DX_LPC_REGS)
        DX_CASE(6, DX_LPC_REGS)
        DX_CASE(7, DX_LPC_HYBRID)
        DX_CASE(8, DX_LPC_HYBRID)
        DX_CASE(9, DX_LPC_HYBRID)
        DX_CASE(10, DX_LPC_HYBRID)
        DX_CASE(11, DX_LPC_HYBRID)
        DX_CASE(12, DX_LPC_HYBRID)
#undef DX_CASE
        default: return DRAG_EINVAL_SIZE;
    }
}
