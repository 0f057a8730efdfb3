// Forward EXP drag update: v_out = exp(dt Omega_v) v_in per cell
// (Eq. ExacSolEqu in velocity form; Algorithm 6 with Algorithm 2).
//
// Warp-per-cell kernel. One warp owns one cell at a time (persistent loop);
// the cell's (N+1)x(N+1) matrix lives in shared memory. The similarity
// E = D^(1/2) P D^(-1/2) (D = diag(rho)) of the propagator P = exp(dt Omega_v)
// is symmetric because rho_i P_ij = rho_j P_ji, and it is a polynomial in the
// symmetric arrowhead X = 2^-s D^(1/2) dt Omega_v D^(-1/2):
//   X_00 = -2^-s sum_i eps_i alpha_i dt,  X_0i = X_i0 = 2^-s sqrt(eps_i) alpha_i dt,
//   X_ii = -2^-s alpha_i dt.
// With sigma = (1, sqrt(eps_1), ...) one has X sigma = 0, hence E sigma = sigma:
// the symmetric form of "rows of P sum to one". The kernel
//   1. selects (k*, s*) by Algorithm 2 from the 1-norm of A = dt Omega_v,
//      summed in a fixed order so the choice is reproducible;
//   2. evaluates T_m(X), m = m_{k*}, by Horner's rule in X: each step
//      F <- F X + b_j I costs O(n^2) because X is an arrowhead;
//   3. squares s* times, computing only the strict upper triangle of E^2
//      (n(n-1)/2 dot products) and setting the diagonal from E sigma = sigma:
//      E_ii = 1 - (1/sigma_i) sum_{j != i} E_ij sigma_j (row-sum restoration);
//   4. applies P = D^(-1/2) E D^(1/2) to the three velocity components with
//      P_ii = E_ii, P_ij = E_ij sigma_j / sigma_i.
#include <cmath>

#include "dx_modes.h"
#include "dx_wpc.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kCellsPerBlock = 16;

struct FwdArgs {
    long long C;           // ncells
    int N;                 // species
    const double *rho_g, *rho_d, *t_s, *v_in;
    double *v_out;
    double dt;
    uint32_t *status;
    double *heat;          // optional per-cell dissipated kinetic energy
};

// Adjoint tape of a launch (hdr null: none): cell c's fingerprint at hdr[c],
// its level t at m + (c * levels + t) * P.
struct FwdTape {
    long long *hdr;
    double *m;
    int levels, P;
};

// Cells of up to 16 species take their set-up two at a time
// (dx_wpc_setup_pair): each warp then holds a second cell's vectors (4 n
// doubles) while it runs the first.
__host__ __device__ constexpr bool fwd_paired(int N) { return dx_wpc_pairs(N); }

// Per-warp shared memory of the FP64 forward (doubles), and the block's pair
// tables: n(n-1)/2 + n(n+1)/2 - 1 shorts after the warps' slices.
__host__ __device__ inline int fwd_warp_doubles(int n) {
    return dx_wpc_fwd_warp_doubles(n) + (fwd_paired(n - 1) ? 4 * n : 0);
}
__host__ __device__ inline int fwd_pair_shorts(int n) { return n * (n - 1) / 2 + n * (n + 1) / 2 - 1; }

template <bool TAPE>
__device__ __forceinline__ void fwd_wpc_body(const FwdArgs &a, const DxConsts &K, const FwdTape &tp) {
    extern __shared__ double smem[];
    const int n = a.N + 1, ns = dx_stride(n);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wd = fwd_warp_doubles(n);
    unsigned short *od = reinterpret_cast<unsigned short *>(smem + kWarpsPerBlock * wd);
    unsigned short *hp = od + n * (n - 1) / 2;
    dx_build_pairs(n, od, hp);
    __syncthreads();
    double *wsm = smem + wib * wd;
    // Each block owns kCellsPerBlock consecutive cells; its warps take them (one
    // or two at a time) from a shared counter, so cells of different cost (s*
    // varies per cell) balance inside the block, and the hardware block
    // scheduler balances blocks across the SMs.
    __shared__ int next;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kCellsPerBlock;
    if (!fwd_paired(a.N)) {
        for (int it = 0; it < kCellsPerBlock; it++) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&next, 1);
            k = __shfl_sync(DX_FULL, k, 0);
            const long long c = base + k;
            if (k >= kCellsPerBlock || c >= a.C) break;
            DxTapeCell tc{nullptr, nullptr, 0, 0};
            if (TAPE) tc = DxTapeCell{tp.hdr + c, tp.m + (size_t)c * tp.levels * tp.P, tp.levels, tp.P};
            dx_wpc_forward_cell(lane, a.N, a.rho_g + c, a.rho_d + c, a.t_s + c, a.v_in + c, a.v_out + c, a.C, a.dt,
                                K, wsm, od, hp, a.status, a.heat ? a.heat + c : nullptr, (double *)nullptr, tc);
        }
        return;
    }
    double *E0 = wsm, *E1 = wsm + n * ns;
    DxVecs V0;
    DxFwdBufs B;
    dx_wpc_fwd_layout(E1 + n * ns, n, V0, B);
    double *v1 = wsm + dx_wpc_fwd_warp_doubles(n);
    const DxVecs V1{v1, v1 + n, v1 + 2 * n, v1 + 3 * n};
    const int h = lane >> 4, l = lane & 15;
    for (int it = 0; it < kCellsPerBlock; it += 2) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&next, 2);
        k = __shfl_sync(DX_FULL, k, 0);
        const long long cA = base + k;
        if (k >= kCellsPerBlock || cA >= a.C) break;
        const int cells = (k + 1 < kCellsPerBlock && cA + 1 < a.C) ? 2 : 1;
        // set-up inputs: half h takes cell cA + h (half 1 repeats cell cA when there is no
        // second cell; its result is not used), lane 16 h + i - 1 its species i
        const long long ch = cA + (h < cells ? h : 0);
        const double rg = a.rho_g[ch];
        double rd = 0.0, ts = INFINITY;
        if (l < a.N) {
            rd = a.rho_d[(long long)l * a.C + ch];
            ts = a.t_s[(long long)l * a.C + ch];
        }
        int k0, s0, k1, s1;
        const unsigned valid = dx_wpc_setup_pair(lane, a.N, rg, rd, ts, a.dt, K, V0, V1, k0, s0, k1, s1);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            if (e >= cells) break;
            const long long c = cA + e;
            const DxVecs &V = e ? V1 : V0;
            double *heat = a.heat ? a.heat + c : nullptr;
            if (!((valid >> e) & 1u)) {
                dx_wpc_fail_cell(lane, n, a.v_out + c, a.C, a.status, heat);
                continue;
            }
            DxCellIn ci;
            dx_wpc_load_cell(lane, a.N, a.rho_g + c, a.rho_d + c, a.t_s + c, a.v_in + c, a.C, ci);
            DxTapeCell tc{nullptr, nullptr, 0, 0};
            if (TAPE) tc = DxTapeCell{tp.hdr + c, tp.m + (size_t)c * tp.levels * tp.P, tp.levels, tp.P};
            const double sg = lane < n ? V.sig[lane] : 1.0;
            dx_wpc_forward_run(lane, a.N, V, E0, E1, B, e ? k1 : k0, e ? s1 : s0, sg, ci, a.v_out + c, a.C, a.dt, K,
                               od, hp, heat, (double *)nullptr, tc);
        }
    }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, 7)
dx_forward_wpc(FwdArgs a, DxConsts K) {
    fwd_wpc_body<false>(a, K, FwdTape{nullptr, nullptr, 0, 0});
}

// The same update, also recording each cell's adjoint tape.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 7)
dx_forward_wpc_taped(FwdArgs a, DxConsts K, FwdTape tp) {
    fwd_wpc_body<true>(a, K, tp);
}

// Mixed-precision forward: FP64 inputs, outputs, set-up and Algorithm 2 (on
// the theta table of u = 2^-24, Eq. B8's single-precision target), FP32
// Taylor, squarings and applications. FP32 issues 64x faster than FP64 on this
// part; the result carries FP32 rounding.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 8)
dx_forward_wpc_f32(FwdArgs a, DxConsts K) {
    extern __shared__ float smemf[];
    const int n = a.N + 1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wd = dx_wpc_fwd_warp_doubles(n) + n * dx_stride(n);   // + the restoration weight table
    unsigned short *od = reinterpret_cast<unsigned short *>(smemf + kWarpsPerBlock * wd);
    unsigned short *hp = od + kPairSlots;
    dx_build_pairs(n, od, hp);
    __syncthreads();
    float *wsm = smemf + wib * wd;
    float *wz = wsm + dx_wpc_fwd_warp_doubles(n);
    __shared__ int next;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kCellsPerBlock;
    for (int it = 0; it < kCellsPerBlock; it++) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&next, 1);
        k = __shfl_sync(DX_FULL, k, 0);
        const long long c = base + k;
        if (k >= kCellsPerBlock || c >= a.C) break;
        dx_wpc_forward_cell(lane, a.N, a.rho_g + c, a.rho_d + c, a.t_s + c, a.v_in + c, a.v_out + c, a.C, a.dt, K, wsm,
                            od, hp, a.status, (double *)nullptr, wz);
    }
}

// (k*, s*) per cell, one thread per cell (diagnostics and FLOP accounting).
__global__ void dx_select_kernel(long long C, int N, const double *rho_g, const double *rho_d, const double *t_s,
                                 double dt, int8_t *k_out, int16_t *s_out, uint32_t *status, DxConsts K) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double rg = rho_g[c];
    bool ok = dx_pos_finite(rg);
    double s1 = 0.0, col0, cmax = 0.0;
    for (int i = 0; i < N && ok; i++) {
        const double rd = rho_d[(long long)i * C + c], ts = t_s[(long long)i * C + c];
        ok = dx_nonneg_finite(rd) && dx_pos_or_inf(ts);
    }
    int kk = 0, s = -1;
    if (ok) {
        for (int i = 0; i < N; i++) {
            const double eps = __ddiv_rn(rho_d[(long long)i * C + c], rg);
            const double alpha = __ddiv_rn(1.0, t_s[(long long)i * C + c]);
            s1 = __dadd_rn(s1, __dmul_rn(__dmul_rn(eps, alpha), dt));
        }
        col0 = s1;
        for (int i = 0; i < N; i++) {
            const double eps = __ddiv_rn(rho_d[(long long)i * C + c], rg);
            const double alpha = __ddiv_rn(1.0, t_s[(long long)i * C + c]);
            const double ai0 = __dmul_rn(alpha, dt);
            col0 = __dadd_rn(col0, ai0);
            const double cj = __dadd_rn(__dmul_rn(__dmul_rn(eps, alpha), dt), ai0);
            cmax = dx_bits(cj) > dx_bits(cmax) ? cj : cmax;
        }
        const double norm = dx_bits(col0) > dx_bits(cmax) ? col0 : cmax;
        if (dx_norm_ok(dx_bits(norm)))
            dx_select(norm, K, kk, s);
        else
            ok = false;
    }
    if (!ok) atomicOr(status, DRAG_STATUS_BAD_CELL);
    if (k_out) k_out[c] = (int8_t)kk;
    if (s_out) s_out[c] = (int16_t)s;
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

int check_common(long long C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt) {
    if (C < 0 || N < 1 || N > DRAG_EXPM_NMAX || !(dt >= 0.0) || !std::isfinite(dt)) return DRAG_EINVAL_SIZE;
    if (C == 0) return DRAG_OK;
    if (!rho_g || !rho_d || !t_s) return DRAG_ENULL;
    if (!aligned8(rho_g) || !aligned8(rho_d) || !aligned8(t_s)) return DRAG_EALIGN;
    return DRAG_OK;
}

}  // namespace

size_t dx_forward_smem_bytes(int n) {
    return sizeof(double) * (size_t)kWarpsPerBlock * fwd_warp_doubles(n) + fwd_pair_shorts(n) * sizeof(unsigned short);
}

size_t dx_forward_f32_smem_bytes(int n) {
    return sizeof(float) * (size_t)kWarpsPerBlock * (dx_wpc_fwd_warp_doubles(n) + n * dx_stride(n)) +
           2 * kPairSlots * sizeof(unsigned short);
}

static int apply_impl(const DxConsts &K, int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                      const double *t_s, double dt, const double *v_in, double *v_out, double *heat,
                      cudaStream_t stream) {
    int rc = check_common(ncells, nspecies, rho_g, rho_d, t_s, dt);
    if (rc != DRAG_OK || ncells == 0) return rc;
    if (!v_in || !v_out) return DRAG_ENULL;
    if (!aligned8(v_in) || !aligned8(v_out) || (heat && !aligned8(heat))) return DRAG_EALIGN;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    const int n = nspecies + 1;
    const int mode = dx_mode_for(n);
    if (mode != DX_MODE_WPC) {
        if (!heat && dx_binned_eligible(n, mode, ncells)) {
            const int rc = dx_binned_forward(K, ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, st, stream);
            if (rc != DX_BINNED_UNAVAILABLE) return rc;
        }
        return dx_launch_forward_lpc(K, n, dx_lpc_store(mode), ncells, rho_g, rho_d, t_s, v_in, v_out, dt, st, heat,
                                     stream);
    }
    const size_t smem = dx_forward_smem_bytes(n);
    if (!dx_once_per_device(0, [] {
            return cudaFuncSetAttribute(dx_forward_wpc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dx_forward_smem_bytes(DX_NMAXF)) == cudaSuccess;
        }))
        return DRAG_ECUDA;
    FwdArgs a{ncells, nspecies, rho_g, rho_d, t_s, v_in, v_out, dt, st, heat};
    const long long grid = (ncells + kCellsPerBlock - 1) / kCellsPerBlock;
    dx_forward_wpc<<<(unsigned)grid, kWarpsPerBlock * 32, smem, stream>>>(a, K);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" int drag_expm_apply(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                               const double *t_s, double dt, const double *v_in, double *v_out,
                               cudaStream_t stream) {
    return apply_impl(dx_consts(), ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, nullptr, stream);
}

extern "C" size_t drag_expm_tape_bytes(int64_t ncells, int32_t nspecies, int32_t levels) {
    if (ncells < 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX || levels < 1 || levels > DRAG_TAPE_MAX_LEVELS)
        return 0;
    return dx_tape_hdr_bytes(ncells) + sizeof(double) * (size_t)ncells * (size_t)levels * dx_tape_slot(nspecies + 1);
}

extern "C" int32_t drag_expm_tape_levels(int32_t sstar) { return sstar < 0 ? 0 : dx_tape_levels(sstar); }

extern "C" int drag_expm_apply_taped(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                     const double *t_s, double dt, const double *v_in, double *v_out, int32_t levels,
                                     void *tape, size_t tape_bytes, cudaStream_t stream) {
    int rc = check_common(ncells, nspecies, rho_g, rho_d, t_s, dt);
    if (rc != DRAG_OK) return rc;
    if (levels < 1 || levels > DRAG_TAPE_MAX_LEVELS) return DRAG_EINVAL_SIZE;
    if (ncells == 0) return DRAG_OK;
    if (!v_in || !v_out || !tape) return DRAG_ENULL;
    if (!aligned8(v_in) || !aligned8(v_out) || (reinterpret_cast<uintptr_t>(tape) & 255) != 0) return DRAG_EALIGN;
    if (tape_bytes < drag_expm_tape_bytes(ncells, nspecies, levels)) return DRAG_EWORKSPACE;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    if (!dx_once_per_device(5, [] {
            return cudaFuncSetAttribute(dx_forward_wpc_taped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dx_forward_smem_bytes(DX_NMAXF)) == cudaSuccess;
        }))
        return DRAG_ECUDA;
    const int n = nspecies + 1;
    FwdArgs a{ncells, nspecies, rho_g, rho_d, t_s, v_in, v_out, dt, st, nullptr};
    FwdTape tp{static_cast<long long *>(tape),
               reinterpret_cast<double *>(static_cast<char *>(tape) + dx_tape_hdr_bytes(ncells)), levels,
               dx_tape_slot(n)};
    // small n: the lane-per-cell forward writes the tape (when the mode table has
    // its default storage there), far cheaper than warp per cell at these sizes
    const int mode = dx_mode_for(n);
    if (n <= DX_LPC_TAPE_NMAX &&
        mode == (n <= DX_LPC_REG_NMAX ? DX_MODE_LPC_REG : DX_MODE_LPC_HYB)) {
        if (dx_binned_eligible(n, mode, ncells)) {   // large inputs: binned, as drag_expm_apply
            const int rc2 = dx_binned_forward(dx_consts(), ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, st,
                                              stream, tp.hdr, tp.m, levels, tp.P);
            if (rc2 != DX_BINNED_UNAVAILABLE) return rc2;
        }
        return dx_launch_forward_lpc_taped(dx_consts(), n, ncells, rho_g, rho_d, t_s, v_in, v_out, dt, st, tp.hdr,
                                           tp.m, levels, tp.P, stream);
    }
    const long long grid = (ncells + kCellsPerBlock - 1) / kCellsPerBlock;
    dx_forward_wpc_taped<<<(unsigned)grid, kWarpsPerBlock * 32, dx_forward_smem_bytes(n), stream>>>(a, dx_consts(), tp);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

int dx_launch_forward_f32(const DxConsts &K, long long ncells, int nspecies, const double *rho_g,
                          const double *rho_d, const double *t_s, double dt, const double *v_in, double *v_out,
                          cudaStream_t stream) {
    int rc = check_common(ncells, nspecies, rho_g, rho_d, t_s, dt);
    if (rc != DRAG_OK || ncells == 0) return rc;
    if (!v_in || !v_out) return DRAG_ENULL;
    if (!aligned8(v_in) || !aligned8(v_out)) return DRAG_EALIGN;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    if (!dx_once_per_device(4, [] {
            return cudaFuncSetAttribute(dx_forward_wpc_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dx_forward_f32_smem_bytes(DX_NMAXF)) == cudaSuccess;
        }))
        return DRAG_ECUDA;
    FwdArgs a{ncells, nspecies, rho_g, rho_d, t_s, v_in, v_out, dt, st, nullptr};
    const long long grid = (ncells + kCellsPerBlock - 1) / kCellsPerBlock;
    const size_t smem = dx_forward_f32_smem_bytes(nspecies + 1);
    dx_forward_wpc_f32<<<(unsigned)grid, kWarpsPerBlock * 32, smem, stream>>>(a, K);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" int drag_expm_apply_target(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                      const double *t_s, double dt, const double *v_in, double *v_out, int32_t ubits,
                                      cudaStream_t stream) {
    const DxConsts *K = dx_consts_for(ubits);
    if (!K) return DRAG_EINVAL_TARGET;
    return apply_impl(*K, ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, nullptr, stream);
}

extern "C" int drag_expm_apply_heat(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                    const double *t_s, double dt, const double *v_in, double *v_out, double *heat_out,
                                    cudaStream_t stream) {
    if (!heat_out && ncells > 0) return DRAG_ENULL;
    return apply_impl(dx_consts(), ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, heat_out, stream);
}

extern "C" int drag_expm_select(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                const double *t_s, double dt, int8_t *k_out, int16_t *s_out, cudaStream_t stream) {
    return drag_expm_select_target(ncells, nspecies, rho_g, rho_d, t_s, dt, 53, k_out, s_out, stream);
}

extern "C" int drag_expm_select_target(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                       const double *t_s, double dt, int32_t ubits, int8_t *k_out, int16_t *s_out,
                                       cudaStream_t stream) {
    const DxConsts *K = dx_consts_for(ubits);
    if (!K) return DRAG_EINVAL_TARGET;
    int rc = check_common(ncells, nspecies, rho_g, rho_d, t_s, dt);
    if (rc != DRAG_OK || ncells == 0) return rc;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    const int threads = 256;
    const long long blocks = (ncells + threads - 1) / threads;
    dx_select_kernel<<<(unsigned)blocks, threads, 0, stream>>>(ncells, nspecies, rho_g, rho_d, t_s, dt, k_out, s_out,
                                                              st, *K);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}
