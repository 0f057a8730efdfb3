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

#include "dx_wpc.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;

struct FwdArgs {
    long long C;           // ncells
    int N;                 // species
    const double *rho_g, *rho_d, *t_s, *v_in;
    double *v_out;
    double dt;
    uint32_t *status;
};

// Per-warp shared-memory footprint (doubles): E0, E1, sigma, tau, X_0f, X_ff,
// sigma v (3 components) and v (3 components).
__host__ __device__ __forceinline__ int warp_smem_doubles(int n) {
    return 2 * n * dx_stride(n) + 10 * DX_NMAXF;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
dx_forward_wpc(FwdArgs a, DxConsts K) {
    extern __shared__ double smem[];
    const int n = a.N + 1, N = a.N, ns = dx_stride(n);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n_od = n * (n - 1) / 2;
    const int n_hp = n * (n + 1) / 2 - 1;

    unsigned short *od = reinterpret_cast<unsigned short *>(smem + kWarpsPerBlock * warp_smem_doubles(n));
    unsigned short *hp = od + kPairSlots;
    dx_build_pairs(n, od, hp);
    __syncthreads();

    double *E0 = smem + wib * warp_smem_doubles(n);
    double *E1 = E0 + n * ns;
    DxVecs V;
    V.sig = E1 + n * ns;
    V.tau = V.sig + DX_NMAXF;
    V.xs = V.tau + DX_NMAXF;
    V.ds = V.xs + DX_NMAXF;
    double *yv = V.ds + DX_NMAXF;      // sigma_f v_f, three components
    double *vv = yv + 3 * DX_NMAXF;    // v_f, three components

    const long long C = a.C;
    const long long nwarps = (long long)gridDim.x * kWarpsPerBlock;
    for (long long c = (long long)blockIdx.x * kWarpsPerBlock + wib; c < C; c += nwarps) {
        const double rg = a.rho_g[c];
        double rd = 0.0, ts = INFINITY;
        if (lane >= 1 && lane <= N) {
            rd = a.rho_d[(long long)(lane - 1) * C + c];
            ts = a.t_s[(long long)(lane - 1) * C + c];
        }
        double vin[3] = {0.0, 0.0, 0.0};
        if (lane < n) {
#pragma unroll
            for (int d = 0; d < 3; d++) vin[d] = a.v_in[((long long)d * n + lane) * C + c];
        }
        DxLane L;
        if (!dx_wpc_setup(lane, N, rg, rd, ts, a.dt, K, V, L)) {
            if (lane < n) {
#pragma unroll
                for (int d = 0; d < 3; d++) a.v_out[((long long)d * n + lane) * C + c] = NAN;
            }
            if (lane == 0) atomicOr(a.status, DRAG_STATUS_BAD_CELL);
            continue;
        }
        const int m = K.mk[L.k];

        // Taylor polynomial T_m(X) by Horner's rule in X
        double *F = E0, *G = E1;
        dx_wpc_taylor_init(lane, n, ns, m, K, V, F);
        for (int j = m - 2; j >= 0; j--) {
            dx_wpc_horner_step(lane, n, ns, n_hp, hp, V, K.b[j], F, G);
            __syncwarp();
            double *tmp = F; F = G; G = tmp;
        }
        dx_wpc_restore(lane, n, ns, V, F);
        __syncwarp();

        // s squarings (Eq. ExpEq1 with n = 2^s), row sums restored each time
        for (int it = 0; it < L.s; it++) {
            dx_wpc_square_offdiag(lane, n, ns, n_od, od, F, G);
            __syncwarp();
            dx_wpc_restore(lane, n, ns, V, G);
            __syncwarp();
            double *tmp = F; F = G; G = tmp;
        }

        // v_out_i = E_ii v_i + tau_i sum_{j != i} E_ij sigma_j v_j  (P = D_sigma^-1 E D_sigma)
        if (lane < n) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                yv[d * DX_NMAXF + lane] = L.sg * vin[d];
                vv[d * DX_NMAXF + lane] = vin[d];
            }
        }
        __syncwarp();
        for (int t = lane; t < 3 * n; t += 32) {
            const int d = t / n, i = t - d * n;
            const double *y = yv + d * DX_NMAXF;
            double acc = 0.0;
            for (int q = 0; q < n - 1; q++) {
                const int k = q + (q >= i);
                acc = fma(F[i * ns + k], y[k], acc);
            }
            a.v_out[((long long)d * n + i) * C + c] = fma(V.tau[i], acc, F[i * ns + i] * vv[d * DX_NMAXF + i]);
        }
        __syncwarp();
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
        dx_select(norm, K, kk, s);
    } else {
        atomicOr(status, DRAG_STATUS_BAD_CELL);
    }
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
    return sizeof(double) * (size_t)kWarpsPerBlock * warp_smem_doubles(n) + 2 * kPairSlots * sizeof(unsigned short);
}

extern "C" int drag_expm_apply(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                               const double *t_s, double dt, const double *v_in, double *v_out,
                               cudaStream_t stream) {
    int rc = check_common(ncells, nspecies, rho_g, rho_d, t_s, dt);
    if (rc != DRAG_OK || ncells == 0) return rc;
    if (!v_in || !v_out) return DRAG_ENULL;
    if (!aligned8(v_in) || !aligned8(v_out)) return DRAG_EALIGN;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    const int n = nspecies + 1;
    const size_t smem = dx_forward_smem_bytes(n);
    if (!dx_once_per_device(0, [] {
            return cudaFuncSetAttribute(dx_forward_wpc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dx_forward_smem_bytes(DX_NMAXF)) == cudaSuccess;
        }))
        return DRAG_ECUDA;
    FwdArgs a{ncells, nspecies, rho_g, rho_d, t_s, v_in, v_out, dt, st};
    const long long want = (ncells + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const long long cap = (long long)dx_sm_count() * 8;
    const int grid = (int)(want < cap ? want : cap);
    dx_forward_wpc<<<grid, kWarpsPerBlock * 32, smem, stream>>>(a, dx_consts());
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" int drag_expm_select(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                const double *t_s, double dt, int8_t *k_out, int16_t *s_out, cudaStream_t stream) {
    int rc = check_common(ncells, nspecies, rho_g, rho_d, t_s, dt);
    if (rc != DRAG_OK || ncells == 0) return rc;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    const int threads = 256;
    const long long blocks = (ncells + threads - 1) / threads;
    dx_select_kernel<<<(unsigned)blocks, threads, 0, stream>>>(ncells, nspecies, rho_g, rho_d, t_s, dt, k_out, s_out,
                                                              st, dx_consts());
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}
