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

#include "dx_common.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kPairSlots = 544;   // >= n(n+1)/2 for n <= 32

struct FwdArgs {
    long long C;           // ncells
    int N;                 // species
    const double *rho_g, *rho_d, *t_s, *v_in;
    double *v_out;
    double dt;
    uint32_t *status;
};

// Row stride of the n x n shared-memory matrices: odd, to spread banks.
__host__ __device__ __forceinline__ int dx_stride(int n) { return n | 1; }

// Per-warp shared-memory footprint (doubles).
__host__ __device__ __forceinline__ int warp_smem_doubles(int n) {
    return 2 * n * dx_stride(n) + 10 * DX_NMAXF;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
dx_forward_wpc(FwdArgs a, DxConsts K) {
    extern __shared__ double smem[];
    const int n = a.N + 1, N = a.N, ns = dx_stride(n);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n_od = n * (n - 1) / 2;           // strict upper pairs (squaring)
    const int n_hp = n * (n + 1) / 2 - 1;       // upper pairs except (0,0) (Horner)

    // Pair tables (shared by the block): od[t] = (i<<8)|j with i<j; hp[t] with i<=j, (i,j) != (0,0).
    unsigned short *od = reinterpret_cast<unsigned short *>(smem + kWarpsPerBlock * warp_smem_doubles(n));
    unsigned short *hp = od + kPairSlots;
    for (int t = threadIdx.x; t < n_od; t += blockDim.x) {
        int i = 0, r = t;
        while (r >= n - 1 - i) { r -= n - 1 - i; i++; }
        od[t] = (unsigned short)((i << 8) | (i + 1 + r));
    }
    for (int t = threadIdx.x; t < n_hp; t += blockDim.x) {
        int i = 0, r = t + 1;                  // skip (0,0)
        while (r >= n - i) { r -= n - i; i++; }
        hp[t] = (unsigned short)((i << 8) | (i + r));
    }
    __syncthreads();

    double *E0 = smem + wib * warp_smem_doubles(n);
    double *E1 = E0 + n * ns;
    double *sig = E1 + n * ns;         // sigma_f
    double *tau = sig + DX_NMAXF;      // 1/sigma_f
    double *xs = tau + DX_NMAXF;       // X_0f (f >= 1), xs[0] = X_00
    double *ds = xs + DX_NMAXF;        // X_ff (f >= 1)
    double *yv = ds + DX_NMAXF;        // sigma_f v_f, three components
    double *vv = yv + 3 * DX_NMAXF;    // v_f, three components

    const long long C = a.C;
    const long long nwarps = (long long)gridDim.x * kWarpsPerBlock;
    for (long long c = (long long)blockIdx.x * kWarpsPerBlock + wib; c < C; c += nwarps) {
        // ---------------- load (lane f holds fluid f; species i on lane i)
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
        const bool okl = (lane == 0 || lane > N) || (dx_nonneg_finite(rd) && dx_pos_or_inf(ts));
        const bool ok = __all_sync(DX_FULL, okl) && dx_pos_finite(rg);
        if (!ok) {
            if (lane < n) {
#pragma unroll
                for (int d = 0; d < 3; d++) a.v_out[((long long)d * n + lane) * C + c] = NAN;
            }
            if (lane == 0) atomicOr(a.status, DRAG_STATUS_BAD_CELL);
            continue;
        }

        // ---------------- A = dt Omega_v entries (Eqs. DragEqVar2/3, jacobian)
        const bool sp = lane >= 1 && lane <= N;
        const double eps = sp ? __ddiv_rn(rd, rg) : 0.0;
        const double alpha = sp ? __ddiv_rn(1.0, ts) : 0.0;
        const double a0i = __dmul_rn(__dmul_rn(eps, alpha), a.dt);   // A_0i
        const double ai0 = __dmul_rn(alpha, a.dt);                   // A_i0 = -A_ii

        // 1-norm, summed in ascending species order: column 0 is
        // |A_00| + sum_i A_i0 with A_00 = -sum_i A_0i; column i is A_0i + A_i0.
        double s1 = 0.0;
        for (int i = 1; i <= N; i++) s1 = __dadd_rn(s1, dx_shfl(a0i, i));
        double col0 = s1;
        for (int i = 1; i <= N; i++) col0 = __dadd_rn(col0, dx_shfl(ai0, i));
        const double colj = sp ? __dadd_rn(a0i, ai0) : 0.0;
        long long nb = dx_warp_max_ll(dx_bits(colj));
        nb = nb > dx_bits(col0) ? nb : dx_bits(col0);
        int kk, s;
        dx_select(__longlong_as_double(nb), K, kk, s);
        const int m = K.mk[kk];

        // ---------------- symmetric arrowhead X = 2^-s D^(1/2) A D^(-1/2)
        const double p2 = dx_pow2(-s);
        double sg = 1.0, tu = 1.0;
        if (sp) {
            const double e = dx_bits(eps) < dx_bits(DX_EPS_FLOOR) ? DX_EPS_FLOOR : eps;
            sg = __dsqrt_rn(e);
            tu = __ddiv_rn(1.0, sg);
        }
        if (lane < n) {
            sig[lane] = sg;
            tau[lane] = tu;
            xs[lane] = lane == 0 ? -s1 * p2 : __dmul_rn(__dmul_rn(sg, alpha), a.dt * p2);
            ds[lane] = -(ai0 * p2);
        }
        __syncwarp();

        // ---------------- Taylor: F = b_m X + b_{m-1} I, then F <- F X + b_j I
        double *F = E0, *G = E1;
        for (int t = lane; t < n * ns; t += 32) F[t] = 0.0;
        __syncwarp();
        if (lane < n) {
            const double x = xs[lane];
            if (lane == 0) {
                F[0] = fma(K.b[m], x, K.b[m - 1]);
            } else {
                F[lane] = F[lane * ns] = K.b[m] * x;
                F[lane * ns + lane] = fma(K.b[m], ds[lane], K.b[m - 1]);
            }
        }
        __syncwarp();
        for (int j = m - 2; j >= 0; j--) {
            const double bj = K.b[j];
            // G_ij = F_i0 X_0j + F_ij X_jj (+ b_j on the diagonal), i <= j, (i,j) != (0,0)
            for (int t = lane; t < n_hp; t += 32) {
                const int p = hp[t], i = p >> 8, jj = p & 255;
                double acc = fma(F[i * ns], xs[jj], i == jj ? bj : 0.0);
                acc = fma(F[i * ns + jj], ds[jj], acc);
                G[i * ns + jj] = acc;
                G[jj * ns + i] = acc;
            }
            // G_00 = sum_k F_0k X_k0 + b_j
            double part = lane < n ? F[lane] * xs[lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(DX_FULL, part, o);
            if (lane == 0) G[0] = part + bj;
            __syncwarp();
            double *tmp = F; F = G; G = tmp;
        }

        // ---------------- restore: E_ii = 1 - tau_i sum_{k != i} E_ik sigma_k
        if (lane < n) {
            double acc = 0.0;
            for (int q = 0; q < n - 1; q++) {
                const int k = q + (q >= lane);
                acc = fma(F[lane * ns + k], sig[k], acc);
            }
            F[lane * ns + lane] = fma(-tau[lane], acc, 1.0);
        }
        __syncwarp();

        // ---------------- s squarings (Eq. ExpEq1 with n = 2^s)
        for (int it = 0; it < s; it++) {
            for (int t = lane; t < n_od; t += 32) {
                const int p = od[t], i = p >> 8, jj = p & 255;
                const double *ri = F + i * ns, *rj = F + jj * ns;
                double acc = 0.0;
                for (int k = 0; k < n; k++) acc = fma(ri[k], rj[k], acc);
                G[i * ns + jj] = acc;
                G[jj * ns + i] = acc;
            }
            __syncwarp();
            if (lane < n) {
                double acc = 0.0;
                for (int q = 0; q < n - 1; q++) {
                    const int k = q + (q >= lane);
                    acc = fma(G[lane * ns + k], sig[k], acc);
                }
                G[lane * ns + lane] = fma(-tau[lane], acc, 1.0);
            }
            __syncwarp();
            double *tmp = F; F = G; G = tmp;
        }

        // ---------------- apply: v_out_i = E_ii v_i + tau_i sum_{j != i} E_ij sigma_j v_j
        if (lane < n) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                yv[d * DX_NMAXF + lane] = sg * vin[d];
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
            a.v_out[((long long)d * n + i) * C + c] = fma(tau[i], acc, F[i * ns + i] * vv[d * DX_NMAXF + i]);
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
