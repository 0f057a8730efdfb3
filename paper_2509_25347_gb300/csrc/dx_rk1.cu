// First-order implicit (backward Euler) drag step with the analytic solution
// of App. A.2 (Eqs. analytic_1-4): the paper's O(N) cost reference for EXP.
//
// For a drag-only step (U^(n+1/2) = U^n in Eq. eq_rk1_2) the update is
// v' = (I - dt Omega_v)^-1 v. With c_i = alpha_i dt / (1 + alpha_i dt)
// = dt / (t_s,i + dt), Eq. analytic_4 divided by rho_g and Eq. analytic_3
// divided by rho_d,i read
//   v_g' = (rho_g v_g + sum_i rho_d,i c_i v_i) / (rho_g + sum_i rho_d,i c_i),
//   v_i' = v_i + c_i (v_g' - v_i),
// which needs one division per species, none by rho_d (zero dust densities
// are fine) and conserves momentum. One thread per cell; consecutive threads
// read consecutive cells of every SoA array.
#include <cmath>

#include "dx_common.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
dx_rk1_lpc(long long C, int N, const double *rho_g, const double *rho_d, const double *t_s, double dt,
           const double *v_in, double *v_out, uint32_t *status) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int n = N + 1;
    const double rg = rho_g[c];
    bool ok = dx_pos_finite(rg);
    for (int i = 0; i < N; i++) ok = ok && dx_nonneg_finite(rho_d[i * C + c]) && dx_pos_or_inf(t_s[i * C + c]);
    if (!ok) {
        for (int e = 0; e < 3 * n; e++) v_out[e * C + c] = NAN;
        atomicOr(status, DRAG_STATUS_BAD_CELL);
        return;
    }
    double den = rg;
    double num[3];
    for (int d = 0; d < 3; d++) num[d] = rg * v_in[(d * n) * C + c];
    double cs[DRAG_EXPM_NMAX];
    for (int i = 0; i < N; i++) {
        const double ci = __ddiv_rn(dt, t_s[i * C + c] + dt);   // t_s = +inf gives 0
        const double e = rho_d[i * C + c] * ci;
        cs[i] = ci;
        den += e;
        for (int d = 0; d < 3; d++) num[d] = fma(e, v_in[(d * n + i + 1) * C + c], num[d]);
    }
    const double inv = __ddiv_rn(1.0, den);
    for (int d = 0; d < 3; d++) {
        const double w0 = num[d] * inv;
        for (int i = 0; i < N; i++) {
            const double vi = v_in[(d * n + i + 1) * C + c];
            v_out[(d * n + i + 1) * C + c] = fma(cs[i], w0 - vi, vi);
        }
        v_out[(d * n) * C + c] = w0;
    }
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

}  // namespace

extern "C" int drag_rk1_apply(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                              const double *t_s, double dt, const double *v_in, double *v_out, cudaStream_t stream) {
    if (ncells < 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX || !(dt >= 0.0) || !std::isfinite(dt))
        return DRAG_EINVAL_SIZE;
    if (ncells == 0) return DRAG_OK;
    if (!rho_g || !rho_d || !t_s || !v_in || !v_out) return DRAG_ENULL;
    if (!aligned8(rho_g) || !aligned8(rho_d) || !aligned8(t_s) || !aligned8(v_in) || !aligned8(v_out))
        return DRAG_EALIGN;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;
    const long long blocks = (ncells + kThreads - 1) / kThreads;
    dx_rk1_lpc<<<(unsigned)blocks, kThreads, 0, stream>>>(ncells, nspecies, rho_g, rho_d, t_s, dt, v_in, v_out, st);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}
