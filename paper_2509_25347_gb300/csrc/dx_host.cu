// Host-side set-up of libdragexpm: the theta_m constants of Eq. B8, the
// Taylor coefficients, the device status word and small query entry points.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dx_common.cuh"
#include "dx_modes.h"

// Sticky status bits, one word per device (DRAG_STATUS_*).
__device__ uint32_t g_dx_status;

namespace {

// Table B.1: m_k, q_k, r_k for k = 1..9.
const int kMk[DX_K + 1] = {0, 2, 4, 6, 9, 12, 16, 20, 25, 30};
const int kQk[DX_K + 1] = {0, 1, 2, 2, 3, 3, 4, 4, 5, 5};
const int kRk[DX_K + 1] = {0, 2, 2, 3, 3, 4, 4, 5, 5, 6};

// f_m(theta)/theta with f_m of Eq. B6. The coefficients of
// rho(x) = e^-x T_m(x) - 1 (Eq. B5) satisfy |c_j| = C(j-1, m)/j!, so
// f_m(theta) = sum_{t>=0} theta^(m+1+t) / ((m+1+t) m! t!): all terms positive.
double fm(int m, double th) {
    double inv_mfact = 1.0;
    for (int a = 2; a <= m; a++) inv_mfact /= a;
    double term = std::pow(th, m + 1) * inv_mfact;   // theta^(m+1)/(m! 0!)
    double f = 0.0;
    for (int t = 0; t < 120; t++) {
        f += term / (m + 1 + t);
        term *= th / (t + 1);
    }
    return f;
}

// theta_m = max{theta : -log(1 - f_m(theta))/theta <= u} (Eq. B8), bisection.
double theta_of(int m, double u) {
    double lo = 0.0, hi = 64.0;
    for (int it = 0; it < 300; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = fm(m, mid);
        bool ok = f < 1.0 && -std::log1p(-f) / mid <= u;
        (ok ? lo : hi) = mid;
    }
    return lo;
}

long long bits(double x) {
    long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
}

DxConsts make_consts(int ubits) {
    DxConsts K;
    std::memset(&K, 0, sizeof K);
    const double u = std::ldexp(1.0, -ubits);
    for (int k = 1; k <= DX_K; k++) {
        double th = theta_of(kMk[k], u);
        K.th[k] = bits(th);
        K.th2[k] = bits(2.0 * th);
        K.th4[k] = bits(4.0 * th);
        K.mk[k] = kMk[k];
        K.qk[k] = kQk[k];
        K.rk[k] = kRk[k];
    }
    K.b[0] = 1.0;
    for (int i = 1; i < 32; i++) K.b[i] = K.b[i - 1] / i;
    K.u = u;
    return K;
}

// ---- Pade variant: coefficients and theta_m (host, double-double series)

// Unevaluated sum hi + lo with |lo| <= ulp(hi)/2; the operations are
// error-free transformations (two-sum, fma two-product), identical on every
// IEEE-754 host.
struct Dd {
    double hi = 0.0, lo = 0.0;
};
Dd dd_norm(double a, double b) {
    Dd r;
    r.hi = a + b;
    r.lo = b - (r.hi - a);
    return r;
}
Dd operator+(Dd a, Dd b) {
    const double s = a.hi + b.hi, v = s - a.hi;
    const double err = (a.hi - (s - v)) + (b.hi - v);
    return dd_norm(s, err + a.lo + b.lo);
}
Dd operator-(Dd a) { return Dd{-a.hi, -a.lo}; }
Dd operator*(Dd a, Dd b) {
    const double p = a.hi * b.hi;
    return dd_norm(p, std::fma(a.hi, b.hi, -p) + a.hi * b.lo + a.lo * b.hi);
}
Dd dd_from_ratio(double num, double den) {       // num / den for integers below 2^53
    const double q = num / den;
    return dd_norm(q, std::fma(-q, den, num) / den);
}

// rho(x) = e^-x R_mm(x) - 1 = -E(x) G(x) with
//   E(x) = e^x D(x) - N(x) = (-1)^m x^(2m+1)/(2m)! int_0^1 e^(tx) t^m (1-t)^m dt
//        = sum_k e_k x^(2m+1+k),  e_k = (-1)^m m! (m+k)! / ((2m)! k! (2m+k+1)!)
//   G(x) = e^-x / D(x):  D G = e^-x, i.e. G_k = (-1)^k/k! - sum_{i>=1} d_i G_{k-i}.
// Returns |rho_j| for j = 2m+1 .. 2m+L (index j - 2m - 1).
void pade_rho_abs(int m, int L, double *out) {
    std::vector<Dd> d(m + 1), G(L), e(L);
    for (int j = 0; j <= m; j++) {             // d_j = (-1)^j (2m-j)! m! / ((2m)! j! (m-j)!)
        Dd v{1.0, 0.0};
        for (int a = 0; a < j; a++) v = v * dd_from_ratio(m - a, (2 * m - a) * (double)(a + 1));
        d[j] = (j & 1) ? -v : v;
    }
    Dd inv_fact{1.0, 0.0};
    for (int k = 0; k < L; k++) {
        if (k > 0) inv_fact = inv_fact * dd_from_ratio(1.0, k);
        Dd g = (k & 1) ? -inv_fact : inv_fact;
        for (int i = 1; i <= m && i <= k; i++) g = g + -(d[i] * G[k - i]);
        G[k] = g;
    }
    Dd ek{1.0, 0.0};                          // |e_0| = m! m! / ((2m)! (2m+1)!)
    for (int a = 1; a <= m; a++) ek = ek * dd_from_ratio(a, m + a);        // m! m! / (2m)!
    for (int a = 2; a <= 2 * m + 1; a++) ek = ek * dd_from_ratio(1.0, a);   // / (2m+1)!
    for (int k = 0; k < L; k++) {
        e[k] = (m & 1) ? -ek : ek;
        ek = ek * dd_from_ratio(m + k + 1, (double)(k + 1) * (2 * m + k + 2));   // e_{k+1}/e_k
    }
    for (int j = 0; j < L; j++) {
        Dd acc;
        for (int k = 0; k <= j; k++) acc = acc + e[k] * G[j - k];
        out[j] = std::fabs(acc.hi + acc.lo);
    }
}

double pade_theta_of(int m, double u) {
    const int L = 200;
    std::vector<double> a(L);
    pade_rho_abs(m, L, a.data());
    double lo = 0.0, hi = 16.0;
    for (int it = 0; it < 300; it++) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = 0.0, p = std::pow(mid, 2 * m + 1);
        for (int j = 0; j < L; j++) {
            f += a[j] * p;
            p *= mid;
        }
        const bool ok = f < 1.0 && -std::log1p(-f) / mid <= u;
        (ok ? lo : hi) = mid;
    }
    return lo;
}

DxPade make_pade(int ubits) {
    static const int kPm[DX_PADE_NM] = {3, 5, 7, 9, 13};
    DxPade P;
    std::memset(&P, 0, sizeof P);
    const double u = std::ldexp(1.0, -ubits);
    for (int i = 0; i < DX_PADE_NM; i++) {
        const int m = kPm[i];
        P.m[i] = m;
        P.th[i] = bits(pade_theta_of(m, u));
        double v = 1.0;                       // c_j = (2m-j)! m! / ((2m)! j! (m-j)!)
        for (int j = 0; j <= m; j++) {
            P.c[i][j] = v;
            v = v * (m - j) / ((2.0 * m - j) * (j + 1));
        }
    }
    return P;
}

std::mutex g_mu;
uint32_t *g_status_ptr[64];
int g_sm_count[64];
bool g_once[64][16];
int g_mode[64][DX_NMAXF + 1];
bool g_mode_init[64];

// Measured on GB300 (stiff MRN-like cells, cost-sorted lane-per-cell tiles,
// 1,048,576 cells): lane per cell with both matrices in registers is fastest
// up to n = 6; from n = 7 to 12 the hybrid storage (current matrix in
// registers, next one in shared memory) beats both all-shared storage (4 % at
// n = 7, 9 % at n = 9, 26 % at n = 10: half the shared memory per warp, twice
// the resident warps) and warp per cell (15 % at n = 12); warp per cell above.
int default_mode(int n) {
    if (n <= DX_LPC_REG_NMAX) return DX_MODE_LPC_REG;
    if (n <= DX_LPC_NMAX) return DX_MODE_LPC_HYB;
    return DX_MODE_WPC;
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return dev;
}

}  // namespace

const DxConsts &dx_consts() {
    static const DxConsts K = make_consts(53);
    return K;
}

const DxPade *dx_pade_for(int ubits) {
    static const DxPade P53 = make_pade(53), P24 = make_pade(24);
    switch (ubits) {
        case 53: return &P53;
        case 24: return &P24;
        default: return nullptr;
    }
}

const DxConsts *dx_consts_for(int ubits) {
    static const DxConsts K24 = make_consts(24), K11 = make_consts(11);
    switch (ubits) {
        case 53: return &dx_consts();
        case 24: return &K24;
        case 11: return &K11;
        default: return nullptr;
    }
}

uint32_t *dx_status_ptr() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dx_status) != cudaSuccess) return nullptr;
        g_status_ptr[dev] = static_cast<uint32_t *>(p);
    }
    return g_status_ptr[dev];
}

int dx_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sm_count[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        g_sm_count[dev] = v;
    }
    return g_sm_count[dev];
}

bool dx_mode_valid(int n, int mode) {
    if (n < 2 || n > DX_NMAXF) return false;
    if (mode == DX_MODE_WPC) return true;
    if (mode == DX_MODE_LPC_REG) return n <= DX_LPC_REG_NMAX;
    if (mode == DX_MODE_LPC_SMEM) return n <= DX_LPC_NMAX;
    if (mode == DX_MODE_LPC_HYB) return n > DX_LPC_REG_NMAX && n <= DX_LPC_NMAX;
    return false;
}

int dx_mode_for(int n) {
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_mode_init[dev]) {
        for (int k = 0; k <= DX_NMAXF; k++) g_mode[dev][k] = default_mode(k);
        g_mode_init[dev] = true;
    }
    return (n >= 0 && n <= DX_NMAXF) ? g_mode[dev][n] : DX_MODE_WPC;
}

void dx_set_mode(int n, int mode) {
    if (!dx_mode_valid(n, mode)) return;
    dx_mode_for(n);   // initialise the table
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    g_mode[dev][n] = mode;
}

bool dx_once_per_device(int slot, bool (*fn)()) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || slot < 0 || slot >= 16) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_once[dev][slot]) return true;
    if (!fn()) return false;
    g_once[dev][slot] = true;
    return true;
}

extern "C" {

int drag_expm_get_status(cudaStream_t stream, uint32_t *status_out) {
    if (!status_out) return DRAG_ENULL;
    uint32_t *p = dx_status_ptr();
    if (!p) return DRAG_ECUDA;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, p, sizeof v, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return DRAG_ECUDA;
    if (cudaMemsetAsync(p, 0, sizeof v, stream) != cudaSuccess) return DRAG_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return DRAG_ECUDA;
    *status_out = v;
    return DRAG_OK;
}

int drag_expm_theta(int32_t k, double *theta_out) { return drag_expm_theta_target(k, 53, theta_out); }

int drag_expm_theta_target(int32_t k, int32_t ubits, double *theta_out) {
    if (!theta_out) return DRAG_ENULL;
    if (k < 1 || k > DX_K) return DRAG_EINVAL_SIZE;
    const DxConsts *K = dx_consts_for(ubits);
    if (!K) return DRAG_EINVAL_TARGET;
    long long b = K->th[k];
    std::memcpy(theta_out, &b, sizeof b);
    return DRAG_OK;
}

int drag_expm_pade_theta(int32_t m, int32_t ubits, double *theta_out) {
    if (!theta_out) return DRAG_ENULL;
    const DxPade *P = dx_pade_for(ubits);
    if (!P) return DRAG_EINVAL_TARGET;
    for (int i = 0; i < DX_PADE_NM; i++)
        if (P->m[i] == m) {
            const long long b = P->th[i];
            std::memcpy(theta_out, &b, sizeof b);
            return DRAG_OK;
        }
    return DRAG_EINVAL_SIZE;
}

const char *drag_expm_strerror(int code) {
    switch (code) {
        case DRAG_OK: return "success";
        case DRAG_EINVAL_SIZE: return "invalid size: ncells < 0, nspecies outside [1, DRAG_EXPM_NMAX] or bad dt";
        case DRAG_ENULL: return "a required pointer is NULL";
        case DRAG_EALIGN: return "a pointer is not 8-byte aligned";
        case DRAG_ECUDA: return "a CUDA runtime call or kernel launch failed";
        case DRAG_EWORKSPACE: return "workspace missing or too small";
        case DRAG_EBLOCKS: return "invalid block count or block descriptor array";
        case DRAG_EINVAL_TARGET: return "unsupported unit round-off target (use 53, 24 or 11; Pade: 53 or 24)";
        case DRAG_EINVAL_OPTION: return "invalid option combination (method, bound_test, arith)";
        case DRAG_ENOALLOC_LIMIT:
            return "batch exceeds the fixed scratch of drag_expm_apply_batched_noalloc "
                   "(DRAG_NOALLOC_MAX_BLOCKS / DRAG_NOALLOC_MAX_CELLS); use drag_expm_apply_batched with a workspace";
        default: return "unknown error code";
    }
}

int drag_expm_version(void) { return DRAG_EXPM_VERSION; }

}  // extern "C"
