// Measurement probes: what bounds the drag update on this GPU.
//
// The update is bound by the FP64 pipe (App. B, "Numerical cost", counts its
// work as n x n matrix products; the squarings of Eq. ExpEq1 dominate). These
// kernels measure the two FP64 paths an sm_103a core offers:
//
//   - DFMA (fma.rn.f64 on the FP64 pipe), the path every drag kernel uses;
//   - DMMA (mma.sync m8n8k4 f64 on the tensor cores),
//
// first as raw throughput (independent chains, one full wave of warps), then
// on the operation that matters, s squarings with row-sum restoration of a
// symmetric n x n matrix E (the similarity form of the propagator):
//   kind 0: the forward's own routine (dx_wpc_square_chain: the strict upper
//           triangle's dot products and the restorations on the build-time
//           round schedule, one warp per matrix);
//   kind 1: DMMA tiles: E padded to a multiple of 8, the 8 x 8 output tiles
//           on and above the diagonal (the product is symmetric) as 8 x 8 x 4
//           MMAs, then the same restorations on the FP64 pipe.
// Both write the squared matrices back, so the host can check that they agree.
// Nothing here is on the update's path; bench.py uses it for the roofline peak.
#include "dx_wpc.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kDfmaChains = 8;
constexpr int kDmmaChains = 4;
constexpr int kSqWarps = 4;

// D = A B + D for one warp: A 8x4 (row major), B 4x8 (column major), D 8x8,
// FP64. Lane l holds A[l/4][l%4], B[l%4][l/4] and D[l/4][2(l%4) + {0,1}].
__device__ __forceinline__ void dx_dmma_8x8x4(double &d0, double &d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kProbeThreads) dx_probe_dfma(long long iters, double seed, double *sink) {
    double a[kDfmaChains];
    const double b = 1.0 - 1e-9 * (double)(threadIdx.x & 7);
    const double c = 1e-12 * (double)((threadIdx.x + blockIdx.x) & 15);
#pragma unroll
    for (int j = 0; j < kDfmaChains; j++) a[j] = seed + j;
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < kDfmaChains; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kDfmaChains; j++) s += a[j];
    if (s == -1.0) *sink = s;   // never true for a positive seed; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) dx_probe_dmma(long long iters, double seed, double *sink) {
    double d[kDmmaChains][2];
    const double a = seed + 1e-3 * (double)(threadIdx.x & 31);
    const double b = 1e-6 * (double)((threadIdx.x + blockIdx.x) & 7);
#pragma unroll
    for (int j = 0; j < kDmmaChains; j++) d[j][0] = d[j][1] = (double)j;
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < kDmmaChains; j++) dx_dmma_8x8x4(d[j][0], d[j][1], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kDmmaChains; j++) s += d[j][0] + d[j][1];
    if (s == -1.0) *sink = s;
}

// Per-warp shared memory of the two squaring kernels (doubles).
__host__ __device__ __forceinline__ int sq_pad(int n) { return (n + 7) & ~7; }
__host__ __device__ __forceinline__ int sq_dmma_stride(int n) { return sq_pad(n) + 1; }
__host__ __device__ __forceinline__ int sq_warp_doubles(int kind, int n) {
    return kind == 0 ? 2 * n * dx_stride(n) + 2 * n : 2 * sq_pad(n) * sq_dmma_stride(n) + 2 * n;
}

__global__ void __launch_bounds__(kSqWarps * 32) dx_probe_square_dfma(int n, long long nmat, int reps,
                                                                     const double *E_in, const double *sig,
                                                                     double *E_out) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, ns = dx_stride(n);
    double *E0 = smem + wib * sq_warp_doubles(0, n), *E1 = E0 + n * ns;
    DxVecs V;
    V.sig = E1 + n * ns;
    V.tau = V.sig + n;
    V.xs = V.ds = nullptr;
    const long long warps = (long long)gridDim.x * kSqWarps;
    for (long long m = (long long)blockIdx.x * kSqWarps + wib; m < nmat; m += warps) {
        const double *src = E_in + m * n * n;
        for (int t = lane; t < n * n; t += 32) E0[(t / n) * ns + t % n] = src[t];
        if (lane < n) {
            const double sg = sig[m * n + lane];
            V.sig[lane] = sg;
            V.tau[lane] = 1.0 / sg;
        }
        __syncwarp();
        const double *R = dx_wpc_square_chain(lane, n, ns, reps, E0, E1, 0, V) ? E1 : E0;
        double *dst = E_out + m * n * n;
        for (int t = lane; t < n * n; t += 32) dst[t] = R[(t / n) * ns + t % n];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kSqWarps * 32, 1) dx_probe_square_dmma(int n, long long nmat, int reps,
                                                                     const double *E_in, const double *sig,
                                                                     double *E_out) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int P = sq_pad(n), ps = sq_dmma_stride(n), tiles = P / 8;
    const int g = lane >> 2, q = lane & 3;
    double *B0 = smem + wib * sq_warp_doubles(1, n), *B1 = B0 + P * ps;
    double *sg = B1 + P * ps, *tu = sg + n;
    const long long warps = (long long)gridDim.x * kSqWarps;
    for (long long m = (long long)blockIdx.x * kSqWarps + wib; m < nmat; m += warps) {
        const double *src = E_in + m * n * n;
        for (int t = lane; t < P * ps; t += 32) {
            const int i = t / ps, j = t - i * ps;
            B0[t] = (i < n && j < n) ? src[i * n + j] : 0.0;
            B1[t] = 0.0;
        }
        if (lane < n) {
            sg[lane] = sig[m * n + lane];
            tu[lane] = 1.0 / sg[lane];
        }
        __syncwarp();
        double *S = B0, *D = B1;
        for (int r = 0; r < reps; r++) {
            // upper tiles (I <= J) of S^2; S is symmetric, so its column-major
            // B operand B[k][c] = S[k][c] reads like the row-major A operand
            for (int I = 0; I < tiles; I++) {
                for (int J = I; J < tiles; J++) {
                    double d0 = 0.0, d1 = 0.0;
                    for (int kk = 0; kk < P; kk += 4) {
                        const double a = S[(8 * I + g) * ps + kk + q];
                        const double b = S[(kk + q) * ps + 8 * J + g];
                        dx_dmma_8x8x4(d0, d1, a, b);
                    }
                    // each entry on or above the diagonal, mirrored below it
                    const int row = 8 * I + g, c0 = 8 * J + 2 * q;
                    if (c0 >= row) {
                        D[row * ps + c0] = d0;
                        D[c0 * ps + row] = d0;
                    }
                    if (c0 + 1 >= row) {
                        D[row * ps + c0 + 1] = d1;
                        D[(c0 + 1) * ps + row] = d1;
                    }
                }
            }
            __syncwarp();
            // row-sum restoration E_ii = 1 - tau_i sum_{k != i} E_ik sigma_k
            if (lane < n) {
                double acc = 0.0;
                for (int k = 0; k < n; k++)
                    if (k != lane) acc = fma(D[lane * ps + k], sg[k], acc);
                D[lane * ps + lane] = fma(-tu[lane], acc, 1.0);
            }
            __syncwarp();
            double *t = S; S = D; D = t;
        }
        double *dst = E_out + m * n * n;
        for (int t = lane; t < n * n; t += 32) dst[t] = S[(t / n) * ps + t % n];
        __syncwarp();
    }
}

}  // namespace

extern "C" int drag_expm_probe_fp64_rate(int32_t kind, int64_t iters, double *sink, double *flop_out,
                                         cudaStream_t stream) {
    if ((kind != 0 && kind != 1) || iters < 1 || iters > (1LL << 40)) return DRAG_EINVAL_SIZE;
    if (!sink || !flop_out) return DRAG_ENULL;
    const int sms = dx_sm_count();
    if (sms < 1) return DRAG_ECUDA;
    const long long blocks = (long long)sms * kProbeBlocksPerSm;
    const double threads = (double)blocks * kProbeThreads;
    if (kind == 0) {
        dx_probe_dfma<<<(unsigned)blocks, kProbeThreads, 0, stream>>>(iters, 1.0, sink);
        *flop_out = 2.0 * kDfmaChains * (double)iters * threads;
    } else {
        dx_probe_dmma<<<(unsigned)blocks, kProbeThreads, 0, stream>>>(iters, 1.0, sink);
        *flop_out = 2.0 * 8 * 8 * 4 * kDmmaChains * (double)iters * (threads / 32);
    }
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" int drag_expm_probe_square(int32_t kind, int32_t n, int64_t nmat, int32_t reps, const double *E_in,
                                      const double *sig, double *E_out, cudaStream_t stream) {
    if ((kind != 0 && kind != 1) || n < 2 || n > DX_NMAXF || nmat < 0 || reps < 0 || reps > 4096)
        return DRAG_EINVAL_SIZE;
    if (nmat == 0) return DRAG_OK;
    if (!E_in || !sig || !E_out) return DRAG_ENULL;
    if ((reinterpret_cast<uintptr_t>(E_in) | reinterpret_cast<uintptr_t>(sig) | reinterpret_cast<uintptr_t>(E_out)) & 7)
        return DRAG_EALIGN;
    const int sms = dx_sm_count();
    if (sms < 1) return DRAG_ECUDA;
    const size_t smem = sizeof(double) * (size_t)kSqWarps * sq_warp_doubles(kind, n);
    void (*kern)(int, long long, int, const double *, const double *, double *) =
        kind == 0 ? dx_probe_square_dfma : dx_probe_square_dmma;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DRAG_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSqWarps * 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long want = (nmat + kSqWarps - 1) / kSqWarps;
    const long long grid = want < (long long)sms * per_sm ? want : (long long)sms * per_sm;
    kern<<<(unsigned)grid, kSqWarps * 32, smem, stream>>>(n, nmat, reps, E_in, sig, E_out);
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}
