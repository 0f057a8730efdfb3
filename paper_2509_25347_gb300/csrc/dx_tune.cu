// Autotuner for the execution mode of each matrix size n = N + 1: lane per
// cell with the matrix in registers, lane per cell with it in shared memory,
// or warp per cell. It times every valid mode on synthetic MRN-like cells
// generated on the device and keeps the fastest per n, per device. Results
// can be cached in a text file keyed by the device name and SM count.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "dx_common.cuh"
#include "dx_modes.h"

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float unit(unsigned long long &st) {
    st = mix64(st);
    return (float)((st >> 40) + 0.5) * (1.0f / 16777216.0f);   // (0, 1)
}

// MRN-like tuning cells: log-normal rho_g, total dust-to-gas U[0.01, 1] spread
// as a_j^0.5 over four decades of grain size, dt/t_s,j = 10^(x0 + 4) / a_j
// with x0 ~ U[-4, 4], v ~ U(-1, 1). Single-precision maths is enough here.
__global__ void tune_cells(long long C, int N, unsigned long long seed, double *rg, double *rd, double *ts,
                           double *v) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    unsigned long long st = seed ^ ((unsigned long long)c * 0x2545f4914f6cdd1dull);
    const float u1 = unit(st), u2 = unit(st);
    const float g = sqrtf(-2.0f * logf(u1)) * cosf(6.2831853f * u2);
    rg[c] = (double)expf(g);
    const float eps_tot = 0.01f + 0.99f * unit(st);
    const float x0 = -4.0f + 8.0f * unit(st);
    float wsum = 0.0f;
    for (int j = 0; j < N; j++) wsum += powf(10.0f, N > 1 ? 2.0f * j / (N - 1) : 0.0f);
    for (int j = 0; j < N; j++) {
        const float a = powf(10.0f, N > 1 ? 4.0f * j / (N - 1) : 0.0f);
        rd[(long long)j * C + c] = (double)(expf(g) * eps_tot * sqrtf(a) / wsum);
        ts[(long long)j * C + c] = (double)(a * powf(10.0f, -(x0 + 4.0f)));
    }
    for (int e = 0; e < 3 * (N + 1); e++) v[(long long)e * C + c] = (double)(2.0f * unit(st) - 1.0f);
}

std::string device_key() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::string name = p.name;
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    return name + "/sm" + std::to_string(p.major) + std::to_string(p.minor) + "/" + std::to_string(sms);
}

// Cache file: lines "<device_key> <n> <mode>".
bool load_cache(const char *path, int nmax, int *modes) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    const std::string key = device_key();
    char kbuf[256];
    int n, m, found = 0;
    while (std::fscanf(f, "%255s %d %d", kbuf, &n, &m) == 3) {
        if (key == kbuf && n >= 2 && n <= nmax && dx_mode_valid(n, m)) {
            modes[n] = m;
            found++;
        }
    }
    std::fclose(f);
    return found == nmax - 1;
}

void save_cache(const char *path, int nmax, const int *modes) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    const std::string key = device_key();
    for (int n = 2; n <= nmax; n++) std::fprintf(f, "%s %d %d\n", key.c_str(), n, modes[n]);
    std::fclose(f);
}

}  // namespace

extern "C" int drag_expm_set_mode(int32_t nspecies, int32_t mode) {
    if (nspecies < 1 || nspecies > DRAG_EXPM_NMAX) return DRAG_EINVAL_SIZE;
    if (!dx_mode_valid(nspecies + 1, mode)) return DRAG_EINVAL_SIZE;
    dx_set_mode(nspecies + 1, mode);
    return DRAG_OK;
}

extern "C" int drag_expm_get_mode(int32_t nspecies, int32_t *mode) {
    if (!mode) return DRAG_ENULL;
    if (nspecies < 1 || nspecies > DRAG_EXPM_NMAX) return DRAG_EINVAL_SIZE;
    *mode = dx_mode_for(nspecies + 1);
    return DRAG_OK;
}

extern "C" int drag_expm_autotune(int32_t nspecies_max, const char *cache_path, cudaStream_t stream) {
    if (nspecies_max < 1 || nspecies_max > DRAG_EXPM_NMAX) return DRAG_EINVAL_SIZE;
    const int nmax = nspecies_max + 1;
    int modes[DX_NMAXF + 1] = {0};
    if (cache_path && load_cache(cache_path, nmax, modes)) {
        for (int n = 2; n <= nmax; n++) dx_set_mode(n, modes[n]);
        return DRAG_OK;
    }
    const long long C = 32768;
    double *buf = nullptr;
    const size_t per_cell = 1 + 2 * (size_t)nspecies_max + 2 * 3 * (size_t)nmax;
    if (cudaMalloc(&buf, sizeof(double) * per_cell * C) != cudaSuccess) return DRAG_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = DRAG_OK;
    for (int n = 2; n <= nmax && rc == DRAG_OK; n++) {
        const int N = n - 1;
        double *rg = buf, *rd = rg + C, *ts = rd + N * C, *v = ts + N * C, *vo = v + 3 * n * C;
        tune_cells<<<(unsigned)((C + 255) / 256), 256, 0, stream>>>(C, N, 0x5eedull + n, rg, rd, ts, v);
        const int prev = dx_mode_for(n);
        float best = 1e30f;
        int best_mode = prev;
        for (int mode = 0; mode < DX_NMODES; mode++) {
            if (!dx_mode_valid(n, mode)) continue;
            dx_set_mode(n, mode);
            if ((rc = drag_expm_apply(C, N, rg, rd, ts, 1.0, v, vo, stream)) != DRAG_OK) break;   // warm-up
            cudaEventRecord(e0, stream);
            for (int r = 0; r < 3 && rc == DRAG_OK; r++) rc = drag_expm_apply(C, N, rg, rd, ts, 1.0, v, vo, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = DRAG_ECUDA;
            if (rc != DRAG_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_mode = mode;
            }
        }
        dx_set_mode(n, rc == DRAG_OK ? best_mode : prev);
        modes[n] = rc == DRAG_OK ? best_mode : prev;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc == DRAG_OK && cache_path) save_cache(cache_path, nmax, modes);
    return rc;
}
