// Forward update on HOST arrays: the cells are cut into chunks that move
// through a two-stream pipeline (host-to-device copies of chunk k + 1 and the
// device-to-host copy of chunk k - 1 overlap the update of chunk k). Each
// chunk is a column block of every SoA row (rho_g, the N rows of rho_d and
// t_s, the 3(N+1) velocity rows), so one pitched copy moves a whole array
// group. The update itself is drag_expm_apply on the chunk's device slab.
#include <cmath>
#include <cstring>
#include <mutex>

#include "dx_common.cuh"
#include "dx_modes.h"

namespace {

constexpr long long kDefaultChunk = 131072;
constexpr long long kBinnedChunk = 262144;   // chunks of lane-per-cell sizes take the binned forward

struct Pipe {
    std::mutex mu;   // held while a call enqueues its work (the fork / join events are shared)
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
};

std::mutex g_pipe_mu;
Pipe g_pipe[64];

// Internal streams and events of the current device (created once).
Pipe *pipe_for_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    Pipe &p = g_pipe[dev];
    if (!p.fork) {
        for (int i = 0; i < 2; i++) {
            if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
            if (cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
        }
        if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    return &p;
}

// Doubles of one chunk slab: rho_g, rho_d (N), t_s (N), v (3n).
size_t slab_doubles(int N, long long chunk) { return (size_t)chunk * (1 + 2 * (size_t)N + 3 * (size_t)(N + 1)); }

// Default chunk: the binned forward's threshold where that path applies, else
// smaller chunks (less copy time exposed at the ends of the pipeline).
long long chunk_of(long long chunk_cells, int nspecies) {
    if (chunk_cells > 0) return chunk_cells;
    const int n = nspecies + 1;
    return dx_binned_eligible(n, dx_mode_for(n), kBinnedChunk) ? kBinnedChunk : kDefaultChunk;
}

}  // namespace

extern "C" size_t drag_expm_host_workspace_bytes(int32_t nspecies, int64_t chunk_cells) {
    if (nspecies < 1 || nspecies > DRAG_EXPM_NMAX || chunk_cells < 0) return 0;
    return 2 * sizeof(double) * slab_doubles(nspecies, chunk_of(chunk_cells, nspecies));
}

extern "C" int drag_expm_apply_host(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                                    const double *t_s, double dt, const double *v_in, double *v_out,
                                    int64_t chunk_cells, void *workspace, size_t workspace_bytes,
                                    cudaStream_t stream) {
    if (ncells < 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX || chunk_cells < 0 || !(dt >= 0.0) ||
        !std::isfinite(dt))
        return DRAG_EINVAL_SIZE;
    if (ncells == 0) return DRAG_OK;
    if (!rho_g || !rho_d || !t_s || !v_in || !v_out || !workspace) return DRAG_ENULL;
    const long long chunk = chunk_of(chunk_cells, nspecies);
    const int N = nspecies, n = N + 1;
    if (workspace_bytes < drag_expm_host_workspace_bytes(nspecies, chunk)) return DRAG_EWORKSPACE;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return DRAG_EALIGN;
    Pipe *P = pipe_for_device();
    if (!P) return DRAG_ECUDA;
    std::lock_guard<std::mutex> lk(P->mu);
    if (cudaEventRecord(P->fork, stream) != cudaSuccess) return DRAG_ECUDA;
    for (int i = 0; i < 2; i++)
        if (cudaStreamWaitEvent(P->s[i], P->fork, 0) != cudaSuccess) return DRAG_ECUDA;

    const size_t hpitch = sizeof(double) * (size_t)ncells;    // host row pitch (SoA, stride ncells)
    int rc = DRAG_OK;
    long long k = 0;
    for (long long c0 = 0; c0 < ncells && rc == DRAG_OK; c0 += chunk, k++) {
        const long long cn = (ncells - c0) < chunk ? (ncells - c0) : chunk;
        cudaStream_t st = P->s[k & 1];
        double *slab = static_cast<double *>(workspace) + (size_t)(k & 1) * slab_doubles(N, chunk);
        double *drg = slab, *drd = drg + cn, *dts = drd + (size_t)N * cn, *dv = dts + (size_t)N * cn;
        const size_t w = sizeof(double) * (size_t)cn, dpitch = w;
        bool ok = cudaMemcpyAsync(drg, rho_g + c0, w, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpy2DAsync(drd, dpitch, rho_d + c0, hpitch, w, N, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpy2DAsync(dts, dpitch, t_s + c0, hpitch, w, N, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpy2DAsync(dv, dpitch, v_in + c0, hpitch, w, 3 * n, cudaMemcpyHostToDevice, st) ==
                       cudaSuccess;
        if (!ok) {
            rc = DRAG_ECUDA;
            break;
        }
        rc = drag_expm_apply(cn, N, drg, drd, dts, dt, dv, dv, st);
        if (rc != DRAG_OK) break;
        if (cudaMemcpy2DAsync(v_out + c0, hpitch, dv, dpitch, w, 3 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = DRAG_ECUDA;
    }
    // join both pipeline streams back into the caller's stream (also after an error, so the
    // caller's stream never runs ahead of work already queued)
    for (int i = 0; i < 2; i++) {
        if (cudaEventRecord(P->join[i], P->s[i]) != cudaSuccess ||
            cudaStreamWaitEvent(stream, P->join[i], 0) != cudaSuccess)
            rc = DRAG_ECUDA;
    }
    return rc;
}
