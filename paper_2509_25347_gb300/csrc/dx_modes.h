// Execution-mode table shared by the host-side dispatchers: for each matrix
// size n = N + 1 which kernel family runs a cell (lane per cell with the
// matrices in registers, in shared memory, or the current one in registers and
// the next in shared memory; or warp per cell). Defaults are set at load time;
// drag_expm_autotune() overwrites them from measurements.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dx_common.cuh"
#include "dx_lpc.cuh"

enum DxMode : int { DX_MODE_WPC = 0, DX_MODE_LPC_REG = 1, DX_MODE_LPC_SMEM = 2, DX_MODE_LPC_HYB = 3 };
#define DX_NMODES 4

#define DX_LPC_NMAX 12   // largest n with a lane-per-cell kernel
#define DX_LPC_REG_NMAX 6

int dx_mode_for(int n);            // current mode for matrix size n (current device)
// Lane-per-cell storage of a lane-per-cell mode.
inline int dx_lpc_store(int mode) {
    return mode == DX_MODE_LPC_REG ? DX_LPC_REGS : (mode == DX_MODE_LPC_HYB ? DX_LPC_HYBRID : DX_LPC_SHARED);
}
void dx_set_mode(int n, int mode);  // used by the autotuner
bool dx_mode_valid(int n, int mode);

int dx_launch_forward_f32(const DxConsts &K, long long ncells, int nspecies, const double *rho_g,
                          const double *rho_d, const double *t_s, double dt, const double *v_in, double *v_out,
                          cudaStream_t stream);
// store: DX_LPC_REGS / DX_LPC_SHARED / DX_LPC_HYBRID (dx_lpc.cuh) for the lane-per-cell modes.
int dx_launch_forward_lpc(const DxConsts &K, int n, int store, long long C, const double *rho_g,
                          const double *rho_d, const double *t_s, const double *v_in, double *v_out, double dt,
                          uint32_t *status, double *heat, cudaStream_t stream);

// Mixed-precision (FP32 matrix work) lane-per-cell forward for n <= DX_LPC_F32_NMAX
// (dx_forward_lpc.cu); arguments already checked by the caller.
#define DX_LPC_F32_NMAX 17
int dx_launch_forward_lpc_f32(const DxConsts &K, int n, long long C, const double *rho_g, const double *rho_d,
                              const double *t_s, const double *v_in, double *v_out, double dt, uint32_t *status,
                              cudaStream_t stream);

// Binned lane-per-cell forward (dx_batched.cu): the batched pipeline with one
// block over the whole input, for sizes whose batched mode is the current mode
// (n <= 9) and at least dx_binned_min_cells(n, false) cells. The lane-per-cell
// adjoint bins from dx_binned_min_cells(n, true) cells. DX_BINNED_UNAVAILABLE:
// no scratch could be had; the caller runs the tile-sorted kernel instead.
#define DX_BINNED_UNAVAILABLE 1
long long dx_binned_min_cells(int n, bool adjoint);
bool dx_binned_eligible(int n, int mode, long long C);
// thdr (null: none): also writes the adjoint tape (geometry as in drag_expm_apply_taped).
int dx_binned_forward(const DxConsts &K, long long C, int N, const double *rho_g, const double *rho_d,
                      const double *t_s, double dt, const double *v_in, double *v_out, uint32_t *status,
                      cudaStream_t stream, long long *thdr = nullptr, double *tm = nullptr, int tlevels = 0,
                      int tP = 0);

// Lane-per-cell forward that also writes the adjoint tape (dx_tape.cuh), for
// n <= DX_LPC_TAPE_NMAX with the default storage of each n (registers up to
// DX_LPC_REG_NMAX, hybrid above); the tape geometry as in drag_expm_apply_taped.
#define DX_LPC_TAPE_NMAX 12
int dx_launch_forward_lpc_taped(const DxConsts &K, int n, long long C, const double *rho_g, const double *rho_d,
                                const double *t_s, const double *v_in, double *v_out, double dt, uint32_t *status,
                                long long *hdr, double *m, int levels, int P, cudaStream_t stream);

// The cells of one input (C cells, N species, one dt) in bin order, binned by
// (k*, s*) as the binned forward bins them: *perm (device, C entries) holds
// each cell's index in its low 32 bits, bins in ascending (k*, s*). Scratch
// comes from the library's stream-ordered pool; the return value (null: no
// scratch could be had, nothing launched) is released with dx_binned_release
// on the same stream after the kernels that read *perm. 5 launches.
void *dx_binned_perm(const DxConsts &K, long long C, int N, const double *rho_g, const double *rho_d,
                     const double *t_s, double dt, uint32_t *status, cudaStream_t stream,
                     const unsigned long long **perm);
int dx_binned_release(void *scratch, cudaStream_t stream);

// Lane-per-cell adjoint (dx_backward_lpc.cu) for n <= DX_BWD_LPC_NMAX, run by
// drag_expm_backward(_taped) when the mode of n is a lane-per-cell one: cells
// binned by (k*, s*) over the whole input from DX_BINNED_MIN_CELLS cells on
// (6 launches), tile-sorted below (1 launch). thdr
// (null: none) is the tape the forward wrote (geometry as in
// drag_expm_backward_taped; tm its first level).
#define DX_BWD_LPC_NMAX 9
int dx_launch_backward_lpc(int n, long long C, const double *rho_g, const double *rho_d, const double *t_s,
                           double dt, const double *v_in, const double *grad_v_out, double *grad_v_in,
                           double *grad_rho_g, double *grad_rho_d, double *grad_t_s, uint32_t *status,
                           const long long *thdr, const double *tm, int levels, int P, cudaStream_t stream);
