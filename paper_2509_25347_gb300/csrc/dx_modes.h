// Execution-mode table shared by the host-side dispatchers: for each matrix
// size n = N + 1 which kernel family runs a cell (lane per cell with the
// matrix in registers or shared memory, or warp per cell). Defaults are set at
// load time; drag_expm_autotune() overwrites them from measurements.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dx_common.cuh"

enum DxMode : int { DX_MODE_WPC = 0, DX_MODE_LPC_REG = 1, DX_MODE_LPC_SMEM = 2 };

#define DX_LPC_NMAX 12   // largest n with a lane-per-cell kernel
#define DX_LPC_REG_NMAX 6

int dx_mode_for(int n);            // current mode for matrix size n (current device)
void dx_set_mode(int n, int mode);  // used by the autotuner
bool dx_mode_valid(int n, int mode);

int dx_launch_forward_f32(const DxConsts &K, long long ncells, int nspecies, const double *rho_g,
                          const double *rho_d, const double *t_s, double dt, const double *v_in, double *v_out,
                          cudaStream_t stream);
int dx_launch_forward_lpc(const DxConsts &K, int n, bool smem, long long C, const double *rho_g,
                          const double *rho_d, const double *t_s, const double *v_in, double *v_out, double dt,
                          uint32_t *status, double *heat, cudaStream_t stream);
