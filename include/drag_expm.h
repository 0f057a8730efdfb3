/*
 * drag_expm.h — C ABI of libdragexpm.so, the GB300 (sm_103a) FP64 exponential
 * drag update for a gas plus N pressureless dust species.
 *
 * What is computed (Sec. 2.2-2.3 of arXiv:2509.25347). Per cell, with
 * eps_i = rho_d,i / rho_g (Eq. DragEqVar2) and alpha_i = 1 / t_s,i
 * (Eq. DragEqVar3), the drag sub-system dU/dt = Omega U on the momenta
 * U = [rho_g v_g, rho_d,i v_d,i] (Eqs. DragEq, DragEqBis, jacobian) is solved
 * exactly over one step dt: U(t0 + dt) = exp(dt Omega) U(t0) (Eq. ExacSolEqu).
 * The densities do not change during the drag step, so the library works on
 * velocities: v_out = exp(dt Omega_v) v_in with Omega_v = Omega^T
 * (= D^-1 Omega D, D = diag(rho)), applied to the x, y and z components.
 * exp(dt Omega_v) is formed by Taylor scaling and squaring: Algorithm 2 picks
 * the Taylor order m* = m_{k*} (Table B.1) and the squaring count s* from the
 * 1-norm of A = dt Omega_v and the theta_m of Eq. B8 (u = 2^-53, K = 9); the
 * order-m Taylor polynomial of 2^-s* A is evaluated and squared s* times
 * (Eq. ExpEq1, Algorithm 6). Row sums of the propagator are kept equal to one
 * after the Taylor step and after every squaring (momentum conservation).
 *
 * Array layout (all FP64, structure of arrays, cell index fastest):
 *   rho_g [c]                      gas density, c = 0..ncells-1
 *   rho_d [i*ncells + c]           dust density of species i+1, i = 0..N-1
 *   t_s   [i*ncells + c]           stopping time of species i+1
 *   v     [(d*(N+1) + f)*ncells + c]  velocity component d (0=x,1=y,2=z) of
 *                                  fluid f (0 = gas, f = i >= 1 dust species i)
 *
 * Ownership: every pointer is caller-owned; the library never frees, keeps or
 * reallocates caller memory. Pointers documented as DEVICE must be device
 * (or managed) memory of the current CUDA device.
 *
 * Errors: functions return 0 on success or a negative DRAG_E* code for errors
 * found on the host, before anything is launched. Kernels run asynchronously
 * on `stream` (NULL = legacy default stream). Bad cell DATA is not a return
 * code: such a cell gets NaN outputs and sets a sticky bit that
 * drag_expm_get_status() reads. Valid data: rho_g > 0 finite, rho_d >= 0
 * finite, t_s > 0 (t_s = +inf is a species with alpha = 0), dt >= 0 finite.
 * A dust density below 1e-200 * rho_g is treated as 1e-200 * rho_g
 * (its feedback on the other fluids is then below FP64 resolution).
 */
#ifndef DRAG_EXPM_H
#define DRAG_EXPM_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DRAG_EXPM_VERSION 1

/* Largest supported number of dust species (matrix size N+1 <= 32). */
#define DRAG_EXPM_NMAX 31

/* Host-detected error codes. */
#define DRAG_OK 0
#define DRAG_EINVAL_SIZE (-1)   /* ncells < 0, nspecies outside [1, DRAG_EXPM_NMAX], dt < 0 or not finite */
#define DRAG_ENULL (-2)         /* a required pointer is NULL while ncells > 0 */
#define DRAG_EALIGN (-3)        /* a pointer is not 8-byte aligned */
#define DRAG_ECUDA (-4)         /* a CUDA runtime call or kernel launch failed */
#define DRAG_EWORKSPACE (-5)    /* workspace missing or smaller than required */
#define DRAG_EBLOCKS (-6)       /* bad block count in the batched entry point */
#define DRAG_ENOALLOC_LIMIT (-7) /* batch larger than drag_expm_apply_batched_noalloc's fixed scratch */
#define DRAG_EINVAL_TARGET (-8)  /* unit round-off target other than 53, 24 or 11 bits (Pade: 53, 24) */
#define DRAG_EINVAL_OPTION (-9)  /* bad drag_expm_options_t combination (see drag_expm_apply_opts) */

/* Sticky device status bits (drag_expm_get_status). */
#define DRAG_STATUS_BAD_CELL 0x1u      /* some cell had invalid data; its outputs are NaN */
#define DRAG_STATUS_BAD_BLOCK 0x2u     /* a batched block descriptor was out of range; it was skipped */
#define DRAG_STATUS_QUEUE_GUARD 0x4u   /* a persistent work loop hit its iteration guard */

/*
 * drag_expm_apply — forward drag update (Eq. ExacSolEqu) for ncells cells with
 * the same nspecies N and time step dt.
 *   ncells   : number of cells (0 is a no-op).
 *   nspecies : N, 1 <= N <= DRAG_EXPM_NMAX.
 *   rho_g, rho_d, t_s : DEVICE, layout above, read only.
 *   dt       : time step, >= 0 (dt = 0 returns v_in unchanged).
 *   v_in     : DEVICE, 3*(N+1)*ncells doubles, read only.
 *   v_out    : DEVICE, 3*(N+1)*ncells doubles, written. v_out == v_in (in
 *              place) is allowed; other overlaps are not.
 *   stream   : CUDA stream for the launches.
 * Returns DRAG_OK or a DRAG_E* code (nothing launched on error).
 * Lane-per-cell sizes (N <= 11 with the default modes) on enough cells run the
 * batched pipeline over one block: the cells are binned by (k*, s*) first, so
 * each warp runs 32 cells of equal cost. "Enough" is where that measured
 * faster than one tile-sorted launch on GB300: 196,608 cells at N = 2,
 * 131,072 at N = 3, 98,304 at N = 4 and 5, 40,960 at N = 6 and 7, 28,672 at
 * N = 8, 26,624 at N = 9 and 10, 24,576 at N = 11; never at N = 1, whose
 * single launch (a few dozen FP64 operations a
 * cell) was the faster at every size measured (drag_expm_apply_launches
 * reports the choice). Its scratch (12 bytes per
 * cell) is taken stream-ordered from a memory pool private to the library,
 * which keeps what it once allocated; the launches stay capturable in a CUDA
 * graph. If no scratch can be had, the single tile-sorted kernel runs instead.
 * The results are the same either way.
 */
int drag_expm_apply(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d, const double *t_s,
                    double dt, const double *v_in, double *v_out, cudaStream_t stream);

/* drag_expm_apply_launches — number of kernels drag_expm_apply launches for
 * (ncells, nspecies) with the current device's mode table (0 for bad sizes). */
int32_t drag_expm_apply_launches(int64_t ncells, int32_t nspecies);

/*
 * drag_expm_apply_target — drag_expm_apply for a lower accuracy target.
 * Eq. B8 defines theta_m for any unit round-off u (the paper names 2^-11,
 * 2^-24, 2^-113 and 2^-237 besides 2^-53); this entry point runs Algorithm 2
 * on the theta_{m_k} table of u = 2^-ubits, so cells take fewer Taylor terms
 * and squarings, and then the same FP64 arithmetic as drag_expm_apply. The
 * result is exp(dt Omega_v + dA) v_in with a backward error |dA| <= u |A| of
 * the Taylor step (App. B), plus FP64 rounding.
 *   ubits : 53 (same as drag_expm_apply), 24 (single-precision target) or
 *           11 (half-precision target); other values return DRAG_EINVAL_TARGET.
 * Other arguments as drag_expm_apply (in place allowed).
 */
int drag_expm_apply_target(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                           const double *t_s, double dt, const double *v_in, double *v_out, int32_t ubits,
                           cudaStream_t stream);

/* Methods of drag_expm_apply_opts. */
#define DRAG_METHOD_TAYLOR 0   /* the paper's Taylor scaling and squaring (Algorithm 2) */
#define DRAG_METHOD_PADE 1     /* diagonal Pade approximant (Eq. PadeEqu) with scaling and squaring */


typedef struct {
    int32_t ubits;       /* accuracy target u = 2^-ubits: 53, 24 or 11 (Pade: 53 or 24) */
    int32_t method;      /* DRAG_METHOD_TAYLOR or DRAG_METHOD_PADE */
    int32_t bound_test;  /* Taylor only: 1 = the paper's second modification (bound test) */
    int32_t arith;       /* DRAG_ARITH_FP64 (0) or DRAG_ARITH_FP32 (1, the mixed-precision path) */
} drag_expm_options_t;

/* Arithmetic of the matrix work in drag_expm_apply_opts. */
#define DRAG_ARITH_FP64 0
#define DRAG_ARITH_FP32 1   /* FP64 in/out, set-up and selection; FP32 Taylor, squarings, applications */

/*
 * drag_expm_apply_opts — forward update with the paper's variants of the
 * Taylor method and its Pade alternative. Host-side validation as
 * drag_expm_apply; opts is a HOST pointer.
 *   method = DRAG_METHOD_TAYLOR, bound_test = 0: drag_expm_apply_target.
 *   method = DRAG_METHOD_TAYLOR, bound_test = 1: after Algorithm 2, the
 *     Paterson-Stockmeyer blocks of T_m are bounded as in Eqs. Pat_Stk5 and
 *     Pat_Stk6 (Algorithm 8's b_exp) and the highest ones dropped while the
 *     bound holds, so the Taylor step has fewer terms (App. B, second
 *     modification); the 1-norms are those of the velocity-form matrices.
 *   method = DRAG_METHOD_PADE: R_mm(X) = D_mm(X)^-1 N_mm(X) (Eq. PadeEqu),
 *     m in {3, 5, 7, 9, 13} and the scaling s chosen with theta_m from the
 *     construction of Eqs. B5-B8 applied to R_mm (drag_expm_pade_theta): the
 *     smallest m with |A|_1 <= theta_m and s = 0, else m = 13 and the smallest
 *     s with 2^-s |A|_1 <= theta_13.
 *   arith = DRAG_ARITH_FP32 (the mixed-precision path of the lower targets):
 *     Taylor without the bound test at ubits = 24 only (Eq. B8 pairs
 *     u = 2^-24 with single precision), and no m_out / s_out. Inputs, outputs, the set-up and Algorithm 2 stay FP64; the Taylor
 *     step, the squarings and the applications run in FP32 (dust-to-gas ratios
 *     below 1e-30 are raised to it there, as 1e-200 in FP64). The result then
 *     carries FP32 rounding, ~1e-6 of the velocity scale.
 *   All variants restore the row sums after the approximant and every squaring.
 *   m_out : DEVICE int8[ncells] or NULL, receives the polynomial degree
 *           evaluated per cell (Taylor: m_{k*} or fewer terms after the bound
 *           test; Pade: m); 0 for invalid cells.
 *   s_out : DEVICE int16[ncells] or NULL, receives s* (-1 for invalid cells).
 * Both variants (and the plain Taylor method when m_out or s_out is asked
 * for) run one lane per cell for N = 1..5 under a lane-per-cell mode (the
 * default there; cells ordered by cost within tiles, 1 launch) and one warp
 * per cell otherwise; the mixed-precision path runs one lane per cell for N <= 11 under
 * a lane-per-cell mode (the default there) and for N = 12..16 always, one warp
 * per cell otherwise.
 * Returns DRAG_ENULL (opts NULL), DRAG_EINVAL_OPTION, DRAG_EINVAL_TARGET, or as
 * drag_expm_apply.
 */
int drag_expm_apply_opts(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                         const double *t_s, double dt, const double *v_in, double *v_out,
                         const drag_expm_options_t *opts, int8_t *m_out, int16_t *s_out, cudaStream_t stream);

/*
 * drag_expm_apply_host — drag_expm_apply on HOST arrays (same SoA layout,
 * stride ncells): the cells are processed in chunks of chunk_cells (0: 262,144
 * where drag_expm_apply bins that many cells, N = 2..11 with the default
 * modes, see there, else 131,072)
 * through a two-stream pipeline, so the host-to-device copies of one chunk
 * and the device-to-host copy of another overlap the update of a third. The
 * copies are asynchronous only from page-locked (pinned) host memory; with
 * pageable memory the call still works but the copies do not overlap.
 *   rho_g, rho_d, t_s, v_in : HOST, read only;  v_out : HOST, written (may be v_in).
 *   workspace : DEVICE, 256-byte aligned, >= drag_expm_host_workspace_bytes(nspecies,
 *               chunk_cells) bytes (two chunk slabs), owned by the caller.
 *   stream    : the work is ordered after the work already on `stream`, and
 *               `stream` waits for it (fork and join through internal streams of the
 *               library). v_out is valid once `stream` has reached that point.
 * Calls from several host threads on one device are serialised while they enqueue.
 * Returns as drag_expm_apply, or DRAG_EWORKSPACE / DRAG_EALIGN for the workspace.
 */
size_t drag_expm_host_workspace_bytes(int32_t nspecies, int64_t chunk_cells);
int drag_expm_apply_host(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                         const double *t_s, double dt, const double *v_in, double *v_out, int64_t chunk_cells,
                         void *workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * drag_expm_apply_heat — drag_expm_apply plus the energy epilogue: heat_out[c]
 * receives the kinetic energy (per unit volume) the drag step dissipates in
 * cell c, sum_f 1/2 rho_f (|v_in,f - V|^2 - |v_out,f - V|^2) with V the
 * centre-of-mass velocity (Eq. V_cm), which is >= 0. The frictional-heating
 * term of Eqs. GenEq_3 / CompVar4 integrated over the exact step is w * heat;
 * the gas energy changes by 1/2 rho_g (|v_g,out|^2 - |v_g,in|^2) + w * heat
 * (w = 1 deposits all dissipation into the gas). The paper does not spell out
 * EXP's energy update; this is the exact integral of its source terms.
 *   heat_out : DEVICE, ncells doubles, written (NaN for invalid cells).
 * Other arguments as drag_expm_apply (in place allowed).
 */
int drag_expm_apply_heat(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                         const double *t_s, double dt, const double *v_in, double *v_out, double *heat_out,
                         cudaStream_t stream);

/*
 * drag_expm_select — the (k*, s*) that drag_expm_apply uses for each cell:
 * Algorithm 2 with K = 9 on the 1-norm of A = dt Omega_v. The Taylor order is
 * m* = m_{k*} of Table B.1 and the cell costs k* + s* matrix products
 * (App. B, "Numerical cost").
 *   k_out : DEVICE int8[ncells], s_out : DEVICE int16[ncells] (either may be NULL).
 * Cells with invalid data get k = 0, s = -1 and set DRAG_STATUS_BAD_CELL.
 */
int drag_expm_select(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d, const double *t_s,
                     double dt, int8_t *k_out, int16_t *s_out, cudaStream_t stream);

/*
 * drag_expm_select_target — drag_expm_select with the theta table of
 * u = 2^-ubits (the (k*, s*) drag_expm_apply_target uses). ubits as
 * drag_expm_apply_target; other values return DRAG_EINVAL_TARGET.
 */
int drag_expm_select_target(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                            const double *t_s, double dt, int32_t ubits, int8_t *k_out, int16_t *s_out,
                            cudaStream_t stream);

/*
 * drag_expm_backward — adjoint of drag_expm_apply (reverse mode). Given
 * grad_v_out = dL/dv_out for a scalar loss L of v_out, returns
 *   grad_v_in  = dL/dv_in  = P^T grad_v_out per component, P = exp(dt Omega_v);
 *   grad_rho_d = dL/drho_d, grad_t_s = dL/dt_s, grad_rho_g = dL/drho_g,
 * through the Frechet derivative of the exponential, Z = L(A^T, G) with
 * A = dt Omega_v and G = sum_d grad_v_out,d v_in,d^T, and the dependence of
 * Omega on eps_i = rho_d,i/rho_g and alpha_i = 1/t_s,i (Eqs. DragEqVar2,
 * DragEqVar3, jacobian). The Frechet derivative is carried through the same
 * Algorithm 2 / Taylor / squaring steps as the forward (block-triangular
 * form [[A, E], [0, A]]), recomputing the forward on the fly (no storage).
 * Kernel family: one warp per cell, or, for N <= 8 under a lane-per-cell mode
 * (the default there), one lane per cell. The lane-per-cell adjoint bins the
 * cells by (k*, s*) over the whole input, with scratch from the library's
 * private stream-ordered pool (graph-capturable, 6 launches), from 32,768
 * cells at N = 1, 24,576 at N = 2 and 4,096 at N = 3..8, and sorts them by
 * cost within tiles below (1 launch; drag_expm_backward_launches reports the
 * choice); both give the same bits.
 *   rho_g, rho_d, t_s, v_in : DEVICE inputs of the forward call (read only).
 *   grad_v_out : DEVICE, 3*(N+1)*ncells doubles, layout of v (read only).
 *   grad_v_in  : DEVICE, layout of v, written (may be NULL).
 *   grad_rho_g : DEVICE, ncells doubles, written (may be NULL).
 *   grad_rho_d, grad_t_s : DEVICE, N*ncells doubles, layout of rho_d (may be NULL).
 * Outputs must not overlap inputs. Invalid cells get NaN gradients and set
 * DRAG_STATUS_BAD_CELL. Returns DRAG_OK or a DRAG_E* code.
 */
int drag_expm_backward(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                       const double *t_s, double dt, const double *v_in, const double *grad_v_out,
                       double *grad_v_in, double *grad_rho_g, double *grad_rho_d, double *grad_t_s,
                       cudaStream_t stream);

/* drag_expm_backward_launches — number of kernels drag_expm_backward (and
 * drag_expm_backward_taped) launch for (ncells, nspecies) with the current
 * device's mode table (0 for bad sizes). */
int32_t drag_expm_backward_launches(int64_t ncells, int32_t nspecies);

/*
 * Adjoint tape. The adjoint needs every restored iterate E_t = exp(2^(t-s*) S)
 * (S the symmetric similarity form of A = dt Omega_v, t = 0 .. s*-1) that the
 * forward's Taylor step and squarings (Algorithm 2 choices, Eq. ExpEq1) form;
 * drag_expm_backward recomputes them. drag_expm_apply_taped stores the ones
 * the forward forms, E_0 .. E_{s*-2} (E_0 alone for s* <= 1), in a tape, and
 * drag_expm_backward_taped reads them instead: it then forms neither the
 * Taylor polynomial nor those products. Where forward and adjoint run the same
 * kernel family (N >= 12, any N whose mode is warp per cell, and N <= 5 under
 * a lane-per-cell mode) the forward forms each E_t by the adjoint's own FP64
 * operations, and the gradients are identical to drag_expm_backward's. For
 * 6 <= N <= 11 with the default modes the lane-per-cell forward writes the
 * tape that the warp-per-cell adjoint reads, and the gradients agree with
 * drag_expm_backward's to rounding. The tape trades HBM for FP64 work:
 *   drag_expm_tape_bytes(ncells, nspecies, levels) bytes, about
 *   ncells * levels * 8 * (N+1)(N+2)/2 (rounded up to 128-byte slots),
 * where `levels` is the capacity per cell; a cell needs
 * drag_expm_tape_levels(s*) = max(s* - 1, 1) of them (drag_expm_select gives
 * s*). A cell that needs more is not recorded and its adjoint recomputes.
 * Layout (opaque to callers): ncells 8-byte fingerprint words, padded to a
 * 256-byte multiple, then per cell `levels` slots of packed upper triangles.
 * Each cell's fingerprint covers rho_g, rho_d, t_s, dt and the tape geometry;
 * the adjoint uses a cell's entries only if its own inputs reproduce the
 * fingerprint, so a stale or foreign tape gives correct gradients (at the
 * recomputing cost), up to 64-bit hash collisions.
 * drag_expm_tape_bytes returns 0 for bad sizes or levels outside
 * [1, DRAG_TAPE_MAX_LEVELS]; drag_expm_tape_levels returns 0 for s* < 0.
 */
#define DRAG_TAPE_MAX_LEVELS 2048
size_t drag_expm_tape_bytes(int64_t ncells, int32_t nspecies, int32_t levels);
int32_t drag_expm_tape_levels(int32_t sstar);

/*
 * drag_expm_apply_taped — drag_expm_apply that also writes the adjoint tape.
 * v_out is bit-identical to drag_expm_apply's under the same mode table: the
 * taped forward runs the same kernel family, lane per cell for N <= 11 with the
 * default modes (binned from the sizes drag_expm_apply bins,
 * tile-sorted otherwise),
 * one warp per cell for other sizes.
 *   levels : tape capacity per cell, 1 .. DRAG_TAPE_MAX_LEVELS.
 *   tape   : DEVICE, 256-byte aligned, >= drag_expm_tape_bytes(ncells,
 *            nspecies, levels) bytes, owned by the caller, written; must not
 *            overlap the other arrays.
 * Returns as drag_expm_apply, or DRAG_EINVAL_SIZE (levels), DRAG_ENULL (tape),
 * DRAG_EALIGN (tape alignment), DRAG_EWORKSPACE (tape_bytes too small).
 */
int drag_expm_apply_taped(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                          const double *t_s, double dt, const double *v_in, double *v_out, int32_t levels,
                          void *tape, size_t tape_bytes, cudaStream_t stream);

/*
 * drag_expm_backward_taped — drag_expm_backward reading the tape written by
 * drag_expm_apply_taped with the same ncells, nspecies and levels (read only).
 * Arguments and errors as drag_expm_backward, plus those of the tape as in
 * drag_expm_apply_taped.
 */
int drag_expm_backward_taped(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d,
                             const double *t_s, double dt, const double *v_in, const double *grad_v_out,
                             double *grad_v_in, double *grad_rho_g, double *grad_rho_d, double *grad_t_s,
                             int32_t levels, const void *tape, size_t tape_bytes, cudaStream_t stream);

/*
 * Batched drag update over AMR-like blocks. Block b holds ncells cells that
 * share nspecies N and time step dt. Its data live in slabs of the caller's
 * arrays, each laid out like a plain call with C = ncells:
 *   rho_g[cell_offset + c]
 *   rho_d[dust_offset + i*ncells + c],  t_s[dust_offset + i*ncells + c]
 *   v_in/v_out[vel_offset + (d*(N+1) + f)*ncells + c]
 * Blocks must not overlap. 40 bytes, 8-byte aligned.
 */
typedef struct drag_block {
    int64_t cell_offset;
    int64_t dust_offset;
    int64_t vel_offset;
    int32_t ncells;
    int32_t nspecies;
    double dt;
} drag_block_t;

/*
 * drag_rk1_apply — first-order implicit drag step with the analytic solution
 * of App. A.2 (Eqs. analytic_1-4), the paper's O(N) cost reference for EXP:
 * v_out = (I - dt Omega_v)^-1 v_in per cell (backward Euler; drag-only split
 * step, U^(n+1/2) = U^n in Eq. eq_rk1_2). First-order accurate in dt,
 * unconditionally stable, conserves momentum. Arguments, layout, in-place use
 * and error behaviour as drag_expm_apply.
 */
int drag_rk1_apply(int64_t ncells, int32_t nspecies, const double *rho_g, const double *rho_d, const double *t_s,
                   double dt, const double *v_in, double *v_out, cudaStream_t stream);

/*
 * drag_expm_batched_workspace_bytes — scratch bytes drag_expm_apply_batched
 * needs for nblocks blocks over arrays of total_cells gas cells (about
 * 12 bytes per cell plus 300 KB). Host only, no CUDA call.
 */
size_t drag_expm_batched_workspace_bytes(int64_t nblocks, int64_t total_cells);

/*
 * drag_expm_apply_batched — forward drag update (Eq. ExacSolEqu, Algorithm 6
 * with Algorithm 2) of every cell of every block in one pass. Cells are
 * binned by (N, k*, s*) on the device and processed by one persistent kernel,
 * so cells with different N and dt (hence different Taylor order and squaring
 * count) share the GPU without idle lanes. Results per cell equal those of
 * drag_expm_apply on the same cell (same arithmetic).
 *   nblocks     : number of descriptors (0 is a no-op).
 *   blocks      : DEVICE array of nblocks drag_block_t (read only).
 *   total_cells, rho_d_len, v_len : lengths (in doubles) of rho_g, of rho_d
 *                 and t_s, and of v_in/v_out; blocks outside them are skipped
 *                 and set DRAG_STATUS_BAD_BLOCK, as are blocks with bad N or dt.
 *   nspecies_max: upper bound on the blocks' N (sizes the shared memory); a
 *                 block with N > nspecies_max is skipped (its v_out slice is
 *                 left untouched) and sets DRAG_STATUS_BAD_BLOCK.
 *   rho_g, rho_d, t_s, v_in : DEVICE inputs; v_out : DEVICE output (may equal v_in).
 *   workspace   : DEVICE scratch of at least drag_expm_batched_workspace_bytes()
 *                 bytes, 256-byte aligned, caller-owned; contents are
 *                 overwritten. Must not be shared by calls in flight at once.
 * All work is queued on `stream` with no host synchronisation and no
 * allocation, so the call can be captured in a CUDA graph.
 * Returns DRAG_OK or DRAG_EBLOCKS / DRAG_EINVAL_SIZE / DRAG_ENULL /
 * DRAG_EALIGN / DRAG_EWORKSPACE / DRAG_ECUDA (nothing launched on error).
 */
int drag_expm_apply_batched(int64_t nblocks, const drag_block_t *blocks, int64_t total_cells, int64_t rho_d_len,
                            int64_t v_len, int32_t nspecies_max, const double *rho_g, const double *rho_d,
                            const double *t_s, const double *v_in, double *v_out, void *workspace,
                            size_t workspace_bytes, cudaStream_t stream);

/*
 * drag_expm_apply_batched_noalloc — drag_expm_apply_batched for callers that
 * cannot provide scratch memory. The paper has no counterpart; this is a
 * library-integration entry point. Some host codes cannot allocate device
 * memory for a library: their device memory is owned entirely by their own
 * pool or arena allocator reserved at start-up, or they must not call
 * cudaMalloc/cudaFree inside a time step because those calls synchronise the
 * device and stall the step's other streams, or they reach this library
 * through a thin binding that only passes the input and output arrays. This
 * entry point allocates nothing: it runs the same pipeline on a fixed scratch
 * array compiled into the library, which every GPU that loads the library
 * holds in global memory until the process exits.
 *   Limits: nblocks <= DRAG_NOALLOC_MAX_BLOCKS and total_cells <=
 *   DRAG_NOALLOC_MAX_CELLS; larger batches return DRAG_ENOALLOC_LIMIT and
 *   launch nothing. All other arguments and errors are those of
 *   drag_expm_apply_batched.
 *   The first call on each device looks up the array's device address (with
 *   that device current; cudaGetSymbolAddress allocates nothing) and keeps it
 *   for the process: make that first call before any stream capture, and do
 *   not call this entry point again after a cudaDeviceReset of that device
 *   (the kept address belongs to the old context).
 *   Calls share the array: each call clears what must start at zero, but two
 *   calls whose work overlaps on the GPU race on it, so order them (same
 *   stream, or an event between streams).
 */
#define DRAG_NOALLOC_MAX_BLOCKS 16384
#define DRAG_NOALLOC_MAX_CELLS 262144
int drag_expm_apply_batched_noalloc(int64_t nblocks, const drag_block_t *blocks, int64_t total_cells,
                                    int64_t rho_d_len, int64_t v_len, int32_t nspecies_max, const double *rho_g,
                                    const double *rho_d, const double *t_s, const double *v_in, double *v_out,
                                    cudaStream_t stream);

/*
 * Execution modes. Each matrix size n = N + 1 runs in one of the kernel
 * families below (all compute the same update, Eq. ExacSolEqu by Algorithm 6):
 * one lane per cell with its matrices in registers (n <= 6), in shared memory
 * (n <= 12), or the current one in registers and the next in shared memory
 * (n = 7..12); or one warp per cell (any n). Defaults: registers up to n = 6,
 * hybrid up to n = 12, warp above. The mode of n also picks the family of the
 * batched path (n <= 9), of the adjoint (lane per cell for n <= 6 under any
 * lane-per-cell mode) and of the mixed-precision path (lane per cell for
 * n <= 12 likewise, and for n = 13..17 always); drag_expm_autotune times the
 * forward only.
 */
#define DRAG_MODE_WARP_PER_CELL 0
#define DRAG_MODE_LANE_REGISTERS 1
#define DRAG_MODE_LANE_SHARED 2
#define DRAG_MODE_LANE_HYBRID 3   /* lane per cell, current matrix in registers, next in shared memory (n = 7..12) */

/* drag_expm_set_mode / drag_expm_get_mode — mode for nspecies on the current
 * device (host only). set returns DRAG_EINVAL_SIZE for an invalid pair. */
int drag_expm_set_mode(int32_t nspecies, int32_t mode);
int drag_expm_get_mode(int32_t nspecies, int32_t *mode);

/*
 * drag_expm_autotune — time every valid mode for N = 1..nspecies_max on
 * 32,768 synthetic MRN-like cells (dt/t_s over 1e-4..1e8) generated on the
 * current device, and keep the fastest per N. cache_path (may be NULL): a
 * text file; if it holds entries for this device (name, compute capability,
 * SM count) they are loaded instead of measuring, otherwise the measured
 * modes are appended. Allocates and frees ~12*(N+1)*256 KB of device memory
 * and synchronises `stream`; call it outside timed or captured regions.
 */
int drag_expm_autotune(int32_t nspecies_max, const char *cache_path, cudaStream_t stream);

/*
 * drag_expm_get_status — copy the current device's sticky status bits
 * (DRAG_STATUS_*) into *status_out and clear them. Synchronises `stream`.
 */
int drag_expm_get_status(cudaStream_t stream, uint32_t *status_out);

/*
 * drag_expm_theta — theta_{m_k} (Eq. B8, u = 2^-53) that the library uses
 * for k = 1..9 (Table B.1 prints these to five digits). Host only.
 */
int drag_expm_theta(int32_t k, double *theta_out);

/*
 * drag_expm_theta_target — theta_{m_k} of Eq. B8 for u = 2^-ubits (53, 24 or
 * 11; DRAG_EINVAL_TARGET otherwise), k = 1..9. Host only.
 */
int drag_expm_theta_target(int32_t k, int32_t ubits, double *theta_out);

/*
 * drag_expm_pade_theta — theta_m of the Pade variant (Eq. PadeEqu; the
 * construction of Eqs. B5-B8 applied to the [m/m] approximant) for
 * m in {3, 5, 7, 9, 13} and u = 2^-ubits, ubits in {53, 24}. Host only.
 * Returns DRAG_EINVAL_SIZE for another m, DRAG_EINVAL_TARGET for another ubits.
 */
int drag_expm_pade_theta(int32_t m, int32_t ubits, double *theta_out);

/*
 * Measurement probes. Not part of the drag update: they measure the resource
 * that bounds it, the FP64 rate of the GPU (App. B, "Numerical cost", counts
 * the update's work as n x n matrix products), for the roofline's peak and for
 * the choice between the FP64 pipe and the FP64 tensor cores.
 *
 * drag_expm_probe_fp64_rate — one launch of independent FP64 operation chains,
 * one full wave (4 blocks of 256 threads per SM), `iters` steps per chain.
 *   kind 0: DFMA (fma.rn.f64, the FP64 pipe); kind 1: DMMA (mma.sync
 *   m8n8k4 f64, the tensor cores).
 *   sink     : DEVICE, 1 double; written only by a result that never occurs.
 *   flop_out : HOST, receives the launch's FP64 FLOPs (an FMA is 2).
 * Time the launch with CUDA events on `stream`. Returns DRAG_OK, or
 * DRAG_EINVAL_SIZE (kind, iters outside 1..2^40) / DRAG_ENULL / DRAG_ECUDA.
 */
int drag_expm_probe_fp64_rate(int32_t kind, int64_t iters, double *sink, double *flop_out, cudaStream_t stream);

/*
 * drag_expm_probe_square — `reps` squarings, each followed by the row-sum
 * restoration E_ii = 1 - (1/sigma_i) sum_{k != i} E_ik sigma_k, of nmat
 * symmetric n x n matrices (the similarity form of the propagator, Eq. ExpEq1
 * with the restoration of the structured method), one warp per matrix.
 *   kind 0: the forward kernels' own routine (upper-triangle dot products and
 *           restorations on the FP64 pipe, build-time round schedule);
 *   kind 1: the products as 8x8x4 DMMA tiles (E padded to a multiple of 8,
 *           tiles on and above the diagonal), the restorations on the FP64 pipe.
 *   E_in  : DEVICE, nmat x n x n doubles, row major (read only).
 *   sig   : DEVICE, nmat x n doubles, sigma > 0 (read only).
 *   E_out : DEVICE, nmat x n x n doubles, the result (must not alias E_in).
 * n in 2..32, reps in 0..4096. Returns DRAG_OK or DRAG_EINVAL_SIZE /
 * DRAG_ENULL / DRAG_EALIGN / DRAG_ECUDA.
 */
int drag_expm_probe_square(int32_t kind, int32_t n, int64_t nmat, int32_t reps, const double *E_in,
                           const double *sig, double *E_out, cudaStream_t stream);

/* drag_expm_strerror — static text for a DRAG_E* code. */
const char *drag_expm_strerror(int code);

/* drag_expm_version — DRAG_EXPM_VERSION of the loaded library. */
int drag_expm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DRAG_EXPM_H */
