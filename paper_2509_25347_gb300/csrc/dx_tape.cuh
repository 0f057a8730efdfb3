// Adjoint tape shared by the forward kernels that write it (warp per cell and
// lane per cell) and the adjoint that reads it.
#pragma once

#include "dx_common.cuh"

// The warp-per-cell forward replaces its last squarings by repeated
// applications: P^(2^q) v is computed as P (P (... P v)) with q = min(s*, DX_APPLY_Q). One squaring costs
// n(n+1)/2 tasks of n FP64 operations, one application 3n tasks of n + 2, so
// for n = 17 two squarings and one application (~206 warp-level FP64
// instructions) become four applications (~152).
#define DX_APPLY_Q 2

// ------------------------------------------------------------ adjoint tape
// The forward can record the restored symmetric iterates E_0 .. E_{s-q} it
// forms (q = min(s, DX_APPLY_Q); E_t = exp(2^(t-s) S) up to rounding), so the
// adjoint, which needs every E_t of the squaring phase, reads them instead of
// recomputing the Taylor step and the squarings. Level t of a cell is its
// upper triangle, row major with the diagonal, in a slot of dx_tape_slot(n)
// doubles; entry (i, j), i <= j, at dx_tape_index(n, i, j).
__host__ __device__ __forceinline__ int dx_tape_index(int n, int i, int j) { return i * (2 * n - i + 1) / 2 + j - i; }
__host__ __device__ __forceinline__ int dx_tape_slot(int n) { return (n * (n + 1) / 2 + 15) & ~15; }   // 128-byte slots
// Levels a cell with s* = s stores: E_0 .. E_{s-q}.
__host__ __device__ __forceinline__ int dx_tape_levels(int s) { return s - (s < DX_APPLY_Q ? s : DX_APPLY_Q) + 1; }
// Bytes of the fingerprint words that open a tape of C cells (256-byte multiple).
__host__ __device__ __forceinline__ size_t dx_tape_hdr_bytes(long long C) {
    return ((size_t)C * sizeof(long long) + 255) & ~(size_t)255;
}

// splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long dx_mix64(unsigned long long x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ULL;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebULL;
    x ^= x >> 31;
    return x;
}

// Fingerprint of a cell's inputs (rho_g, dt, and rho_d, t_s of species f on
// lane f), salted with the tape geometry; warp collective, same value on every
// lane. A tape entry is used only where the adjoint's inputs reproduce the
// fingerprint the forward stored, so a stale tape costs time, not accuracy.
// Species f contributes a term of its own, combined by XOR (order free).
__device__ __forceinline__ unsigned long long dx_fingerprint_term(int f, double rd, double ts) {
    return dx_mix64((unsigned long long)dx_bits(rd) + 0x9e3779b97f4a7c15ULL * (unsigned long long)f) ^
           dx_mix64((unsigned long long)dx_bits(ts) ^ (0xd1b54a32d192ed03ULL * (unsigned long long)f));
}
__device__ __forceinline__ long long dx_fingerprint_final(unsigned long long h, double rg, double dt,
                                                          unsigned long long salt) {
    return (long long)dx_mix64(h ^ dx_mix64((unsigned long long)dx_bits(rg) ^
                                            dx_mix64((unsigned long long)dx_bits(dt) ^ salt)));
}
__device__ __forceinline__ long long dx_cell_fingerprint(int lane, int N, double rg, double rd, double ts, double dt,
                                                         unsigned long long salt) {
    unsigned long long h = (lane >= 1 && lane <= N) ? dx_fingerprint_term(lane, rd, ts) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(DX_FULL, h, o);
    return dx_fingerprint_final(h, rg, dt, salt);
}

// The same fingerprint computed by one thread (species i + 1 at rd[i * stride], ts[i * stride]).
__device__ __forceinline__ long long dx_cell_fingerprint_serial(int N, double rg, const double *rd, const double *ts,
                                                                long long stride, double dt,
                                                                unsigned long long salt) {
    unsigned long long h = 0;
    for (int i = 0; i < N; i++) h ^= dx_fingerprint_term(i + 1, rd[i * stride], ts[i * stride]);
    return dx_fingerprint_final(h, rg, dt, salt);
}

// Salt of a tape's geometry.
__host__ __device__ __forceinline__ unsigned long long dx_tape_salt(int levels, int n) {
    return ((unsigned long long)levels << 8) | (unsigned long long)n;
}

// One cell's view of a tape (pointers already offset to the cell; m null: no tape).
struct DxTapeCell {
    long long *hdr;   // fingerprint word
    double *m;        // level 0; level t at m + t * P
    int levels, P;
};
