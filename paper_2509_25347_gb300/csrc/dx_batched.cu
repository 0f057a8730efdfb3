// Batched forward drag update over AMR-like blocks whose cells differ in
// species count N and time step dt, hence in Taylor order m* and squaring
// count s* (Algorithm 2). The drag step is cell local (Sec. 3.5: each cell
// solves its own drag equation), so the batch is re-ordered freely:
//
//   1. prepare  (1 CTA)  : validate descriptors, prefix-sum block sizes, clear counters;
//   2. count    (grid)   : per cell, Algorithm 2 -> bin (n, k*, min(s*, 63)), histogram;
//   3. bins     (1 CTA)  : prefix sums of bin counts and of work items per bin;
//   4. scatter  (grid)   : cells -> bin-sorted permutation;
//   5. main     (persistent grids) : warps pull work items from atomic counters.
//      An item is 32 cells of one bin run lane-per-cell (small n, the lanes
//      of a warp share m* and s*, so no lane idles) or one cell run
//      warp-per-cell (large n), per n as dx_batch_modes() reads the mode table.
//      The two kinds of item run in two kernels, each with its own queue, so
//      that the register-heavy lane-per-cell code does not set the occupancy
//      of the warp-per-cell work.
//
// Every launch goes to the caller's stream; there is no host synchronisation
// and no allocation (scratch is the caller's workspace), so the whole call can
// be captured in a CUDA graph and replayed.
//
// The same pipeline also serves drag_expm_apply for lane-per-cell sizes on
// large inputs (dx_binned_forward): one block, scratch from a library-private
// stream-ordered memory pool. Binning by (k*, s*) over the whole input gives
// every warp 32 cells of one Taylor order and squaring count, where the plain
// lane-per-cell kernel can only sort within a tile of 512 cells.
#include <climits>
#include <cmath>
#include <mutex>

#include "dx_lpc.cuh"
#include "dx_modes.h"
#include "dx_wpc.cuh"

namespace {

constexpr int kSBins = 64;
constexpr int kBinsPerN = DX_K * kSBins;
constexpr int kNBins = (DX_NMAXF - 1) * kBinsPerN;   // n = 2..32
constexpr int kLpcWarps = 2;                         // warps per CTA, lane-per-cell kernel
constexpr int kWpcWarps = 4;                         // warps per CTA, warp-per-cell kernel
constexpr int kWpcMinBlocks = 6;                     // resident CTAs per SM the latter is compiled for
constexpr int kScanThreads = 1024;
constexpr int kBatchLpcNMax = 9;                     // largest n run lane-per-cell in the batched kernel
// Largest n the binned single-N forward runs lane per cell. Its n = 10..12
// items (hybrid storage, registers near the limit) have a kernel instance of
// their own, so that they do not set the register use of the n <= 9 items.
constexpr int kBinnedLpcNMax = 12;
// One n (the binned drag_expm_apply and adjoint): the bins are chunk-major,
// (chunk of consecutive cells, k*, s*), so that the items run one chunk after
// the other and a chunk's cells, scattered over its bins, are read from DRAM
// once and then from L2 (65,536 cells of N = 8 hold 37 MB). At most
// kMaxChunks chunks, so that the bin scans stay short.
constexpr long long kChunkMin = 65536;
constexpr long long kMaxChunks = 64;

struct Desc {
    long long cell_offset, dust_offset, vel_offset;
    int ncells, nspecies;
    double dt;
};
static_assert(sizeof(Desc) == sizeof(drag_block_t), "descriptor layout");

struct Work {
    unsigned long long *perm;   // (block << 32) | local cell, bin-sorted
    unsigned int *key;          // bin of each enumerated cell
    long long *blk_start;       // exclusive prefix of valid block sizes [nblocks + 1]
    unsigned int *hist, *offs, *cursor;               // [nbins + 1]
    unsigned int *item_w, *item_l;   // [nbins + 1] first item of each bin among warp- / lane-per-cell items
    unsigned int *ctr;   // [0] / [1] warp-per-cell queue counter / items, [2] enumerated cells,
                         // [3] / [4] lane-per-cell queue counter / items
    int nbins;           // kNBins (bins by n, k*, s*) or chunks x kBinsPerN (one n: chunk, k*, s*)
    int n_fixed;         // 0, or the n of every cell (chunk-major bins)
    long long chunk;     // cells per chunk (n_fixed only)
};

struct Modes {
    int m[DX_NMAXF + 1];
};

__device__ __forceinline__ int bin_of(int n, int k, int s) {
    return ((n - 2) * DX_K + (k - 1)) * kSBins + (s < kSBins - 1 ? s : kSBins - 1);
}

// Bin of enumerated cell g with (n, k*, s*) under the work's binning.
__device__ __forceinline__ unsigned int bin_of(const Work &W, long long g, int n, int k, int s) {
    if (!W.n_fixed) return (unsigned int)bin_of(n, k, s);
    return (unsigned int)((g / W.chunk) * kBinsPerN + (k - 1) * kSBins + (s < kSBins - 1 ? s : kSBins - 1));
}

// Matrix size of the cells in a bin.
__device__ __forceinline__ int n_of_bin(const Work &W, int bin) { return W.n_fixed ? W.n_fixed : bin / kBinsPerN + 2; }

// Warp-per-cell items of a bin of c cells of size n: pairs of cells where the
// forward sets up two at a time (dx_wpc_pairs), single cells above.
__host__ __device__ __forceinline__ unsigned int wpc_items(int n, unsigned int c) {
    return dx_wpc_pairs(n - 1) ? (c + 1) / 2 : c;
}

// A block is run only if its record is in range. N above nspecies_max is
// rejected too: the main kernels' per-warp shared-memory slices are sized for
// matrices up to nspecies_max + 1.
__device__ __forceinline__ bool desc_valid(const Desc &d, int nspecies_max, long long total_cells, long long rho_d_len,
                                           long long v_len) {
    if (d.ncells < 0 || d.nspecies < 1 || d.nspecies > nspecies_max || d.nspecies > DRAG_EXPM_NMAX) return false;
    const long long b = __double_as_longlong(d.dt);
    if (!((b & 0x7fffffffffffffffLL) == 0 || (b > 0 && b < 0x7ff0000000000000LL))) return false;   // dt >= 0 finite
    const long long C = d.ncells, N = d.nspecies;
    if (d.cell_offset < 0 || d.cell_offset + C > total_cells) return false;
    if (d.dust_offset < 0 || d.dust_offset + N * C > rho_d_len) return false;
    if (d.vel_offset < 0 || d.vel_offset + 3 * (N + 1) * C > v_len) return false;
    return true;
}

// Block-wide exclusive scan of one value per thread (kScanThreads threads).
template <typename T>
__device__ T block_exclusive_scan(T v, T *sh, T &total) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        T add = t >= o ? sh[t - o] : T(0);
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    total = sh[kScanThreads - 1];
    T ex = sh[t] - v;
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(kScanThreads)
dx_batch_prepare(long long nblocks, const Desc *blocks, int nspecies_max, long long total_cells, long long rho_d_len,
                 long long v_len, Work W, uint32_t *status) {
    __shared__ long long sh[kScanThreads];
    const int t = threadIdx.x;
    for (int i = t; i < W.nbins; i += kScanThreads) W.hist[i] = 0;
    if (t < 8) W.ctr[t] = 0;
    const long long per = (nblocks + kScanThreads - 1) / kScanThreads;
    const long long b0 = t * per, b1 = b0 + per < nblocks ? b0 + per : nblocks;
    long long sum = 0;
    bool bad = false;
    for (long long b = b0; b < b1; b++) {
        const Desc d = blocks[b];
        const bool ok = desc_valid(d, nspecies_max, total_cells, rho_d_len, v_len);
        bad |= !ok;
        sum += ok ? d.ncells : 0;
    }
    long long total;
    long long run = block_exclusive_scan(sum, sh, total);
    for (long long b = b0; b < b1; b++) {
        W.blk_start[b] = run;
        const Desc d = blocks[b];
        run += desc_valid(d, nspecies_max, total_cells, rho_d_len, v_len) ? d.ncells : 0;
    }
    if (t == 0) {
        W.blk_start[nblocks] = total;
        // non-overlapping valid blocks never hold more cells than rho_g
        W.ctr[2] = (unsigned int)(total < total_cells ? total : total_cells);
        if (total > total_cells) bad = true;
    }
    if (bad) atomicOr(status, DRAG_STATUS_BAD_BLOCK);
}

// Block b with blk_start[b] <= g < blk_start[b + 1] (blocks of size 0 are skipped).
__device__ __forceinline__ long long find_block(const long long *bs, long long nblocks, long long g) {
    long long lo = 0, hi = nblocks;   // invariant: bs[lo] <= g < bs[hi]
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (bs[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void dx_batch_count(long long nblocks, const Desc *blocks, const double *rho_g, const double *rho_d,
                               const double *t_s, Work W, DxConsts K) {
    const long long total = W.ctr[2];
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long b = find_block(W.blk_start, nblocks, g);
        const Desc d = blocks[b];
        const long long c = g - W.blk_start[b], C = d.ncells;
        const int N = d.nspecies;
        const double rg = rho_g[d.cell_offset + c];
        const double *rd = rho_d + d.dust_offset + c, *ts = t_s + d.dust_offset + c;
        bool ok = dx_pos_finite(rg);
        for (int i = 0; i < N && ok; i++) ok = dx_nonneg_finite(rd[i * C]) && dx_pos_or_inf(ts[i * C]);
        int kk = 1, s = 0;
        if (ok) {
            // 1-norm of A = dt Omega_v in ascending species order (as the apply kernels do)
            double s1 = 0.0, ai0s[DRAG_EXPM_NMAX];
            long long cmax = 0;
            for (int i = 0; i < N; i++) {
                const double eps = __ddiv_rn(rd[i * C], rg), alpha = __ddiv_rn(1.0, ts[i * C]);
                const double a0i = __dmul_rn(__dmul_rn(eps, alpha), d.dt), ai0 = __dmul_rn(alpha, d.dt);
                s1 = __dadd_rn(s1, a0i);
                ai0s[i] = ai0;
                const long long cb = dx_bits(__dadd_rn(a0i, ai0));
                cmax = cb > cmax ? cb : cmax;
            }
            double col0 = s1;
            for (int i = 0; i < N; i++) col0 = __dadd_rn(col0, ai0s[i]);
            const long long nb = dx_bits(col0) > cmax ? dx_bits(col0) : cmax;
            if (dx_norm_ok(nb)) dx_select(__longlong_as_double(nb), K, kk, s);   // else the cell routine flags it
        }
        const unsigned int key = bin_of(W, g, N + 1, kk, s);
        W.key[g] = key;
        atomicAdd(&W.hist[key], 1u);
    }
}

__global__ void __launch_bounds__(kScanThreads) dx_batch_bins(Work W, Modes M) {
    __shared__ long long sh[kScanThreads];
    const int t = threadIdx.x;
    const int nb = W.nbins;
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int i0 = t * per < nb ? t * per : nb, i1 = i0 + per < nb ? i0 + per : nb;
    long long cs = 0, ws = 0, ls = 0;
    for (int i = i0; i < i1; i++) {
        const unsigned int c = W.hist[i];
        const bool wpc = M.m[n_of_bin(W, i)] == DX_MODE_WPC;
        cs += c;
        ws += wpc ? wpc_items(n_of_bin(W, i), c) : 0;
        ls += wpc ? 0 : (c + 31) / 32;
    }
    long long ctot, wtot, ltot;
    long long crun = block_exclusive_scan(cs, sh, ctot);
    long long wrun = block_exclusive_scan(ws, sh, wtot);
    long long lrun = block_exclusive_scan(ls, sh, ltot);
    for (int i = i0; i < i1; i++) {
        const unsigned int c = W.hist[i];
        const bool wpc = M.m[n_of_bin(W, i)] == DX_MODE_WPC;
        W.offs[i] = (unsigned int)crun;
        W.cursor[i] = (unsigned int)crun;
        W.item_w[i] = (unsigned int)wrun;
        W.item_l[i] = (unsigned int)lrun;
        crun += c;
        wrun += wpc ? wpc_items(n_of_bin(W, i), c) : 0;
        lrun += wpc ? 0 : (c + 31) / 32;
    }
    if (t == 0) {
        W.offs[nb] = (unsigned int)ctot;
        W.item_w[nb] = (unsigned int)wtot;
        W.item_l[nb] = (unsigned int)ltot;
        W.ctr[1] = (unsigned int)wtot;
        W.ctr[4] = (unsigned int)ltot;
    }
}

__global__ void dx_batch_scatter(long long nblocks, Work W) {
    const long long total = W.ctr[2];
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long b = find_block(W.blk_start, nblocks, g);
        const unsigned long long local = (unsigned long long)(g - W.blk_start[b]);
        const unsigned int pos = atomicAdd(&W.cursor[W.key[g]], 1u);
        W.perm[pos] = ((unsigned long long)b << 32) | local;
    }
}

struct MainArgs {
    const Desc *blocks;
    const double *rho_g, *rho_d, *t_s, *v_in;
    double *v_out;
    uint32_t *status;
    int warp_doubles;   // per-warp shared-memory slice (doubles)
    int pair_od, pair_doubles;   // warp-per-cell kernel: the pair tables after each slice (od entries, doubles)
    // adjoint tape (taped lane-per-cell kernel only): the cell at cell_offset +
    // c of its block has its fingerprint at thdr[cell], its level t at
    // tm + (cell * tlevels + t) * tP
    long long *thdr;
    double *tm;
    int tlevels, tP;
};

template <int NF, int ST, bool TAPE>
__device__ __forceinline__ void lpc_item(int lane, const MainArgs &a, const Desc &d, long long c, const DxConsts &K,
                                         const double *bsh, double *wsm) {
    const long long C = d.ncells;
    DxTapeCell tc{nullptr, nullptr, 0, 0};
    if (TAPE) {
        const long long cell = d.cell_offset + c;
        tc = DxTapeCell{a.thdr + cell, a.tm + (size_t)cell * a.tlevels * a.tP, a.tlevels, a.tP};
    }
    dx_lpc_forward_cell<NF, ST>(lane, a.rho_g + d.cell_offset + c, a.rho_d + d.dust_offset + c,
                                  a.t_s + d.dust_offset + c, a.v_in + d.vel_offset + c, a.v_out + d.vel_offset + c, C,
                                  d.dt, K, bsh, wsm, a.status, nullptr, tc);
}

template <bool TAPE, bool BIG>
__device__ __forceinline__ void lpc_dispatch(int n, int lane, const MainArgs &a, const Desc &d, long long c,
                                             const DxConsts &K, const double *bsh, double *wsm) {
    // the storage per n is compiled in: registers up to n = 6, hybrid above;
    // BIG: the n = 10..12 items of the binned single-N forward
    switch (n) {
#define DX_ITEM(NF, ST) \
    case NF: lpc_item<NF, ST, TAPE>(lane, a, d, c, K, bsh, wsm); break;
#define DX_ITEM_SMALL(NF, ST) \
    case NF: if constexpr (!BIG) lpc_item<NF, ST, TAPE>(lane, a, d, c, K, bsh, wsm); break;
#define DX_ITEM_BIG(NF, ST) \
    case NF: if constexpr (BIG) lpc_item<NF, ST, TAPE>(lane, a, d, c, K, bsh, wsm); break;
        DX_ITEM_SMALL(2, DX_LPC_REGS)
        DX_ITEM_SMALL(3, DX_LPC_REGS)
        DX_ITEM_SMALL(4, DX_LPC_REGS)
        DX_ITEM_SMALL(5, DX_LPC_REGS)
        DX_ITEM_SMALL(6, DX_LPC_REGS)
        DX_ITEM_SMALL(7, DX_LPC_HYBRID)
        DX_ITEM_SMALL(8, DX_LPC_HYBRID)
        DX_ITEM_SMALL(9, DX_LPC_HYBRID)
        DX_ITEM_BIG(10, DX_LPC_HYBRID)
        DX_ITEM_BIG(11, DX_LPC_HYBRID)
        DX_ITEM_BIG(12, DX_LPC_HYBRID)
#undef DX_ITEM_BIG
#undef DX_ITEM_SMALL
#undef DX_ITEM
        default: break;
    }
}

// Pulls items of one kind (warp- or lane-per-cell) from that kind's queue;
// item_offs numbers the items of that kind bin by bin. Returns when the queue
// is empty. Each claim takes a fresh item, so a warp runs at most nitems + 1
// of them.
template <typename F>
__device__ __forceinline__ void dx_batch_queue(unsigned int *counter, unsigned int nitems,
                                               const unsigned int *item_offs, int nbins, uint32_t *status,
                                               F &&run) {
    const int lane = threadIdx.x & 31;
    for (unsigned int guard = 0;; guard++) {
        if (guard > nitems) {
            if (lane == 0) atomicOr(status, DRAG_STATUS_QUEUE_GUARD);
            break;
        }
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(DX_FULL, item, 0);
        if (item >= nitems) break;
        // bin holding this item: last bin with item_offs[bin] <= item
        int lo = 0, hi = nbins;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (item_offs[mid] <= item) lo = mid; else hi = mid;
        }
        run(lo, item - item_offs[lo]);
    }
}

// Warp-per-cell items: one cell, or for sizes set up two at a time
// (dx_wpc_pairs) two consecutive cells of the bin, which may belong to
// different blocks (their own slabs and dt).
__global__ void __launch_bounds__(kWpcWarps * 32, kWpcMinBlocks)
dx_batch_main_wpc(MainArgs a, Work W, DxConsts K) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *wsm = smem + wib * (a.warp_doubles + a.pair_doubles);
    unsigned short *od = reinterpret_cast<unsigned short *>(wsm + a.warp_doubles);
    unsigned short *hp = od + a.pair_od;
    int table_n = 0;
    dx_batch_queue(&W.ctr[0], W.ctr[1], W.item_w, W.nbins, a.status, [&](int bin, unsigned int sub) {
        const int n = n_of_bin(W, bin), N = n - 1;
        if (table_n != n) {
            dx_build_pairs_warp(lane, n, od, hp);
            table_n = n;
        }
        if (!dx_wpc_pairs(N)) {
            const unsigned long long p = W.perm[W.offs[bin] + sub];
            const Desc d = a.blocks[p >> 32];
            const long long c = (long long)(p & 0xffffffffull);
            dx_wpc_forward_cell(lane, d.nspecies, a.rho_g + d.cell_offset + c, a.rho_d + d.dust_offset + c,
                                a.t_s + d.dust_offset + c, a.v_in + d.vel_offset + c, a.v_out + d.vel_offset + c,
                                d.ncells, d.dt, K, wsm, od, hp, a.status);
            return;
        }
        const int ns = dx_stride(n);
        double *E0 = wsm, *E1 = wsm + n * ns;
        DxVecs V0;
        DxFwdBufs B;
        dx_wpc_fwd_layout(E1 + n * ns, n, V0, B);
        double *v1 = wsm + dx_wpc_fwd_warp_doubles(n);
        const DxVecs V1{v1, v1 + n, v1 + 2 * n, v1 + 3 * n};
        const unsigned int pos0 = W.offs[bin] + 2 * sub;
        const int cells = pos0 + 1 < W.offs[bin + 1] ? 2 : 1;
        // set-up inputs: half h takes the item's cell h (half 1 repeats cell 0 when the
        // item holds one cell; its result is not used), lane 16 h + i - 1 its species i
        const int h = lane >> 4, l = lane & 15;
        const unsigned long long ph = W.perm[pos0 + (h < cells ? h : 0)];
        const Desc dh = a.blocks[ph >> 32];
        const long long ch = (long long)(ph & 0xffffffffull);
        const double rg = a.rho_g[dh.cell_offset + ch];
        double rd = 0.0, ts = INFINITY;
        if (l < N) {
            rd = a.rho_d[dh.dust_offset + ch + (long long)l * dh.ncells];
            ts = a.t_s[dh.dust_offset + ch + (long long)l * dh.ncells];
        }
        int k0, s0, k1, s1;
        const unsigned valid = dx_wpc_setup_pair(lane, N, rg, rd, ts, dh.dt, K, V0, V1, k0, s0, k1, s1);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            if (e >= cells) break;
            const unsigned long long p = W.perm[pos0 + e];
            const Desc d = a.blocks[p >> 32];
            const long long c = (long long)(p & 0xffffffffull);
            double *vop = a.v_out + d.vel_offset + c;
            if (!((valid >> e) & 1u)) {
                dx_wpc_fail_cell(lane, n, vop, d.ncells, a.status, nullptr);
                continue;
            }
            DxCellIn ci;
            dx_wpc_load_cell(lane, N, a.rho_g + d.cell_offset + c, a.rho_d + d.dust_offset + c,
                             a.t_s + d.dust_offset + c, a.v_in + d.vel_offset + c, d.ncells, ci);
            const DxVecs &V = e ? V1 : V0;
            const double sg = lane < n ? V.sig[lane] : 1.0;
            dx_wpc_forward_run(lane, N, V, E0, E1, B, e ? k1 : k0, e ? s1 : s0, sg, ci, vop, d.ncells, d.dt, K,
                               od, hp, (double *)nullptr, (double *)nullptr, DxTapeCell{nullptr, nullptr, 0, 0});
        }
    });
}

template <bool TAPE, bool BIG>
__global__ void __launch_bounds__(kLpcWarps * 32)
dx_batch_main_lpc(MainArgs a, Work W, Modes M, DxConsts K) {
    (void)M;   // lane-per-cell items only (the bins already carry the mode)
    extern __shared__ double smem[];
    double *bsh = smem;
    for (int t = threadIdx.x; t < 32; t += blockDim.x) bsh[t] = K.b[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *wsm = smem + 32 + wib * a.warp_doubles;
    dx_batch_queue(&W.ctr[3], W.ctr[4], W.item_l, W.nbins, a.status, [&](int bin, unsigned int sub) {
        const int n = n_of_bin(W, bin);
        const unsigned int pos = W.offs[bin] + 32 * sub + lane;
        if (pos < W.offs[bin + 1]) {
            const unsigned long long p = W.perm[pos];
            const Desc d = a.blocks[p >> 32];
            lpc_dispatch<TAPE, BIG>(n, lane, a, d, (long long)(p & 0xffffffffull), K, bsh, wsm);
        }
        __syncwarp();
    });
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t perm, key, blk_start, hist, offs, cursor, item_w, item_l, ctr, total;
};

Layout layout(long long nblocks, long long total_cells, int nbins = kNBins) {
    Layout L;
    size_t o = 0;
    L.perm = o; o += align256(sizeof(unsigned long long) * (size_t)total_cells);
    L.key = o; o += align256(sizeof(unsigned int) * (size_t)total_cells);
    L.blk_start = o; o += align256(sizeof(long long) * (size_t)(nblocks + 1));
    L.hist = o; o += align256(sizeof(unsigned int) * ((size_t)nbins + 1));
    L.offs = o; o += align256(sizeof(unsigned int) * ((size_t)nbins + 1));
    L.cursor = o; o += align256(sizeof(unsigned int) * ((size_t)nbins + 1));
    L.item_w = o; o += align256(sizeof(unsigned int) * ((size_t)nbins + 1));
    L.item_l = o; o += align256(sizeof(unsigned int) * ((size_t)nbins + 1));
    L.ctr = o; o += align256(sizeof(unsigned int) * 8);
    L.total = o;
    return L;
}

// Per-warp shared memory (doubles) each main kernel needs for matrices of
// n_min..n_max; *has_wpc / *has_lpc tell whether any of them runs that way.
void warp_doubles_for(const Modes &M, int n_min, int n_max, int *wpc, int *lpc, bool *has_wpc, bool *has_lpc) {
    *wpc = *lpc = 0;
    *has_wpc = *has_lpc = false;
    for (int n = n_min; n <= n_max; n++) {
        int need = 0;
        if (M.m[n] == DX_MODE_WPC) {
            *has_wpc = true;
            need = dx_wpc_fwd_warp_doubles(n) + (dx_wpc_pairs(n - 1) ? 4 * n : 0);   // + a second cell's vectors
            *wpc = need > *wpc ? need : *wpc;
            continue;
        }
        *has_lpc = true;
        const bool hyb = M.m[n] == DX_MODE_LPC_HYB;
        if (M.m[n] == DX_MODE_LPC_SMEM || hyb) {
            switch (n) {
#define DX_NEED(NF) \
    case NF: need = hyb ? dx_lpc_warp_smem_doubles<NF, DX_LPC_HYBRID>() : dx_lpc_warp_smem_doubles<NF, DX_LPC_SHARED>(); break;
                DX_NEED(2)
                DX_NEED(3)
                DX_NEED(4)
                DX_NEED(5)
                DX_NEED(6)
                DX_NEED(7)
                DX_NEED(8)
                DX_NEED(9)
                DX_NEED(10)
                DX_NEED(11)
                DX_NEED(12)
#undef DX_NEED
                default: break;
            }
        }
        *lpc = need > *lpc ? need : *lpc;
    }
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

}  // namespace

// Kernel family per n for the batched path: 32 cells per warp (lane per cell)
// or one (warp per cell) as the device's mode table says (drag_expm_autotune
// sets it from measurements), for n <= kBatchLpcNMax; warp per cell above.
// The lane-per-cell storage here is the one compiled into dx_batch_main_lpc:
// registers up to DX_LPC_REG_NMAX, the hybrid storage above. Items are binned
// by (n, k*, s*), so the 32 lanes of a lane-per-cell item run exactly their
// own Taylor order and squaring count.
Modes dx_batch_modes() {
    Modes M;
    for (int n = 0; n <= DX_NMAXF; n++) {
        if (n < 2 || n > kBatchLpcNMax || dx_mode_for(n) == DX_MODE_WPC)
            M.m[n] = DX_MODE_WPC;
        else
            M.m[n] = n <= DX_LPC_REG_NMAX ? DX_MODE_LPC_REG : DX_MODE_LPC_HYB;
    }
    return M;
}

// Chunk-major binning of C cells of one n: cells per chunk and bins.
long long fixed_n_chunk(long long C) {
    const long long by_count = (C + kMaxChunks - 1) / kMaxChunks;
    return by_count > kChunkMin ? by_count : kChunkMin;
}
int fixed_n_bins(long long C) { return (int)((C + fixed_n_chunk(C) - 1) / fixed_n_chunk(C)) * kBinsPerN; }

Work work_at(char *ws, const Layout &L, int nbins = kNBins, int n_fixed = 0, long long chunk = 0) {
    Work W;
    W.nbins = nbins;
    W.n_fixed = n_fixed;
    W.chunk = chunk;
    W.perm = reinterpret_cast<unsigned long long *>(ws + L.perm);
    W.key = reinterpret_cast<unsigned int *>(ws + L.key);
    W.blk_start = reinterpret_cast<long long *>(ws + L.blk_start);
    W.hist = reinterpret_cast<unsigned int *>(ws + L.hist);
    W.offs = reinterpret_cast<unsigned int *>(ws + L.offs);
    W.cursor = reinterpret_cast<unsigned int *>(ws + L.cursor);
    W.item_w = reinterpret_cast<unsigned int *>(ws + L.item_w);
    W.item_l = reinterpret_cast<unsigned int *>(ws + L.item_l);
    W.ctr = reinterpret_cast<unsigned int *>(ws + L.ctr);
    return W;
}

// The binning stages of the pipeline: block offsets, (k*, s*) of every cell,
// bin offsets and item tables, then the bin-sorted permutation W.perm.
void launch_binning(const DxConsts &K, long long nblocks, const Desc *D, int nspecies_max, long long total_cells,
                    long long rho_d_len, long long v_len, const double *rho_g, const double *rho_d, const double *t_s, const Work &W,
                    const Modes &M, uint32_t *st, cudaStream_t stream) {
    const int sms = dx_sm_count();
    const long long cgrid_want = (total_cells + 255) / 256;
    const int cgrid = (int)(cgrid_want < (long long)sms * 16 ? cgrid_want : (long long)sms * 16);
    dx_batch_prepare<<<1, kScanThreads, 0, stream>>>(nblocks, D, nspecies_max, total_cells, rho_d_len, v_len, W, st);
    dx_batch_count<<<cgrid, 256, 0, stream>>>(nblocks, D, rho_g, rho_d, t_s, W, K);
    dx_batch_bins<<<1, kScanThreads, 0, stream>>>(W, M);
    dx_batch_scatter<<<cgrid, 256, 0, stream>>>(nblocks, W);
}

// The five-kernel pipeline on a checked workspace ws with layout L. thdr
// (null: none): adjoint tape written by the lane-per-cell items (see MainArgs).
static int batched_run(const DxConsts &K, long long nblocks, const Desc *D, long long total_cells, long long rho_d_len,
                       long long v_len, int nspecies_max, const double *rho_g, const double *rho_d,
                       const double *t_s, const double *v_in, double *v_out, char *ws, const Layout &L,
                       uint32_t *st, cudaStream_t stream, long long *thdr = nullptr, double *tm = nullptr,
                       int tlevels = 0, int tP = 0, int n_fixed = 0) {
    const Work W = n_fixed ? work_at(ws, L, fixed_n_bins(total_cells), n_fixed, fixed_n_chunk(total_cells))
                           : work_at(ws, L);
    Modes M = dx_batch_modes();
    if (n_fixed > kBatchLpcNMax && n_fixed <= kBinnedLpcNMax && dx_mode_for(n_fixed) == DX_MODE_LPC_HYB)
        M.m[n_fixed] = DX_MODE_LPC_HYB;   // the binned single-N forward's n = 10..12 items
    const int sms = dx_sm_count();
    launch_binning(K, nblocks, D, nspecies_max, total_cells, rho_d_len, v_len, rho_g, rho_d, t_s, W, M, st, stream);

    int wd_wpc = 0, wd_lpc = 0;
    bool has_wpc = false, has_lpc = false;
    // one n (n_fixed): only its own kernel family runs
    warp_doubles_for(M, n_fixed ? n_fixed : 2, n_fixed ? n_fixed : nspecies_max + 1, &wd_wpc, &wd_lpc, &has_wpc,
                     &has_lpc);
    if (has_lpc) {
        MainArgs a{D, rho_g, rho_d, t_s, v_in, v_out, st, wd_lpc, 0, 0, thdr, tm, tlevels, tP};
        const bool big = n_fixed > kBatchLpcNMax;
        void (*kern)(MainArgs, Work, Modes, DxConsts) =
            big ? (thdr ? dx_batch_main_lpc<true, true> : dx_batch_main_lpc<false, true>)
                : (thdr ? dx_batch_main_lpc<true, false> : dx_batch_main_lpc<false, false>);
        const size_t smem = sizeof(double) * (32 + (size_t)kLpcWarps * wd_lpc);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return DRAG_ECUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLpcWarps * 32, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        kern<<<sms * per_sm, kLpcWarps * 32, smem, stream>>>(a, W, M, K);
        if (cudaGetLastError() != cudaSuccess) return DRAG_ECUDA;
    }
    if (has_wpc) {
        // pair tables of the largest size (the warp rebuilds them when an item's n changes)
        const int nm = nspecies_max + 1;
        const int pod = nm * (nm - 1) / 2, phs = nm * (nm + 1) / 2 - 1;
        const int pdbl = (pod + phs + 3) / 4;
        MainArgs a{D, rho_g, rho_d, t_s, v_in, v_out, st, wd_wpc, pod, pdbl, nullptr, nullptr, 0, 0};
        const size_t smem = sizeof(double) * (size_t)kWpcWarps * (wd_wpc + pdbl);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(dx_batch_main_wpc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return DRAG_ECUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dx_batch_main_wpc, kWpcWarps * 32, smem) !=
                cudaSuccess || per_sm < 1)
            per_sm = 1;
        dx_batch_main_wpc<<<sms * per_sm, kWpcWarps * 32, smem, stream>>>(a, W, K);
    }
    return cudaGetLastError() == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" size_t drag_expm_batched_workspace_bytes(int64_t nblocks, int64_t total_cells) {
    if (nblocks < 0 || total_cells < 0) return 0;
    return layout(nblocks, total_cells).total;
}

extern "C" int drag_expm_apply_batched(int64_t nblocks, const drag_block_t *blocks, int64_t total_cells, int64_t rho_d_len,
                                       int64_t v_len, int32_t nspecies_max, const double *rho_g, const double *rho_d,
                                       const double *t_s, const double *v_in, double *v_out, void *workspace,
                                       size_t workspace_bytes, cudaStream_t stream) {
    if (nblocks < 0 || nblocks > (1LL << 31) - 1) return DRAG_EBLOCKS;
    if (total_cells < 0 || total_cells > (1LL << 32) - 1 || rho_d_len < 0 || v_len < 0) return DRAG_EINVAL_SIZE;
    if (nspecies_max < 1 || nspecies_max > DRAG_EXPM_NMAX) return DRAG_EINVAL_SIZE;
    if (nblocks == 0 || total_cells == 0) return DRAG_OK;
    if (!blocks || !rho_g || !rho_d || !t_s || !v_in || !v_out) return DRAG_ENULL;
    if (!aligned8(blocks) || !aligned8(rho_g) || !aligned8(rho_d) || !aligned8(t_s) || !aligned8(v_in) ||
        !aligned8(v_out))
        return DRAG_EALIGN;
    const Layout L = layout(nblocks, total_cells);
    if (!workspace || workspace_bytes < L.total) return DRAG_EWORKSPACE;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return DRAG_EALIGN;
    uint32_t *st = dx_status_ptr();
    if (!st) return DRAG_ECUDA;

    return batched_run(dx_consts(), nblocks, reinterpret_cast<const Desc *>(blocks), total_cells, rho_d_len, v_len,
                       nspecies_max, rho_g, rho_d, t_s, v_in, v_out, static_cast<char *>(workspace), L, st, stream);
}

// ---------------------------------------------------------------------------
// Batched update without caller scratch.
//
// Some callers cannot hand this library a workspace: host codes whose device
// memory is owned entirely by their own pool or arena allocator (reserved at
// start-up, with no hook through which a library could obtain scratch), codes
// that must not call cudaMalloc/cudaFree inside a time step because those
// calls synchronise the device and stall the other streams of the step, and
// thin foreign-language bindings that only exchange the input and output
// arrays. For them this entry point runs the same five-kernel pipeline as
// drag_expm_apply_batched on a fixed scratch array compiled into the library.
//
// The array lives in device global memory of every GPU that loads the library
// and stays there until the process exits. In host code its name only stands
// in for it, so its device address is looked up once per device (first call on
// that device, with that device current) and passed to the kernels. The
// cached address belongs to that device's context: it does not survive a
// cudaDeviceReset. Every call
// uses the same array: the first kernel of the pipeline clears the histogram
// and the counters, and every other part is written before it is read, so no
// stale contents leak from one call to the next; but two calls whose work
// overlaps on the GPU (different streams, no ordering) would race on it.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNoAllocBytes =
    na_align(sizeof(unsigned long long) * (size_t)DRAG_NOALLOC_MAX_CELLS) +
    na_align(sizeof(unsigned int) * (size_t)DRAG_NOALLOC_MAX_CELLS) +
    na_align(sizeof(long long) * ((size_t)DRAG_NOALLOC_MAX_BLOCKS + 1)) +
    5 * na_align(sizeof(unsigned int) * (kNBins + 1)) + na_align(sizeof(unsigned int) * 8);

std::mutex g_noalloc_mu;
void *g_noalloc_addr[64];

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

extern "C" int drag_expm_apply_batched_noalloc(int64_t nblocks, const drag_block_t *blocks, int64_t total_cells,
                                               int64_t rho_d_len, int64_t v_len, int32_t nspecies_max,
                                               const double *rho_g, const double *rho_d, const double *t_s,
                                               const double *v_in, double *v_out, cudaStream_t stream) {
    if (nblocks > DRAG_NOALLOC_MAX_BLOCKS || total_cells > DRAG_NOALLOC_MAX_CELLS) return DRAG_ENOALLOC_LIMIT;
    if (nblocks >= 0 && total_cells >= 0 && drag_expm_batched_workspace_bytes(nblocks, total_cells) > kNoAllocBytes)
        return DRAG_ENOALLOC_LIMIT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DRAG_ECUDA;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DRAG_ECUDA;
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    return drag_expm_apply_batched(nblocks, blocks, total_cells, rho_d_len, v_len, nspecies_max, rho_g, rho_d, t_s,
                                   v_in, v_out, scratch, kNoAllocBytes, stream);
}

// ---------------------------------------------------------------------------
// Binned forward: drag_expm_apply for lane-per-cell sizes on large inputs runs
// the pipeline above with one block, its bins chunk-major (chunk, k*, s*). Its scratch (12 bytes per cell) comes
// from a library-private, stream-ordered memory pool that keeps what it has
// once allocated (release threshold: never), so calls on different streams
// never share scratch, repeated calls do not reallocate, and stream capture
// records the allocation as graph nodes.
// ---------------------------------------------------------------------------

namespace {


std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];

cudaMemPool_t scratch_pool() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return nullptr;
        }
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

__global__ void dx_batch_single_desc(Desc *d, long long C, int N, double dt) {
    d->cell_offset = 0;
    d->dust_offset = 0;
    d->vel_offset = 0;
    d->ncells = (int)C;
    d->nspecies = N;
    d->dt = dt;
}

}  // namespace

// Smallest input from which binning the whole input by (chunk, k*, s*) beats
// one tile-sorted launch: the crossovers measured on GB300 (CUDA events, cold
// L2, the MRN-like workloads, n = 2..12). Binning pays earlier for larger n,
// whose per-warp work varies more with (k*, s*), and much earlier for the
// adjoint, whose squarings cost 5x the forward's. At n = 2 the forward runs in
// the velocity form, a few dozen FP64 operations a cell: its single launch beat
// the binned pipeline at every size measured (411.7 against 685.0 us at
// 2,097,152 cells), so it never bins. Building with
// -DDX_BINNED_MIN_CELLS=<cells> sets one threshold for every n (measurements).
long long dx_binned_min_cells(int n, bool adjoint) {
#ifdef DX_BINNED_MIN_CELLS
    return n >= 2 && n <= (adjoint ? kBatchLpcNMax : kBinnedLpcNMax) ? (long long)(DX_BINNED_MIN_CELLS) : LLONG_MAX;
#else
    static constexpr long long kForward[kBinnedLpcNMax + 1] = {0, 0, LLONG_MAX, 196608, 131072, 98304, 98304,
                                                               40960, 40960, 28672, 26624, 26624, 24576};
    static constexpr long long kAdjoint[kBatchLpcNMax + 1] = {0, 0, 32768, 24576, 4096, 4096, 4096,
                                                              4096, 4096, 4096};
    if (n < 2 || n > (adjoint ? kBatchLpcNMax : kBinnedLpcNMax)) return LLONG_MAX;
    return adjoint ? kAdjoint[n] : kForward[n];
#endif
}

bool dx_binned_eligible(int n, int mode, long long C) {
    // the storage the binned kernel compiles for n: registers up to DX_LPC_REG_NMAX, hybrid above
    const int binned_mode = n <= DX_LPC_REG_NMAX ? DX_MODE_LPC_REG : DX_MODE_LPC_HYB;
    return n >= 2 && n <= kBinnedLpcNMax && mode == binned_mode && C >= dx_binned_min_cells(n, false) &&
           C <= 0x7fffffffLL;
}

int dx_binned_forward(const DxConsts &K, long long C, int N, const double *rho_g, const double *rho_d,
                      const double *t_s, double dt, const double *v_in, double *v_out, uint32_t *status,
                      cudaStream_t stream, long long *thdr, double *tm, int tlevels, int tP) {
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return DX_BINNED_UNAVAILABLE;
    const Layout L = layout(1, C, fixed_n_bins(C));
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, L.total + 256, pool, stream) != cudaSuccess || !p) {
        cudaGetLastError();
        return DX_BINNED_UNAVAILABLE;
    }
    int rc = DRAG_OK;
    if ((reinterpret_cast<uintptr_t>(p) & 255) != 0) {
        rc = DX_BINNED_UNAVAILABLE;
    } else {
        Desc *D = reinterpret_cast<Desc *>(static_cast<char *>(p) + L.total);
        dx_batch_single_desc<<<1, 1, 0, stream>>>(D, C, N, dt);
        rc = batched_run(K, 1, D, C, (long long)N * C, 3LL * (N + 1) * C, N, rho_g, rho_d, t_s, v_in, v_out,
                         static_cast<char *>(p), L, status, stream, thdr, tm, tlevels, tP, N + 1);
    }
    if (cudaFreeAsync(p, stream) != cudaSuccess && rc == DRAG_OK) rc = DRAG_ECUDA;
    return rc;
}

void *dx_binned_perm(const DxConsts &K, long long C, int N, const double *rho_g, const double *rho_d,
                     const double *t_s, double dt, uint32_t *status, cudaStream_t stream,
                     const unsigned long long **perm) {
    cudaMemPool_t pool = scratch_pool();
    if (!pool || C < 1 || C > 0x7fffffffLL) return nullptr;
    const Layout L = layout(1, C, fixed_n_bins(C));
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, L.total + 256, pool, stream) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    if ((reinterpret_cast<uintptr_t>(p) & 255) != 0) {
        cudaFreeAsync(p, stream);
        return nullptr;
    }
    char *ws = static_cast<char *>(p);
    Desc *D = reinterpret_cast<Desc *>(ws + L.total);
    const Work W = work_at(ws, L, fixed_n_bins(C), N + 1, fixed_n_chunk(C));
    dx_batch_single_desc<<<1, 1, 0, stream>>>(D, C, N, dt);
    launch_binning(K, 1, D, N, C, (long long)N * C, 3LL * (N + 1) * C, rho_g, rho_d, t_s, W, dx_batch_modes(), status,
                   stream);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(p, stream);
        return nullptr;
    }
    *perm = W.perm;
    return p;
}

int dx_binned_release(void *scratch, cudaStream_t stream) {
    return cudaFreeAsync(scratch, stream) == cudaSuccess ? DRAG_OK : DRAG_ECUDA;
}

extern "C" int32_t drag_expm_apply_launches(int64_t ncells, int32_t nspecies) {
    if (ncells <= 0 || nspecies < 1 || nspecies > DRAG_EXPM_NMAX) return 0;
    const int n = nspecies + 1;
    return dx_binned_eligible(n, dx_mode_for(n), ncells) ? 6 : 1;
}
