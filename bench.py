#!/usr/bin/env python3
"""Throughput benchmark of the FP64 EXP drag update on GB300.

One step = one forward drag update (drag_expm_apply) over the whole headline
workload: the N=16 MRN-like workload of 128^3 = 2,097,152 cells (17x17 drag
matrices, dt/t_s in [1e-4, 1e8]). Inputs are synthetic and seeded
(paper_2509_25347_gb300.workloads) and larger than L2, so no flush is needed.

The same run measures the other four workloads under "configs": N=1 Dustybox
(32,768 cells, L2 flushed between launches), N=4 (128^3), the AMR-like batch
(1,048,576 cells, one CUDA-graph replay of drag_expm_apply_batched) and N=8
forward and forward + adjoint (128^3), each with its clocks, roofline and the
CPU oracle timed on the same arrays.

Roofline: the FP64 pipe binds everywhere (1.7-195 FLOP per byte against a
balance point of 0.19). `achieved` counts the FP64 FLOPs of the update as the
kernels compute it (symmetric squarings, Horner in the arrowhead,
applications; shard.built_flops) from each cell's (k*, s*), over the FP64
peak measured in the same run by the DFMA probe (drag_expm_probe_fp64_rate).
The paper's dense cost model (App. B: k* + s* dense n x n products) is
reported beside it as context.

Prints one JSON line (rank 0). Under torchrun each rank runs its own copy of
every workload (independent draws, weak scaling, no collective on the data
path); with --partition the ranks split one workload instead (contiguous cell
ranges, or whole AMR blocks balanced by cost: strong scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--configs none]
  python bench.py --fp64-peak          # DFMA / DMMA throughput and squaring comparison only
  python bench.py --impl reference ... # the CPU oracle, timed on host cores
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_25347_gb300 import shard  # noqa: E402
from paper_2509_25347_gb300 import workloads as W  # noqa: E402

METRIC = "FP64 cell drag updates/sec at N=16 (fwd, fwd+adjoint) and % of FP64/HBM roofline"
UNIT = "cell-updates/s"
HEADLINE = "mrn_n16_128cube"
CONFIG_LEGS = ("dustybox_n1_32k", "mrn_n4_128cube", "batched_amr_1m", "mrn_n8_128cube_adjoint")
# FP64 pipe of one GB300 by unit count: 152 SMs x 4 sub-partitions x 0.5 DFMA/clk x 2 flop = 608 flop/clk,
# at the 2070 MHz maximum SM clock (context beside the measured peak).
FP64_FLOP_PER_CLK = 152 * 4 * 0.5 * 2
SM_MAX_MHZ = 2070.0

# DRAM traffic of the dominant kernel per cell, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one 262,144-cell launch of
# the same kernel and launch shape, divided by its cells; the summary under
# profiles/ gives the command). It holds only for the sources it was taken on:
# the entry carries a SHA-256 of them and is reported as null once they change.
KERNEL_SOURCES = {
    "dx_forward_wpc": ["csrc/dx_forward.cu", "csrc/dx_wpc.cuh", "csrc/dx_tape.cuh", "csrc/dx_common.cuh", "sched.py"],
}
MEASURED_TRAFFIC = {
    ("mrn_n16_128cube", "dx_forward_wpc"): {
        "sources_sha256": "d37f403c45f46a356c12b2910a0d3cde745a84644ff5ad8d67f2c99a52d7c0e3",
        "bytes_per_cell": (188641024 + 81163264) / 262144,
        # FP64 FLOPs the kernel executes: thread-level 2 DFMA + DADD + DMUL (sm__sass_thread_inst_executed_op_*)
        "executed_flop_per_cell": (2 * 11389688778 + 642554274 + 99185602) / 262144,
        "capture": "profiles/dx_forward_wpc_mrn_n16.md",
    },
}


def sources_digest(kernel):
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2509_25347_gb300", rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(workload, kernel, cells, key="bytes_per_cell"):
    """Per-launch DRAM bytes (or, with key="executed_flop_per_cell", executed FP64
    FLOPs) of `kernel` on `cells` cells of `workload`, or None."""
    e = MEASURED_TRAFFIC.get((workload, kernel))
    if e is None or kernel not in KERNEL_SOURCES or sources_digest(kernel) != e["sources_sha256"]:
        return None
    return e[key] * cells


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=HEADLINE, choices=list(W.WORKLOADS))
    p.add_argument("--configs", default="all", choices=["all", "none"],
                   help="also measure the other four workloads (default with the headline workload)")
    p.add_argument("--partition", action="store_true",
                   help="under torchrun: split one workload over the ranks (strong scaling)")
    p.add_argument("--fp64-peak", action="store_true", help="only the FP64 probes (DFMA/DMMA, squaring comparison)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--ncells", type=int, default=None, help="truncate the workload (profiling runs only)")
    p.add_argument("--nblocks", type=int, default=2048, help="blocks of the batched workload (profiling runs only)")
    p.add_argument("--no-plain-baseline", action="store_true", help="batched workload: skip the per-block comparison")
    return p.parse_args()


# ------------------------------------------------------------------ helpers ---

def max_over_ranks(values, world, device="cpu"):
    """Element-wise max of per-rank timings (ms) over all ranks; the job is as
    slow as its slowest rank. Identity when world == 1."""
    import torch
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_per_rank, world, ms):
    """Weak scaling: every rank processes its own full workload, so the
    whole-job throughput is the units of all ranks over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def dense_counts(N, k, s):
    """Per-cell FLOPs of the paper's dense cost model (2 n^3 (k* + s*) + 6 n^2:
    k* + s* dense n x n products, App. B "Numerical cost", plus three mat-vecs)
    and algorithmic bytes (8 (1 + 2N) inputs + 24 n in + 24 n out)."""
    n = N + 1
    flops = 2.0 * n ** 3 * (k.astype(np.float64) + s.astype(np.float64)) + 6.0 * n * n
    bytes_per_cell = 8 * (1 + 2 * N) + 48 * n
    return flops, bytes_per_cell


def read_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get("hbm_gbs")
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ["uuid", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, uuid):
        self.uuid = uuid
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8 or (self.uuid and f[0] != self.uuid):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(pw) if pw else None}


def gpu_uuid(local):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        return None


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------ CPU oracle ---

def _oracle_chunk(args):
    import oracle
    rg, rd, ts, dt, v = args
    oracle.drag_apply(rg, rd, ts, dt, v)
    return rg.shape[0]


def _oracle_chunk_fb(args):
    import oracle
    rg, rd, ts, dt, v, g = args
    oracle.drag_apply(rg, rd, ts, dt, v)
    oracle.drag_backward(rg, rd, ts, dt, v, g)
    return rg.shape[0]


def _host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_oracle_rate(cells, seconds, steps=1, adjoint=False, min_wall=1.0):
    """Oracle cell-updates/s on the host cores (spawned worker processes, one
    chunk of contiguous cells each), forward or forward + adjoint. A step
    repeats its pass over the sample until it has run min_wall seconds (a
    small workload's single pass is dominated by the pool's dispatch).
    Returns (rate, cores, sample_cells, wall_per_step, passes_per_step)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    cores = _host_cores()
    probe = cells.subset(np.arange(min(64, cells.ncells)))
    g = W.adjoint_target(cells.ncells, cells.rho_d.shape[0]) if adjoint else None
    t0 = time.perf_counter()
    oracle.drag_apply(probe.rho_g, probe.rho_d, probe.t_s, probe.dt, probe.v)
    if adjoint:
        oracle.drag_backward(probe.rho_g, probe.rho_d, probe.t_s, probe.dt, probe.v, g[:, :, :probe.ncells])
    per_cell = (time.perf_counter() - t0) / probe.ncells
    sample = int(min(cells.ncells, max(cores * 16, seconds * cores / max(per_cell, 1e-9))))
    sub = cells.subset(np.arange(sample))
    bounds = np.linspace(0, sample, cores + 1).astype(int)
    chunks = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        if b > a:
            c = (sub.rho_g[a:b].copy(), sub.rho_d[:, a:b].copy(), sub.t_s[:, a:b].copy(), sub.dt,
                 sub.v[:, :, a:b].copy())
            chunks.append(c + ((g[:, :, a:b].copy(),) if adjoint else ()))
    fn = _oracle_chunk_fb if adjoint else _oracle_chunk
    ctx = mp.get_context("spawn")
    walls = []
    total = 0
    passes = 0
    with ctx.Pool(cores) as pool:
        pool.map(fn, [tuple(x[..., :1] if isinstance(x, np.ndarray) else x for x in c) for c in chunks])
        for _ in range(steps):
            t0 = time.perf_counter()
            while True:
                total += sum(pool.map(fn, chunks))
                passes += 1
                if time.perf_counter() - t0 >= min_wall:
                    break
            walls.append(time.perf_counter() - t0)
    wall = float(np.mean(walls))
    return total / float(np.sum(walls)), cores, sample, wall, passes // steps


def cpu_oracle_single_core_rate(cells, seconds):
    """Oracle cell-updates/s in this process alone (one core), on a prefix of
    the workload sized for about `seconds` of work. Returns (rate, sample_cells)."""
    import oracle
    oracle.build()
    probe = cells.subset(np.arange(min(32, cells.ncells)))
    t0 = time.perf_counter()
    oracle.drag_apply(probe.rho_g, probe.rho_d, probe.t_s, probe.dt, probe.v)
    per_cell = (time.perf_counter() - t0) / probe.ncells
    sample = int(min(cells.ncells, max(32, seconds / max(per_cell, 1e-9))))
    sub = cells.subset(np.arange(sample))
    t0 = time.perf_counter()
    oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    return sample / (time.perf_counter() - t0), sample


def _oracle_blocks(args):
    import oracle
    desc, rg, rd, ts, v = args
    oracle.drag_apply_batched(desc, rg, rd, ts, v)
    return int(desc["ncells"].sum())


def cpu_oracle_batched_rate(batch, seconds, steps=1):
    """Oracle cell-updates/s on the batched workload: a prefix of the blocks,
    one contiguous group of blocks per spawned worker."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    cores = _host_cores()
    t0 = time.perf_counter()
    probe = W.Batch(batch.blocks[:8])
    oracle.drag_apply_batched(*probe.pack())
    per_cell = (time.perf_counter() - t0) / max(1, probe.ncells)
    want_cells = seconds * cores / max(per_cell, 1e-9)
    bc = max(1, batch.blocks[0][2].ncells)
    nb = int(min(len(batch.blocks), max(cores, want_cells / bc)))
    groups = np.array_split(np.arange(nb), cores)
    jobs = [W.Batch([batch.blocks[i] for i in g]).pack() for g in groups if len(g)]
    ctx = mp.get_context("spawn")
    walls = []
    with ctx.Pool(cores) as pool:
        for _ in range(steps):
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_blocks, jobs))
            walls.append(time.perf_counter() - t0)
    wall = float(np.mean(walls))
    return done / wall, cores, nb, wall


def cpu_baseline_entry(cells, name, seconds, adjoint=False):
    rate, cores, sample, _, passes = cpu_oracle_rate(cells, seconds=seconds)
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {sample} cells of {name}, {passes} pass{'es' if passes > 1 else ''} "
                     f"(same seeded arrays as the GPU leg)"}
    if adjoint:
        fr, fc, fs, _, fp = cpu_oracle_rate(cells, seconds=seconds, adjoint=True)
        out["fwd_adjoint"] = {"value": fr, "unit": UNIT, "cores": fc,
                              "sample": f"first {fs} cells of {name}: orc forward + orc adjoint, {fp} "
                                        f"pass{'es' if fp > 1 else ''}"}
    return out


# ---------------------------------------------------------------- reference ---

def run_reference(args, rank):
    if rank != 0:
        return
    secs = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    if args.workload == "batched_amr_1m":
        batch = W.batched(nblocks=args.nblocks)
        C, N = batch.ncells, "{1,4,8,16}"
        rate, cores, nb, wall = cpu_oracle_batched_rate(batch, secs, steps=args.steps)
        sample = nb * 512
    else:
        cells = W.workload(args.workload)
        _, C, N, _ = W.WORKLOADS[args.workload]
        rate, cores, sample, wall, passes = cpu_oracle_rate(cells, seconds=secs, steps=args.steps)
        sample *= passes
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "ncells": C, "nspecies": N, "step_sample_cells": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {sample} cells of {args.workload} per step"},
            "gpu_launches": 0,
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- FP64 probes ---

def symmetric_propagators(n, nmat, seed=0):
    """E = exp(2^-6 S) for random symmetric arrowheads S (the similarity form of
    A = dt Omega_v), and their sigma; E sigma = sigma."""
    rng = np.random.default_rng(seed)
    eps = 10.0 ** rng.uniform(-2, 0, (nmat, n - 1))
    alpha = 10.0 ** rng.uniform(-1, 1, (nmat, n - 1))
    S = np.zeros((nmat, n, n))
    S[:, 0, 0] = -np.sum(eps * alpha, axis=1)
    S[:, 0, 1:] = S[:, 1:, 0] = np.sqrt(eps) * alpha
    idx = np.arange(1, n)
    S[:, idx, idx] = -alpha
    lam, Q = np.linalg.eigh(S / 64.0)
    E = np.einsum("mij,mj,mkj->mik", Q, np.exp(lam), Q)
    sig = np.concatenate([np.ones((nmat, 1)), np.sqrt(eps)], axis=1)
    return np.ascontiguousarray(E), np.ascontiguousarray(sig)


def fp64_rates(dx, stream, repeats=5):
    """DFMA and DMMA throughput (TFLOP/s, best of `repeats` launches after two
    warm-ups), each launch timed alone with CUDA events on `stream`."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = {}
    for kind, iters in (("dfma", 16384), ("dmma", 4096)):
        with torch.cuda.stream(stream):
            for _ in range(2):
                dx.probe_fp64_rate(kind, iters, sink, stream=stream)
            best = 0.0
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                flop = dx.probe_fp64_rate(kind, iters, sink, stream=stream)
                e1.record(stream)
                e1.synchronize()
                best = max(best, flop / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[kind] = best
    return out


def square_comparison(dx, stream, n, nmat=19456, reps=64):
    """Time per restored squaring of one n x n symmetric matrix: the forward
    kernels' DFMA routine against DMMA tiles (same matrices, CUDA events), and
    the largest difference between their results."""
    import torch
    E, sig = symmetric_propagators(n, nmat, seed=n)
    tE, ts = torch.from_numpy(E).cuda(), torch.from_numpy(sig).cuda()
    res, outs = {}, {}
    for kind in ("dfma", "dmma"):
        out = torch.empty_like(tE)
        with torch.cuda.stream(stream):
            dx.probe_square(tE, ts, reps, kind=kind, out=out, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = float("inf")
            for _ in range(3):
                e0.record(stream)
                dx.probe_square(tE, ts, reps, kind=kind, out=out, stream=stream)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        outs[kind] = out
        per_sq_ns = best * 1e6 / (nmat * reps)
        useful = n * n * (n + 1.0) * nmat * reps / (best * 1e-3) / 1e12   # symmetric-form FLOPs
        res[kind] = {"ms": best, "ns_per_squaring_per_matrix": per_sq_ns, "useful_tflops": useful}
    res["dmma_over_dfma_time"] = res["dmma"]["ms"] / res["dfma"]["ms"]
    res["max_abs_diff"] = float((outs["dfma"] - outs["dmma"]).abs().max())
    res.update({"n": n, "matrices": nmat, "squarings_each": reps,
                "useful_flop_per_squaring": n * n * (n + 1)})
    return res


def peak_entry(rates):
    unit_count = FP64_FLOP_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
    return {"dfma_tflops": rates["dfma"], "dmma_tflops": rates["dmma"], "unit_count_tflops": unit_count,
            "dfma_frac_of_unit_count": rates["dfma"] / unit_count,
            "source": "drag_expm_probe_fp64_rate: independent FMA chains (DFMA) or m8n8k4 MMA chains (DMMA), "
                      "one wave of 4 x 256 threads per SM, best of 5 launches timed alone with CUDA events"}


def run_fp64_peak(args, rank, world):
    import torch

    import paper_2509_25347_gb300 as dx
    from paper_2509_25347_gb300 import build as dxbuild
    if rank != 0:
        return
    torch.cuda.set_device(0)
    dxbuild.build()
    dx.load_library()
    stream = torch.cuda.Stream()
    sampler = ClockSampler(gpu_uuid(0))
    sampler.start()
    rates = fp64_rates(dx, stream)
    squares = {f"n={n}": square_comparison(dx, stream, n) for n in (5, 9, 17)}
    clocks = sampler.stop()
    if dx.get_status():
        raise RuntimeError("device status set after the probes")
    print(json.dumps({"probe": "fp64_peak", "peak": peak_entry(rates), "square": squares, "clocks": clocks}),
          flush=True)


# --------------------------------------------------------------- GPU legs ---

def time_steps(fn, steps, stream, flush=None):
    """Per-step CUDA-event times (ms) on `stream`. flush = (w, r, out): between
    steps, outside the events, w (twice L2) is written, which evicts every
    input line, then r (twice L2) is read, which writes the dirty lines of w
    back, so a launch starts with none of its inputs and no dirty line in L2."""
    import torch
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush[0].fill_(float(i))
            torch.sum(flush[1], dim=0, out=flush[2])
        ev0[i].record(stream)
        fn()
        ev1[i].record(stream)
    torch.cuda.synchronize()
    return [ev0[i].elapsed_time(ev1[i]) for i in range(steps)]


def c_abi_forward(dx, C, N, rg, rd, ts, dt, v, vout, stream):
    """drag_expm_apply through the C ABI with its arguments marshalled once, so
    that a timed step enqueues the launch within microseconds of its start
    event (the Python binding's checks would otherwise sit between the event
    and a 30 us launch). Raises on a non-zero return code."""
    import ctypes
    lib = dx.load_library()
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    args = (C, N, p(rg), p(rd), p(ts), float(dt), p(v), p(vout), ctypes.c_void_p(stream.cuda_stream))
    fn = lib.drag_expm_apply

    def call():
        rc = fn(*args)
        if rc:
            raise RuntimeError(f"drag_expm_apply returned {rc}")
    return call


def roofline_entry(built_flop, dense_flop, alg_bytes, mean_s, peak, hbm_peak, family):
    achieved = built_flop / mean_s / 1e12
    gbs = alg_bytes / mean_s / 1e9
    return {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
        "peak_source": "FP64 DFMA rate measured in this run (drag_expm_probe_fp64_rate, burst); the unit count "
                       "152 SMs x 608/152 flop/clk x 2070 MHz = %.4f TFLOP/s is context" %
                       (FP64_FLOP_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12),
        "flop_per_launch": built_flop,
        "flop_model": "the update as the kernels compute it, from each cell's (k*, s*): set-up 13N, Horner in the "
                      "arrowhead (m* - 1) (2n^2 + 4n - 4), restorations 2n^2, symmetric squarings n^2 (n+1), "
                      "applications 6n^2 + 6n (%s; warp per cell: 2^q applications 2^q 6n^2 + 9n, sigma o v carried "
                      "between them); n = 2 lane per cell in the velocity form: set-up 10, "
                      "Taylor 2 (m* - 1) + 3, 4 per squaring, 15 for the application" % family,
        "dense_model": {"flop_per_launch": dense_flop, "achieved": dense_flop / mean_s / 1e12,
                        "frac": dense_flop / mean_s / 1e12 / peak,
                        "model": "paper's cost model (App. B): k* + s* dense n x n products, 2n^3 (k* + s*) + 6n^2 "
                                 "per cell; more work than the kernels do, so not a headroom measure"},
        "kernel_mean_ms": mean_s * 1e3,
        "algorithmic_bytes_per_launch": float(alg_bytes),
        "hbm_gbs": gbs, "hbm_frac_of_measured": (gbs / hbm_peak) if hbm_peak else None,
    }


def family_of(dx, N):
    wpc = dx.get_mode(N) == dx.MODE_WARP_PER_CELL
    return wpc, ("warp per cell: s* - min(s*, 2) squarings, 2^min(s*, 2) applications" if wpc
                 else "lane per cell: s* squarings, one application")


def load_cells(name, rank, world, partition, ncells=None):
    """This rank's cells of a single-N workload and the total over ranks."""
    if partition and world > 1:
        full = W.workload(name, ncells=ncells)
        a, b = shard.cell_range(full.ncells, rank, world)
        return full.subset(np.arange(a, b)), full.ncells
    cells = W.workload(name, ncells=ncells, replica=rank)
    return cells, cells.ncells * world


def leg_single(dx, args, name, rank, world, stream, peak, hbm_peak, local, steps, adjoint=False, cpu_seconds=5.0,
               ncells=None):
    """Forward (and optionally forward + adjoint) of one single-N workload."""
    import torch
    _, _, N, _ = W.WORKLOADS[name]
    cells, total = load_cells(name, rank, world, args.partition, ncells)
    C = cells.ncells
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rg, rd, ts, v = dev(cells.rho_g), dev(cells.rho_d), dev(cells.t_s), dev(cells.v)
    vout = torch.empty_like(v)
    k, s = dx.select(rg, rd, ts, cells.dt)
    k, s = k.cpu().numpy(), s.cpu().numpy()
    wpc, fam = family_of(dx, N)
    built = float(shard.built_flops(N, k, s, wpc).sum())
    dense, bytes_cell = dense_counts(N, k, s)
    dense = float(dense.sum())
    l2 = getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 0) or 129 * 2 ** 20
    flush = None
    if bytes_cell * C < 2 * l2:
        flush = (torch.empty(2 * l2 // 4, dtype=torch.float32, device="cuda"),
                 torch.ones((2 * l2 // 4 // 1024, 1024), dtype=torch.float32, device="cuda"),
                 torch.empty(1024, dtype=torch.float32, device="cuda"))
    fwd = c_abi_forward(dx, C, N, rg, rd, ts, cells.dt, v, vout, stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            fwd()
    torch.cuda.synchronize()
    dx.get_status()
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        per = time_steps(fwd, steps, stream, flush)
    barrier(world)
    clocks = sampler.stop()
    if dx.get_status():
        raise RuntimeError(f"device status set after the {name} forward")
    fb_ms = ft_ms = None
    levels = tape_nbytes = 0
    if adjoint:
        vt = dev(W.adjoint_target(C, N))
        gvi, grg = torch.empty_like(v), torch.empty_like(rg)
        grd, gts = torch.empty_like(rd), torch.empty_like(ts)

        def fwd_bwd():
            dx.apply(rg, rd, ts, cells.dt, v, vout, stream=stream)
            torch.sub(vout, vt, out=gvi)
            dx.backward(rg, rd, ts, cells.dt, v, gvi, out=(vout, grg, grd, gts), stream=stream)

        with torch.cuda.stream(stream):
            fwd_bwd()
            torch.cuda.synchronize()
            fb_steps = max(1, min(steps, 3))
            fb = time_steps(fwd_bwd, fb_steps, stream)
        fb_ms = float(np.mean(fb))
        if dx.get_status():
            raise RuntimeError(f"device status set after the {name} forward + adjoint")
        # the same step through the adjoint tape (the forward stores E_0 .. E_{s*-2})
        levels = dx.tape_levels_needed(rg, rd, ts, cells.dt)
        tape_nbytes = dx.tape_bytes(C, N, levels)
        ft_ms = None
        if tape_nbytes < 0.8 * torch.cuda.mem_get_info()[0]:
            holder = [None]

            def fwd_bwd_taped():
                _, holder[0] = dx.apply_taped(rg, rd, ts, cells.dt, v, vout, levels=levels, tape=holder[0],
                                              stream=stream)
                torch.sub(vout, vt, out=gvi)
                dx.backward(rg, rd, ts, cells.dt, v, gvi, out=(vout, grg, grd, gts), tape=holder[0], stream=stream)

            with torch.cuda.stream(stream):
                fwd_bwd_taped()
                torch.cuda.synchronize()
                ft_ms = float(np.mean(time_steps(fwd_bwd_taped, fb_steps, stream)))
            holder[0] = None
            if dx.get_status():
                raise RuntimeError(f"device status set after the {name} taped forward + adjoint")
    # the paper's variants at N = 4 (lane per cell there, one launch each), outside the timed region
    var_ms = {}
    if name == "mrn_n4_128cube":
        for vname, kw in (("pade", {"method": "pade"}), ("taylor_bound_test", {"bound_test": True})):
            run_var = (lambda kw=kw: dx.apply_opts(rg, rd, ts, cells.dt, v, vout, stream=stream, **kw))
            with torch.cuda.stream(stream):
                run_var()
                torch.cuda.synchronize()
                var_ms[vname] = float(np.mean(time_steps(run_var, max(3, min(steps, 5)), stream, flush)))
        if dx.get_status():
            raise RuntimeError(f"device status set after the {name} variants")
    mean_ms = float(np.mean(per))
    vals = [float(np.sum(per)), mean_ms] + ([fb_ms, ft_ms or 0.0] if adjoint else []) + list(var_ms.values())
    red = max_over_ranks(vals, world, device="cuda")
    ms_step = red[0] / steps
    entry = {
        "workload": name, "ncells": total, "nspecies": N, "matrix": f"{N + 1}x{N + 1}",
        "value": total / (ms_step * 1e-3),
        "unit": UNIT, "ms_per_step": ms_step, "steps": steps, "warmup": args.warmup,
        "mean_k_star": float(k.mean()), "mean_s_star": float(s.mean()), "max_s_star": int(s.max()),
        "l2": ("inputs (%.3f GB) larger than L2, no flush" % (bytes_cell * C / 1e9)) if flush is None else
              ("inputs (%.4f GB) below 2 x L2: between timed launches a %.0f MB buffer is written (evicting the "
               "inputs) and a second one read (writing the dirty lines back), each launch timed alone"
               % (bytes_cell * C / 1e9, 2 * l2 / 1e6)),
        "roofline": roofline_entry(built, dense, bytes_cell * C, red[1] * 1e-3, peak, hbm_peak, fam),
        "clocks": clocks,
        "gpu_launches": dx.apply_launches(C, N) * steps,
    }
    if adjoint:
        entry["fwd_adjoint"] = {"value": total / (red[2] * 1e-3), "unit": UNIT, "ms_per_step": red[2],
                                "adjoint_over_forward_time": red[2] / ms_step,
                                "note": "forward + dL/dv_out (torch sub) + drag_expm_backward, CUDA events"}
        if ft_ms is not None:
            entry["fwd_adjoint_taped"] = {
                "value": total / (red[3] * 1e-3), "unit": UNIT, "ms_per_step": red[3],
                "adjoint_over_forward_time": red[3] / ms_step, "tape_levels": levels, "tape_bytes": tape_nbytes,
                "note": "drag_expm_apply_taped + dL/dv_out (torch sub) + drag_expm_backward_taped, CUDA events"}
    if var_ms:
        red_var = red[2 + (2 if adjoint else 0):]
        entry["variants"] = {
            "note": "drag_expm_apply_opts: the Pade variant (Eq. PadeEqu) and the paper's second modification "
                    "(bound test), one cell per lane at this N; outside the timed region",
            **{vn: {"value": total / (t * 1e-3), "unit": UNIT, "ms_per_step": t}
               for vn, t in zip(var_ms.keys(), red_var)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        entry["cpu_baseline"] = cpu_baseline_entry(cells, name, cpu_seconds, adjoint=adjoint)
    return entry, (cells, rg, rd, ts, v, vout, k, s, per, total)


def leg_batched(dx, args, rank, world, stream, peak, hbm_peak, local, steps, cpu_seconds=5.0):
    """AMR-like batch: one step = one CUDA-graph replay of
    drag_expm_apply_batched over 2048 blocks of 8^3 cells (N in {1,4,8,16},
    dt = 2^-k). The plain single-N entry point, launched once per block and
    captured in a graph too, is timed alongside."""
    import torch
    batch_full = W.batched(nblocks=args.nblocks, seed=W.replica_seed(3, 0 if args.partition else rank))
    blocks = batch_full.blocks
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def per_cell_ks(batch):
        desc, rg_h, rd_h, ts_h, _ = batch.pack()
        rg_, rd_, ts_ = dev(rg_h), dev(rd_h), dev(ts_h)
        k = np.zeros(rg_h.size, dtype=np.int64)
        s = np.zeros(rg_h.size, dtype=np.int64)
        for (N, dt, cells), d in zip(batch.blocks, desc):
            co, do, C = int(d["cell_offset"]), int(d["dust_offset"]), cells.ncells
            kk, ss = dx.select(rg_[co:co + C], rd_[do:do + N * C].view(N, C), ts_[do:do + N * C].view(N, C), dt)
            k[co:co + C], s[co:co + C] = kk.cpu().numpy(), ss.cpu().numpy()
        return desc, k, s

    wpc_of = lambda N: dx.get_mode(N) == dx.MODE_WARP_PER_CELL
    total = batch_full.ncells * (1 if args.partition else world)
    if args.partition and world > 1:
        desc_f, k_f, s_f = per_cell_ks(batch_full)
        mine = shard.balance_blocks(shard.block_cost(desc_f, k_f, s_f, wpc_of), world)[rank]
        batch = W.Batch([blocks[i] for i in mine])
    else:
        batch = batch_full
    desc, k, s = per_cell_ks(batch)
    _, rg_h, rd_h, ts_h, v_h = batch.pack()
    C = rg_h.size
    nmax = int(desc["nspecies"].max())
    rg, rd, ts, v = dev(rg_h), dev(rd_h), dev(ts_h), dev(v_h)
    dblocks = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
    vout = torch.empty_like(v)
    ws = torch.empty(dx.batched_workspace_bytes(len(desc), C), dtype=torch.uint8, device="cuda")
    built = dense = 0.0
    bytes_step = 0.0
    for d in desc:
        N, c0, Cb = int(d["nspecies"]), int(d["cell_offset"]), int(d["ncells"])
        built += float(shard.built_flops(N, k[c0:c0 + Cb], s[c0:c0 + Cb], wpc_of(N)).sum())
        fl, bc = dense_counts(N, k[c0:c0 + Cb], s[c0:c0 + Cb])
        dense += float(fl.sum())
        bytes_step += bc * Cb

    def batched_call():
        dx.apply_batched(dblocks, rg, rd, ts, v, vout, nspecies_max=nmax, workspace=ws, stream=stream)

    views = []
    for (N, dt, cells), d in zip(batch.blocks, desc):
        c0, c1 = int(d["cell_offset"]), int(d["cell_offset"]) + cells.ncells
        d0, d1 = int(d["dust_offset"]), int(d["dust_offset"]) + N * cells.ncells
        v0, v1 = int(d["vel_offset"]), int(d["vel_offset"]) + 3 * (N + 1) * cells.ncells
        shp = (3, N + 1, cells.ncells)
        views.append((rg[c0:c1], rd[d0:d1].view(N, -1), ts[d0:d1].view(N, -1), dt, v[v0:v1].view(shp),
                      vout[v0:v1].view(shp)))

    def plain_calls():
        for a, b_, c_, dt, vi, vo in views:
            dx.apply(a, b_, c_, dt, vi, vo, stream=stream)

    plain = not args.no_plain_baseline
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            batched_call()
            if plain:
                plain_calls()
    torch.cuda.synchronize()
    g_b, g_p = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_b, stream=stream):
        batched_call()
    if plain:
        with torch.cuda.graph(g_p, stream=stream):
            plain_calls()
    torch.cuda.synchronize()
    if dx.get_status():
        raise RuntimeError("device status set after the batched warm-up")

    def time_graph(g, nsteps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for i in range(nsteps):
                g.replay()
                ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[-1]), [ev[i].elapsed_time(ev[i + 1]) for i in range(nsteps)]

    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    total_ms, per = time_graph(g_b, steps)
    barrier(world)
    clocks = sampler.stop()
    plain_ms = float("nan")
    if plain:
        psteps = max(1, min(steps, 5))
        plain_ms, _ = time_graph(g_p, psteps)
        plain_ms /= psteps
    if dx.get_status():
        raise RuntimeError("device status set after the batched timed region")
    total_ms, mean_ms, plain_ms = max_over_ranks([total_ms, float(np.mean(per)), plain_ms], world, device="cuda")
    ms = total_ms / steps
    rate = lambda t: total / (t * 1e-3)    # cells of all ranks over the slowest rank's time
    entry = {
        "workload": "batched_amr_1m" if args.nblocks == 2048 else f"batched_amr_{args.nblocks}_blocks",
        "ncells": total, "nblocks": len(desc) * (1 if args.partition else world), "block_cells": 512,
        "nspecies": "{1,4,8,16}", "dt": "2^-k, k in 0..6",
        "value": rate(ms), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": args.warmup,
        "launch": "one CUDA-graph replay of drag_expm_apply_batched: 4 binning kernels + 2 persistent kernels",
        "l2": "inputs (%.2f GB) larger than L2, no flush" % (bytes_step / 1e9),
        "roofline": roofline_entry(built, dense, bytes_step, mean_ms * 1e-3, peak, hbm_peak,
                                   "per block by its N's mode"),
        "plain_per_block": ({"value": rate(plain_ms), "unit": UNIT, "ms_per_step": plain_ms,
                             "batched_speedup": plain_ms / ms,
                             "note": "drag_expm_apply once per block, all launches captured in one CUDA graph"}
                            if plain else None),
        "clocks": clocks,
        "gpu_launches": 6 * steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nb, _ = cpu_oracle_batched_rate(batch, cpu_seconds)
        entry["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"first {nb} blocks of the batch, one pass (same seeded arrays)"}
    state = (desc, rg_h, rd_h, ts_h, v_h, rg, rd, ts, v, vout, dblocks, ws, batched_call, nmax)
    return entry, state


# ------------------------------------------------------------ headline extras ---

def headline_extras(dx, args, rank, world, stream, name, state, local):
    """e2e through the host-array entry point, the adjoint (recomputing and
    taped), RK1, the lower accuracy targets and the paper's variants, all on
    the headline cells."""
    import torch
    cells, rg, rd, ts, v, vout, k, s, per, total = state
    C = cells.ncells
    N = cells.rho_d.shape[0]
    steps = args.steps
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def timed(fn, nsteps):
        with torch.cuda.stream(stream):
            fn()
            torch.cuda.synchronize()
            return float(np.mean(time_steps(fn, nsteps, stream)))

    # e2e: the C-ABI call on pinned HOST buffers (drag_expm_apply_host): every
    # step copies the inputs host-to-device and v_out device-to-host, in chunks
    # pipelined against the updates
    h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hrg, hrd, hts, hv = h(cells.rho_g), h(cells.rho_d), h(cells.t_s), h(cells.v)
    hout = torch.empty_like(hv).pin_memory()
    h2d = sum(x.numel() * 8 for x in (hrg, hrd, hts, hv))
    d2h = hout.numel() * 8
    hws = torch.empty(dx.host_workspace_bytes(N), dtype=torch.uint8, device="cuda")
    e2e_ms = timed(lambda: dx.apply_host(hrg, hrd, hts, cells.dt, hv, hout, workspace=hws, stream=stream),
                   max(1, min(steps, 5)))

    vt = dev(W.adjoint_target(C, N))
    gvi, grg = torch.empty_like(v), torch.empty_like(rg)
    grd, gts = torch.empty_like(rd), torch.empty_like(ts)
    fb_steps = max(1, min(steps, 3))

    def fwd_bwd():
        dx.apply(rg, rd, ts, cells.dt, v, vout, stream=stream)
        torch.sub(vout, vt, out=gvi)
        dx.backward(rg, rd, ts, cells.dt, v, gvi, out=(vout, grg, grd, gts), stream=stream)

    fb_ms = timed(fwd_bwd, fb_steps)
    if dx.get_status():
        raise RuntimeError("device status set after forward + adjoint")

    tape_levels = dx.tape_levels_needed(rg, rd, ts, cells.dt)
    tape_nbytes = dx.tape_bytes(C, N, tape_levels)
    taped = {"levels": tape_levels, "tape_bytes": tape_nbytes}
    ft_ms = None
    if tape_nbytes < 0.8 * torch.cuda.mem_get_info()[0]:
        holder = [None]
        mids = []

        def fwd_bwd_taped():
            _, holder[0] = dx.apply_taped(rg, rd, ts, cells.dt, v, vout, levels=tape_levels, tape=holder[0],
                                          stream=stream)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            mids.append(ev)
            torch.sub(vout, vt, out=gvi)
            dx.backward(rg, rd, ts, cells.dt, v, gvi, out=(vout, grg, grd, gts), tape=holder[0], stream=stream)

        with torch.cuda.stream(stream):
            fwd_bwd_taped()
            torch.cuda.synchronize()
            mids.clear()
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(fb_steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(fb_steps)]
            for i in range(fb_steps):
                starts[i].record(stream)
                fwd_bwd_taped()
                ends[i].record(stream)
            torch.cuda.synchronize()
        ft_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / fb_steps
        fwd_t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, mids)) / fb_steps
        holder[0] = None
        if dx.get_status():
            raise RuntimeError("device status set after taped forward + adjoint")
        taped.update({"forward_taped_ms": fwd_t_ms, "adjoint_and_sub_ms": ft_ms - fwd_t_ms, "steps": fb_steps,
                      "note": "drag_expm_apply_taped + dL/dv_out (torch sub) + drag_expm_backward_taped, "
                              "outside the headline timed region"})
    else:
        taped["skipped"] = "tape larger than 80 % of free device memory"

    rk_steps = max(3, steps)
    rk_ms = timed(lambda: dx.rk1_apply(rg, rd, ts, cells.dt, v, vout, stream=stream), rk_steps)

    target_ms, target_ks = {}, {}
    for ub in (24, 11):
        kt, st_ = dx.select(rg, rd, ts, cells.dt, ubits=ub)
        target_ks[ub] = (float(kt.double().mean()), float(st_.double().mean()))
        target_ms[ub] = timed(lambda: dx.apply(rg, rd, ts, cells.dt, v, vout, ubits=ub, stream=stream), rk_steps)
    if dx.get_status():
        raise RuntimeError("device status set after the accuracy-target runs")

    variant_ms, variant_deg = {}, {}
    for vname, kw in (("taylor_bound_test", {"bound_test": True}), ("pade", {"method": "pade"}),
                      ("mixed_fp32_u24", {"ubits": 24, "arith": "fp32"})):
        if vname.startswith("mixed"):
            variant_deg[vname] = None
        else:
            _, mdeg, _ = dx.apply_opts(rg, rd, ts, cells.dt, v, vout, return_ms=True, **kw)
            variant_deg[vname] = float(mdeg.double().mean())
        variant_ms[vname] = timed(lambda: dx.apply_opts(rg, rd, ts, cells.dt, v, vout, stream=stream, **kw),
                                  rk_steps)
    if dx.get_status():
        raise RuntimeError("device status set after the variant runs")

    vals = [e2e_ms, fb_ms, ft_ms or 0.0, rk_ms, target_ms[24], target_ms[11], variant_ms["taylor_bound_test"],
            variant_ms["pade"], variant_ms["mixed_fp32_u24"]]
    (e2e_ms, fb_ms, ft_red, rk_ms, t24, t11, bt, pd, mx) = max_over_ranks(vals, world, device="cuda")
    rate = lambda t: total / (t * 1e-3)    # cells of all ranks over the slowest rank's time
    fwd_ms = float(np.mean(per))
    if ft_ms is not None:
        taped.update({"value": rate(ft_red), "unit": UNIT, "ms_per_step": ft_red})
    return {
        "e2e": {"value": rate(e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "drag_expm_apply_host (pinned host buffers, chunked copy/compute pipeline)"},
        "fwd_adjoint": {"value": rate(fb_ms), "unit": UNIT, "ms_per_step": fb_ms, "steps": fb_steps,
                        "adjoint_over_forward_time": fb_ms / fwd_ms,
                        "note": "forward + dL/dv_out (torch sub) + drag_expm_backward, outside the headline timed "
                                "region"},
        "fwd_adjoint_taped": taped,
        "rk1": {"value": rate(rk_ms), "unit": UNIT, "ms_per_step": rk_ms, "exp_over_rk1_time": fwd_ms / rk_ms,
                "note": "drag_rk1_apply (analytic implicit RK1, App. A.2), outside the headline timed region"},
        "precision_targets": {
            "note": "drag_expm_apply_target: Algorithm 2 on the theta table of u (Eq. B8), FP64 arithmetic; "
                    "outside the headline timed region",
            **{f"u=2^-{ub}": {"value": rate(t), "unit": UNIT, "ms_per_step": t, "mean_k_star": target_ks[ub][0],
                               "mean_s_star": target_ks[ub][1]} for ub, t in ((24, t24), (11, t11))}},
        "variants": {
            "note": "drag_expm_apply_opts: the paper's second modification (bound test), the Pade variant "
                    "(Eq. PadeEqu) and the mixed-precision path (FP32 matrix work at the u = 2^-24 target); "
                    "outside the headline timed region",
            **{vn: {"value": rate(t), "unit": UNIT, "ms_per_step": t, "mean_degree": variant_deg[vn]}
               for vn, t in (("taylor_bound_test", bt), ("pade", pd), ("mixed_fp32_u24", mx))}},
    }


def run_ours(args, rank, world):
    import torch

    import paper_2509_25347_gb300 as dx
    from paper_2509_25347_gb300 import build as dxbuild

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        dxbuild.build()
    barrier(world)
    dx.load_library()
    stream = torch.cuda.Stream()
    hbm_peak = read_hbm_peak()
    rates = fp64_rates(dx, stream)
    peak = rates["dfma"]                      # this rank's GPU; rank 0 prints its own
    square17 = square_comparison(dx, stream, 17)
    scaling = "strong" if (args.partition and world > 1) else "weak"

    if args.workload == "batched_amr_1m":
        head, _ = leg_batched(dx, args, rank, world, stream, peak, hbm_peak, local, args.steps, args.cpu_seconds)
        extras = {}
    else:
        adj = args.workload == "mrn_n8_128cube_adjoint"
        head, state = leg_single(dx, args, args.workload, rank, world, stream, peak, hbm_peak, local, args.steps,
                                 adjoint=adj, cpu_seconds=args.cpu_seconds, ncells=args.ncells)
        if args.workload == HEADLINE:
            wpc, _ = family_of(dx, 16)
            C_rank = state[0].ncells
            mean_s = head["roofline"]["kernel_mean_ms"] * 1e-3
            exec_flop = measured_traffic(args.workload, "dx_forward_wpc", C_rank, "executed_flop_per_cell") \
                if wpc else None
            head["roofline"]["traffic"] = measured_traffic(args.workload, "dx_forward_wpc", C_rank) if wpc else None
            head["roofline"]["traffic_unit"] = "bytes per launch (ncu dram read + write, per cell x cells)"
            head["roofline"]["executed"] = None if exec_flop is None else {
                "flop_per_launch": exec_flop, "achieved": exec_flop / mean_s / 1e12, "unit": "TFLOP/s",
                "frac": exec_flop / mean_s / 1e12 / peak,
                "source": "ncu thread-level DFMA x 2 + DADD + DMUL of the kernel per cell (profiles/); includes "
                          "the operations the kernel issues beyond the built count (padding, zero terms)"}
            extras = headline_extras(dx, args, rank, world, stream, args.workload, state, local)
        else:
            extras = {}
        del state
    torch.cuda.empty_cache()

    configs = {}
    if args.configs == "all" and args.workload == HEADLINE and not args.ncells:
        for name in CONFIG_LEGS:
            if name == "batched_amr_1m":
                e, st = leg_batched(dx, args, rank, world, stream, peak, hbm_peak, local, max(args.steps, 10))
            else:
                e, st = leg_single(dx, args, name, rank, world, stream, peak, hbm_peak, local,
                                   max(args.steps, 20) if name == "dustybox_n1_32k" else args.steps,
                                   adjoint=name == "mrn_n8_128cube_adjoint", cpu_seconds=5.0)
            del st
            torch.cuda.empty_cache()
            configs[name] = e

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": scaling,
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {k_: head[k_] for k_ in ("workload", "ncells", "nspecies", "matrix", "l2", "mean_k_star",
                                                "mean_s_star", "max_s_star", "nblocks", "dt", "launch")
                       if k_ in head},
            "roofline": head["roofline"],
            **extras,
            "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"],
            "fp64_peak": {**peak_entry(rates), "square_n17_dfma_vs_dmma": square17},
        }
        line["config"]["partition"] = ("contiguous cell ranges / cost-balanced whole blocks over ranks"
                                       if scaling == "strong" else
                                       "each rank its own independent draw of the workload")
        for k_ in ("fwd_adjoint", "fwd_adjoint_taped", "plain_per_block", "cpu_baseline", "variants"):
            if k_ in head and k_ not in line:
                line[k_] = head[k_]
        if "e2e" not in line:
            line["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                           "note": "measured on the headline workload only"}
        if world == 1 and not args.no_cpu_baseline and "cpu_baseline" in head:
            cb = head["cpu_baseline"]
            if args.workload != "batched_amr_1m":
                r1, s1 = cpu_oracle_single_core_rate(W.workload(args.workload, ncells=args.ncells),
                                                     seconds=args.cpu_seconds / 4)
                cb["single_core"] = {"value": r1, "unit": UNIT, "cores": 1,
                                     "sample": f"first {s1} cells of {args.workload}, one pass"}
            line["cpu_baseline"] = cb
        if configs:
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.fp64_peak:
        run_fp64_peak(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
