#!/usr/bin/env python3
"""Throughput benchmark of the FP64 EXP drag update on GB300.

One step = one forward drag update (drag_expm_apply) over the whole
workload: the N=16 MRN-like workload of 128^3 = 2,097,152 cells by default
(17x17 drag matrices, dt/t_s in [1e-4, 1e8]). Inputs are synthetic and seeded
(paper_2509_25347_gb300.workloads) and larger than L2, so no flush is needed.

Prints one JSON line (rank 0). Launch N>1 with torchrun; each rank then runs
its own full copy of the workload (independent cells, weak scaling, no
collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_25347_gb300 import workloads as W  # noqa: E402

METRIC = "FP64 cell drag updates/sec at N=16 (fwd, fwd+adjoint) and % of FP64/HBM roofline"
UNIT = "cell-updates/s"
# FP64 pipe of one GB300: 152 SMs x 4 sub-partitions x 0.5 DFMA/clk x 2 flop = 608 flop/clk
# (measured: one warp-wide DFMA per 64 cycles per sub-partition), at the 2070 MHz maximum SM clock.
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
        "sources_sha256": "f950f6c493d2a33d0c91a98262307d52299e93c66fbed3697cfecb38b8e7fd88",
        "bytes_per_cell": (188.071936e6 + 81.039104e6) / 262144,
        # FP64 FLOPs the kernel executes: thread-level (2 DFMA + DADD + DMUL) per cycle x elapsed cycles
        "executed_flop_per_cell": (2 * 231.801724 + 15.894142 + 3.616074) * 49135479.171 / 262144,
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
    p.add_argument("--workload", default="mrn_n16_128cube", choices=list(W.WORKLOADS))
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


def algorithmic_counts(N, k, s):
    """Per-cell algorithmic FLOPs (2 n^3 (k* + s*) + 6 n^2: k* + s* dense n x n
    products, App. B "Numerical cost", plus three mat-vecs) and bytes
    (8 (1 + 2N) inputs + 24 n in + 24 n out)."""
    n = N + 1
    flops = 2.0 * n ** 3 * (k.astype(np.float64) + s.astype(np.float64)) + 6.0 * n * n
    bytes_per_cell = 8 * (1 + 2 * N) + 48 * n
    return flops, bytes_per_cell


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


def _oracle_chunk(args):
    import oracle
    rg, rd, ts, dt, v = args
    oracle.drag_apply(rg, rd, ts, dt, v)
    return rg.shape[0]


def cpu_oracle_rate(cells, seconds, steps=1):
    """Oracle cell-updates/s on the host cores (spawned worker processes, one
    chunk of contiguous cells each). Returns (rate, cores, sample_cells, wall_per_step)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    probe = cells.subset(np.arange(min(64, cells.ncells)))
    t0 = time.perf_counter()
    oracle.drag_apply(probe.rho_g, probe.rho_d, probe.t_s, probe.dt, probe.v)
    per_cell = (time.perf_counter() - t0) / probe.ncells
    sample = int(min(cells.ncells, max(cores * 16, seconds * cores / max(per_cell, 1e-9))))
    sub = cells.subset(np.arange(sample))
    bounds = np.linspace(0, sample, cores + 1).astype(int)
    chunks = [(sub.rho_g[a:b].copy(), sub.rho_d[:, a:b].copy(), sub.t_s[:, a:b].copy(), sub.dt,
               sub.v[:, :, a:b].copy()) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    ctx = mp.get_context("spawn")
    walls = []
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(c[0][:1], c[1][:, :1], c[2][:, :1], c[3], c[4][:, :, :1]) for c in chunks])
        for _ in range(steps):
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_chunk, chunks))
            walls.append(time.perf_counter() - t0)
    wall = float(np.mean(walls))
    return done / wall, cores, sample, wall


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


# ---------------------------------------------------------------- reference ---

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
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    probe = W.Batch(batch.blocks[:8])
    oracle.drag_apply_batched(*probe.pack())
    per_cell = (time.perf_counter() - t0) / max(1, probe.ncells)
    want_cells = seconds * cores / max(per_cell, 1e-9)
    nb = int(min(len(batch.blocks), max(cores, want_cells / 512)))
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
        rate, cores, sample, wall = cpu_oracle_rate(cells, seconds=secs, steps=args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "ncells": C, "nspecies": N, "step_sample_cells": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {sample} cells of {args.workload} per step"},
            "gpu_launches": 0,
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours ---

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
    if world > 1:
        torch.distributed.barrier()
    dx.load_library()

    _, C, N, _ = W.WORKLOADS[args.workload]
    if args.ncells:
        C = min(C, args.ncells)
    cells = W.workload(args.workload, ncells=C)
    n = N + 1
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rg, rd, ts, v = dev(cells.rho_g), dev(cells.rho_d), dev(cells.t_s), dev(cells.v)
    vout = torch.empty_like(v)
    stream = torch.cuda.current_stream()

    k, s = dx.select(rg, rd, ts, cells.dt)
    k, s = k.cpu().numpy(), s.cpu().numpy()
    flops_cell, bytes_cell = algorithmic_counts(N, k, s)
    flops_launch = float(flops_cell.sum())

    for _ in range(args.warmup):
        dx.apply(rg, rd, ts, cells.dt, v, vout)
    torch.cuda.synchronize()
    dx.get_status()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # Inputs smaller than twice L2 (the small N = 1 workload, truncated profiling
    # runs) would be re-read from L2 by the next launch: write a buffer of twice
    # L2 between timed launches and time each launch on its own.
    l2 = getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 0) or 129 * 2 ** 20
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device="cuda") if bytes_cell * C < 2 * l2 else None
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(float(i))
        ev0[i].record(stream)
        dx.apply(rg, rd, ts, cells.dt, v, vout)
        ev1[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    per_launch = [ev0[i].elapsed_time(ev1[i]) for i in range(args.steps)]
    total_ms = float(np.sum(per_launch))
    status = dx.get_status()
    if status:
        raise RuntimeError(f"device status {status:#x} after timed region")

    # e2e: the C-ABI call on pinned HOST buffers (drag_expm_apply_host): every
    # step copies the inputs host-to-device and v_out device-to-host, in chunks
    # pipelined against the updates
    h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hrg, hrd, hts, hv = h(cells.rho_g), h(cells.rho_d), h(cells.t_s), h(cells.v)
    hout = torch.empty_like(hv).pin_memory()
    h2d = sum(x.numel() * 8 for x in (hrg, hrd, hts, hv))
    d2h = hout.numel() * 8
    e2e_steps = max(1, min(args.steps, 5))
    hws = torch.empty(dx.host_workspace_bytes(N), dtype=torch.uint8, device="cuda")
    dx.apply_host(hrg, hrd, hts, cells.dt, hv, hout, workspace=hws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        dx.apply_host(hrg, hrd, hts, cells.dt, hv, hout, workspace=hws)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    # forward + adjoint: loss 0.5 ||v_out - v_target||^2, v_target ~ N(0,1)
    vt = dev(W.adjoint_target(C, N))
    gvi = torch.empty_like(v)
    grd, gts = torch.empty_like(rd), torch.empty_like(ts)
    grg = torch.empty_like(rg)
    fb_steps = max(1, min(args.steps, 3))

    def fwd_bwd():
        dx.apply(rg, rd, ts, cells.dt, v, vout)
        torch.sub(vout, vt, out=gvi)                     # dL/dv_out
        dx.backward(rg, rd, ts, cells.dt, v, gvi, out=(vout, grg, grd, gts))

    fwd_bwd()
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(fb_steps):
        fwd_bwd()
    b1.record(stream)
    torch.cuda.synchronize()
    fb_ms = b0.elapsed_time(b1) / fb_steps
    if dx.get_status():
        raise RuntimeError("device status set after forward + adjoint")

    # forward + adjoint through the adjoint tape: the forward records
    # E_0 .. E_{s*-2}, the adjoint reads them (same gradients, fewer FP64 ops)
    tape_levels = dx.tape_levels_needed(rg, rd, ts, cells.dt)
    tape_nbytes = dx.tape_bytes(C, N, tape_levels)
    fwd_adj_taped = {"levels": tape_levels, "tape_bytes": tape_nbytes}
    if tape_nbytes < 0.8 * torch.cuda.mem_get_info()[0]:
        holder = [None]

        def fwd_bwd_taped(ev=None):
            _, holder[0] = dx.apply_taped(rg, rd, ts, cells.dt, v, vout, levels=tape_levels, tape=holder[0])
            if ev is not None:
                ev.record(stream)
            torch.sub(vout, vt, out=gvi)
            dx.backward(rg, rd, ts, cells.dt, v, gvi, out=(vout, grg, grd, gts), tape=holder[0])

        fwd_bwd_taped()
        torch.cuda.synchronize()
        mids = [torch.cuda.Event(enable_timing=True) for _ in range(fb_steps)]
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(fb_steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(fb_steps)]
        for i in range(fb_steps):
            starts[i].record(stream)
            fwd_bwd_taped(mids[i])
            ends[i].record(stream)
        torch.cuda.synchronize()
        ft_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / fb_steps
        fwd_t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, mids)) / fb_steps
        holder[0] = None
        if dx.get_status():
            raise RuntimeError("device status set after taped forward + adjoint")
        fwd_adj_taped.update({"value": whole_job_rate(C, world, ft_ms), "unit": UNIT, "ms_per_step": ft_ms,
                              "forward_taped_ms": fwd_t_ms, "adjoint_and_sub_ms": ft_ms - fwd_t_ms,
                              "steps": fb_steps,
                              "note": "drag_expm_apply_taped + dL/dv_out (torch sub) + drag_expm_backward_taped, "
                                      "outside the headline timed region"})
    else:
        fwd_adj_taped["skipped"] = "tape larger than 80 % of free device memory"

    # analytic implicit RK1 (App. A.2): the paper's cost reference for EXP
    rk_steps = max(3, args.steps)
    for _ in range(2):
        dx.rk1_apply(rg, rd, ts, cells.dt, v, vout)
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(rk_steps):
        dx.rk1_apply(rg, rd, ts, cells.dt, v, vout)
    r1.record(stream)
    torch.cuda.synchronize()
    rk_ms = r0.elapsed_time(r1) / rk_steps

    # lower accuracy targets (Eq. B8 with u = 2^-24, 2^-11): Algorithm 2 on
    # that theta table, FP64 arithmetic
    target_ms, target_ks = {}, {}
    for ub in (24, 11):
        kt, st_ = dx.select(rg, rd, ts, cells.dt, ubits=ub)
        target_ks[ub] = (float(kt.double().mean()), float(st_.double().mean()))
        dx.apply(rg, rd, ts, cells.dt, v, vout, ubits=ub)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(rk_steps):
            dx.apply(rg, rd, ts, cells.dt, v, vout, ubits=ub)
        t1.record(stream)
        torch.cuda.synchronize()
        target_ms[ub] = t0.elapsed_time(t1) / rk_steps
    if dx.get_status():
        raise RuntimeError("device status set after the accuracy-target runs")

    # the paper's variants: second modification (bound test) and Pade
    variant_ms, variant_deg = {}, {}
    for name, kw in (("taylor_bound_test", {"bound_test": True}), ("pade", {"method": "pade"}),
                     ("mixed_fp32_u24", {"ubits": 24, "arith": "fp32"})):
        if name.startswith("mixed"):
            dx.apply_opts(rg, rd, ts, cells.dt, v, vout, **kw)
            variant_deg[name] = None
        else:
            _, mdeg, _ = dx.apply_opts(rg, rd, ts, cells.dt, v, vout, return_ms=True, **kw)
            variant_deg[name] = float(mdeg.double().mean())
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(rk_steps):
            dx.apply_opts(rg, rd, ts, cells.dt, v, vout, **kw)
        t1.record(stream)
        torch.cuda.synchronize()
        variant_ms[name] = t0.elapsed_time(t1) / rk_steps
    if dx.get_status():
        raise RuntimeError("device status set after the variant runs")

    total_ms, e2e_ms, fb_ms, rk_ms, t24_ms, t11_ms, bt_ms, pd_ms, mx_ms = max_over_ranks(
        [total_ms, e2e_ms, fb_ms, rk_ms, target_ms[24], target_ms[11], variant_ms["taylor_bound_test"],
         variant_ms["pade"], variant_ms["mixed_fp32_u24"]], world, device="cuda")
    target_ms = {24: t24_ms, 11: t11_ms}
    variant_ms = {"taylor_bound_test": bt_ms, "pade": pd_ms, "mixed_fp32_u24": mx_ms}
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(C, world, ms_per_step)
    e2e_value = whole_job_rate(C, world, e2e_ms)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    mean_launch_s = float(np.mean(per_launch)) * 1e-3
    achieved_tf = flops_launch / mean_launch_s / 1e12
    peak_tf = FP64_FLOP_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except Exception:
        pass
    gbs = bytes_cell * C / mean_launch_s / 1e9
    wpc = dx.get_mode(N) == dx.MODE_WARP_PER_CELL
    exec_flop = measured_traffic(args.workload, "dx_forward_wpc", C, "executed_flop_per_cell") if wpc else None
    executed = None if exec_flop is None else {
        "flop_per_launch": exec_flop, "achieved": exec_flop / mean_launch_s / 1e12, "unit": "TFLOP/s",
        "frac": exec_flop / mean_launch_s / 1e12 / peak_tf,
        "source": "ncu thread-level DFMA x 2 + DADD + DMUL of the kernel, per cell, from the capture in profiles/",
        "note": "the symmetric-form kernel executes fewer FLOPs than the dense cost model 2n^3 (k* + s*) + 6n^2 "
                "behind `achieved`; this is the pipe's own load"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "ncells": C, "nspecies": N, "matrix": f"{n}x{n}",
                   "dt_over_ts": W.WORKLOADS[args.workload][0].split("dt/t_s in ")[-1],
                   "l2": ("inputs (%.2f GB) larger than L2, no flush" % (bytes_cell * C / 1e9)) if flush is None
                   else ("inputs (%.4f GB) below 2 x L2: a %.0f MB buffer written between timed launches, each "
                         "launch timed alone" % (bytes_cell * C / 1e9, 2 * l2 / 1e6)),
                   "mean_k_star": float(k.mean()), "mean_s_star": float(s.mean()), "max_s_star": int(s.max())},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / peak_tf,
                     "traffic": measured_traffic(args.workload, "dx_forward_wpc", C) if wpc else None,
                     "traffic_unit": "bytes per launch (ncu dram read + write, per cell x cells)",
                     "algorithmic_bytes_per_launch": float(bytes_cell * C),
                     "peak_source": "FP64 pipe: 152 SMs x 608/152 flop/clk x 2070 MHz (unit count x max clock)",
                     "algorithmic_flop_per_launch": flops_launch,
                     "algorithmic_flop_model": "paper's cost model (App. B): k* + s* dense n x n products per cell, "
                                               "2n^3 (k* + s*) + 6n^2 FLOPs; frac > 1 because the kernel exploits "
                                               "symmetry and the arrowhead (see `executed` for the pipe's own load)",
                     "kernel_mean_ms": mean_launch_s * 1e3,
                     "hbm_gbs": gbs, "hbm_frac_of_measured": (gbs / hbm_peak) if hbm_peak else None,
                     "executed": executed},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "drag_expm_apply_host (pinned host buffers, chunked copy/compute pipeline)"},
        "fwd_adjoint": {"value": whole_job_rate(C, world, fb_ms), "unit": UNIT, "ms_per_step": fb_ms, "steps": fb_steps,
                        "note": "forward + dL/dv_out (torch sub) + drag_expm_backward, outside the headline timed region"},
        "fwd_adjoint_taped": fwd_adj_taped,
        "rk1": {"value": whole_job_rate(C, world, rk_ms), "unit": UNIT, "ms_per_step": rk_ms,
                "exp_over_rk1_time": ms_per_step / rk_ms, "hbm_gbs": bytes_cell * C / (rk_ms * 1e-3) / 1e9,
                "hbm_frac_of_measured": (bytes_cell * C / (rk_ms * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None,
                "note": "drag_rk1_apply (analytic implicit RK1, App. A.2), outside the headline timed region"},
        "precision_targets": {
            "note": "drag_expm_apply_target: Algorithm 2 on the theta table of u (Eq. B8), FP64 arithmetic; "
                    "outside the headline timed region",
            **{f"u=2^-{ub}": {"value": whole_job_rate(C, world, target_ms[ub]), "unit": UNIT,
                               "ms_per_step": target_ms[ub], "mean_k_star": target_ks[ub][0],
                               "mean_s_star": target_ks[ub][1]}
               for ub in (24, 11)}},
        "variants": {
            "note": "drag_expm_apply_opts: the paper's second modification (bound test), the Pade variant "
                    "(Eq. PadeEqu) and the mixed-precision path (FP32 matrix work at the u = 2^-24 target), "
                    "warp per cell; outside the headline timed region",
            **{name: {"value": whole_job_rate(C, world, variant_ms[name]), "unit": UNIT,
                      "ms_per_step": variant_ms[name], "mean_degree": variant_deg[name]}
               for name in ("taylor_bound_test", "pade", "mixed_fp32_u24")}},
        "gpu_launches": dx.apply_launches(C, N) * args.steps,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        rate, cores, sample, _ = cpu_oracle_rate(cells, seconds=args.cpu_seconds)
        rate1, sample1 = cpu_oracle_single_core_rate(cells, seconds=args.cpu_seconds / 4)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {sample} cells of {args.workload}, one pass",
                                "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                                "sample": f"first {sample1} cells of {args.workload}, one pass"}}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(args, rank, world):
    """AMR-like batched workload: one step = one CUDA-graph replay of
    drag_expm_apply_batched over 2048 blocks of 8^3 cells (N in {1,4,8,16},
    dt = 2^-k). The plain single-N entry point, launched once per block and
    captured in a graph too, is timed alongside for comparison."""
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
    if world > 1:
        torch.distributed.barrier()
    dx.load_library()

    batch = W.batched(nblocks=args.nblocks)
    desc, rg_h, rd_h, ts_h, v_h = batch.pack()
    C = rg_h.size
    nmax = int(desc["nspecies"].max())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rg, rd, ts, v = dev(rg_h), dev(rd_h), dev(ts_h), dev(v_h)
    dblocks = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
    vout = torch.empty_like(v)
    ws = torch.empty(dx.batched_workspace_bytes(len(desc), C), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()

    # algorithmic FLOPs from each block's (k*, s*)
    flops = 0.0
    for (N, dt, cells), d in zip(batch.blocks, desc):
        co, do = int(d["cell_offset"]), int(d["dust_offset"])
        k, s = dx.select(rg[co:co + cells.ncells], rd[do:do + N * cells.ncells].view(N, cells.ncells),
                         ts[do:do + N * cells.ncells].view(N, cells.ncells), dt)
        flops += float(algorithmic_counts(N, k.cpu().numpy(), s.cpu().numpy())[0].sum())
    bytes_step = float(sum(8 * (1 + 2 * N) + 48 * (N + 1) for N in desc["nspecies"]) * 512)

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
        raise RuntimeError("device status set after warm-up")

    def time_graph(g, steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for i in range(steps):
                g.replay()
                ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[-1]), [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms, per = time_graph(g_b, args.steps)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    plain_ms = float("nan")
    if plain:
        plain_ms, _ = time_graph(g_p, max(1, min(args.steps, 5)))
        plain_ms /= max(1, min(args.steps, 5))
    if dx.get_status():
        raise RuntimeError("device status set after timed region")

    # e2e: host inputs -> device, batched call, v_out -> host
    h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hrg, hrd, hts, hv, hdesc = h(rg_h), h(rd_h), h(ts_h), h(v_h), h(desc.view(np.uint8))
    hout = torch.empty_like(hv).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in (hrg, hrd, hts, hv, hdesc))
    d2h = hout.numel() * 8
    e2e_steps = max(1, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(e2e_steps):
            for dst, src in ((rg, hrg), (rd, hrd), (ts, hts), (v, hv), (dblocks, hdesc)):
                dst.copy_(src, non_blocking=True)
            batched_call()
            hout.copy_(vout, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    total_ms, e2e_ms, plain_ms = max_over_ranks([total_ms, e2e_ms, plain_ms], world, device="cuda")
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    ms = total_ms / args.steps
    mean_s = float(np.mean(per)) * 1e-3
    achieved = flops / mean_s / 1e12
    peak = FP64_FLOP_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": whole_job_rate(C, world, ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched_amr_1m" if args.nblocks == 2048 else f"batched_amr_{args.nblocks}_blocks",
                   "ncells": C, "nblocks": len(desc), "block_cells": 512,
                   "nspecies": "{1,4,8,16}", "dt": "2^-k, k in 0..6",
                   "l2": "inputs (%.2f GB) larger than L2, no flush" % (bytes_step / 1e9),
                   "launch": "one CUDA-graph replay: 4 binning kernels + 1 persistent kernel"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "algorithmic_flop_per_launch": flops, "step_mean_ms": mean_s * 1e3,
                     "peak_source": "FP64 pipe: 152 SMs x 608/152 flop/clk x 2070 MHz (unit count x max clock)"},
        "plain_per_block": ({"value": whole_job_rate(C, world, plain_ms), "unit": UNIT, "ms_per_step": plain_ms,
                             "note": "drag_expm_apply once per block, all launches captured in one CUDA graph"}
                            if plain else None),
        "e2e": {"value": whole_job_rate(C, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 5 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.workload == "batched_amr_1m":
        run_batched(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
