#!/usr/bin/env python3
"""Benchmark of the adjoint-guided AMR hot path on GB300.

A step is one complete forward solve of the 2D layered-acoustics workload
(coarse 100^2, ratios 2 and 4, t_f = 8; adjoint-flagged regridding every 2
steps of each level; J at t_f) against the device-resident adjoint snapshot
set (400^2 x 200 snapshots, solved once on the GPU before timing).  The
metric is FP64 forward cell-updates per second.  Alongside: the batched
4096-patch configuration (fused work-list launch vs one launch per patch),
the roofline of the step kernel against the live-measured FP64 pipe peak,
an end-to-end figure through the public API from pinned host buffers, and
the CPU oracle as the reported baseline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 (under torchrun): independent replicas, one per GPU (the path has no
data exchange between solves); value = all ranks' cell-updates / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FP64 cell-updates/s (fused batched vs per-patch, same GPU); serve p50/p99 latency"
UNIT = "cell-updates/s"

# FP64 operations per cell-update in the canonical operation order, one per
# IEEE operation (fma, division, min and max count one each; negation and
# absolute value are free; a cell owns one x-edge and one y-edge); counted by
# running that sequence on a counting number type (tests/test_op_count.py).
#  2D acoustics, per edge: jump 2, decomposition 6, fluctuations 4, two MC
#   limiters 20, correction coefficients 4, second-order flux 12, CFL 3
#   (max |s|, product, running max), two transverse splits 16 and their
#   accumulation 4 = 71; per cell: entering sums 6 (component 0, the one the
#   transverse splits take), update 18.  2*71 + 24 = 166.
#  2D linearised shallow water (f-wave): jump 3, decomposition 6, no
#   fluctuation products, limiters 20, coefficients 2, flux 12, CFL 3,
#   transverse 16 + 4 = 66 per edge; 2*66 + 24 = 156.
#  1D acoustics: per edge 2 + 6 + 4 + 20 + 4 + 12 + 3 = 51; update 9; 60.
# The FP64 pipe issues one such operation per instruction, so the roofline
# peak is the pipe's instruction rate (the DFMA micro-benchmark's flop rate / 2).
OPS_PER_CELL = {"acoustics2d": 166, "shallow_water2d": 156, "acoustics1d": 60}
OPS_PER_CELL_2D = OPS_PER_CELL["acoustics2d"]
# algorithmic bytes per cell-update: read q (m doubles) and the cell's
# coefficients (aux), write q
BYTES_PER_CELL = {"acoustics2d": 24 + 32 + 24, "shallow_water2d": 24 + 48 + 24, "acoustics1d": 16 + 24 + 16}
# DRAM bytes per cell-update of a finest-level step launch, from an ncu
# capture of one such launch (the 601st finest-level launch of the config-2
# solve to t = 2: 53,424 cells, 3.67 MB read, 0 written): 69 B, 1.2x the 56
# algorithmic bytes read (tile halos and descriptors); written lines stay in
# L2 within the launch.  The capture predates the current k_step2d, which
# reads its work-list entry before the wait for the kernel ahead, so the
# roofline reports no traffic for it and names the capture instead.
TRAFFIC_PER_CELL_L2 = 3.665152e6 / 53424.0
TRAFFIC_IS_CURRENT = False


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(td, local_ms, local_cells, device):
    """Replicas: whole-job time is the slowest rank's, work is the sum over
    ranks.  Returns (max ms, total cell-updates)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(local_cells)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    td.all_reduce(c, op=td.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def workload():
    from paper_1511_03645_gb300 import workloads as W
    return W.config2(seed=0, ts=0.0, tol=1e-3)


# ------------------------------------------------------------------ oracle
def oracle_sample(wl, snaps, budget_s=15.0):
    """The CPU oracle (as it stands) on the same workload: coarse steps from
    t_0 until the time budget is used; returns (cell-updates/s, description)."""
    from oracle import oracle as O
    h = O.OracleHierarchy(wl)
    h.set_adjoint(snaps)
    t0 = time.perf_counter()
    h.regrid(0, init=True)
    n = 0
    ntot = h.nsteps_total()
    while n < ntot and time.perf_counter() - t0 < budget_s:
        h.advance(1)
        n += 1
    dt = time.perf_counter() - t0
    cu = h.cell_updates()
    return cu / dt, f"first {n} of {ntot} level-0 steps of the forward AMR solve ({cu} cell-updates, {dt:.1f} s)"


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    from oracle import oracle as O
    wl = workload()
    # the oracle's own adjoint on a bounded grid would take minutes; the
    # snapshot set is an input of the forward solve, so it is built here
    # (untimed) by the oracle at the workload's size
    t = time.perf_counter()
    snaps = O.adjoint_solve(wl)
    log(f"reference: oracle adjoint solve {time.perf_counter() - t:.1f} s")
    per = []
    cus = []
    desc = ""
    for k in range(args.warmup + args.steps):
        v, desc = oracle_sample(wl, snaps, budget_s=max(2.0, 60.0 / max(1, args.warmup + args.steps)))
        if k >= args.warmup:
            per.append(v)
    val = statistics.median(per)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name + " config 2 (100^2, ratios 2,4, t_f=8, adjoint 400^2x200)",
                       "sample": desc},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ configs 1 and 3
def measure_config(A, W, wl, s, peak_ops, cpu_budget, adj_medium=None, label=""):
    """One more workload of the benchmark measured whole: its adjoint solved on
    the GPU (untimed), one warm-up and one timed forward solve (CUDA events on
    the solve's stream, inputs resident), one instrumented solve for the
    step-kernel roofline, and the CPU oracle on a bounded sample of the same
    solve (its first coarse steps)."""
    import torch
    sp = s.cuda_stream
    t = time.perf_counter()
    adj = A.solve_adjoint(wl, stream=sp, medium_dense=adj_medium)
    torch.cuda.synchronize()
    adj_s = time.perf_counter() - t

    def run(timing):
        h = A.Hierarchy(wl, stream=sp)
        h.set_adjoint(adj)
        h.set_timing(timing)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        h.regrid(0, init=True)
        h.advance(h.nsteps_total())
        J = h.functional()
        e1.record(s)
        e1.synchronize()
        st = h.stats()
        h.close()
        return e0.elapsed_time(e1), st, J

    run(False)
    ms, st, J = run(False)
    _, sti, _ = run(True)
    ops = OPS_PER_CELL[wl.name]
    nbytes = BYTES_PER_CELL[wl.name]
    step_s = sti["step_kernel_ms"] * 1e-3
    achieved = ops * sti["cell_updates"] / step_s / 1e12 if step_s > 0 else None
    out = {"workload": label, "value": st["cell_updates"] / (ms * 1e-3), "unit": UNIT, "ms_per_solve": ms,
           "cell_updates": st["cell_updates"], "J": J, "adjoint_solve_s": adj_s,
           "roofline": {"bound": "alu", "kernel": "k_step1d" if wl.dim == 1 else "k_step2d", "achieved": achieved,
                        "peak": peak_ops, "unit": "TOP/s (FP64 operations)",
                        "frac": achieved / peak_ops if achieved else None, "ops_per_cell_update": ops,
                        "algorithmic_bytes_per_cell_update": nbytes,
                        "step_kernel_ms": sti["step_kernel_ms"], "step_launches": sti["step_kernel_launches"],
                        "per_level_tops": [ops * c / (m * 1e-3) / 1e12 if m > 0 else None
                                           for c, m in zip(sti["level_cell_updates"][:wl.nlevels],
                                                           sti["level_step_ms"][:wl.nlevels])]}}
    if cpu_budget > 0:
        snaps = adj.read()
        v, desc = oracle_sample(wl, snaps, budget_s=cpu_budget)
        del snaps
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                               "sample": desc}
    adj.release()
    return out


def measure_adjoint_amr(A, W, wl, s, fixed_s, ratios=(2,), tol=0.01):
    """The adjoint of config 2 solved with AMR (its 400^2 grid as level 0,
    finer levels by undivided-difference flags): wall time (the host
    regrids included), adjoint cell-updates/s, and the largest difference of
    its snapshots from the fixed-grid ones."""
    import torch
    sp = s.cuda_stream
    fixed = A.solve_adjoint(wl, stream=sp)
    best = None
    for _ in range(2):
        h = A.Hierarchy(wl, stream=sp)
        torch.cuda.synchronize()
        t = time.perf_counter()
        a = A.solve_adjoint(wl, stream=sp, ctx=h, amr=(ratios, W.FLAG_DIFFERENCE, tol))
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        cu = h.stats()["adjoint_cell_updates"]
        h.close()
        if best is None or el < best[0]:
            if best is not None:
                best[2].release()
            best = (el, cu, a)
        else:
            a.release()
    el, cu, a = best
    diff = float(np.max(np.abs(a.read() - fixed.read())))
    a.release()
    fixed.release()
    return {"workload": "config-2 adjoint, 400^2 x 200 snapshots as level 0, ratios " + str(list(ratios))
                        + f", undivided-difference flags tol {tol}",
            "s": el, "cell_updates": cu, "value": cu / el, "unit": UNIT, "fixed_grid_s": fixed_s,
            "max_abs_snapshot_change_vs_fixed_grid": diff}


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world):
    import torch
    from paper_1511_03645_gb300 import adjamr as A
    from paper_1511_03645_gb300 import workloads as W

    dist = world > 1
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    A.load()
    wl = workload()
    s = torch.cuda.Stream()
    sp = s.cuda_stream

    # FP64 pipe peak (live)
    peak_fma, _ = A.fp64_peak(0, 8192)
    peak_add, _ = A.fp64_peak(1, 8192)

    t = time.perf_counter()
    adj = A.solve_adjoint(wl, stream=sp)
    torch.cuda.synchronize()
    adj_s = time.perf_counter() - t
    log(f"adjoint solve on GPU: {adj_s:.3f} s")

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    # step-kernel tile per level (same bits for every tile; speed only)
    from paper_1511_03645_gb300 import autotune as AT
    tuned = AT.tune_amr(wl, adj, key="acoustics2d-100-r2r4", stream=s, use_cache=False)
    log(f"tiles per level: {tuned['best_per_level']}")

    def make(timing=False):
        h = A.Hierarchy(wl, stream=sp)
        h.set_adjoint(adj)
        h.set_timing(timing)
        AT.apply_amr(h, tuned)
        return h

    def solve(h):
        h.regrid(0, init=True)
        h.advance(h.nsteps_total())
        return h.functional()

    for _ in range(args.warmup):
        h = make()
        solve(h)
        h.close()
    hs = [make() for _ in range(args.steps)]
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    times = []
    cu = 0
    launches = 0
    step_ms = 0.0
    step_launches = 0
    Js = []
    regrid_ms = 0.0
    cluster_ms = 0.0
    rebuilds = kept = 0
    phases = [0.0] * 6
    cphases = [0.0] * 4
    lev_ms = [0.0] * wl.nlevels
    lev_launch = [0] * wl.nlevels
    lev_cells = [0] * wl.nlevels
    lev_ghost = [0.0] * wl.nlevels
    for h in hs:
        with torch.cuda.stream(s):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(s)
        J = solve(h)
        ev1.record(s)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        st = h.stats()
        cu += st["cell_updates"]
        launches += st["kernel_launches"]
        regrid_ms += st["regrid_host_ms"]
        cluster_ms += st["cluster_host_ms"]
        rebuilds += st["level_rebuilds"]
        kept += st["level_rebuilds_skipped"]
        phases = [a + b for a, b in zip(phases, st["regrid_phase_ms"])]
        cphases = [a + b for a, b in zip(cphases, st["cluster_phase_ms"])]
        Js.append(J)
    torch.cuda.synchronize()
    if dist:
        td.barrier()
    ck = clocks.stop()
    # step-kernel times from one more solve with CUDA events around every
    # level's launches (kept out of the timed solves: an event between two
    # kernels also stops the next one from launching early)
    hi = make(timing=True)
    solve(hi)
    torch.cuda.synchronize()
    st = hi.stats()
    hi.close()
    step_ms = st["step_kernel_ms"] * args.steps
    step_launches = st["step_kernel_launches"] * args.steps
    for lev in range(wl.nlevels):
        lev_ms[lev] = st["level_step_ms"][lev] * args.steps
        lev_launch[lev] = st["level_step_launches"][lev] * args.steps
        lev_cells[lev] = st["level_cell_updates"][lev] * args.steps
        lev_ghost[lev] = st["level_ghost_ms"][lev] * args.steps
    total_ms = sum(times)
    if dist:
        total_ms, cu_all = aggregate(td, total_ms, cu, "cuda")
    else:
        cu_all = float(cu)
    value = cu_all / (total_ms * 1e-3)
    for h in hs:
        h.close()

    # roofline of the step kernel (FP64-pipe bound)
    cells_per_launch = cu / max(step_launches, 1)
    avg_launch_s = step_ms * 1e-3 / max(step_launches, 1)
    achieved = OPS_PER_CELL_2D * cells_per_launch / avg_launch_s / 1e12
    # peak: FP64 instructions per second of the pipe, measured live with DFMA
    # chains (flop rate / 2: one operation per instruction)
    peak = peak_fma / 2 / 1e12

    # batched patches: fused work-list vs one launch per patch (same GPU)
    batched = None
    if rank == 0:
        pb = W.config4(seed=0)
        b = A.Batch(pb, stream=sp)
        cells = b.cells()
        res = {}
        for name, mode, graph in (("fused_worklist", 0, False), ("fused_persistent", 1, False),
                                  ("fused_graph", 0, True), ("per_patch", 2, False)):
            b.step(2, mode=mode, graph=graph)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            nst = 20
            e0.record(s)
            b.step(nst, mode=mode, graph=graph)
            e1.record(s)
            e1.synchronize()
            res[name] = cells * nst / (e0.elapsed_time(e1) * 1e-3)
        b.close()
        # autotuned: work-list order x tile x launch mode x ghost fusion, then
        # the best configuration replayed from a CUDA graph
        tb = AT.tune_batch(pb, key="config4-seed0", stream=s, use_cache=False)
        best = tb["best"]
        b = A.Batch(pb, stream=sp)
        b.set_order(AT.batch_orders(pb)[best["order"]])
        b.set_ghost_fusion(best["fuse_ghosts"])
        tile = tuple(best["tile"])
        b.step(2, mode=best["mode"], tile=tile, graph=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        nst = 20
        e0.record(s)
        b.step(nst, mode=best["mode"], tile=tile, graph=True)
        e1.record(s)
        e1.synchronize()
        res["fused_tuned_graph"] = cells * nst / (e0.elapsed_time(e1) * 1e-3)
        b.close()
        tuned_batch = {k: best[k] for k in ("order", "tile", "mode", "fuse_ghosts")}
        best_fused = max(v for k, v in res.items() if k != "per_patch")
        batched = {"patches": pb.npatch, "cells": cells, **{k: v for k, v in res.items()},
                   "tuned_config": tuned_batch,
                   "fp64_roofline_frac_best": OPS_PER_CELL_2D * best_fused / (peak_fma / 2),
                   "fused_over_per_patch": res["fused_worklist"] / res["per_patch"],
                   "best_fused_over_per_patch": best_fused / res["per_patch"]}

    # end to end through the public API from pinned host buffers
    e2e = None
    if rank == 0:
        snaps_host = torch.empty(adj.shape, dtype=torch.float64, pin_memory=True)
        snaps_host.numpy()[...] = adj.read()
        h2d = snaps_host.numel() * 8 + wl.m * wl.n0[0] * wl.n0[1] * 8
        d2h = 8
        ne = max(1, min(args.steps, 2))
        # one context for the run, as a user solving repeatedly keeps it:
        # each step starts a new solve in it (adjamr_reset)
        he = A.Hierarchy(wl, stream=sp)
        AT.apply_amr(he, tuned)
        torch.cuda.synchronize()
        t = time.perf_counter()
        cu_e = 0
        for _ in range(ne):
            he.reset()
            he.load_adjoint(snaps_host.numpy())
            solve(he)
            cu_e += he.stats()["cell_updates"]
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        he.close()
        e2e = {"value": cu_e / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "note": "per step, in one context (reset between solves): snapshot set + level-0 state "
                       "host->device, J device->host; regrid flag bitmaps also cross (internal)"}

    flaggers = None
    paper = None
    configs = None
    if rank == 0:
        flaggers = compare_flaggers(A, W, wl, adj, adj_s, s, tuned)
        paper = paper_table(A, W, s)
        configs = {}
        if not args.no_configs:
            w1 = W.config1()
            configs["config1"] = measure_config(
                A, W, w1, s, peak, args.cpu_budget / 3,
                label="acoustics1d config 1: 200 cells, ratio 4, t_f=20, adjoint 800 x 100 snapshots, tol 1e-3, "
                      "time range [0, t_f]")
            w3 = W.config3(seed=0)
            configs["config3"] = measure_config(
                A, W, w3, s, peak, args.cpu_budget / 3, adj_medium=W.config3_adjoint_medium(w3),
                label="shallow_water2d config 3: 2000 km square, coarse 200^2, ratios 4,4,2, t_f=4 h, adjoint "
                      "1000^2 x 300 snapshots, tol 4e-3, time range [t_f/2, t_f]")
            for k, v in configs.items():
                log(f"{k}: {v['value']:.3e} cell-updates/s, frac {v['roofline']['frac']}")
        # the adjoint solved with AMR (config 2's adjoint grid as level 0,
        # one ratio-2 level flagged by undivided differences) against the
        # fixed-grid adjoint
        configs["adjoint_amr"] = measure_adjoint_amr(A, W, wl, s, adj_s)

    serving = None
    if rank == 0 and args.serve_sample > 0:
        serving = serve_stream(A, W, args.serve_sample, [0.8], args.slots, nmin=64, nmax=256)
        serving["note"] = ("bounded sample of the serving configuration (n0 64..256); the full 512-request stream "
                           "is `bench.py --case serve`")

    if rank != 0:
        return
    # CPU baseline: the oracle as it stands, bounded sample
    cpu = None
    if not args.no_cpu:
        v, desc = oracle_sample(wl, adj.read(), budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle", "sample": desc}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "acoustics2d config 2: coarse 100^2, ratios 2,4, t_f=8, adjoint 400^2 x 200 "
                               "snapshots (device-resident, solved once), tol 1e-3, time range [0, t_f]",
                   "step": "one full adjoint-flagged forward AMR solve to t_f plus J",
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "step_kernel_per_level": tuned["best_per_level"]},
        "roofline": {"bound": "alu", "kernel": "k_step2d (fused wave-propagation step)",
                     "achieved": achieved, "peak": peak, "unit": "TOP/s (FP64 operations)",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_PER_CELL_L2 * cells_per_launch if TRAFFIC_IS_CURRENT else None,
                     "traffic_note": None if TRAFFIC_IS_CURRENT else
                     "the last ncu capture (profiles/k_step2d_amr_level2_config2.md) predates this build's k_step2d "
                     "(work-list entry now read before the wait for the kernel ahead); it measured "
                     f"{TRAFFIC_PER_CELL_L2:.1f} B read per cell-update, 1.2x the algorithmic bytes",
                     "peak_source": "FP64 instruction rate of the project DFMA micro-benchmark, measured live "
                                    "(its flop rate / 2)",
                     "ops_per_cell_update": OPS_PER_CELL_2D,
                     "cells_per_launch": cells_per_launch, "avg_launch_us": avg_launch_s * 1e6,
                     "per_level": [{"level": lev, **tuned["best_per_level"][lev],
                                    "launches_per_step": lev_launch[lev] / args.steps,
                                    "cells_per_launch": lev_cells[lev] / max(lev_launch[lev], 1),
                                    "avg_launch_us": lev_ms[lev] * 1e3 / max(lev_launch[lev], 1),
                                    "ghost_ms_per_step": lev_ghost[lev] / args.steps,
                                    "tops": (OPS_PER_CELL_2D * lev_cells[lev] / (lev_ms[lev] * 1e-3) / 1e12
                                               if lev_ms[lev] > 0 else None)}
                                   for lev in range(wl.nlevels)]},
        "fp64_peak": {"dfma_tflops": peak_fma / 1e12, "dadd_tflops": peak_add / 1e12},
        "batched": batched,
        "configs": configs,
        "flaggers": flaggers,
        "paper_sec_5_2": paper,
        "serving": serving,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": ck,
        "gpu_launches": int(launches),
        "breakdown_per_step_ms": {"step_kernels": step_ms / args.steps, "regrid_host_wall": regrid_ms / args.steps,
                                  "of_which_clustering": cluster_ms / args.steps,
                                  "level_rebuilds": rebuilds / args.steps,
                                  "levels_kept_unchanged": kept / args.steps,
                                  "regrid_phases": dict(zip(["flag_and_wait", "window_copy", "clustering",
                                                             "arena_alloc_upload", "builder_kernels", "release_old"],
                                                            [v / args.steps for v in phases])),
                                  "clustering_phases": dict(zip(["dilate_nest", "integral_images", "bisection",
                                                                 "split_sort"], [v / args.steps for v in cphases]))},
        "adjoint_solve_s": adj_s,
        "J": Js[0],
    }
    # the headline figures of every measured configuration in a few hundred
    # characters, last in the line so that a truncated record still holds them
    def rnd(x, n=4):
        return float(f"{x:.{n}g}") if isinstance(x, (int, float)) else x

    summ = {"config2_cell_updates_per_s": rnd(value), "config2_step_frac": rnd(achieved / peak, 3),
            "config2_e2e": rnd(e2e["value"]) if e2e else None}
    if batched:
        summ["config4_batched_cell_updates_per_s"] = rnd(max(
            batched[k] for k in ("fused_worklist", "fused_persistent", "fused_graph", "fused_tuned_graph")))
        summ["config4_batched_frac"] = rnd(batched.get("fp64_roofline_frac_best"), 3)
        summ["config4_fused_over_per_patch"] = rnd(batched.get("fused_over_per_patch"), 3)
    for k in ("config1", "config3"):
        if configs and k in configs:
            c = configs[k]
            summ[k] = {"value": rnd(c["value"]), "step_frac": rnd(c["roofline"]["frac"], 3),
                       "cpu_oracle": rnd(c["cpu_baseline"]["value"]) if "cpu_baseline" in c else None}
    if configs and "adjoint_amr" in configs:
        summ["adjoint_amr_cell_updates_per_s"] = rnd(configs["adjoint_amr"]["value"])
    if serving and serving.get("runs"):
        summ["serve_sample_p50_s"] = rnd(serving["runs"][0]["p50_latency_s"], 3)
        summ["serve_sample_p99_s"] = rnd(serving["runs"][0]["p99_latency_s"], 3)
    if paper:
        summ["sec_5_2_gauge_err_adjoint_vs_fine"] = [
            rnd(r["adjoint_flagging"]["gauge_max_abs_err_vs_uniform_fine"], 3) for r in paper.values()]
        summ["sec_5_2_gauge_err_pressure_vs_fine"] = [
            rnd(r["pressure_flagging"]["gauge_max_abs_err_vs_uniform_fine"], 3) for r in paper.values()]
        summ["sec_5_2_J_err_error_flagging_vs_fine"] = [
            rnd(r["error_flagging_reflux"]["J_rel_err_vs_uniform_fine"], 3) for r in paper.values()]
        summ["sec_5_2_J_err_richardson_vs_fine"] = [
            rnd(r["richardson_flagging_reflux"]["J_rel_err_vs_uniform_fine"], 3) for r in paper.values()]
    if flaggers and flaggers.get("error_estimate"):
        summ["config2_error_flagging"] = [[r["tol"], rnd(r["J_rel_err_vs_uniform_fine"], 3), rnd(r["ms_per_solve"], 4)]
                                          for r in flaggers["error_estimate"]]
    if flaggers and flaggers.get("richardson"):
        summ["config2_richardson"] = [[r["tol"], rnd(r["J_rel_err_vs_uniform_fine"], 3), rnd(r["ms_per_solve"], 4)]
                                      for r in flaggers["richardson"]]
    line["summary"] = summ
    log("autotune (ms of the timed coarse steps per candidate, by level): " + json.dumps(
        {f"level{r['level']}": {f"{c['tile'][0]}x{c['tile'][1]}{'' if c['fuse_ghosts'] else '+fill'}": round(c["ms"], 2)
                                for c in r["candidates"]} for r in tuned["candidates"]}))
    print(json.dumps(line), flush=True)


def serve_stream(A, W, nreq, rate_factors, slots, seed=0, nmin=64, nmax=512, budget=120 << 30, log_fn=log):
    """Serving (config 5): requests from a seeded Poisson process, each a 2D
    acoustics AMR solve flagged against the device-resident adjoint set of its
    medium; admission by a device-memory budget.  First the saturation
    throughput is measured with all requests submitted at once; then the
    stream is replayed at each rate factor times that throughput.  Returns a
    dict with p50/p99 latency (completion - arrival) per rate."""
    import torch
    media, reqs = W.config5(seed=seed, nreq=nreq, rate=1.0, nmin=nmin, nmax=nmax)
    wls = [W.request_workload(r, media) for r in reqs]
    for wl in wls:
        wl.ts = 0.0
        wl.tol = 1e-3
    t = time.perf_counter()
    adjs = {}
    for r, wl in zip(reqs, wls):
        if r.medium_id not in adjs:
            adjs[r.medium_id] = A.solve_adjoint(wl)
    torch.cuda.synchronize()
    adj_s = time.perf_counter() - t
    out = {"requests": nreq, "slots": slots, "budget_bytes": int(budget), "media": len(adjs),
           "adjoint_sets_s": adj_s, "n0_range": [nmin, nmax]}
    # saturation: everything at once
    srv = A.Server(budget, slots)
    t0 = srv.now()
    tks = [srv.submit(wl, adjs[r.medium_id]) for r, wl in zip(reqs, wls)]
    res = [srv.wait(tk) for tk in tks]
    t1 = max(x["t_finish"] for x in res)
    srv.close()
    assert all(x["status"] == 0 for x in res), [x["error"] for x in res if x["status"]]
    sat = nreq / (t1 - t0)
    cells = sum(x["cell_updates"] for x in res)
    out["saturation_req_per_s"] = sat
    out["saturation_cell_updates_per_s"] = cells / (t1 - t0)
    J_alone = {tk: x["J"] for tk, x in zip(range(nreq), res)}
    runs = []
    gaps = np.diff([r.arrival for r in reqs])
    for fac in rate_factors:
        rate = fac * sat
        arr = np.concatenate([[0.0], np.cumsum(gaps)]) / rate   # unit-rate stream scaled to this rate
        srv = A.Server(budget, slots)
        start = srv.now()
        tks = []
        for k, (r, wl) in enumerate(zip(reqs, wls)):
            while srv.now() - start < arr[k]:
                time.sleep(min(0.001, max(0.0, arr[k] - (srv.now() - start))))
            tks.append(srv.submit(wl, adjs[r.medium_id]))
        res = [srv.wait(tk) for tk in tks]
        srv.close()
        lat = np.array([x["t_finish"] - x["t_submit"] for x in res])
        span = max(x["t_finish"] for x in res) - start
        same = all(x["J"] == J_alone[k] for k, x in enumerate(res))
        runs.append({"rate_factor": fac, "offered_req_per_s": rate, "p50_latency_s": float(np.percentile(lat, 50)),
                     "p99_latency_s": float(np.percentile(lat, 99)), "achieved_req_per_s": nreq / span,
                     "cell_updates_per_s": sum(x["cell_updates"] for x in res) / span,
                     "results_equal_to_saturation_run": bool(same)})
        log_fn(f"serve rate x{fac}: p50 {runs[-1]['p50_latency_s']:.3f} s p99 {runs[-1]['p99_latency_s']:.3f} s")
    out["runs"] = runs
    return out


def run_case_serve(args):
    """Full serving configuration (512 requests, n0 64..512, 8 media)."""
    import torch
    from paper_1511_03645_gb300 import adjamr as A
    from paper_1511_03645_gb300 import workloads as W
    torch.cuda.set_device(0)
    A.load()
    res = serve_stream(A, W, args.nreq, [float(v) for v in args.rates.split(",")], args.slots)
    print(json.dumps({"case": "serve", **res}), flush=True)


def run_case_batch(args):
    """Profiling case: the 4096-patch batch (about 2.7 GB on the device, larger
    than L2), fused work-list steps only."""
    import torch
    from paper_1511_03645_gb300 import adjamr as A
    from paper_1511_03645_gb300 import workloads as W
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    b = A.Batch(W.config4(seed=0), stream=s.cuda_stream)
    b.step(args.warmup, mode=0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    b.step(args.steps, mode=0)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"case": "batch", "cells": b.cells(), "ms_per_step": ms,
                      "cell_updates_per_s": b.cells() / (ms * 1e-3)}), flush=True)
    b.close()


def compare_flaggers(A, W, wl, adj, adj_s, s, tuned=None, diff_tols=(0.1, 0.03, 0.01, 0.003),
                     err_tols=(1e-6, 1e-7, 1e-8), rich_tols=(1e-3, 1e-4, 1e-5)):
    """The paper's comparison (Sec. 5.2.4): the same forward solve refined by
    adjoint flagging and by the standard undivided-difference ("pressure")
    flagging over a range of tolerances (0.1 is the paper's), by the
    adjoint-weighted error estimate (Sec. 7) and by the estimate alone (the
    standard Richardson flagger, Sec. 1); GPU time per solve,
    cell-updates, and the error of J and of the gauge at the centre of the
    target region against the uniform run on the finest grid."""
    import copy
    import torch
    from paper_1511_03645_gb300 import autotune as AT
    gx = [0.5 * (wl.target.x0 + wl.target.x1)]
    gy = [0.5 * (wl.target.y0 + wl.target.y1)]

    def one(mode, tol):
        w = copy.copy(wl)
        w.flag_mode, w.tol = mode, tol
        h = A.Hierarchy(w, stream=s.cuda_stream)
        if tuned:
            AT.apply_amr(h, tuned)
        h.set_adjoint(adj)
        h.set_gauges(gx, gy)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        h.regrid(0, init=True)
        h.advance(h.nsteps_total())
        J = h.functional()
        e1.record(s)
        e1.synchronize()
        res = {"tol": tol, "ms_per_solve": e0.elapsed_time(e1), "cell_updates": h.stats()["cell_updates"], "J": J}
        g = h.gauges()[:, 0, 1]
        h.close()
        return res, g

    # reference: the uniform run on the finest grid (every cell refined)
    h0 = A.Hierarchy(wl, stream=s.cuda_stream)
    dt0, n0 = h0.time_info()
    h0.close()
    rf = int(np.prod(wl.ratios))
    fine = A.Hierarchy(wl, nlevels=1, n0=wl.level_shape(wl.nlevels - 1), dt0=dt0 / rf, stream=s.cuda_stream)
    fine.set_gauges(gx, gy)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fine.advance(n0 * rf)
    J_fine = fine.functional()
    e1.record(s)
    e1.synchronize()
    g_fine = fine.gauges()[rf - 1::rf, 0, 1]
    ref = {"ms_per_solve": e0.elapsed_time(e1), "cell_updates": fine.stats()["cell_updates"], "J": J_fine}
    fine.close()

    def accuracy(res, g):
        res["J_rel_err_vs_uniform_fine"] = abs(res["J"] - J_fine) / max(abs(J_fine), 1e-300)
        res["gauge_max_abs_err_vs_uniform_fine"] = float(np.max(np.abs(g - g_fine)))

    adj_runs = [one(wl.flag_mode, wl.tol) for _ in range(2)]
    ra, ga = min(adj_runs, key=lambda r: r[0]["ms_per_solve"])
    ra["adjoint_solve_ms"] = adj_s * 1e3
    accuracy(ra, ga)
    out = {"uniform_fine": ref, "adjoint": ra,
           "gauge": {"x": gx[0], "y": gy[0], "records": int(ga.size), "peak_abs_p_fine": float(np.max(np.abs(g_fine)))},
           "difference": []}
    for tol in diff_tols:
        rd, gd = one(W.FLAG_DIFFERENCE, tol)
        accuracy(rd, gd)
        rd["time_over_adjoint_forward"] = rd["ms_per_solve"] / ra["ms_per_solve"]
        out["difference"].append(rd)
    out["error_estimate"] = []
    for tol in err_tols:
        re_, ge = one(W.FLAG_ERROR, tol)
        accuracy(re_, ge)
        re_["time_over_adjoint_forward"] = re_["ms_per_solve"] / ra["ms_per_solve"]
        out["error_estimate"].append(re_)
    out["richardson"] = []
    for tol in rich_tols:
        rr, gr = one(W.FLAG_RICHARDSON, tol)
        accuracy(rr, gr)
        rr["time_over_adjoint_forward"] = rr["ms_per_solve"] / ra["ms_per_solve"]
        out["richardson"].append(rr)
    out["paper_context"] = ("Sec. 5.2.4 (laptop): pressure-flagging 3.1-15.7 s vs adjoint-flagging forward "
                            "1.3-6.9 s + adjoint 0.47-0.68 s")
    return out


PAPER_TABLE_5_2_4 = {  # Sec. 5.2.4 (a laptop): pressure-flagging; adjoint-flagging forward, adjoint solve (s)
    "timepoint_walls": (3.137, 1.325, 0.465),
    "range_walls": (15.664, 6.866, 0.683),
    "range_mixed": (13.504, 5.492, 0.666),
}


def paper_table(A, W, s, reps=3):
    """The Sec. 5.2 examples at the paper's sizes on this GPU: adjoint solve,
    adjoint-flagged forward solve (tol 0.02; also with the conservation
    fix-up), pressure-flagged forward solve (undivided differences, tol
    0.1), the forward solve flagged by the adjoint-weighted error estimate
    (Sec. 7; tol 1e-4, with the fix-up) and by the estimate alone (Sec. 1's
    Richardson flagging; tol 1e-3, with the fix-up), best of `reps` wall
    times each; J
    and the gauge at (3.5, 0.5) of every run against the uniform run on the
    finest grid (200^2 with the finest time step)."""
    import copy
    import torch
    out = {}
    for v in W.PAPER_5_2_VARIANTS:
        wl = W.paper_5_2(v)
        gx, gy = wl.extra["gauge"]
        best_adj = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            adj = A.solve_adjoint(wl, stream=s.cuda_stream)
            torch.cuda.synchronize()
            el = time.perf_counter() - t
            if best_adj is None or el < best_adj[0]:
                if best_adj is not None:
                    best_adj[1].release()
                best_adj = (el, adj)
            else:
                adj.release()
        res = {"adjoint_solve_s": best_adj[0]}
        # reference: every cell refined, i.e. the uniform finest grid
        h0 = A.Hierarchy(wl, stream=s.cuda_stream)
        dt0, n0 = h0.time_info()
        h0.close()
        rf = int(np.prod(wl.ratios))
        fine = A.Hierarchy(wl, nlevels=1, n0=wl.level_shape(wl.nlevels - 1), dt0=dt0 / rf, stream=s.cuda_stream)
        fine.set_gauges([gx], [gy])
        fine.advance(n0 * rf)
        J_fine = fine.functional()
        g_fine = fine.gauges()[rf - 1::rf, 0, 1]
        fine.close()
        res["uniform_fine"] = {"J": J_fine, "gauge_peak_abs": float(np.max(np.abs(g_fine)))}
        gauges = {}
        for name, mode, tol, reflux in (("adjoint_flagging", W.FLAG_BRACKET_MAX, wl.tol, 0),
                                        ("adjoint_flagging_reflux", W.FLAG_BRACKET_MAX, wl.tol, 1),
                                        ("pressure_flagging", W.FLAG_DIFFERENCE, 0.1, 0),
                                        ("error_flagging_reflux", W.FLAG_ERROR, 1e-4, 1),
                                        ("richardson_flagging_reflux", W.FLAG_RICHARDSON, 1e-3, 1)):
            w = copy.copy(wl)
            w.flag_mode, w.tol, w.reflux = mode, tol, reflux
            best = None
            for _ in range(reps):
                h = A.Hierarchy(w, stream=s.cuda_stream)
                h.set_adjoint(best_adj[1])
                h.set_gauges([gx], [gy])
                torch.cuda.synchronize()
                t = time.perf_counter()
                h.regrid(0, init=True)
                h.advance(h.nsteps_total())
                J = h.functional()
                torch.cuda.synchronize()
                el = time.perf_counter() - t
                if best is None or el < best[0]:
                    best = (el, h.stats()["cell_updates"], J, h.gauges()[:, 0, 1])
                h.close()
            g = best[3]
            res[name] = {"tol": tol, "forward_s": best[0], "cell_updates": best[1], "J": best[2],
                         "J_rel_err_vs_uniform_fine": abs(best[2] - J_fine) / max(abs(J_fine), 1e-300),
                         "gauge_max_abs_err_vs_uniform_fine": float(np.max(np.abs(g - g_fine))),
                         "gauge_peak_abs": float(np.max(np.abs(g)))}
            gauges[name] = g
        res["gauge_max_abs_diff_adjoint_vs_pressure"] = float(
            np.max(np.abs(gauges["adjoint_flagging"] - gauges["pressure_flagging"])))
        pp, pf, pa = PAPER_TABLE_5_2_4[v]
        res["paper_laptop_s"] = {"pressure_flagging": pp, "adjoint_flagging_forward": pf, "adjoint_solve": pa}
        best_adj[1].release()
        out[v] = res
    return out


def run_case_paper(args):
    """The paper's Sec. 5.2.4 timing table, reproduced on this GPU."""
    import torch
    from paper_1511_03645_gb300 import adjamr as A
    from paper_1511_03645_gb300 import workloads as W
    torch.cuda.set_device(0)
    A.load()
    s = torch.cuda.Stream()
    print(json.dumps({"case": "paper", "sec_5_2": paper_table(A, W, s)}), flush=True)


def run_case_solve(args):
    """Profiling case: one config-2 forward solve to --tf (adjoint solved
    first) with the step-kernel tile and ghost mode of every level given by
    --kernels (default: the configuration the autotuner picks on a GB300,
    12x8 fused, 8x8 fused, 16x12 with a separate ghost fill); prints
    per-level step statistics.  --flag error --tol T: flagged by the
    adjoint-weighted error estimate (Sec. 7) instead; --config 1 or 3: that
    workload instead of config 2 (config 1 with its default kernels)."""
    import torch
    from paper_1511_03645_gb300 import adjamr as A
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    from paper_1511_03645_gb300 import workloads as W
    wl = {"2": workload, "1": W.config1, "3": lambda: W.config3(seed=0)}[args.config]()
    if args.tf:
        wl.tf = args.tf
    if args.flag != "adjoint":
        from paper_1511_03645_gb300 import workloads as W
        wl.flag_mode = W.FLAG_ERROR if args.flag == "error" else W.FLAG_RICHARDSON
    if args.tol > 0:
        wl.tol = args.tol
    adj = A.solve_adjoint(wl, stream=s.cuda_stream,
                          medium_dense=W.config3_adjoint_medium(wl) if args.config == "3" else None)
    for rep in range(1 + args.warmup):
        h = A.Hierarchy(wl, stream=s.cuda_stream)
        for lev, spec in enumerate(args.kernels.split(",")[:wl.nlevels] if args.config != "1" else []):
            # suffix f: ghost ring in the step kernel; s: substep launches (finest level)
            fused, sub = spec.endswith("f"), spec.endswith("s")
            tx, ty = (int(v) for v in spec.rstrip("fs").split("x"))
            h.set_level_kernel(lev, (tx, ty), fused or sub, A.LAUNCH_SUBSTEPS if sub else A.LAUNCH_WORKLIST)
        h.set_adjoint(adj)
        h.set_timing(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.regrid(0, init=True)
        h.advance(h.nsteps_total())
        J = h.functional()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        st = h.stats()
        h.close()
    print(json.dumps({"case": "solve", "tf": wl.tf, "s": el, "J": J, "cell_updates": st["cell_updates"],
                      "kernel_launches": st["kernel_launches"], "step_kernel_ms": st["step_kernel_ms"],
                      "level_step_ms": st["level_step_ms"][:wl.nlevels],
                      "level_step_launches": st["level_step_launches"][:wl.nlevels],
                      "level_cell_updates": st["level_cell_updates"][:wl.nlevels],
                      "regrid_phase_ms": st["regrid_phase_ms"], "regrids": st["regrids"],
                      "level_rebuilds": st["level_rebuilds"],
                      "levels_kept_unchanged": st["level_rebuilds_skipped"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--case", default="main", choices=["main", "batch", "serve", "solve", "paper"])
    ap.add_argument("--tf", type=float, default=0.0, help="solve case: final time (0: the workload's)")
    ap.add_argument("--flag", default="adjoint", choices=["adjoint", "error", "richardson"],
                    help="solve case: adjoint flagging (bracket rule), the adjoint-weighted error estimate, or "
                         "the estimate alone (Richardson)")
    ap.add_argument("--tol", type=float, default=0.0, help="solve case: flag tolerance (0: the workload's)")
    ap.add_argument("--config", default="2", choices=["1", "2", "3"],
                    help="solve case: the workload (config 1 runs with the default 1D kernels)")
    ap.add_argument("--kernels", default="12x8f,8x8f,16x12",
                    help="solve case: per-level step tile, suffix f = ghost ring computed in the step kernel")
    ap.add_argument("--nreq", type=int, default=512)
    ap.add_argument("--rates", default="0.5,0.8,1.0", help="serve case: offered rates as fractions of saturation")
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--serve-sample", type=int, default=32)
    ap.add_argument("--no-configs", action="store_true", help="skip the config-1 and config-3 solves")
    args = ap.parse_args()
    if args.case == "batch":
        run_case_batch(args)
        return
    if args.case == "serve":
        run_case_serve(args)
        return
    if args.case == "solve":
        run_case_solve(args)
        return
    if args.case == "paper":
        run_case_paper(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
