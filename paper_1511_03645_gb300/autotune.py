"""Autotuner for the fused step kernel: tile shape x work-list order x launch
mode, measured with CUDA events on the GPU in use and cached per (GPU,
workload key) in ``_build/autotune.json``.

Every tile shape, order and launch mode computes the same bits (the work of
a tile does not depend on the schedule), so tuning changes speed only.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

import numpy as np

from . import adjamr as A

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_build", "autotune.json")
# tile sizes the patches are cut to (the kernel compiled for the smallest of
# 8x8, 16x8, 16x12, 32x8, 16x16, 64x8, 32x16 holding them runs them): the compiled
# shapes and cuts between them, which move a level's tile count towards whole
# waves of resident CTAs
TILES = [(32, 8), (16, 8), (16, 16), (32, 16), (64, 8), (8, 8), (12, 8), (16, 12), (24, 8), (24, 16), (48, 8),
         (12, 12)]
_lock = threading.Lock()


def _gpu_key():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}"


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    with _lock:
        d = _load()
        d[key] = value
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)


def _time(stream, fn, reps=1):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def batch_orders(pb):
    """Candidate work-list orders for a batch of patches."""
    n = pb.npatch
    cells = pb.nx.astype(np.int64) * pb.ny
    return {
        "natural": np.arange(n, dtype=np.int32),
        "shuffled": np.asarray(pb.order, dtype=np.int32),
        "largest_first": np.argsort(-cells, kind="stable").astype(np.int32),
    }


def tune_batch(pb, key: str, stream=None, steps: int = 4, use_cache: bool = True) -> dict:
    """Best (work-list order, tile size, launch mode) for a batch, ghost ring
    from its own kernel (the measured faster way for this batch; the fused
    ring, the shuffled order and the dynamic tile counter never won); returns
    a dict with the choice and the measured cell-updates/s of every
    candidate."""
    import torch
    ck = f"{_gpu_key()}|batch|{key}"
    if use_cache:
        hit = _load().get(ck)
        if hit:
            return hit
    s = torch.cuda.Stream() if stream is None else stream
    b = A.Batch(pb, stream=s.cuda_stream)
    cells = b.cells()
    results = []
    for oname, order in batch_orders(pb).items():
        if oname == "shuffled":
            continue
        b.set_order(order)
        for tile in TILES:
            for mode in (A.LAUNCH_WORKLIST, A.LAUNCH_PERSISTENT):
                for fuse in (False,):
                    b.set_ghost_fusion(fuse)
                    b.step(1, mode=mode, tile=tile)
                    ms = _time(s, lambda: b.step(steps, mode=mode, tile=tile)) / steps
                    results.append({"order": oname, "tile": list(tile), "mode": mode, "fuse_ghosts": fuse,
                                    "ms": ms, "cell_updates_per_s": cells / (ms * 1e-3)})
    b.close()
    best = max(results, key=lambda r: r["cell_updates_per_s"])
    out = {"best": best, "candidates": results}
    _store(ck, out)
    return out


def tune_amr(wl, adj, key: str, stream=None, coarse_steps: int = 60, skip_steps: int = 40,
             use_cache: bool = True) -> dict:
    """Best step-kernel configuration (tile size, ghost ring fused into the
    step or filled by its own kernel; one work-list launch per level: the
    dynamic tile counter never won, and substep launches save less kernel
    time than their host-side dependency lists cost) of every level of an
    AMR solve.

    Each candidate runs part of the solve (after `skip_steps` coarse steps,
    so that the finest levels have grown) with the candidate on one level and
    the best configuration found so far on the others, finest level first;
    the whole run is timed with one pair of CUDA events and no events between
    launches, which would stop a launch from starting early behind the one
    before it (the separate ghost fill overlaps the previous step's tail that
    way).  The hierarchy evolves bit-identically under every candidate, so the
    times compare directly."""
    import torch
    ck = f"{_gpu_key()}|amr|{key}"
    if use_cache:
        hit = _load().get(ck)
        if hit:
            return hit
    s = torch.cuda.Stream() if stream is None else stream
    cands = list(itertools.product(TILES, (True, False)))
    best = [((16, 12), False) for _ in range(wl.nlevels)]

    def run(cfg):
        h = A.Hierarchy(wl, stream=s.cuda_stream)
        for lev, (tile, fuse) in enumerate(cfg):
            h.set_level_kernel(lev, tile, fuse, A.LAUNCH_WORKLIST)
        h.set_adjoint(adj)
        h.regrid(0, init=True)
        h.advance(skip_steps)
        torch.cuda.synchronize()
        ms = _time(s, lambda: h.advance(coarse_steps))
        h.close()
        return ms

    results = []
    for lev in reversed(range(wl.nlevels)):
        per = []
        for tile, fuse in cands:
            cfg = list(best)
            cfg[lev] = (tile, fuse)
            ms = run(cfg)
            per.append({"tile": list(tile), "fuse_ghosts": fuse, "ms": ms})
        b = min(per, key=lambda r: r["ms"])
        best[lev] = (tuple(b["tile"]), b["fuse_ghosts"])
        results.append({"level": lev, "candidates": per})
    out = {"best_per_level": [{"tile": list(t), "fuse_ghosts": f, "mode": A.LAUNCH_WORKLIST} for t, f in best],
           "candidates": results, "coarse_steps": coarse_steps, "skip_steps": skip_steps}
    _store(ck, out)
    return out


def apply_amr(h, tuned: dict) -> None:
    """Set the tuned per-level step-kernel configuration on a hierarchy."""
    for lev, b in enumerate(tuned["best_per_level"]):
        h.set_level_kernel(lev, b["tile"], b["fuse_ghosts"], b.get("mode", -1))
