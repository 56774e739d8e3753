"""Per-workload choice of the block size (8, 16 or 32 cells per side) and of
the fused kernel variant (one cell per thread, or 4 cells per thread, 8 in
16-bit storage, with vector loads above a launch size, optionally with the
blocks staged in shared memory by bulk copies) and of programmatic dependent
launch, by timing coarse steps on the device.

The block size trades halo and mailbox waste (large blocks refine more cells
than the body boxes ask for) against per-block overhead (small blocks mean
more blocks, more neighbour lookups and no vector path); the best choice
depends on the grid, the refinement and the storage, so it is measured
rather than modelled.  Only sizes that divide every instance's coarsest grid
and that the planner accepts are tried.
"""
from __future__ import annotations

import time
from dataclasses import replace

from . import workloads as wl

BLOCKS = (8, 16, 32)
VEC_THRESHOLDS = (-1, 0, 1 << 14, 1 << 16, 1 << 19, 1 << 22)  # -1: never the vector kernel, 0: always


def with_block(spec: wl.DomainSpec, block: int) -> wl.DomainSpec:
    """``spec`` with another block size (the grid itself unchanged)."""
    return replace(spec, block=block, boxes=list(spec.boxes),
                   body=replace(spec.body) if spec.body is not None else None)


def block_candidates(specs, blocks=BLOCKS) -> list:
    """Block sizes that divide every instance's coarsest grid and that the
    planner accepts for every instance (host only, no GPU)."""
    from .native import SbotError, plan_blocks

    out = []
    for b in blocks:
        ok = True
        for s in specs:
            if s.nx0 % b or s.ny0 % b:
                ok = False
                break
            try:
                plan_blocks(with_block(s, b), 0)
            except SbotError:
                ok = False
                break
        if ok:
            out.append(b)
    return out


def time_config(specs, block: int, vec_min_cells: int, storage: int, steps: int = 20, warmup: int = 5,
                stream=None, repeats: int = 3, staged: int = 0, pdl: int = 0) -> float:
    """Milliseconds per coarse step of all ``specs`` advanced together (the
    best of ``repeats`` runs of ``steps`` steps)."""
    import torch

    from .native import TUNE_PDL, TUNE_STAGED, TUNE_VECTOR_MIN_CELLS, Batch

    stream = stream if stream is not None else torch.cuda.Stream()
    b = Batch(len(specs), block=block, storage=storage, stream=stream)
    try:
        for s in specs:
            b.admit(wl.replace_storage(with_block(s, block), storage))
        b.set_tuning(TUNE_VECTOR_MIN_CELLS, vec_min_cells)
        b.set_tuning(TUNE_STAGED, staged)
        b.set_tuning(TUNE_PDL, pdl)
        b.step(warmup)
        best = float("inf")
        for _ in range(repeats):  # the best of a few short runs: trials are brief and the GPU is shared
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                e0.record(stream)
                b.step(steps)
                e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / steps)
        return best
    finally:
        b.close()


def tune(specs, storage: int | None = None, steps: int = 20, warmup: int = 5, blocks=BLOCKS,
         thresholds=VEC_THRESHOLDS, stream=None, timer=None) -> dict:
    """Try every feasible block size at the default kernel threshold, then
    every threshold at the best size, then the staged variant and
    programmatic dependent launch on the best so far.  Returns the best
    configuration and all trials (milliseconds per coarse step).  ``timer``
    defaults to ``time_config`` (device timing); the host-side tests pass a
    cost model with the same arguments."""
    specs = list(specs) if isinstance(specs, (list, tuple)) else [specs]
    storage = specs[0].storage if storage is None else storage
    cands = block_candidates(specs, blocks)
    if not cands:
        raise ValueError("no block size divides every grid")
    timer = timer or time_config
    default = 1 << 19
    trials = []
    t0 = time.perf_counter()
    for b in cands:
        trials.append({"block": b, "vec_min_cells": default,
                       "ms_per_step": timer(specs, b, default, storage, steps, warmup, stream)})
    best = min(trials, key=lambda t: t["ms_per_step"])
    if best["block"] in (16, 32):
        for v in thresholds:
            if v == default:
                continue
            trials.append({"block": best["block"], "vec_min_cells": v,
                           "ms_per_step": timer(specs, best["block"], v, storage, steps, warmup, stream)})
        best = min(trials, key=lambda t: t["ms_per_step"])
        if best["vec_min_cells"] >= 0:  # the shared-memory staged variant of the vector kernel
            trials.append({"block": best["block"], "vec_min_cells": best["vec_min_cells"], "staged": 1,
                           "ms_per_step": timer(specs, best["block"], best["vec_min_cells"], storage, steps,
                                                      warmup, stream, staged=1)})
            best = min(trials, key=lambda t: t["ms_per_step"])
    # programmatic dependent launch on the best configuration
    trials.append({"block": best["block"], "vec_min_cells": best["vec_min_cells"], "staged": best.get("staged", 0),
                   "pdl": 1, "ms_per_step": timer(specs, best["block"], best["vec_min_cells"], storage, steps,
                                                        warmup, stream, staged=best.get("staged", 0), pdl=1)})
    best = min(trials, key=lambda t: t["ms_per_step"])
    for t in trials:
        t.setdefault("staged", 0)
        t.setdefault("pdl", 0)
    return {"best": best, "trials": trials, "seconds": time.perf_counter() - t0}
