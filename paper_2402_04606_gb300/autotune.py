"""Per-workload choice of the block size (8, 16 or 32 cells per side), of
the fused kernel variant (one cell per thread, or 4 cells per thread, 8 in
16-bit storage, with vector loads above a launch size, optionally with the
blocks staged in shared memory by bulk copies), of programmatic dependent
launch, of the IBM's threads per body, and of the persistent step kernel
(with its thread-block size and task sizes) against the per-phase
graphs, by timing coarse steps on the device.

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


KNOBS = ("staged", "pdl", "ibm_threads", "persistent", "step_threads", "bulk_rounds", "crit_blocks",
         "steps_per_launch", "vec_waves")
DEFAULTS = {"staged": 0, "pdl": 0, "ibm_threads": 1024, "persistent": 0, "step_threads": 0, "bulk_rounds": 8,
            "crit_blocks": 0, "steps_per_launch": 8, "vec_waves": 8}


def knob_ids() -> dict:
    """The library's tuning parameter of each knob name (and of the
    vector-kernel threshold, ``vec_min_cells``)."""
    from . import native as nv

    return {"vec_min_cells": nv.TUNE_VECTOR_MIN_CELLS, "staged": nv.TUNE_STAGED, "pdl": nv.TUNE_PDL,
            "ibm_threads": nv.TUNE_IBM_THREADS, "persistent": nv.TUNE_PERSISTENT,
            "step_threads": nv.TUNE_STEP_THREADS, "bulk_rounds": nv.TUNE_BULK_ROUNDS,
            "crit_blocks": nv.TUNE_CRIT_BLOCKS, "steps_per_launch": nv.TUNE_STEPS_PER_LAUNCH,
            "vec_waves": nv.TUNE_VEC_WAVES}


def time_config(specs, block: int, vec_min_cells: int, storage: int, steps: int = 20, warmup: int = 5,
                stream=None, repeats: int = 3, **knobs) -> float:
    """Milliseconds per coarse step of all ``specs`` advanced together (the
    best of ``repeats`` runs of ``steps`` steps, rounded up to whole launches
    of the persistent kernel); ``knobs`` sets the other tuning parameters by
    name (``KNOBS``)."""
    import torch

    from . import native as nv

    ids = knob_ids()
    stream = stream if stream is not None else torch.cuda.Stream()
    b = nv.Batch(len(specs), block=block, storage=storage, stream=stream)
    try:
        for s in specs:
            b.admit(wl.replace_storage(with_block(s, block), storage))
        b.set_tuning(nv.TUNE_VECTOR_MIN_CELLS, vec_min_cells)
        for k, v in {**DEFAULTS, **knobs}.items():
            b.set_tuning(ids[k], v)
        per = max(1, knobs.get("steps_per_launch", DEFAULTS["steps_per_launch"]))
        if knobs.get("persistent", 0):
            steps = -(-steps // per) * per
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
    """Search, each stage on the best configuration so far: every feasible
    block size (default kernel threshold), every vector-kernel threshold
    (cells per thread: one below it, 4 in 32-bit and 8 in 16-bit storage
    above it), the shared-memory staged variant, programmatic dependent
    launch, the IBM's threads per body (256, 512, 1024), the vector kernel's
    thread blocks (one per list group, or 2 waves of grid-stride blocks,
    against the default 8 waves), then the persistent
    step kernel at three vector-kernel thresholds of its own (the default,
    the graphs' best, never) and, at the best of those, its thread-block size
    768, a bulk task size of 1 or 16 block groups, 1 or 2 blocks per task of
    the sweeps other phases wait for, and 16 coarse steps per launch.  Returns the best configuration and
    every trial (milliseconds per coarse step).  ``timer`` defaults to
    ``time_config`` (device timing); the host-side tests pass a cost model
    with the same arguments."""
    specs = list(specs) if isinstance(specs, (list, tuple)) else [specs]
    storage = specs[0].storage if storage is None else storage
    cands = block_candidates(specs, blocks)
    if not cands:
        raise ValueError("no block size divides every grid")
    timer = timer or time_config
    default = 1 << 19
    trials = []
    t0 = time.perf_counter()

    def trial(block, vec, **knobs):
        cfg = {"block": block, "vec_min_cells": vec, **DEFAULTS, **knobs}
        ms = timer(specs, block, vec, storage, steps, warmup, stream, **{k: cfg[k] for k in KNOBS})
        trials.append({**cfg, "ms_per_step": ms})

    def best():
        return min(trials, key=lambda t: t["ms_per_step"])

    def knobs_of(t):
        return {k: t[k] for k in KNOBS}

    for b in cands:
        trial(b, default)
    if best()["block"] in (16, 32):
        for v in thresholds:
            if v != default:
                trial(best()["block"], v)
        if best()["vec_min_cells"] >= 0:  # the shared-memory staged variant of the vector kernel
            trial(best()["block"], best()["vec_min_cells"], staged=1)
    b0 = best()
    trial(b0["block"], b0["vec_min_cells"], **{**knobs_of(b0), "pdl": 1})
    for threads in (256, 512):
        b0 = best()
        trial(b0["block"], b0["vec_min_cells"], **{**knobs_of(b0), "ibm_threads": threads})
    b0 = best()
    if b0["block"] in (16, 32) and b0["vec_min_cells"] >= 0 and not b0["staged"]:
        for w in (0, 2):  # short-lived vector blocks (0: one per list group), or fewer waves
            trial(b0["block"], b0["vec_min_cells"], **{**knobs_of(b0), "vec_waves": w})
    # the persistent kernel maps cells to threads its own way, so its threshold is searched apart
    b0 = best()
    pv = sorted({default, b0["vec_min_cells"], -1}) if b0["block"] in (16, 32) else [b0["vec_min_cells"]]
    for v in pv:
        trial(b0["block"], v, **{**knobs_of(b0), "staged": 0, "persistent": 1})
    bp = min((t for t in trials if t["persistent"]), key=lambda t: t["ms_per_step"])
    for st, br in ((768, 8), (0, 1), (0, 16)):
        trial(bp["block"], bp["vec_min_cells"], **{**knobs_of(bp), "step_threads": st, "bulk_rounds": br})
    for cb in (1, 2):
        bp = min((t for t in trials if t["persistent"]), key=lambda t: t["ms_per_step"])
        trial(bp["block"], bp["vec_min_cells"], **{**knobs_of(bp), "crit_blocks": cb})
    bp = min((t for t in trials if t["persistent"]), key=lambda t: t["ms_per_step"])
    trial(bp["block"], bp["vec_min_cells"], **{**knobs_of(bp), "steps_per_launch": 16})
    return {"best": best(), "trials": trials, "seconds": time.perf_counter() - t0}


def best_of_form(result: dict, persistent: int) -> dict:
    """the fastest trial of one step form (0 per-phase graphs, 1 persistent kernel)"""
    return min((t for t in result["trials"] if t["persistent"] == persistent), key=lambda t: t["ms_per_step"])
