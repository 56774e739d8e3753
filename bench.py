#!/usr/bin/env python
"""Benchmark of the hot path: one step = one coarse time step (Algorithm 1:
every level's fused stream-collide sweeps, the coarse/fine transfers, the
multi-direct-forcing IBM before every finest collision and the force/moment
reduction) of the refined circular-cylinder workload: Re = 100, D = 40
finest cells, 3 levels (factor 2), coarsest grid 30D x 15D (rounded up to
whole blocks), uniform inflow u = 0.05, 126 markers, K = 5, FP32 storage.

Prints one JSON line.  --impl reference times the CPU oracle (plain FP64 C,
OpenMP) on the same workload instead.

Timing: W untimed warm-up steps; then K steps in calls of the library's
step function, each call bracketed by CUDA events on the library's stream,
with a 512 MiB write between calls to flush the 129 MB L2 (the flush is
outside the events).  A call advances as many coarse steps as one launch of
the persistent step kernel runs (SBOT_TUNE_STEPS_PER_LAUNCH; one step per
call for the per-phase graphs), so the roofline's kernel time is the call's
time.  value = actual cell updates / summed device time.  The same steps in
the other form are reported beside it (other_form).  With extras: the other body cases, the 64-instance batch,
the served request mix (config 5) and, last on the line, the HBM-scale sweep.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("cylinder Re=100, D=40 finest cells, 3 levels, coarsest 30Dx15D rounded to 304x160 cells, "
            "u_in=0.05, 126 markers, K=5, FP32 storage")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "f16dev", "bf16dev"])
    ap.add_argument("--workload", default="cylinder", choices=["cylinder", "sweep", "batch"],
                    help="cylinder: the benchmark workload; sweep: a single-level periodic "
                         "Taylor-Green grid of side --n (fused stream-collide alone); batch: the "
                         "64-instance BF16 batch alone")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner's short trials for the main workload (step form, vector-kernel "
                         "threshold, IBM threads; the block size stays the workload's 16)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (64 uneven instances, BF16) and served (Poisson arrivals) measurements")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--body-steps", type=int, default=40, help="coarse steps timed per body case")
    ap.add_argument("--batch-block", type=int, default=0, help="skip the batch autotuner: use this block size")
    ap.add_argument("--batch-vec", type=int, default=1 << 16, help="with --batch-block: the vector-kernel threshold")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-periods", type=float, default=10.0)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--block", type=int, default=16)
    ap.add_argument("--coll", default="bgk", choices=["bgk", "mrt", "les"],
                    help="collision of the sweep workload (BGK, the MRT or the LES option of Sec. 2.1)")
    return ap.parse_args()


def workload_spec(storage: str, workload: str = "cylinder", n: int = 8192, block: int = 16, coll: str = "bgk"):
    from paper_2402_04606_gb300 import workloads as wl

    st = {"f64": wl.F64, "f32": wl.F32, "f16dev": wl.F16DEV, "bf16dev": wl.BF16DEV}[storage]
    if workload == "sweep":
        spec = wl.tgv(n=n, tau=0.8, u0=0.02, storage=st, block=block)
        return wl.with_mrt(spec) if coll == "mrt" else (wl.with_les(spec) if coll == "les" else spec)
    return wl.cylinder(D=40, levels=3, re=100.0, u=0.05, n_markers=126, K=5, storage=st, block=16)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "k_step_cylinder_D40_m3_f32.md")


def sources_sha256():
    """hash of the library's device and host sources (csrc/*), in name order"""
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2402_04606_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def profiled_traffic(spec):
    """DRAM bytes per coarse step of the step kernel on this workload from
    the committed ncu summary (launches of several steps), or None when the
    sources have changed since it was taken."""
    try:
        text = open(PROFILE_TRAFFIC).read()
    except OSError:
        return None
    import re

    m = re.search(r"traffic_bytes_per_step = ([0-9.eE+]+) \(sources sha256 ([0-9a-f]+)\)", text)
    if not m or m.group(2) != sources_sha256() or spec.block != 16:
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_run(spec, seconds: float, max_steps: int | None = None, warmup: int = 0):
    """Time the FP64 oracle (OpenMP build) on the workload: whole coarse steps
    until `seconds` have elapsed (or max_steps).  Returns (MLUPS, steps, s, cores)."""
    import oracle  # the CPU baseline leg is the one place bench.py runs the oracle

    from tests.helpers import init_oracle, oracle_from_spec

    o = init_oracle(oracle_from_spec(spec, openmp=True), spec)
    cells = 0
    for l in range(spec.levels):
        cells += int((o.types(l) == oracle.T_INT).sum()) << l
    for _ in range(warmup):
        o.step(1)
    steps = 0
    t0 = time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and steps >= max_steps) or (max_steps is None and el >= seconds):
            break
    cores = len(os.sched_getaffinity(0))
    return cells * steps / el / 1e6, steps, el, cores, cells


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    spec = workload_spec("f32", args.workload, args.n, args.block, args.coll)
    mlups, steps, el, cores, cells = cpu_oracle_run(spec, 0.0, max_steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cell_updates_per_step": cells, "l2": "cpu run"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{steps} coarse steps of the workload after {args.warmup} warm-up steps"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args):
    import numpy as np
    import torch

    from paper_2402_04606_gb300 import build as bld
    from paper_2402_04606_gb300.native import TUNE_PERSISTENT, TUNE_VECTOR_MIN_CELLS, Domain
    from paper_2402_04606_gb300.replicas import job_rate, max_over_ranks
    from paper_2402_04606_gb300.workloads import initial_fields

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    bld.build()
    spec = workload_spec(args.storage, args.workload, args.n, args.block, args.coll)
    stream = torch.cuda.Stream()
    from paper_2402_04606_gb300 import autotune as at
    from paper_2402_04606_gb300 import native as nv

    forms = {1: {"vec_min_cells": 1 << 19, **at.DEFAULTS, "persistent": 1},
             0: {"vec_min_cells": 1 << 19, **at.DEFAULTS, "persistent": 0, "pdl": 1}}
    if not args.no_tune:
        # kernel threshold, IBM threads, dependent launch, each step form's own best: short
        # timed trials of this workload with its own block size
        tuned = at.tune([spec], blocks=(spec.block,), steps=20, warmup=5, stream=stream)
        forms = {p: {k: at.best_of_form(tuned, p)[k] for k in ("vec_min_cells", *at.KNOBS)} for p in (0, 1)}
    knobs = forms[1]
    ids = at.knob_ids()

    def domain(persistent=None):
        g = Domain(spec, stream=stream)
        for k, v in (knobs if persistent is None else forms[persistent]).items():
            g.set_tuning(ids[k], v)
        return g

    fields = [initial_fields(spec, l) for l in range(spec.levels)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def per_call(g):
        """coarse steps per timed call: one launch of the persistent kernel, one step of the graphs"""
        return g.tuning(nv.TUNE_STEPS_PER_LAUNCH) if g.tuning(nv.TUNE_PERSISTENT) else 1

    def calls_of(g, steps):
        """`steps` coarse steps as timed calls: per_call(g) steps each, the rest in a last call"""
        per = per_call(g)
        return [per] * (steps // per) + ([steps % per] if steps % per else [])

    def timed_pass(g, steps):
        """device ms summed over exactly `steps` coarse steps in the calls of
        calls_of, each bracketed by events on the library's stream, with the
        L2 flushed between calls"""
        calls = calls_of(g, steps)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k, n in enumerate(calls):
                flush.fill_(k & 255)  # evict the state from L2 between timed calls
                ev[k][0].record(stream)
                g.step(n)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev), time.perf_counter() - t0

    # each form with its own knobs, timed the way the timed region is (L2 flushed between steps):
    # the faster one is the headline, the other is reported beside it
    quick = {}
    for p in (1, 0):
        gq = domain(p)
        for l in range(spec.levels):
            gq.set_fields(l, *fields[l])
        gq.step(args.warmup)
        quick[p] = timed_pass(gq, min(args.steps, 100))[0]
        gq.close()
    form = 1 if quick[1] <= quick[0] else 0
    knobs = forms[form]
    g = domain()
    for l in range(spec.levels):
        g.set_fields(l, *fields[l])
    cells, fine_eq = g.work()
    g.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    g.set_profiling(0)  # zero the library's launch count
    per_call_used = per_call(g)
    with ClockSampler(local) as clk:
        dev_ms, wall = timed_pass(g, args.steps)
    launches = g.profile(4)[0]  # every kernel the library launched inside the timed region
    if world > 1:
        torch.distributed.barrier()
    dev_ms = max_over_ranks(dev_ms)  # the slowest replica times the job
    clocks = clk.summary()
    if form:
        # one traced step: when each phase of the persistent kernel ran
        g.set_profiling(16)
        g.step(1)
        trace = g.step_trace()
        g.set_profiling(0)
        prof = None
    else:
        # the same number of steps again with every kernel's events, captured on one
        # stream so that the kernels' times do not overlap
        trace = []
        g.set_profiling(15)
        prof_ms, _ = timed_pass(g, args.steps)
        prof = {k: g.profile(k) for k in range(4)}
        g.set_profiling(0)
    cs = g.checksum()  # must stay finite (guards against a silently diverged run)
    ok = bool(np.isfinite(cs).all())
    g.close()
    value = job_rate(cells * args.steps, dev_ms * 1e-3, world) / 1e6

    # the same steps in the other form (persistent kernel or per-phase graphs)
    g = domain(1 - form)
    for l in range(spec.levels):
        g.set_fields(l, *fields[l])
    g.step(args.warmup)
    g.set_profiling(0)
    other_ms, _ = timed_pass(g, min(args.steps, 200))
    other_launches = g.profile(4)[0]
    g.close()
    other = {"form": "graphs" if form else "persistent", "ms_per_step": other_ms / min(args.steps, 200),
             "kernels_per_step": other_launches / min(args.steps, 200)}

    # end to end through the public API with host buffers: the initial state
    # uploaded once from pinned host memory, then the steps advanced in the
    # timed region's calls, each call's force history read back to the host
    g2 = domain()
    pinned = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in f] for f in fields]
    h2d = sum(a.nbytes for f in pinned for a in f)
    torch.cuda.synchronize()
    nf = 1 << (spec.levels - 1)
    t0 = time.perf_counter()
    for l in range(spec.levels):
        g2.set_fields(l, *pinned[l])
    for n in calls_of(g2, args.steps):
        g2.step(n)
        g2.forces(cap=nf * n)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    g2.close()
    e2e = {"value": job_rate(cells * args.steps, e2e_s, world) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": nf * 3 * 8,
           "h2d_initial_bytes": h2d,
           "note": "the initial fields (h2d_initial_bytes) are uploaded once at the start of the timed region; "
                   "h2d_bytes_per_step is that upload over the steps; every call reads the force history of its "
                   "steps back"}

    peak, peak_kind = measured_peaks()
    sb = {"f64": 8, "f32": 4}.get(args.storage, 2)
    if form:
        # roofline of the step kernel: the timed region is its launches (several coarse steps each)
        alg_step = cells * 18 * sb  # each population read and written once per cell update
        steps_per_launch = args.steps / max(launches, 1)
        launch_us = 1e3 * dev_ms / max(launches, 1)
        achieved = alg_step * steps_per_launch / (launch_us * 1e-6) / 1e9
        traffic = profiled_traffic(spec) if args.workload == "cylinder" and args.storage == "f32" else None
        if traffic is not None:
            traffic *= steps_per_launch  # the capture's figure is per coarse step
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "kernel": "k_step (persistent: every phase of its coarse steps)",
                    "peak_kind": peak_kind, "launches": launches, "avg_launch_us": launch_us,
                    "steps_per_launch": steps_per_launch, "bytes_per_launch": alg_step * steps_per_launch,
                    "note": "launches x avg_launch_us = the timed region; the state (15 MB) lives in L2 within a "
                            "launch"}
    else:
        # roofline of the sweep kernels (the dominant kind) from the serialised profiling pass
        n_f, ms_f, by_f = prof[0]
        avg_us = 1e3 * ms_f / max(n_f, 1)
        achieved = by_f / (ms_f * 1e-3) / 1e9 if ms_f > 0 else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak if achieved else None, "traffic": None,
                    "kernel": "k_fused / k_fused_v4 (stream-collide sweeps, all levels)", "peak_kind": peak_kind,
                    "launches": n_f, "avg_launch_us": avg_us, "bytes_per_launch": by_f / max(n_f, 1),
                    "kinds_us_per_step": {name: round(1e3 * prof[k][1] / args.steps, 2) for k, name in
                                          ((0, "sweeps"), (1, "c2f"), (3, "ibm"))},
                    "note": "per-launch times from a pass of the same steps captured on one stream (no overlap); "
                            f"that pass took {prof_ms / args.steps:.4f} ms per step"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        mlups, steps, el, cores, _ = cpu_oracle_run(workload_spec("f32", args.workload, args.n, args.block, args.coll),
                                                    args.cpu_seconds)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps} coarse steps ({el:.1f} s) of the same workload, FP64 OpenMP oracle"}
    if rank == 0:
        period_fine = 40 / (0.165 * 0.05) if args.workload == "cylinder" else float("nan")
        spans = {}
        for p in trace:
            if p["tasks"] > 0:
                k = spans.setdefault(p["kind"], [0, 0.0])
                k[0] += 1
                k[1] += p["end_us"] - p["start_us"]
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32"}.get(args.storage, "f32"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "cylinder" else
                       f"single-level periodic Taylor-Green {args.n}x{args.n}, tau=0.8, {args.coll.upper()}, blocks of {args.block}, "
                       f"{args.storage} storage", "cell_updates_per_step": cells,
                       "fine_equivalent_per_step": fine_eq, "levels": spec.levels, "block": spec.block,
                       "storage": args.storage,
                       "l2": f"flushed (512 MiB write) between timed calls of {per_call_used} coarse steps "
                             "(one launch of the step kernel, or one step of the graphs)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "gpu_launches": launches,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "finite": ok,
            "mlups_fine_equivalent": world * fine_eq * args.steps / (dev_ms * 1e-3) / 1e6,
            "periods_per_s": (world * args.steps * nf / period_fine / (dev_ms * 1e-3)
                              if args.workload == "cylinder" else None),
            "wall_s": wall, "step_form": "persistent" if form else "graphs", "other_form": other,
        }
        line["config"]["tuning"] = knobs
        if trace:
            line["step_phases"] = {"phases": len(trace),
                                   "span_us_by_kind": {k: round(v[1], 1) for k, v in spans.items()},
                                   "note": "one traced step; spans of phases of a kind, which can overlap"}
        if not args.no_extras:
            detail = {}
            line["bodies"] = measure_bodies(args, stream)
            batch = measure_batch(args, stream, detail)
            line["batch"] = batch
            line["serving"] = measure_serving(args, stream, batch)
            line["sweep"] = measure_sweep(args, stream)  # last: the record's tail carries these fractions
            print(json.dumps({"detail": detail}), file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_sweep(args, stream):
    """The fused stream-collide kernel alone at HBM scale: one level, 8192^2
    periodic cells (4.8 GB per FP32 step, 2.4 GB in 16-bit storage), against
    the measured copy bandwidth: BGK in FP32, BF16 and FP16, the MRT
    collision (same bytes, about twice the arithmetic) and the LES collision
    (FP32), each per-launch event-timed; and the persistent step kernel on
    the same grid (all of it bulk work), FP32 and BF16, timed per step."""
    import torch

    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import TUNE_PERSISTENT, Domain

    peak, peak_kind = measured_peaks()
    out = {"workload": "single-level periodic 8192x8192, blocks of 16, uniform state", "peak_gbs": peak,
           "peak_kind": peak_kind}
    for name, st, coll in (("f32", wl.F32, 0), ("bf16dev", wl.BF16DEV, 0), ("f16dev", wl.F16DEV, 0),
                           ("f32_mrt", wl.F32, 1), ("bf16dev_mrt", wl.BF16DEV, 1), ("f32_les", wl.F32, 2)):
        spec = wl.tgv(n=8192, storage=st, block=16)
        spec = wl.with_mrt(spec) if coll == 1 else (wl.with_les(spec) if coll == 2 else spec)
        g = Domain(spec, stream=stream)
        g.set_tuning(TUNE_PERSISTENT, 0)
        g.step(3)
        g.set_profiling(1)
        g.step(10)
        torch.cuda.synchronize()
        n, ms, by = g.profile(0)
        g.close()
        gbs = by / (ms * 1e-3) / 1e9
        out[name] = {"frac": round(gbs / peak, 4), "gbs": round(gbs, 1), "avg_launch_us": round(1e3 * ms / n, 1)}
    for name, st in (("f32_persistent", wl.F32), ("bf16dev_persistent", wl.BF16DEV)):
        spec = wl.tgv(n=8192, storage=st, block=16)
        g = Domain(spec, stream=stream)
        g.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.step(10)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        g.close()
        gbs = spec.nx0 * spec.ny0 * 18 * (4 if st == wl.F32 else 2) / (ms * 1e-3) / 1e9
        out[name] = {"frac": round(gbs / peak, 4), "gbs": round(gbs, 1), "ms_per_step": round(ms, 3)}
    return out


def measure_bodies(args, stream):
    """The paper's other body cases at full size, FP32 storage, one instance
    each: the flapping ellipse (Sec. 3.6, config 3), the flat plate in the
    pitch-up ramp (Sec. 3.4), the NACA 0018 section in triangular pitch
    (Sec. 3.5), the Table 1 stationary cylinder at Re 300 (Sec. 3.3,
    static-body path: stored IBM geometry) and the lid-driven cavity with its
    cylinder (Sec. 3.2) by interpolated bounce-back and by the IBM.  Per case:
    device time per coarse step over --body-steps steps (L2 flushed before
    the timed run), actual MLUPS, the persistent kernel's and the graph
    path's times (the faster is the library's choice for a single instance
    when the autotuner runs)."""
    import numpy as np
    import torch

    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import TUNE_PERSISTENT, Domain
    from paper_2402_04606_gb300.workloads import initial_fields

    cases = [("wing_c64_m4_flapping", wl.wing(c=64, levels=4, storage=wl.F32)),
             ("plate_pitch_up_c64_m3", wl.pitch_up(c=64, levels=3, storage=wl.F32)),
             ("naca0018_triangle_pitch_c64_m3", wl.pitching_airfoil(c=64, levels=3, storage=wl.F32)),
             ("cylinder_table1_re300_D128_m4", wl.cylinder_table1(re=300.0, storage=wl.F32)),
             ("cavity_re400_L304_cylinder_bounce_back", wl.cavity(L=304, re=400.0, mode="bounce", storage=wl.F32)),
             ("cavity_re400_L304_cylinder_ibm", wl.cavity(L=304, re=400.0, mode="ibm", storage=wl.F32))]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, spec in cases:
        row = {}
        for persistent in (1, 0):
            g = Domain(spec, stream=stream)
            g.set_tuning(TUNE_PERSISTENT, persistent)
            for l in range(spec.levels):
                g.set_fields(l, *initial_fields(spec, l))
            cells, _ = g.work()
            g.step(5)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.fill_(1)
                e0.record(stream)
                g.step(args.body_steps)
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.body_steps
            finite = bool(np.isfinite(g.checksum()).all()) and (spec.body is None or bool(np.isfinite(g.forces()).all()))
            g.close()
            row["persistent_ms" if persistent else "graph_ms"] = round(ms, 4)
            row.setdefault("finite", True)
            row["finite"] = row["finite"] and finite
        best = min(row["persistent_ms"], row["graph_ms"])
        row["mlups"] = round(cells / (best * 1e-3) / 1e6, 1)
        row["cell_updates_per_step"] = cells
        out[name] = row
    return out


def reduced_precision_errors(stream):
    """Velocity L2 (relative, all levels) of BF16 and FP16 deviation storage
    after 10,000 finest steps of the D = 10, 3-level cylinder at Re = 40 (a
    steady wake: no instability amplifies the rounding), against the same run
    in FP64 on the GPU, which the parity tests hold to the FP64 oracle within
    1e-12."""
    import math

    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import Domain
    from paper_2402_04606_gb300.workloads import initial_fields

    runs = {}
    for st in (wl.F64, wl.F16DEV, wl.BF16DEV):
        spec = wl.cylinder(D=10, levels=3, block=8, storage=st, re=40.0)
        g = Domain(spec, stream=stream)
        for l in range(spec.levels):
            g.set_fields(l, *initial_fields(spec, l))
        g.step(2500)
        runs[st] = [g.fields(l) for l in range(3)], [g.types(l) == 1 for l in range(3)]
        g.close()

    def err(st):
        num = den = 0.0
        for l in range(3):
            m = runs[wl.F64][1][l]
            _, ua, va = runs[st][0][l]
            _, ub, vb = runs[wl.F64][0][l]
            num += (((ua - ub) ** 2 + (va - vb) ** 2)[m]).sum()
            den += ((ub ** 2 + vb ** 2)[m]).sum()
        return math.sqrt(num / den)

    return {"bf16_velocity_l2": err(wl.BF16DEV), "fp16_velocity_l2": err(wl.F16DEV), "target_16bit": 2e-3,
            "case": "cylinder D=10, 3 levels, Re 40, 10,000 finest steps, against FP64 on the GPU"}


def measure_batch(args, stream, detail=None):
    """64 uneven cylinder / flapping instances (seed 0: coarsest 256x128 to
    2048x1024, 2-4 levels, Re in [50, 400], pitch amplitude 16-64 degrees),
    BF16 deviation storage; the autotuner picks block size, kernel variants,
    the IBM's threads per body and the per-phase graphs or the persistent
    step kernel (short trials first); both step forms are then timed."""
    import torch

    from paper_2402_04606_gb300 import autotune as at
    from paper_2402_04606_gb300 import native as nv
    from paper_2402_04606_gb300 import serving as sv
    from paper_2402_04606_gb300 import workloads as wl

    specs = wl.batch(64, seed=0, storage=wl.BF16DEV, block=16)
    if args.batch_block:
        best = {"block": args.batch_block, "vec_min_cells": args.batch_vec, **at.DEFAULTS}
        tuned = {"best": best, "trials": None, "seconds": 0.0}
    else:
        tuned = at.tune(specs, storage=wl.BF16DEV, steps=5, warmup=2, stream=stream)
    best = tuned["best"]
    ids = at.knob_ids()
    block = best["block"]
    periods_per_step = sum((1 << (s.levels - 1)) / sv.body_period_fine(s) for s in specs)

    def run(persistent):
        b = nv.Batch(64, block=block, storage=wl.BF16DEV, stream=stream)
        for s in specs:
            b.admit(at.with_block(s, block))
        b.set_tuning(nv.TUNE_VECTOR_MIN_CELLS, best["vec_min_cells"])
        for k in at.KNOBS:
            b.set_tuning(ids[k], best[k])
        b.set_tuning(nv.TUNE_PERSISTENT, persistent)
        cells = b.info()["cell_updates_per_step"]
        b.step(5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            b.step(args.batch_steps)
            e1.record(stream)
        torch.cuda.synchronize()
        b.close()
        return e0.elapsed_time(e1) / args.batch_steps, cells

    ms, cells = run(best["persistent"])
    other_ms, _ = run(1 - best["persistent"])
    if detail is not None:
        detail["batch_autotune_trials"] = tuned["trials"]
    prec = reduced_precision_errors(stream)
    return {"workload": "64 uneven cylinder/flapping instances, seed 0, BF16 deviation storage",
            "ms_per_step": ms, "mlups": cells / (ms * 1e-3) / 1e6, "cell_updates_per_step": cells,
            "hbm_frac": cells * 36 / (ms * 1e-3) / 1e9 / measured_peaks()[0],
            "solved_periods_per_s": periods_per_step / (ms * 1e-3),
            "step_form": "persistent" if best["persistent"] else "graphs",
            "other_form_ms_per_step": other_ms, "tuning": {k: best[k] for k in ("block", "vec_min_cells", *at.KNOBS)},
            "autotune_s": round(tuned["seconds"], 1), "steps": args.batch_steps,
            "accuracy_16bit": prec, "l2": "state (about 1.7 GB) larger than L2"}


def measure_serving(args, stream, batch=None):
    """Config 5: Poisson arrivals (20/s, seed 1) of --serve-requests solve
    requests drawn like the batch mix, each run to --serve-periods body
    periods, under a 150 GB budget, in three arms on the same arrivals:
    served with continuous batching in FP16 and in FP32 deviation storage,
    and plain FP32 one request at a time on its own context (its context
    set-up timed apart and left out of its clock).  The served batches take
    the kernel choices the autotuner made for the batch mix, when given."""
    from paper_2402_04606_gb300 import autotune as at
    from paper_2402_04606_gb300 import serving as sv
    from paper_2402_04606_gb300 import workloads as wl

    tuning = None
    if batch is not None and batch["tuning"]["block"] == 16:
        t = batch["tuning"]
        tuning = {i: t[k] for k, i in at.knob_ids().items()}
    arrivals, specs = wl.serving_arrivals(args.serve_requests, 20.0, seed=1)
    reqs = sv.requests_from(arrivals, specs, args.serve_periods)
    keep = ("solved_periods_per_s", "p50_time_to_result_s", "p99_time_to_result_s", "wall_s")
    arms = {}
    for name, st in (("served_fp16", wl.F16DEV), ("served_fp32", wl.F32)):
        _, r = sv.run_served(reqs, storage=st, block=16, budget_bytes=150 << 30, chunk=16, stream=stream,
                             tuning=tuning)
        arms[name] = {k: r[k] for k in keep}
    _, r = sv.run_sequential(reqs, storage=wl.F32, block=16, stream=stream)
    arms["plain_fp32"] = {**{k: r[k] for k in keep}, "setup_s_excluded": r["setup_s"]}
    plain = arms["plain_fp32"]["solved_periods_per_s"]
    return {"workload": f"{args.serve_requests} Poisson requests (20/s, seed 1) of the batch mix, "
                        f"{args.serve_periods} body periods each",
            **arms,
            "served_fp16_over_plain_fp32": arms["served_fp16"]["solved_periods_per_s"] / plain,
            "served_fp32_over_plain_fp32": arms["served_fp32"]["solved_periods_per_s"] / plain}


def run_batch_main(args):
    """--workload batch: the 64-instance batch as the line's workload."""
    import torch

    from paper_2402_04606_gb300 import build as bld

    torch.cuda.set_device(dist_env()[2])
    bld.build()
    stream = torch.cuda.Stream()
    b = measure_batch(args, stream)
    line = {"metric": "MLUPS", "value": b["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.batch_steps,
            "warmup": 5, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": b["workload"], **b["tuning"], "l2": b["l2"]}, "batch": b}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_main(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
