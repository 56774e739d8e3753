#!/usr/bin/env python
"""Benchmark of the hot path: one step = one coarse time step (Algorithm 1:
every level's fused stream-collide sweeps, the coarse/fine transfers, the
multi-direct-forcing IBM before every finest collision and the force/moment
reduction) of the refined circular-cylinder workload: Re = 100, D = 40
finest cells, 3 levels (factor 2), coarsest grid 30D x 15D (rounded up to
whole blocks), uniform inflow u = 0.05, 126 markers, K = 5, FP32 storage.

Prints one JSON line.  --impl reference times the CPU oracle (plain FP64 C,
OpenMP) on the same workload instead.

Timing: W untimed warm-up steps; then K steps, each bracketed by CUDA events
on the library's stream, with a 512 MiB write between steps to flush the
129 MB L2 (the flush is outside the events).  value = actual cell updates /
summed device time.  A second pass of the same K steps records the library's
own per-kernel events inside the CUDA graph (kernel roofline and shares).
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
    ap.add_argument("--tune", action="store_true",
                    help="choose the block size and kernel threshold of the main workload by timed trials "
                         "(the cylinder workload is defined with blocks of 16; the batch is always tuned)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (64 uneven instances, BF16) and served (Poisson arrivals) measurements")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--body-steps", type=int, default=40, help="coarse steps timed per body case")
    ap.add_argument("--batch-block", type=int, default=0, help="skip the batch autotuner: use this block size")
    ap.add_argument("--batch-vec", type=int, default=1 << 16, help="with --batch-block: the vector-kernel threshold")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-periods", type=float, default=0.25)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--block", type=int, default=16)
    return ap.parse_args()


def workload_spec(storage: str, workload: str = "cylinder", n: int = 8192, block: int = 16):
    from paper_2402_04606_gb300 import workloads as wl

    st = {"f64": wl.F64, "f32": wl.F32, "f16dev": wl.F16DEV, "bf16dev": wl.BF16DEV}[storage]
    if workload == "sweep":
        return wl.tgv(n=n, tau=0.8, u0=0.02, storage=st, block=block)
    return wl.cylinder(D=40, levels=3, re=100.0, u=0.05, n_markers=126, K=5, storage=st, block=16)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "k_fused_cylinder_D40_m3_f32.md")


def kernels_sha256():
    import hashlib

    with open(os.path.join(ROOT, "paper_2402_04606_gb300", "csrc", "kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profiled_traffic(spec):
    """DRAM bytes per k_fused launch on this workload from the committed ncu
    summary, or None when the kernels have changed since it was taken."""
    try:
        text = open(PROFILE_TRAFFIC).read()
    except OSError:
        return None
    import re

    m = re.search(r"traffic_bytes_per_launch = ([0-9.eE+]+) \(kernels.cu sha256 ([0-9a-f]+)\)", text)
    if not m or m.group(2) != kernels_sha256() or spec.block != 16:
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
    spec = workload_spec("f32", args.workload, args.n, args.block)
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
    from paper_2402_04606_gb300.native import Domain
    from paper_2402_04606_gb300.replicas import job_rate, max_over_ranks
    from paper_2402_04606_gb300.workloads import initial_fields

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    bld.build()
    spec = workload_spec(args.storage, args.workload, args.n, args.block)
    stream = torch.cuda.Stream()
    tuned = None
    if args.tune:
        # block size and fused kernel variant by short timed trials of this workload
        from paper_2402_04606_gb300 import autotune as at

        tuned = at.tune([spec], steps=10, warmup=3, stream=stream)
        spec = at.with_block(spec, tuned["best"]["block"])
    g = Domain(spec, stream=stream)
    if tuned is not None:
        from paper_2402_04606_gb300.native import TUNE_VECTOR_MIN_CELLS

        g.set_tuning(TUNE_VECTOR_MIN_CELLS, tuned["best"]["vec_min_cells"])
    fields = [initial_fields(spec, l) for l in range(spec.levels)]
    for l in range(spec.levels):
        g.set_fields(l, *fields[l])
    cells, fine_eq = g.work()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    g.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    def timed_pass():
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 255)  # evict the state from L2 between timed steps
                ev[k][0].record(stream)
                g.step(1)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev), time.perf_counter() - t0

    # pass 1: the timed region (no profiling events in the graph)
    with ClockSampler(local) as clk:
        dev_ms, wall = timed_pass()
    if world > 1:
        torch.distributed.barrier()
    # pass 2: the same K steps again with the library's per-kernel events
    # recorded inside the CUDA graph, for the per-kernel roofline
    g.set_profiling(15)
    prof_ms, _ = timed_pass()
    n_fused, ms_fused, bytes_fused = g.profile(0)
    launches_profiled = sum(g.profile(kind)[0] for kind in range(4))
    kinds = {}
    for kind, name in enumerate(("fused_stream_collide", "c2f_halo_copy", "f2c_merge", "ibm_mdf")):
        n_k, ms_k, b_k = g.profile(kind)
        kinds[name] = {"launches": n_k, "avg_us": 1e3 * ms_k / max(n_k, 1), "share_of_step": ms_k / prof_ms,
                       "gbs": b_k / (ms_k * 1e-3) / 1e9 if ms_k > 0 else None}
    g.set_profiling(0)
    dev_ms = max_over_ranks(dev_ms)  # the slowest replica times the job
    clocks = clk.summary()
    # checksum must stay finite (guards against a silently diverged run)
    cs = g.checksum()
    ok = bool(np.isfinite(cs).all())
    value = job_rate(cells * args.steps, dev_ms * 1e-3, world) / 1e6

    # end to end through the public API with host buffers: upload the initial
    # state from pinned host memory, then every step advance and read that
    # step's force history back to the host
    e2e = None
    g2 = Domain(spec, stream=stream)
    if tuned is not None:
        g2.set_tuning(TUNE_VECTOR_MIN_CELLS, tuned["best"]["vec_min_cells"])
    pinned = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in f] for f in fields]
    h2d = sum(a.nbytes for f in pinned for a in f)
    torch.cuda.synchronize()
    nf = 1 << (spec.levels - 1)
    t0 = time.perf_counter()
    for l in range(spec.levels):
        g2.set_fields(l, *pinned[l])
    for k in range(args.steps):
        g2.step(1)
        fr = g2.forces(cap=nf)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": job_rate(cells * args.steps, e2e_s, world) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": nf * 3 * 8}
    g2.close()

    peak, peak_kind = measured_peaks()
    achieved = bytes_fused / (ms_fused * 1e-3) / 1e9 if ms_fused > 0 else None
    traffic = profiled_traffic(spec) if args.workload == "cylinder" and args.storage == "f32" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel": "k_fused (stream-collide, all levels)", "peak_kind": peak_kind,
                "launches": n_fused, "avg_launch_us": 1e3 * ms_fused / max(n_fused, 1),
                "bytes_per_launch": bytes_fused / max(n_fused, 1)}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        mlups, steps, el, cores, _ = cpu_oracle_run(workload_spec("f32", args.workload, args.n, args.block),
                                                    args.cpu_seconds)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps} coarse steps ({el:.1f} s) of the same workload, FP64 OpenMP oracle"}
    if rank == 0:
        period_fine = 40 / (0.165 * 0.05) if args.workload == "cylinder" else float("nan")
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32"}.get(args.storage, "f32"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "cylinder" else
                       f"single-level periodic Taylor-Green {args.n}x{args.n}, tau=0.8, blocks of {args.block}, "
                       f"{args.storage} storage", "cell_updates_per_step": cells,
                       "fine_equivalent_per_step": fine_eq, "levels": spec.levels, "block": spec.block,
                       "storage": args.storage, "l2": "flushed between timed steps (512 MiB write)",
                       "vec_min_cells": tuned["best"]["vec_min_cells"] if tuned else 1 << 19,
                       "autotune_trials": tuned["trials"] if tuned else None,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "mlups_fine_equivalent": world * fine_eq * args.steps / (dev_ms * 1e-3) / 1e6,
            "periods_per_s": (world * args.steps * nf / period_fine / (dev_ms * 1e-3)
                              if args.workload == "cylinder" else None),
            "wall_s": wall, "finite": ok,
            "clocks": clocks, "roofline": roofline, "kernels": kinds, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_profiled,
        }
        g.close()
        if not args.no_extras:
            line["sweep"] = measure_sweep(args, stream)
            line["bodies"] = measure_bodies(args, stream)
            line["batch"] = measure_batch(args, stream)
            line["serving"] = measure_serving(args, stream, line["batch"])
        print(json.dumps(line), flush=True)
    else:
        g.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_sweep(args, stream):
    """The fused stream-collide kernel alone at HBM scale: one level, 8192^2
    periodic cells (4.8 GB per FP32 step, 2.4 GB in 16-bit storage), against
    the measured copy bandwidth; BGK in FP32, BF16 and FP16, the MRT collision
    (same bytes, about twice the arithmetic) and the LES collision (FP32)."""
    import torch

    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import Domain

    peak, peak_kind = measured_peaks()
    out = {"workload": "single-level periodic 8192x8192, blocks of 16, uniform state", "peak_gbs": peak,
           "peak_kind": peak_kind}
    for name, st, coll in (("f32", wl.F32, 0), ("bf16dev", wl.BF16DEV, 0), ("f16dev", wl.F16DEV, 0),
                           ("f32_mrt", wl.F32, 1), ("bf16dev_mrt", wl.BF16DEV, 1), ("f32_les", wl.F32, 2)):
        spec = wl.tgv(n=8192, storage=st, block=16)
        spec = wl.with_mrt(spec) if coll == 1 else (wl.with_les(spec) if coll == 2 else spec)
        g = Domain(spec, stream=stream)
        g.step(3)
        g.set_profiling(1)
        g.step(10)
        torch.cuda.synchronize()
        n, ms, by = g.profile(0)
        g.close()
        gbs = by / (ms * 1e-3) / 1e9
        out[name] = {"launches": n, "avg_launch_us": 1e3 * ms / n, "bytes_per_launch": by / n, "gbs": gbs,
                     "frac": gbs / peak, "glups": (by / n) / (18 * (4 if st == wl.F32 else 2)) / (ms / n * 1e-3) / 1e9}
    return out


def measure_bodies(args, stream):
    """The paper's other body cases at full size, FP32 storage, one instance
    each: the flapping ellipse (Sec. 3.6, config 3), the flat plate in the
    pitch-up ramp (Sec. 3.4), the NACA 0018 section in triangular pitch
    (Sec. 3.5), the Table 1 stationary cylinder at Re 300 (Sec. 3.3,
    static-body path: stored IBM geometry) and the lid-driven cavity with its
    cylinder (Sec. 3.2) by interpolated bounce-back and by the IBM.  Per case: device time per
    coarse step over --body-steps steps (L2 flushed before the timed run),
    actual and fine-equivalent MLUPS, and the IBM launch's event time."""
    import numpy as np
    import torch

    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import Domain
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
        g = Domain(spec, stream=stream)
        for l in range(spec.levels):
            g.set_fields(l, *initial_fields(spec, l))
        cells, fine_eq = g.work()
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
        g.set_profiling(8)
        g.step(args.body_steps)
        torch.cuda.synchronize()
        n_i, ms_i, _ = g.profile(3)
        g.set_profiling(0)
        finite = bool(np.isfinite(g.checksum()).all()) and bool(np.isfinite(g.forces()).all())
        g.close()
        out[name] = {"grid": f"{spec.nx0}x{spec.ny0} coarsest, {spec.levels} levels, blocks of {spec.block}",
                     "markers": spec.body.n_markers if spec.body is not None else 0, "ms_per_step": ms,
                     "mlups": cells / (ms * 1e-3) / 1e6,
                     "mlups_fine_equivalent": fine_eq / (ms * 1e-3) / 1e6, "cell_updates_per_step": cells,
                     "ibm_launches": n_i, "ibm_avg_us": 1e3 * ms_i / max(n_i, 1), "finite": finite}
    return out


def measure_batch(args, stream):
    """64 uneven cylinder / flapping instances (seed 0: coarsest 256x128 to
    2048x1024, 2-4 levels, Re in [50, 400], pitch amplitude 16-64 degrees),
    BF16 deviation storage, one graph launch per coarse step; the block size
    and fused kernel variant come from the autotuner (short trials first)."""
    import torch

    from paper_2402_04606_gb300 import autotune as at
    from paper_2402_04606_gb300 import serving as sv
    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import TUNE_PDL, TUNE_STAGED, TUNE_VECTOR_MIN_CELLS, Batch

    specs = wl.batch(64, seed=0, storage=wl.BF16DEV, block=16)
    if args.batch_block:
        tuned = {"best": {"block": args.batch_block, "vec_min_cells": args.batch_vec}, "trials": None, "seconds": 0.0}
    else:
        tuned = at.tune(specs, storage=wl.BF16DEV, steps=5, warmup=2, stream=stream)
    block, vec = tuned["best"]["block"], tuned["best"]["vec_min_cells"]
    staged = tuned["best"].get("staged", 0)
    pdl = tuned["best"].get("pdl", 0)
    b = Batch(64, block=block, storage=wl.BF16DEV, stream=stream)
    for s in specs:
        b.admit(at.with_block(s, block))
    b.set_tuning(TUNE_VECTOR_MIN_CELLS, vec)
    b.set_tuning(TUNE_STAGED, staged)
    b.set_tuning(TUNE_PDL, pdl)
    cells = b.info()["cell_updates_per_step"]
    periods_per_step = sum((1 << (s.levels - 1)) / sv.body_period_fine(s) for s in specs)
    b.step(5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.step(args.batch_steps)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b.set_profiling(15)
    b.step(args.batch_steps)
    torch.cuda.synchronize()
    n_f, ms_f, by_f = b.profile(0)
    b.set_profiling(0)
    b.close()
    return {"workload": "64 uneven cylinder/flapping instances, seed 0, BF16 deviation storage",
            "block": block, "vec_min_cells": vec, "staged": staged, "pdl": pdl, "autotune_trials": tuned["trials"],
            "autotune_s": tuned["seconds"], "steps": args.batch_steps, "ms_per_step": ms / args.batch_steps,
            "mlups": cells * args.batch_steps / (ms * 1e-3) / 1e6, "cell_updates_per_step": cells,
            "solved_periods_per_s": periods_per_step * args.batch_steps / (ms * 1e-3),
            "fused_gbs": by_f / (ms_f * 1e-3) / 1e9 if ms_f > 0 else None,
            "l2": "state (about 1.7 GB) larger than L2"}


def measure_serving(args, stream, batch=None):
    """The batch mix as solve requests of --serve-periods body periods each.
    Poisson arrivals (20/s, seed 1) served with continuous batching in FP16
    deviation storage under a 150 GB budget give the time-to-result
    percentiles; the same requests all present at once measure capacity,
    served (FP16) and one at a time on single-instance FP32 contexts.  The
    served batches take the kernel choices the autotuner made for the same
    mix (the batch measurement), when given."""
    from paper_2402_04606_gb300 import serving as sv
    from paper_2402_04606_gb300 import workloads as wl
    from paper_2402_04606_gb300.native import TUNE_PDL, TUNE_STAGED, TUNE_VECTOR_MIN_CELLS

    tuning = None
    if batch is not None and batch.get("block") == 16:
        tuning = {TUNE_VECTOR_MIN_CELLS: batch["vec_min_cells"], TUNE_STAGED: batch.get("staged", 0),
                  TUNE_PDL: batch.get("pdl", 0)}
    arrivals, specs = wl.serving_arrivals(args.serve_requests, 20.0, seed=1)
    reqs = sv.requests_from(arrivals, specs, args.serve_periods)
    _, poisson = sv.run_served(reqs, storage=wl.F16DEV, block=16, budget_bytes=150 << 30, chunk=16, stream=stream,
                               tuning=tuning)
    at_once = sv.requests_from([0.0] * len(specs), specs, args.serve_periods)
    _, served = sv.run_served(at_once, storage=wl.F16DEV, block=16, budget_bytes=150 << 30, chunk=16, stream=stream,
                              tuning=tuning)
    _, plain = sv.run_sequential(at_once, storage=wl.F32, block=16, stream=stream)
    return {"workload": f"{args.serve_requests} requests of the batch mix, {args.serve_periods} body periods each",
            "served_tuning": {"vec_min_cells": batch["vec_min_cells"], "staged": batch.get("staged", 0),
                              "pdl": batch.get("pdl", 0)} if tuning else None,
            "poisson_20_per_s_fp16": poisson, "all_at_once_served_fp16": served,
            "all_at_once_plain_fp32_one_at_a_time": plain,
            "capacity_ratio_solved_periods_per_s": served["solved_periods_per_s"] / plain["solved_periods_per_s"]}


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
            "config": {"workload": b["workload"], "block": b["block"], "vec_min_cells": b["vec_min_cells"],
                       "l2": b["l2"]}, "batch": b}
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
