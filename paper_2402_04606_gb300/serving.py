"""Continuous-batching request loop over the batch ABI (sbot_batch_*).

Solve requests (a domain, a body and a number of body periods) arrive over
time.  The loop admits each one into the live batch as soon as an instance
slot and the device-memory budget allow it (the library refuses an admission
that does not fit), advances every live solve together (one graph launch per
coarse step covers all of them) with a bounded queue of chunks on the
device, and retires a solve once it has run its periods, draining its force
history, which frees its blocks for the next arrivals.  All arithmetic runs in the library's kernels; this
module only schedules and times.

``run_sequential`` is the plain form the loop is compared with: the same
requests, one at a time, each on its own single-instance context (its
context set-up timed apart).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as wl


@dataclass
class Request:
    rid: int
    spec: wl.DomainSpec
    arrival_s: float  # seconds after the start of the run
    periods: float    # body periods to solve


@dataclass
class Result:
    rid: int
    name: str
    arrival_s: float
    admitted_s: float
    done_s: float
    fine_steps: int
    periods: float
    cd_mean: float  # over the last solved period (or the whole run if shorter)
    cl_rms: float
    forces: np.ndarray = field(repr=False, default=None)

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


# force-history entries (finest steps) an instance may accumulate before the
# loop drains them; the library's ring holds 65536
HIST_DRAIN_FINE = 1 << 15


def body_period_fine(spec: wl.DomainSpec) -> float:
    """Period of the body in finest steps: the prescribed motion's period, or
    for a static cylinder the shedding period D / (St U) with St = 0.165."""
    b = spec.body
    if b is None:
        raise ValueError("a solve request needs a body")
    if b.motion != 0:
        return float(b.period)
    return 2.0 * b.a / (0.165 * b.u_ref)


def coarse_steps_for(spec: wl.DomainSpec, periods: float) -> int:
    return max(1, int(math.ceil(periods * body_period_fine(spec) / (1 << (spec.levels - 1)))))


def coefficients(spec: wl.DomainSpec, forces: np.ndarray, fine_steps: int):
    """Mean drag and rms lift coefficient over the last body period:
    C = 2 F / (rho0 U^2 L) with the body's reference speed and length."""
    b = spec.body
    f = forces[:fine_steps]
    if len(f) == 0:
        return float("nan"), float("nan")
    n = min(len(f), max(1, int(round(body_period_fine(spec)))))
    q = 0.5 * spec.rho0 * b.u_ref ** 2 * b.l_ref
    cd = f[-n:, 0] / q
    cl = f[-n:, 1] / q
    return float(cd.mean()), float(np.sqrt(np.mean(cl ** 2)))


def force_statistics(spec: wl.DomainSpec, forces: np.ndarray, skip: int = 0) -> dict:
    """The statistics of Sec. 3.3, Eq. 19, from a force history (one row per
    finest step, rows from ``skip`` on): mean drag coefficient, the rms of
    the lift coefficient about its mean, and the Strouhal number f D / U of
    the lift's dominant frequency (the peak of its spectrum, refined by
    parabolic interpolation of the log magnitudes), with time in finest
    steps and the body's reference length and speed."""
    b = spec.body
    f = np.asarray(forces, np.float64)[skip:]
    q = 0.5 * spec.rho0 * b.u_ref ** 2 * b.l_ref
    cd = f[:, 0] / q
    cl = f[:, 1] / q
    out = {"cd_mean": float(cd.mean()), "cl_rms": float(np.sqrt(np.mean((cl - cl.mean()) ** 2))),
           "strouhal": float("nan"), "samples": int(len(f))}
    if len(f) >= 16:
        x = (cl - cl.mean()) * np.hanning(len(cl))
        mag = np.abs(np.fft.rfft(x))
        k = int(np.argmax(mag[1:]) + 1)
        shift = 0.0
        if 1 <= k < len(mag) - 1 and min(mag[k - 1], mag[k], mag[k + 1]) > 0:
            lm, l0, lp = np.log(mag[k - 1]), np.log(mag[k]), np.log(mag[k + 1])
            den = lm - 2 * l0 + lp
            shift = 0.5 * (lm - lp) / den if den != 0 else 0.0
        freq = (k + shift) / len(cl)  # cycles per finest step
        out["strouhal"] = float(freq * b.l_ref / b.u_ref)
    return out


def requests_from(arrivals, specs, periods: float):
    return [Request(i, s, float(t), periods) for i, (t, s) in enumerate(zip(arrivals, specs))]


def run_served(requests, storage: int, block: int = 16, budget_bytes: int = 150 << 30, max_instances: int = 256,
               chunk: int = 16, stream=None, keep_forces: bool = False, tuning: dict | None = None,
               in_flight: int = 2, batch_factory=None, event_factory=None):
    """Serve the requests with continuous batching.  Returns (results, stats).

    The loop keeps up to ``in_flight`` chunks of ``chunk`` coarse steps
    queued on the device and synchronises only to hand back a finished solve
    (or to drain a force history before its ring would wrap), so the GPU
    does not wait for the host between chunks.  ``tuning``: library tuning
    knobs (sbot_set_tuning) for the batch, e.g. the autotuner's choice for
    the request mix.  ``batch_factory`` and ``event_factory`` default to the
    library's ``Batch`` and ``torch.cuda.Event`` (the host-side tests pass
    stand-ins with the same calls)."""
    import collections

    from .native import ERR_OOM, SbotError

    if batch_factory is None:
        from .native import Batch as batch_factory
    if event_factory is None:
        import torch

        event_factory = torch.cuda.Event
    b = batch_factory(max_instances, block=block, storage=storage, budget_bytes=budget_bytes, stream=stream)
    for what, value in (tuning or {}).items():
        b.set_tuning(what, value)
    pending = sorted(requests, key=lambda r: r.arrival_s)
    live = {}  # rid -> [request, instance, target coarse steps, admitted_s, force chunks, last drained step]
    queued = collections.deque()  # one event per chunk still on the device
    results = []
    refused = 0
    t0 = time.perf_counter()
    steps_run = 0
    while pending or live:
        now = time.perf_counter() - t0
        while pending and pending[0].arrival_s <= now:
            r = pending[0]
            spec = wl.replace_storage(r.spec, storage, block)
            try:
                inst = b.admit(spec)
            except SbotError as e:
                if e.status != ERR_OOM or not live:
                    raise  # not a lack of room, or it cannot fit even alone
                refused += 1
                break  # wait for a retirement to free memory
            pending.pop(0)
            live[r.rid] = [r, inst, coarse_steps_for(spec, r.periods), time.perf_counter() - t0, [], 0]
        if not live:
            if pending:
                time.sleep(max(0.0, min(pending[0].arrival_s - (time.perf_counter() - t0), 0.05)))
            continue
        b.step(chunk)
        steps_run += chunk
        ev = event_factory()
        ev.record(b.stream)
        queued.append(ev)
        if len(queued) > in_flight:
            queued.popleft().synchronize()
        done = []
        for rid, entry in live.items():
            r, inst, target, adm, chunks, drained = entry
            n = inst.coarse_steps()
            if n >= target:
                done.append(rid)
            elif (n - drained) << (inst.spec.levels - 1) >= HIST_DRAIN_FINE:
                chunks.append(inst.forces(cap=1 << 17))  # before the history ring wraps
                entry[5] = n
        for rid in done:
            r, inst, target, adm, chunks, _ = live.pop(rid)
            chunks.append(inst.forces(cap=1 << 17))  # waits for the instance's last steps
            spec = inst.spec
            fine = target << (spec.levels - 1)
            forces = np.concatenate(chunks, axis=0)
            cd, cl = coefficients(spec, forces, fine)
            t_done = time.perf_counter() - t0
            results.append(Result(r.rid, spec.name, r.arrival_s, adm, t_done, fine, r.periods, cd, cl,
                                  forces[:fine] if keep_forces else None))
            b.retire(inst)
    wall = time.perf_counter() - t0
    b.close()
    return results, summarize(results, wall, extra={"refused_admissions": refused, "batch_coarse_steps": steps_run})


def run_sequential(requests, storage: int = wl.F32, block: int = 16, stream=None, chunk: int = 64,
                   keep_forces: bool = False, domain_factory=None):
    """The plain form: each request alone on its own context, in arrival order.

    The clock stops while a request's context is created and initialised
    (device allocation, planning, the first collision): that set-up is
    reported apart as ``setup_s`` and is not part of the wall time, the
    latencies or the throughput, so the comparison with the served form
    measures the stepping alone.  ``domain_factory`` defaults to the
    library's ``Domain`` (the host-side tests pass a stand-in)."""
    if domain_factory is None:
        from .native import Domain as domain_factory

    results = []
    setup = 0.0
    t0 = time.perf_counter()

    def clock():
        return time.perf_counter() - t0 - setup

    for r in sorted(requests, key=lambda q: q.arrival_s):
        now = clock()
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        adm = clock()
        s0 = time.perf_counter()
        spec = wl.replace_storage(r.spec, storage, block)
        g = domain_factory(spec, stream=stream)
        g.step(0)  # the initial collision: part of the set-up
        g.sync()
        setup += time.perf_counter() - s0
        target = coarse_steps_for(spec, r.periods)
        chunks = []
        n = 0
        while n < target:
            k = min(chunk, target - n)
            g.step(k)
            n += k
            chunks.append(g.forces(cap=1 << 17))
        fine = target << (spec.levels - 1)
        forces = np.concatenate(chunks, axis=0)
        cd, cl = coefficients(spec, forces, fine)
        results.append(Result(r.rid, spec.name, r.arrival_s, adm, clock(), fine, r.periods, cd, cl,
                              forces[:fine] if keep_forces else None))
        s0 = time.perf_counter()
        g.close()
        setup += time.perf_counter() - s0
    wall = clock()
    return results, summarize(results, wall, extra={"setup_s": setup})


def summarize(results, wall_s: float, extra=None) -> dict:
    lat = np.array([r.latency_s for r in results]) if results else np.zeros(1)
    periods = float(sum(r.periods for r in results))
    d = {
        "requests": len(results),
        "wall_s": wall_s,
        "solved_periods_per_s": periods / wall_s if wall_s > 0 else None,
        "solves_per_s": len(results) / wall_s if wall_s > 0 else None,
        "p50_time_to_result_s": float(np.percentile(lat, 50)),
        "p99_time_to_result_s": float(np.percentile(lat, 99)),
    }
    if extra:
        d.update(extra)
    return d
