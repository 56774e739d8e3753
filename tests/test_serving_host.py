"""Host-side logic of the request loop (no GPU): periods, step counts,
force coefficients and latency statistics."""
import math

import numpy as np
import pytest

from paper_2402_04606_gb300 import serving as sv
from paper_2402_04606_gb300 import workloads as wl


def test_body_period_and_steps():
    cyl = wl.cylinder(D=40, levels=3)
    assert sv.body_period_fine(cyl) == pytest.approx(40 / (0.165 * 0.05))  # shedding period D / (St U)
    wing = wl.wing(c=64, levels=4)
    assert sv.body_period_fine(wing) == pytest.approx(2.5 * math.pi * 64 / 0.05)  # Sec. 3.6: T = 2.5 pi c / U
    # coarse steps: each is 2^(m-1) finest steps
    assert sv.coarse_steps_for(wing, 1.0) == math.ceil(2.5 * math.pi * 64 / 0.05 / 8)
    assert sv.coarse_steps_for(cyl, 1e-9) == 1


def test_coefficients_closed_forms():
    spec = wl.cylinder(D=40, levels=3)
    q = 0.5 * spec.rho0 * spec.body.u_ref ** 2 * spec.body.l_ref
    n = int(round(sv.body_period_fine(spec)))
    t = np.arange(3 * n)
    f = np.zeros((3 * n, 3))
    f[:, 0] = 0.7 * q  # constant drag force: C_D = 0.7
    f[:, 1] = 0.3 * q * np.sin(2 * np.pi * t / n)  # lift oscillating with amplitude C_L = 0.3
    cd, cl = sv.coefficients(spec, f, 3 * n)
    assert cd == pytest.approx(0.7, rel=1e-12)
    assert cl == pytest.approx(0.3 / math.sqrt(2), rel=1e-3)


def test_summary_percentiles():
    res = [sv.Result(i, "r", 0.0, 0.0, float(i + 1), 10, 0.5, 0.0, 0.0) for i in range(100)]
    s = sv.summarize(res, 50.0)
    assert s["requests"] == 100
    assert s["solved_periods_per_s"] == pytest.approx(1.0)
    assert s["p50_time_to_result_s"] == pytest.approx(50.5)
    assert s["p99_time_to_result_s"] == pytest.approx(99.01)


def test_requests_and_storage_copies():
    arrivals, specs = wl.serving_arrivals(6, 20.0, seed=1)
    assert np.all(np.diff(arrivals) > 0)
    reqs = sv.requests_from(arrivals, specs, 2.0)
    assert [r.rid for r in reqs] == list(range(6)) and all(r.periods == 2.0 for r in reqs)
    s16 = wl.replace_storage(specs[0], wl.F16DEV)
    assert s16.storage == wl.F16DEV
    assert s16.body is not specs[0].body and s16.boxes is not specs[0].boxes
    with pytest.raises(ValueError):
        wl.replace_storage(specs[0], wl.F32, block=specs[0].block * 2)


def test_force_statistics_of_a_synthetic_history():
    """Eq. 19 statistics on a history with known mean, rms and frequency:
    C_D = 1.33 + 0.01 cos(2 w t), C_L = 0.05 + 0.34 sin(w t), St = 0.2."""
    from paper_2402_04606_gb300 import serving as sv
    from paper_2402_04606_gb300 import workloads as wl

    spec = wl.cylinder(D=40, levels=3)
    b = spec.body
    q = 0.5 * spec.rho0 * b.u_ref ** 2 * b.l_ref
    St = 0.2
    f = St * b.u_ref / b.l_ref  # cycles per finest step
    n = int(round(20 / f))  # 20 whole periods
    t = np.arange(n)
    cd = 1.33 + 0.01 * np.cos(4 * np.pi * f * t)
    cl = 0.05 + 0.34 * np.sin(2 * np.pi * f * t)
    forces = np.stack([cd * q, cl * q, np.zeros(n)], axis=1)
    st = sv.force_statistics(spec, forces)
    assert abs(st["cd_mean"] - 1.33) <= 1e-4
    assert abs(st["cl_rms"] - 0.34 / np.sqrt(2)) <= 1e-3
    assert abs(st["strouhal"] - St) <= 2e-3


class _FakeInstance:
    """Stand-in for a batch instance: counts coarse steps and serves a force
    history whose first column is the finest step index, from a ring of the
    library's 65536 entries."""

    RING = 65536

    def __init__(self, spec, owner):
        self.spec, self.owner, self.n, self.drained = spec, owner, 0, 0

    def coarse_steps(self):
        return self.n

    def forces(self, cap=1 << 20):
        total = self.n << (self.spec.levels - 1)
        rows = np.zeros((total - self.drained, 3))
        rows[:, 0] = np.arange(self.drained, total)
        self.drained = total
        assert len(rows) <= cap
        return rows


class _FakeBatch:
    """Stand-in for the batch ABI: an admission is refused with ERR_OOM when
    the live instances' footprint (cells at the finest resolution) would pass
    the budget, as the library refuses one that does not fit in memory."""

    def __init__(self, max_instances, block, storage, budget_bytes, stream):
        self.budget, self.live, self.stream = budget_bytes, [], None
        self.wrapped, self.closed, self.peak_live = 0, False, 0

    @staticmethod
    def cost(spec):
        return spec.nx0 * spec.ny0 << (2 * (spec.levels - 1))

    def set_tuning(self, what, value):
        pass

    def admit(self, spec):
        from paper_2402_04606_gb300.native import ERR_OOM, SbotError

        if sum(self.cost(i.spec) for i in self.live) + self.cost(spec) > self.budget:
            raise SbotError(ERR_OOM, "over the budget")
        inst = _FakeInstance(spec, self)
        self.live.append(inst)
        self.peak_live = max(self.peak_live, len(self.live))
        return inst

    def step(self, n):
        for i in self.live:
            i.n += n
            if (i.n << (i.spec.levels - 1)) - i.drained > _FakeInstance.RING:
                self.wrapped += 1

    def retire(self, inst):
        self.live.remove(inst)

    def close(self):
        self.closed = True


class _FakeEvent:
    def record(self, stream):
        pass

    def synchronize(self):
        pass


def test_served_loop_admits_retires_and_drains_on_the_host():
    """The request loop with stand-ins for the batch and its events: every
    request is solved once; an admission refused for lack of room waits for
    a retirement; each force history comes back whole, in order, drained
    before the library's ring would wrap (one request runs 60 periods of a
    static cylinder on two levels, about 180k finest steps)."""
    specs = wl.batch(8, seed=3)
    periods = [0.2] * 8
    specs[0] = wl.cylinder(D=40, levels=2)
    periods[0] = 60.0
    reqs = [sv.Request(i, s, 0.001 * i, p) for i, (s, p) in enumerate(zip(specs, periods))]
    budget = max(_FakeBatch.cost(s) for s in specs)  # the largest fits only alone
    made = []

    def factory(*a, **k):
        made.append(_FakeBatch(*a, **k))
        return made[-1]

    results, stats = sv.run_served(reqs, wl.BF16DEV, budget_bytes=budget, keep_forces=True,
                                   batch_factory=factory, event_factory=_FakeEvent)
    b = made[0]
    assert sorted(r.rid for r in results) == list(range(8))
    assert b.closed and not b.live and b.wrapped == 0
    assert stats["refused_admissions"] > 0 and b.peak_live >= 2
    for r in results:
        spec = specs[r.rid]
        assert r.fine_steps == sv.coarse_steps_for(spec, r.periods) << (spec.levels - 1)
        assert np.array_equal(r.forces[:, 0], np.arange(r.fine_steps))
        assert r.admitted_s >= r.arrival_s - 1e-9 and r.done_s >= r.admitted_s


class _FakeDomain:
    """Stand-in for a single-instance context whose creation takes a while."""

    SETUP_S = 0.05

    def __init__(self, spec, stream=None):
        import time

        time.sleep(self.SETUP_S)
        self.spec, self.n, self.drained = spec, 0, 0

    def step(self, n):
        self.n += n

    def sync(self):
        pass

    def forces(self, cap=1 << 20):
        total = self.n << (self.spec.levels - 1)
        rows = np.zeros((total - self.drained, 3))
        rows[:, 0] = np.arange(self.drained, total)
        self.drained = total
        return rows

    def close(self):
        pass


def test_plain_form_times_its_set_up_apart():
    """run_sequential stops its clock while a context is set up: the set-up
    is reported as setup_s and is in neither the wall time nor the latencies;
    every request's force history comes back whole."""
    specs = wl.batch(4, seed=5)
    reqs = [sv.Request(i, s, 0.0, 0.1) for i, s in enumerate(specs)]
    results, stats = sv.run_sequential(reqs, wl.F32, keep_forces=True, domain_factory=_FakeDomain)
    assert stats["setup_s"] >= 4 * _FakeDomain.SETUP_S
    assert stats["wall_s"] < 4 * _FakeDomain.SETUP_S  # the stepping of the stand-in takes no time
    assert max(r.latency_s for r in results) <= stats["wall_s"] + 1e-9
    for r in results:
        assert np.array_equal(r.forces[:, 0], np.arange(r.fine_steps))
