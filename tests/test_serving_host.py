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
