"""The continuous-batching request loop (paper_2402_04606_gb300.serving).

Requests arrive while others run; each result must be the same in the mix as
alone: with the same storage, the force history of every served solve equals,
bit for bit, the one of the same request run on its own context.  Mean drag
with reduced-precision storage is compared with the FP64 oracle.
"""
import numpy as np
import pytest

from paper_2402_04606_gb300 import serving as sv
from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, oracle_from_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def small_requests():
    wing = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=wl.F32,
                   heave_chords=1.0)
    wing.body.period = 400.0
    wing.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    cyl3 = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    cyl2 = wl.cylinder(D=10, levels=2, block=8, storage=wl.F32, re=150.0)
    pitch = wl.wing(c=16, levels=2, re=120.0, n_markers=48, block=8, domain_chords=8.0, storage=wl.F32,
                    heave_chords=0.0)
    pitch.body.motion = 1
    pitch.body.period = 300.0
    pitch.margin = (0.0, 12.0) + (0.0,) * 6
    specs = [cyl3, wing, cyl2, pitch, cyl3]
    arrivals = [0.0, 0.01, 0.03, 0.05, 0.08]
    periods = [0.15, 0.5, 0.1, 0.4, 0.1]
    return [sv.Request(i, s, t, p) for i, (s, t, p) in enumerate(zip(specs, arrivals, periods))]


def test_served_results_equal_alone():
    reqs = small_requests()
    served, stats = sv.run_served(reqs, storage=wl.F32, block=8, chunk=8, max_instances=3, keep_forces=True)
    alone, _ = sv.run_sequential(reqs, storage=wl.F32, block=8, keep_forces=True)
    assert stats["requests"] == len(reqs)
    assert stats["p99_time_to_result_s"] >= stats["p50_time_to_result_s"] > 0
    by_id = {r.rid: r for r in alone}
    for r in served:
        a = by_id[r.rid]
        assert r.fine_steps == a.fine_steps
        assert r.forces.shape == a.forces.shape
        assert np.isfinite(r.forces).all()
        assert np.array_equal(r.forces, a.forces), f"request {r.rid} ({r.name}) differs in the mix"


def test_admission_waits_for_memory():
    """with a budget for one and a half solves, the others wait for retirements"""
    from paper_2402_04606_gb300.native import Batch

    reqs = small_requests()
    for r in reqs:
        r.arrival_s = 0.0  # all at once: the budget, not the arrivals, paces admission
    probe = Batch(1, block=8, storage=wl.F32)
    probe.admit(reqs[0].spec)
    need = probe.info()["bytes"]
    probe.close()
    served, stats = sv.run_served(reqs, storage=wl.F32, block=8, chunk=8, budget_bytes=int(1.5 * need),
                                  keep_forces=True)
    assert stats["requests"] == len(reqs)
    assert stats["refused_admissions"] > 0
    alone, _ = sv.run_sequential(reqs, storage=wl.F32, block=8, keep_forces=True)
    by_id = {r.rid: r for r in alone}
    for r in served:
        assert np.array_equal(r.forces, by_id[r.rid].forces)


@pytest.mark.parametrize("storage", [wl.F32, wl.F16DEV, wl.BF16DEV])
def test_mean_drag_against_fp64_oracle(storage):
    # mean drag over the run of a refined cylinder: reduced storage within
    # 0.5% of the FP64 oracle (the bound the method's precision is held to)
    spec = wl.cylinder(D=10, levels=3, block=8, storage=storage, re=100.0)
    req = [sv.Request(0, spec, 0.0, 0.33)]
    served, _ = sv.run_served(req, storage=storage, block=8, chunk=16, keep_forces=True)
    n = served[0].fine_steps
    o = init_oracle(oracle_from_spec(spec), spec)
    o.step(n >> (spec.levels - 1))
    fo = o.forces()[:n]
    fg = served[0].forces
    cd_o, cd_g = fo[:, 0].mean(), fg[:, 0].mean()
    assert abs(cd_g - cd_o) <= 5e-3 * abs(cd_o), (cd_g, cd_o)
