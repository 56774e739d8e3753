"""The persistent step kernel (SBOT_TUNE_PERSISTENT): one cooperative launch
per coarse step (or per several, SBOT_TUNE_STEPS_PER_LAUNCH) that walks
Algorithm 1's phases over every instance, against the per-phase CUDA graphs
of the same steps.

Each cell's arithmetic is the same code on both paths, so with the same cell
mapping (blocks of 8: one cell per thread everywhere; or the vector mapping
forced everywhere) populations and forces must be equal bit for bit: on the
refined cylinder, the flapping wing whose refinement follows it, and a batch
of uneven instances.  The oracle comparisons of the other GPU tests run on
the persistent path (the default).  A wait limit of zero makes the launch
give up and report SBOT_ERR_TIMEOUT, with no trap and no hang, after which
the device keeps working.
"""
import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, initial_fields, oracle_from_spec, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def small_wing(storage):
    spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=storage,
                   heave_chords=1.0)
    spec.body.period = 400.0
    spec.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    return spec


def pitching_wing(storage):
    """a moving body whose refinement is planned once (no re-tagging): the
    small wing pitching without heave, inside a wider refined margin"""
    spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=storage,
                   heave_chords=0.0)
    spec.body.period = 400.0
    spec.margin = (0.0, 18.0, 10.0) + (0.0,) * 5
    spec.retag = 0
    return spec


def run(spec, persistent, steps, vec=None, per_launch=None, launches=None):
    from paper_2402_04606_gb300.native import (TUNE_PERSISTENT, TUNE_STEPS_PER_LAUNCH, TUNE_VECTOR_MIN_CELLS,
                                               Domain)

    g = Domain(spec)
    g.set_tuning(TUNE_PERSISTENT, persistent)
    if per_launch is not None:
        g.set_tuning(TUNE_STEPS_PER_LAUNCH, per_launch)
    if vec is not None:
        g.set_tuning(TUNE_VECTOR_MIN_CELLS, vec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    g.step(1)
    n0 = g.profile(4)[0]
    g.step(steps - 1)
    if launches is not None:
        launches.append(g.profile(4)[0] - n0)
    out = [g.populations(l) for l in range(spec.levels)], (g.forces() if spec.body is not None else None)
    g.close()
    return out


def same(a, b):
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    if a[1] is not None:
        assert np.array_equal(a[1], b[1])


@pytest.mark.parametrize("storage", [wl.F64, wl.F32, wl.BF16DEV])
@pytest.mark.parametrize("per_launch", [1, 8])
def test_persistent_equals_graphs_cylinder(storage, per_launch):
    spec = wl.cylinder(D=10, levels=3, block=8, storage=storage, re=100.0)
    same(run(spec, 1, 25, per_launch=per_launch), run(spec, 0, 25))


@pytest.mark.parametrize("storage", [wl.F32, wl.F16DEV])
@pytest.mark.parametrize("per_launch", [1, 8])
def test_persistent_equals_graphs_moving_wing(storage, per_launch):
    """the wing whose refinement follows it: several steps go into one launch
    between re-tags of its footprint"""
    spec = small_wing(storage)
    same(run(spec, 1, 30, per_launch=per_launch), run(spec, 0, 30))


@pytest.mark.parametrize("vec", [0, -1])
def test_persistent_equals_graphs_blocks_of_16(vec):
    """blocks of 16 with the vector mapping everywhere (0) or nowhere (-1)"""
    spec = wl.cylinder(D=20, levels=3, block=16, storage=wl.F32, re=100.0)
    same(run(spec, 1, 12, vec), run(spec, 0, 12, vec))


def test_persistent_fp64_matches_oracle_blocks_of_16():
    """the vector mapping inside the persistent kernel against the oracle"""
    spec = wl.cylinder(D=20, levels=3, block=16, storage=wl.F64, re=100.0)
    pops, forces = run(spec, 1, 10, vec=0)
    o = init_oracle(oracle_from_spec(spec), spec)
    o.step(10)
    for l in range(spec.levels):
        m = o.types(l) == 1
        assert rel_l2(pops[l][:, m], o.populations(l)[:, m]) <= 1e-12
    fo = o.forces()
    np.testing.assert_allclose(forces[:, :2], fo[:, :2], rtol=1e-10, atol=1e-11 * np.abs(fo[:, :2]).max())


def test_persistent_batch_equals_graphs():
    from paper_2402_04606_gb300.native import TUNE_PERSISTENT, Batch

    specs = [wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0), small_wing(wl.F32),
             wl.tgv(n=64, block=8, storage=wl.F32),
             wl.DomainSpec("bc", 64, 32, levels=1, block=8, bc=(1, 2, 3, 3), tau_finest=0.6, u_in=(0.05, 0.0),
                           storage=wl.F32)]
    res = []
    for persistent in (1, 0):
        b = Batch(8, block=8, storage=wl.F32)
        b.set_tuning(TUNE_PERSISTENT, persistent)
        insts = []
        for s in specs:
            i = b.admit(s)
            for l in range(s.levels):
                i.set_fields(l, *initial_fields(s, l))
            insts.append(i)
        b.step(16)
        res.append([([i.populations(l) for l in range(s.levels)], i.forces() if s.body is not None else None)
                    for i, s in zip(insts, specs)])
        b.close()
    for a, c in zip(*res):
        same(a, c)


@pytest.mark.parametrize("case", ["cylinder", "pitching_wing"])
def test_several_steps_per_launch_equal_graphs(case):
    """SBOT_TUNE_STEPS_PER_LAUNCH 4: 25 steps after the first as 6 launches
    of 4 steps and one of one, equal bit for bit to the graphs; the
    dependencies between consecutive steps inside one launch (buffers, the
    halo copies, a moving body's poses and geometries, the force sums' term
    slots) are what this checks"""
    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0) if case == "cylinder" \
        else pitching_wing(wl.F32)
    n = []
    a = run(spec, 1, 26, per_launch=4, launches=n)
    same(a, run(spec, 0, 26))
    assert n == [7]


def test_several_steps_per_launch_batch_equals_graphs():
    from paper_2402_04606_gb300.native import TUNE_PERSISTENT, TUNE_STEPS_PER_LAUNCH, Batch

    specs = [wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0), pitching_wing(wl.F32),
             wl.tgv(n=64, block=8, storage=wl.F32)]
    res = []
    for persistent in (1, 0):
        b = Batch(8, block=8, storage=wl.F32)
        b.set_tuning(TUNE_PERSISTENT, persistent)
        b.set_tuning(TUNE_STEPS_PER_LAUNCH, 3)
        insts = []
        for s in specs:
            i = b.admit(s)
            for l in range(s.levels):
                i.set_fields(l, *initial_fields(s, l))
            insts.append(i)
        b.step(16)
        res.append([([i.populations(l) for l in range(s.levels)], i.forces() if s.body is not None else None)
                    for i, s in zip(insts, specs)])
        b.close()
    for a, c in zip(*res):
        same(a, c)


def test_tuning_knobs_validate_and_round_trip():
    """each knob of the step forms takes its documented range, reads back what
    was set, and rejects a value outside it with SBOT_ERR_ARG"""
    from paper_2402_04606_gb300 import native as nv

    g = nv.Domain(wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0))
    cases = [(nv.TUNE_PERSISTENT, 0, 3), (nv.TUNE_STEP_THREADS, 768, 512), (nv.TUNE_SPIN_NS, 10**6, -1),
             (nv.TUNE_BULK_ROUNDS, 4, 0), (nv.TUNE_BULK_ROUNDS, 64, 65), (nv.TUNE_IBM_THREADS, 512, 300),
             (nv.TUNE_CRIT_BLOCKS, 2, -1), (nv.TUNE_CRIT_BLOCKS, 64, 65), (nv.TUNE_STEPS_PER_LAUNCH, 1, 0),
             (nv.TUNE_STEPS_PER_LAUNCH, 16, 17), (nv.TUNE_VEC_WAVES, 2, -2), (nv.TUNE_VEC_WAVES, 64, 65)]
    for what, good, bad in cases:
        g.set_tuning(what, good)
        assert g.tuning(what) == good
        with pytest.raises(nv.SbotError) as e:
            g.set_tuning(what, bad)
        assert e.value.status == nv.ERR_ARG
        assert g.tuning(what) == good
    g.close()


@pytest.mark.parametrize("storage", [wl.F32, wl.BF16DEV])
def test_vector_kernel_waves_do_not_change_results(storage):
    """SBOT_TUNE_VEC_WAVES changes only how many thread blocks sweep a
    vector-kernel launch's list (short-lived blocks, 2 or the default 8 waves
    of grid-stride blocks): the populations and forces are the same bit for
    bit"""
    from paper_2402_04606_gb300 import native as nv

    spec = wl.cylinder(D=40, levels=3, block=16, storage=storage, re=100.0)  # the headline geometry
    res = []
    for waves in (8, 0, 2):
        g = nv.Domain(spec)
        g.set_tuning(nv.TUNE_PERSISTENT, 0)
        g.set_tuning(nv.TUNE_VECTOR_MIN_CELLS, 0)
        g.set_tuning(nv.TUNE_VEC_WAVES, waves)
        assert g.tuning(nv.TUNE_VEC_WAVES) == waves
        for l in range(spec.levels):
            g.set_fields(l, *initial_fields(spec, l))
        g.step(6)
        res.append(([g.populations(l) for l in range(spec.levels)], g.forces()))
        g.close()
    same(res[0], res[1])
    same(res[0], res[2])


def test_fewer_steps_than_a_launch_holds_run_one_by_one():
    """step counts below SBOT_TUNE_STEPS_PER_LAUNCH (and the remainder of a
    longer call) run as one-step launches, with the same result as one call"""
    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    from paper_2402_04606_gb300.native import TUNE_STEPS_PER_LAUNCH, Domain

    def go(calls):
        g = Domain(spec)
        g.set_tuning(TUNE_STEPS_PER_LAUNCH, 4)
        for l in range(spec.levels):
            g.set_fields(l, *initial_fields(spec, l))
        g.step(1)  # the first step also runs the set-up launches
        n0 = g.profile(4)[0]
        for n in calls:
            g.step(n)
        out = [g.populations(l) for l in range(spec.levels)], g.forces()
        n = g.profile(4)[0] - n0
        g.close()
        return out, n

    a, na = go([11])          # 4 + 4 + 1 + 1 + 1
    b, nb = go([3, 3, 5])     # 1 + 1 + 1, 1 + 1 + 1, 4 + 1
    same(a, b)
    assert (na, nb) == (5, 8)


def test_wait_limit_reports_timeout_and_device_recovers():
    from paper_2402_04606_gb300.native import ERR_TIMEOUT, TUNE_SPIN_NS, Domain, SbotError

    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    g = Domain(spec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    g.step(1)
    g.set_tuning(TUNE_SPIN_NS, 0)  # no wait at all: the first dependency not yet met stops the launch
    g.step(2)
    with pytest.raises(SbotError) as e:
        g.checksum()
    assert e.value.status == ERR_TIMEOUT
    g.close()
    # the device and a new context work as before
    a = run(spec, 1, 5)
    b = run(spec, 0, 5)
    same(a, b)
