"""Batches (sbot_batch_*): many instances in one slot pool, stepped together.

Each instance in a mixed batch must evolve exactly as it does alone: its
populations against the FP64 oracle at the parity tolerance (1e-12 relative
L2, all levels), its forces against the oracle's, and -- FP64 and FP32 alike
-- bit for bit against the same instance run alone on the GPU (each cell's
arithmetic does not depend on which other blocks share a launch).
"""
import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, initial_fields, oracle_from_spec, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def set_initial(inst, spec):
    for l in range(spec.levels):
        inst.set_fields(l, *initial_fields(spec, l))


def small_wing(storage=wl.F64):
    spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=storage,
                   heave_chords=1.0)
    spec.body.period = 400.0
    spec.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    return spec


def refined_tgv(storage=wl.F64):
    n0, levels = 32, 2
    nf = n0 << (levels - 1)
    spec = wl.DomainSpec("ref2", n0, n0, levels=levels, block=8, tau_finest=0.7, storage=storage,
                         boxes=[(1, nf * 0.2, nf * 0.25, nf * 0.7, nf * 0.6)], init="tgv", tgv_u0=0.03,
                         tgv_offset=0.5)
    return spec


def mix(storage=wl.F64):
    """instances of different sizes, level counts, boundaries and bodies"""
    return [
        wl.cylinder(D=10, levels=3, block=8, storage=storage, re=100.0),
        wl.tgv(n=64, block=8, storage=storage),
        small_wing(storage),
        refined_tgv(storage),
        wl.DomainSpec("bc", 64, 32, levels=1, block=8, bc=(1, 2, 3, 3), tau_finest=0.6, u_in=(0.05, 0.0),
                      storage=storage),
    ]


def compare_to_oracle(g, o, spec, tol):
    for l in range(spec.levels):
        t = o.types(l)
        assert np.array_equal(g.types(l), t), f"{spec.name}: cell kinds differ on level {l}"
        mask = t == 1
        if not mask.any():
            continue
        err = rel_l2(g.populations(l)[:, mask], o.populations(l)[:, mask])
        assert err <= tol, f"{spec.name} level {l}: rel L2 {err:.3e}"
    if spec.body is not None:
        fg, fo = g.forces(), o.forces()
        assert fg.shape == fo.shape
        scale = np.abs(fo[:, :2]).max()
        np.testing.assert_allclose(fg[:, :2], fo[:, :2], rtol=1e-10, atol=1e-11 * scale)  # as in the parity tests


def test_mixed_batch_matches_oracle_and_alone():
    from paper_2402_04606_gb300.native import Batch, Domain

    specs = mix(wl.F64)
    b = Batch(len(specs) + 2, block=8, storage=wl.F64)
    insts = []
    for s in specs:
        i = b.admit(s)
        set_initial(i, s)
        insts.append(i)
    assert b.info()["live"] == len(specs)
    steps = 24
    b.step(steps)
    for s, i in zip(specs, insts):
        assert i.coarse_steps() == steps
        o = init_oracle(oracle_from_spec(s), s)
        o.step(steps)
        compare_to_oracle(i, o, s, TOL64)
        alone = Domain(s)
        set_initial(alone, s)
        alone.step(steps)
        for l in range(s.levels):
            assert np.array_equal(alone.populations(l), i.populations(l)), f"{s.name}: batch != alone on level {l}"
        alone.close()
    b.close()


def test_fp32_batch_bitwise_equal_to_alone():
    from paper_2402_04606_gb300.native import Batch, Domain

    specs = mix(wl.F32)
    b = Batch(len(specs), block=8, storage=wl.F32)
    insts = []
    for s in specs:
        i = b.admit(s)
        set_initial(i, s)
        insts.append(i)
    b.step(30)
    for s, i in zip(specs, insts):
        alone = Domain(s)
        set_initial(alone, s)
        alone.step(30)
        for l in range(s.levels):
            assert np.array_equal(alone.populations(l), i.populations(l)), f"{s.name}: batch != alone on level {l}"
        if s.body is not None:
            assert np.array_equal(alone.forces(), i.forces())
        alone.close()
    b.close()


def test_admission_mid_run_and_retire():
    """an instance admitted while others run keeps its own clock; retiring
    one leaves the others untouched"""
    from paper_2402_04606_gb300.native import Batch

    s_a = wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=100.0)
    s_b = small_wing(wl.F64)
    s_c = refined_tgv(wl.F64)
    b = Batch(3, block=8, storage=wl.F64)
    a = b.admit(s_a)
    set_initial(a, s_a)
    b.step(7)  # odd: level 0 of the batch now runs on the other buffer parity
    bb = b.admit(s_b)
    set_initial(bb, s_b)
    b.step(10)
    c = b.admit(s_c)
    set_initial(c, s_c)
    b.step(5)
    b.retire(a)
    b.step(4)
    assert bb.coarse_steps() == 19 and c.coarse_steps() == 9
    for s, inst, n in ((s_b, bb, 19), (s_c, c, 9)):
        o = init_oracle(oracle_from_spec(s), s)
        o.step(n)
        compare_to_oracle(inst, o, s, TOL64)
    # the freed slot is reused
    a2 = b.admit(s_a)
    assert a2.slot == 0
    set_initial(a2, s_a)
    b.step(3)
    o = init_oracle(oracle_from_spec(s_a), s_a)
    o.step(3)
    compare_to_oracle(a2, o, s_a, TOL64)
    b.close()


def test_admission_refused_over_budget_or_capacity():
    from paper_2402_04606_gb300.native import ERR_OOM, Batch, SbotError

    s = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    probe = Batch(1, block=8, storage=wl.F32)
    probe.admit(s)
    need = probe.info()["bytes"]
    probe.close()
    b = Batch(4, block=8, storage=wl.F32, budget_bytes=int(need * 2.5))
    b.admit(s)
    b.admit(s)
    with pytest.raises(SbotError) as e:
        b.admit(s)
    assert e.value.status == ERR_OOM
    assert b.info()["live"] == 2
    b.step(2)  # the batch still steps after a refusal
    b.close()
    full = Batch(1, block=8, storage=wl.F32)
    full.admit(s)
    with pytest.raises(SbotError) as e:
        full.admit(s)
    assert e.value.status == ERR_OOM
    full.close()


def test_batch_rejects_mismatched_storage_or_block():
    from paper_2402_04606_gb300.native import ERR_ARG, Batch, SbotError

    b = Batch(2, block=8, storage=wl.F32)
    with pytest.raises(SbotError) as e:
        b.admit(wl.tgv(n=64, block=16, storage=wl.F32))
    assert e.value.status == ERR_ARG
    with pytest.raises(SbotError) as e:
        b.admit(wl.tgv(n=64, block=8, storage=wl.F64))
    assert e.value.status == ERR_ARG
    assert b.info()["live"] == 0
    b.close()
