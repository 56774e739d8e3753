"""The C-ABI library loads without a GPU, exports every function that
include/sbot.h declares, and its host-side topology planner agrees exactly
with the oracle's (integer work: bit-exact)."""
import ctypes as C

import numpy as np
import pytest

from paper_2402_04606_gb300 import build as bld
from paper_2402_04606_gb300 import native
from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import oracle_from_spec, small_pitch_specs


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return native.load()


def test_every_declared_symbol_is_exported(lib):
    names = native.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    spec = wl.tgv(n=32, block=16)
    d, keep = native.domain_desc(spec)
    h = C.c_void_p()
    rc = lib.sbot_create_domain(C.byref(d), None, C.byref(h))
    assert rc != native.OK and not h.value


def test_valid_descriptions_pass_validation(lib):
    # without a GPU a valid description gets past validation and fails only
    # at the device (SBOT_ERR_CUDA), so validation rejects nothing it should take
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for spec in (wl.tgv(n=32, block=16), wl.with_mrt(wl.tgv(n=32, block=16)), wl.with_les(wl.tgv(n=32, block=16)),
                 wl.cavity(L=96, mode="bounce"), wl.cavity(L=96, mode="ibm"), wl.cylinder(D=10, levels=3, block=8),
                 wl.wing(c=16, levels=3, n_markers=50, block=8, domain_chords=8.0)):
        d, keep = native.domain_desc(spec)
        h = C.c_void_p()
        assert lib.sbot_create_domain(C.byref(d), None, C.byref(h)) == native.ERR_CUDA, spec.name
        assert not h.value


def test_invalid_descriptions_are_rejected(lib):
    nan = float("nan")
    for bad in (dict(nx0=30), dict(block=12), dict(levels=0), dict(levels=9), dict(tau_finest=0.5),
                dict(tau_finest=nan), dict(storage=4), dict(bc=(1, 0, 0, 0)), dict(bc=(5, 5, 0, 0)),
                dict(collision=3), dict(collision=-1), dict(les_cs=-0.1), dict(les_cs=1.5), dict(les_cs=nan),
                dict(mrt_rates=(2.5, 1.0, 1.0)), dict(mrt_rates=(1.0, -0.1, 1.0)),
                dict(solid=(3, 0.0, 0.0, 0.0)), dict(solid=(1, 16.0, 16.0, 0.0)),
                dict(solid=(1, 16.0, 16.0, 4.0), retag=1)):
        spec = wl.tgv(n=32, block=16)
        for k, v in bad.items():
            setattr(spec, k, v)
        d, keep = native.domain_desc(spec)
        h = C.c_void_p()
        assert lib.sbot_create_domain(C.byref(d), None, C.byref(h)) == native.ERR_ARG


def _specs():
    out = []
    out.append(wl.DomainSpec("boxes", 16, 16, levels=3, block=8,
                             boxes=[(1, 24.0, 20.0, 70.0, 60.0), (2, 40.0, 36.0, 52.0, 46.0)]))
    out.append(wl.cylinder(D=10, levels=3, block=8))
    out.append(wl.cylinder(D=20, levels=3, block=16))
    w = wl.wing(c=16, levels=3, n_markers=50, block=8, domain_chords=8.0)
    w.body.period = 400.0
    out.append(w)
    out.append(wl.wing(c=32, levels=4, n_markers=100, block=8, domain_chords=10.0))
    out.extend(small_pitch_specs())
    out.append(wl.cylinder_table1(D=16, lx=80.0, ly=60.0, xc=20.0))  # four levels, static body
    out.append(wl.cavity(L=96, re=100.0, mode="ibm"))  # wall sides with an IBM body
    out.append(wl.cavity(L=160, re=100.0, mode="bounce", levels=2))  # wall sides with a solid
    rng = np.random.default_rng(3)
    for k in range(4):
        boxes = []
        for _ in range(3):
            x0, y0 = rng.uniform(0, 200, 2)
            boxes.append((int(rng.integers(1, 4)), x0, y0, x0 + rng.uniform(1, 40), y0 + rng.uniform(1, 40)))
        out.append(wl.DomainSpec(f"rand{k}", 16, 16, levels=4, block=8, boxes=boxes))
    return out


@pytest.mark.parametrize("spec", _specs(), ids=lambda s: s.name)
def test_topology_planner_matches_oracle(lib, spec):
    o = oracle_from_spec(spec)
    for l in range(spec.levels):
        assert np.array_equal(native.plan_blocks(spec, l, coarse_step=0), o.blocks(l)), (spec.name, l)


@pytest.mark.parametrize("spec", small_pitch_specs(), ids=lambda s: s.name)
def test_pitch_motions_planner_matches_oracle(lib, spec):
    from tests.helpers import init_oracle
    o = init_oracle(oracle_from_spec(spec), spec)
    changes = 0
    prev = None
    for n in range(1, 21):
        o.step(1)
        cur = [o.blocks(l) for l in range(spec.levels)]
        for l in range(spec.levels):
            assert np.array_equal(native.plan_blocks(spec, l, coarse_step=n - 1), cur[l]), (n, l)
        if prev is not None and any(not np.array_equal(x, y) for x, y in zip(prev, cur)):
            changes += 1
        prev = cur
    assert changes >= 1


def test_moving_topology_planner_matches_oracle(lib):
    # the oracle re-tags at the start of coarse step n (window [n, n+1]); after
    # n steps its blocks are those of window n-1
    spec = wl.wing(c=16, levels=3, n_markers=50, block=8, domain_chords=8.0)
    spec.body.period = 160.0
    from tests.helpers import init_oracle
    o = init_oracle(oracle_from_spec(spec), spec)
    changes = 0
    prev = None
    for n in range(1, 25):
        o.step(1)
        cur = [o.blocks(l) for l in range(3)]
        for l in range(3):
            assert np.array_equal(native.plan_blocks(spec, l, coarse_step=max(n - 1, 0)), cur[l]), (n, l)
        if prev is not None and any(not np.array_equal(a, b) for a, b in zip(prev, cur)):
            changes += 1
        prev = cur
    assert changes >= 1


@pytest.mark.parametrize("seed", range(24))
def test_random_refinements_match_oracle(lib, seed):
    """Random static refinements (2-5 levels, blocks of 8 or 16, periodic or
    inlet/outlet/symmetry sides): the library's planner and the oracle give
    the same block maps on every level, and refuse the same descriptions (a
    refinement reaching a non-periodic side)."""
    from paper_2402_04606_gb300.native import SbotError

    rng = np.random.default_rng(100 + seed)
    periodic = seed % 2 == 0
    block = int(rng.choice([8, 16]))
    levels = int(rng.integers(2, 6))
    n0 = block * int(rng.integers(2, 5) if periodic else rng.integers(4, 7))
    nf = n0 << (levels - 1)
    # periodic: boxes anywhere (wrapping); other sides: mostly in the middle
    lo, span = (0.0, 0.4) if periodic else (0.3, 0.15)
    boxes = []
    for _ in range(int(rng.integers(1, 5))):
        w, h = rng.uniform(2, span * nf, 2)
        x0 = rng.uniform(lo * nf, (1 - lo) * nf - w)
        y0 = rng.uniform(lo * nf, (1 - lo) * nf - h)
        boxes.append((int(rng.integers(1, levels)), x0, y0, x0 + w, y0 + h))
    bc = (0, 0, 0, 0) if periodic else (1, 2, 3, 3)
    spec = wl.DomainSpec(f"rnd{seed}", n0, n0, levels=levels, block=block, bc=bc, boxes=boxes)
    try:
        o = oracle_from_spec(spec)
    except RuntimeError:
        with pytest.raises(SbotError):
            for l in range(levels):
                native.plan_blocks(spec, l, coarse_step=0)
        return
    for l in range(levels):
        assert np.array_equal(native.plan_blocks(spec, l, coarse_step=0), o.blocks(l)), (seed, l)


@pytest.mark.parametrize("seed", range(6))
def test_random_moving_wings_planner_matches_oracle(lib, seed):
    """Random pitching or flapping wings (amplitude, period, phase, heave and
    stroke angle drawn from a seed): after each of 12 coarse steps the
    oracle's re-tagged block maps equal the library's plan for that step."""
    from tests.helpers import init_oracle

    rng = np.random.default_rng(200 + seed)
    spec = wl.wing(c=16, levels=3, n_markers=50, block=8, domain_chords=8.0,
                   heave_chords=float(rng.uniform(0.0, 1.2)), beta_deg=float(rng.uniform(0.0, 90.0)))
    spec.body.motion = int(rng.choice([1, 2]))
    spec.body.alpha_amp = float(rng.uniform(0.2, 1.1))
    spec.body.period = float(rng.uniform(120.0, 400.0))
    spec.body.phase = float(rng.uniform(0.0, 2.0 * np.pi))
    o = init_oracle(oracle_from_spec(spec), spec)
    for n in range(1, 13):
        o.step(1)
        for l in range(spec.levels):
            assert np.array_equal(native.plan_blocks(spec, l, coarse_step=n - 1), o.blocks(l)), (seed, n, l)
