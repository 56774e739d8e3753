"""The synthetic input recipes: the 64-instance batch and the serving arrivals.

- every batch instance lies in the stated ranges: coarsest nx in {256, 512,
  1024, 2048} with ny = nx / 2, 2-4 levels, a cylinder of D = 40 or an
  ellipse wing of chord 64 and thickness 0.12 c, Re in [50, 400] (recovered
  from the relaxation time of Eq. 9), wing pitch amplitude in [16, 64]
  degrees;
- the recipe is a function of its seed alone;
- the planner gives the batch 48,107,008 cell updates per coarse step;
- the arrivals have the stated mean rate, and their request mix is the batch
  recipe under its own seed.
"""
import math

import numpy as np

from paper_2402_04606_gb300 import native
from paper_2402_04606_gb300 import workloads as wl


def reynolds(spec):
    nu = (spec.tau_finest - 0.5) / 3.0  # Eq. 9 on the finest level
    return spec.body.u_ref * spec.body.l_ref / nu


def test_batch_instances_lie_in_the_stated_ranges():
    specs = wl.batch(64, seed=0)
    assert len(specs) == 64
    kinds = set()
    for s in specs:
        assert s.nx0 in (256, 512, 1024, 2048) and s.ny0 == s.nx0 // 2
        assert 2 <= s.levels <= 4
        assert s.storage == wl.BF16DEV and s.block == 16
        assert 50.0 - 1e-9 <= reynolds(s) <= 400.0 + 1e-9
        b = s.body
        if b.kind == 0:
            assert b.a == b.b == 20.0 and b.motion == 0
        else:
            assert b.kind == 1 and b.a == 32.0 and math.isclose(b.b, 0.12 * 32.0)
            assert math.radians(16.0) - 1e-12 <= b.alpha_amp <= math.radians(64.0) + 1e-12
        kinds.add(b.kind)
    assert kinds == {0, 1}


def test_batch_recipe_depends_on_its_seed_only():
    a, b, c = wl.batch(64, seed=0), wl.batch(64, seed=0), wl.batch(64, seed=1)
    assert [s.name for s in a] == [s.name for s in b]
    assert [s.tau_finest for s in a] == [s.tau_finest for s in b]
    assert [s.name for s in a] != [s.name for s in c]


def test_batch_cell_updates_per_coarse_step():
    total = 0
    for s in wl.batch(64, seed=0):
        for l in range(s.levels):
            interior = int((native.plan_blocks(s, l, coarse_step=0) == 1).sum())
            total += interior * s.block * s.block << l
    assert total == 48_107_008


def test_serving_arrivals_rate_and_mix():
    t, specs = wl.serving_arrivals(4000, 20.0, seed=1)
    assert np.all(np.diff(t) > 0) and len(specs) == 4000
    assert abs(len(t) / t[-1] - 20.0) < 1.0  # 4000 arrivals: rate within 5 %
    t2, specs2 = wl.serving_arrivals(4000, 20.0, seed=1)
    assert np.array_equal(t, t2)
    assert [s.name for s in specs[:16]] == [s.name for s in wl.batch(16, seed=1001)]
