"""Edge cases of the GPU path against the oracle or against itself.

- zero coarse steps change nothing;
- a batch emptied by retirements still steps, and a solve admitted into
  the freed slots equals the same solve alone bit for bit;
- the smallest body the library accepts (3 markers);
- a body whose marker box spans more than 16 blocks per side, which takes
  the IBM's path without the block-slot table (FP32 storage by velocity
  and force against the FP64 oracle);
- FP16 deviation storage through the IBM of a moving body.
"""
import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, oracle_from_spec
from tests.test_gpu_parity import TOL64, compare_forces, compare_populations, gpu_domain, velocity_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def test_zero_steps_change_nothing():
    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=100.0)
    g = gpu_domain(spec)
    g.step(3)
    before = [g.populations(l) for l in range(3)]
    n0 = g.forces().shape[0]
    g.step(0)
    for l in range(3):
        assert np.array_equal(g.populations(l), before[l])
    assert g.forces().shape[0] == 0 and n0 > 0  # nothing new since the last read


def test_emptied_batch_steps_and_reuses_slots():
    from paper_2402_04606_gb300.native import Batch, Domain

    from tests.helpers import initial_fields

    a = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    w = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=wl.F32,
                heave_chords=1.0)
    w.body.period = 400.0
    w.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    b = Batch(2, block=8, storage=wl.F32)
    i0 = b.admit(a)
    b.step(4)
    b.retire(i0)
    b.step(2)  # no live instance
    i1 = b.admit(w)  # into the freed slots
    b.step(6)
    alone = Domain(w)
    for l in range(w.levels):
        alone.set_fields(l, *initial_fields(w, l))
    alone.step(6)
    for l in range(w.levels):
        assert np.array_equal(i1.populations(l), alone.populations(l))
    assert np.array_equal(i1.forces(), alone.forces())
    b.close()


def test_three_marker_body_fp64():
    spec = wl.cylinder(D=10, levels=2, block=8, storage=wl.F64, re=100.0, n_markers=3)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(20)
    g.step(20)
    compare_populations(g, o, 2, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


def test_body_wider_than_the_slot_table_fp32():
    # an ellipse 140 cells long on blocks of 8: its marker box spans 19 blocks
    spec = wl.wing(c=140, levels=2, re=200.0, n_markers=282, block=8, domain_chords=3.0, storage=wl.F64,
                   thickness=10.0 / 140.0, heave_chords=0.0)
    spec.body.motion = 0
    spec.body.alpha_mean = 0.0
    spec.margin = (0.0, 10.0) + (0.0,) * 6
    spec.retag = 0
    spec.init, spec.tgv_u0 = "tgv", 0.02  # a flow past the static body from the first step
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(wl.replace_storage(spec, wl.F32))
    o.step(10)
    g.step(10)
    assert velocity_error(g, o, 2) <= 1e-5
    fo, fg = o.forces(), g.forces()
    np.testing.assert_allclose(fg[:, :2], fo[:, :2], rtol=0, atol=1e-4 * np.abs(fo[:, :2]).max())


def test_fp16_moving_wing_against_fp64():
    spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=wl.F64,
                   heave_chords=1.0)
    spec.body.period = 400.0
    spec.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(wl.replace_storage(spec, wl.F16DEV))
    o.step(30)
    g.step(30)
    assert velocity_error(g, o, 3) <= 5e-3
