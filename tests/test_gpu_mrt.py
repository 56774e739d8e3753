"""The MRT and LES collisions (Sec. 2.1) on the GPU against the FP64 oracle.

FP64 storage: relative L2 of the populations <= 1e-12 on a periodic grid
(scalar and vector kernels, and the shared-memory staged kernel), the
refined cylinder with its forces and the moving wing with the refined region
following it.  Reduced storage: velocity against the oracle as for BGK.  With
every rate equal to 1/tau on one level MRT equals BGK up to rounding.
"""
import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, oracle_from_spec, rel_l2
from tests.test_gpu_parity import TOL64, compare_forces, compare_populations, gpu_domain, velocity_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


@pytest.mark.parametrize("block,vec", [(16, -1), (16, 0), (32, 0)])
def test_mrt_tgv_fp64(block, vec):
    from paper_2402_04606_gb300.native import TUNE_VECTOR_MIN_CELLS

    spec = wl.with_mrt(wl.tgv(n=128, block=block, storage=wl.F64))
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, vec)
    o.step(100)
    g.step(100)
    compare_populations(g, o, 1, TOL64)


def test_mrt_staged_kernel_fp64():
    from paper_2402_04606_gb300.native import TUNE_STAGED, TUNE_VECTOR_MIN_CELLS

    spec = wl.with_mrt(wl.tgv(n=128, block=16, storage=wl.F64), (1.2, 1.1, 1.3))
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
    g.set_tuning(TUNE_STAGED, 1)
    o.step(50)
    g.step(50)
    compare_populations(g, o, 1, TOL64)


def test_mrt_refined_cylinder_fp64():
    spec = wl.with_mrt(wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=300.0))
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(40)
    g.step(40)
    compare_populations(g, o, 3, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


def test_mrt_moving_wing_fp64():
    spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=wl.F64,
                   heave_chords=1.0)
    spec.body.period = 400.0
    spec.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    spec = wl.with_mrt(spec)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(30)
    g.step(30)
    for l in range(3):
        assert np.array_equal(g.blocks(l), o.blocks(l))
    compare_populations(g, o, 3, TOL64)
    fg, fo = g.forces(), o.forces()
    b = spec.body
    atol = max(1e-11 * np.abs(fo[:, :2]).max(), 4.0 * b.n_markers * o.ds() * np.spacing(max(b.x0)))
    np.testing.assert_allclose(fg[:, :2], fo[:, :2], rtol=1e-10, atol=atol)


@pytest.mark.parametrize("storage,tol", [(wl.F32, 1e-5), (wl.F16DEV, 5e-4), (wl.BF16DEV, 2e-3)])
def test_mrt_reduced_storage(storage, tol):
    spec = wl.with_mrt(wl.tgv(n=512, block=16, storage=storage))
    ref = wl.replace_storage(spec, wl.F64)
    o = init_oracle(oracle_from_spec(ref), ref)
    g = gpu_domain(spec)
    o.step(20)
    g.step(20)
    assert velocity_error(g, o, 1) <= tol


def test_mrt_with_equal_rates_is_bgk():
    tau = 0.8
    a = gpu_domain(wl.with_mrt(wl.tgv(n=64, block=16, storage=wl.F64, tau=tau), (1 / tau,) * 3))
    b = gpu_domain(wl.tgv(n=64, block=16, storage=wl.F64, tau=tau))
    a.step(200)
    b.step(200)
    assert rel_l2(a.populations(0), b.populations(0)) <= 1e-13


def test_batch_keeps_one_collision_kind():
    from paper_2402_04606_gb300.native import Batch, SbotError

    b = Batch(2, block=16, storage=wl.F32)
    b.admit(wl.tgv(n=64, block=16, storage=wl.F32))
    with pytest.raises(SbotError):
        b.admit(wl.with_mrt(wl.tgv(n=64, block=16, storage=wl.F32)))
    b.close()


@pytest.mark.parametrize("block,vec", [(16, -1), (32, 0)])
def test_les_tgv_fp64(block, vec):
    """LES (Smagorinsky) near tau = 1/2, where the eddy viscosity matters."""
    from paper_2402_04606_gb300.native import TUNE_VECTOR_MIN_CELLS

    spec = wl.with_les(wl.tgv(n=128, block=block, storage=wl.F64, tau=0.505, u0=0.05), 0.17)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, vec)
    o.step(100)
    g.step(100)
    compare_populations(g, o, 1, TOL64)


def test_les_refined_cylinder_fp64():
    spec = wl.with_les(wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=1000.0), 0.15)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(40)
    g.step(40)
    compare_populations(g, o, 3, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


def test_les_fp32():
    spec = wl.with_les(wl.tgv(n=512, block=16, storage=wl.F32, tau=0.505, u0=0.05))
    ref = wl.replace_storage(spec, wl.F64)
    o = init_oracle(oracle_from_spec(ref), ref)
    g = gpu_domain(spec)
    o.step(20)
    g.step(20)
    assert velocity_error(g, o, 1) <= 1e-5
