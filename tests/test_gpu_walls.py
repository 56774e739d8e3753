"""Walls and solid obstacles (reading R15) on the GPU against the oracle.

FP64 populations <= 1e-12 relative L2 (cell kinds, solid cells included,
equal): plane Couette flow between half-way walls and with the interpolated
flat wall at link fractions below and above one half; the lid-driven cavity
with its cylinder as a solid (one level and two levels, scalar and vector
kernels) and as an IBM body; exact mass conservation in a closed cavity;
FP32 storage by velocity.
"""
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, oracle_from_spec
from tests.test_gpu_parity import TOL32_U, TOL64, compare_forces, compare_populations, gpu_domain, velocity_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def channel(y0=None, tau=0.8, n=32):
    bc = (wl.BC_PERIODIC, wl.BC_PERIODIC, wl.BC_WALL, wl.BC_WALL)
    solid = (0, 0.0, 0.0, 0.0) if y0 is None else (2, y0, 0.0, 0.0)
    return wl.DomainSpec("couette", nx0=n, ny0=n, levels=1, block=16, bc=bc, tau_finest=tau, storage=wl.F64,
                         uwall=(0.0,) * 6 + (0.02, 0.0), solid=solid)


@pytest.mark.parametrize("y0", [None, 2.3, 2.7])
def test_couette_walls_fp64(y0):
    spec = channel(y0)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(300)
    g.step(300)
    compare_populations(g, o, 1, TOL64)


@pytest.mark.parametrize("levels,vec", [(1, -1), (1, 0), (2, -1)])
def test_cavity_solid_cylinder_fp64(levels, vec):
    from paper_2402_04606_gb300.native import TUNE_VECTOR_MIN_CELLS

    # two levels need room between the refined cylinder and the walls
    spec = wl.cavity(L=96 if levels == 1 else 160, re=100.0, mode="bounce", storage=wl.F64, levels=levels)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, vec)
    assert (g.types(levels - 1) == 4).sum() > 0
    o.step(100)
    g.step(100)
    compare_populations(g, o, levels, TOL64)


def test_cavity_ibm_cylinder_fp64():
    spec = wl.cavity(L=96, re=100.0, mode="ibm", storage=wl.F64)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(100)
    g.step(100)
    compare_populations(g, o, 1, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


def test_closed_cavity_conserves_mass_fp64():
    spec = wl.DomainSpec("box", nx0=64, ny0=64, levels=1, block=16, bc=(wl.BC_WALL,) * 4, tau_finest=0.6,
                         storage=wl.F64, uwall=(0.0,) * 6 + (0.05, 0.0))
    g = gpu_domain(spec)
    m0 = g.checksum()[0]
    g.step(500)
    assert abs(g.checksum()[0] - m0) <= 1e-12 * m0


def test_cavity_solid_fp32():
    spec = wl.cavity(L=96, re=100.0, mode="bounce", storage=wl.F32)
    ref = wl.replace_storage(spec, wl.F64)
    o = init_oracle(oracle_from_spec(ref), ref)
    g = gpu_domain(spec)
    o.step(200)
    g.step(200)
    assert velocity_error(g, o, 1) <= TOL32_U
