"""Reduced-precision storage against the FP64 oracle at the stated horizon.

Targets (the precision pattern of this library): velocity relative L2
<= 1e-5 with FP32 storage and <= 2e-3 with FP16 or BF16 deviation storage
after 10,000 finest steps, and mean drag and lift coefficients (Sec. 3.3,
Eq. 19) within 0.5 % of the oracle's.  Compute is FP32 for all three.

Readings of "after 10,000 steps", where a pointwise comparison measures the
arithmetic and not a physical instability:
- the D = 10, 3-level cylinder at Re = 40, below the onset of shedding (its
  steady symmetric wake is stable, so rounding differences are not
  amplified); at Re = 100 the symmetric wake of an exactly centred body is
  unstable and any rounding asymmetry grows into shedding, which the FP64
  oracle never starts;
- the Taylor-Green vortex on 128^2 at tau = 0.52 (it keeps 72 % of its
  amplitude after 10,000 steps; at tau = 0.8 it decays 125-fold and the
  relative error is then a ratio to a vanishing field).
The shedding cylinder (Re = 100, body 0.3 cells off the centre line so that
shedding starts from the geometry, not from round-off) is compared through
its mean coefficients over the last five of 22 periods (developed from about
the 17th; the lift rms carries a slow modulation of about 2 %, so fewer
periods would weigh its phase).

Targets the storage cannot meet are marked as expected failures that state
the measured level; each also has a bound at the measured level, which must
hold.
"""
import math

import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, initial_fields, oracle_from_spec

pytestmark = pytest.mark.gpu

TARGET = {wl.F32: 1e-5, wl.F16DEV: 2e-3, wl.BF16DEV: 2e-3}
NAME = {wl.F32: "f32", wl.F16DEV: "f16dev", wl.BF16DEV: "bf16dev"}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def gpu_run(spec, coarse_steps, chunk=None):
    """the GPU state and force history after `coarse_steps` coarse steps"""
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    forces = []
    done = 0
    chunk = chunk or coarse_steps
    while done < coarse_steps:
        k = min(chunk, coarse_steps - done)
        g.step(k)
        done += k
        if spec.body is not None:
            forces.append(g.forces(cap=1 << 20))
    fields = [g.fields(l) for l in range(spec.levels)]
    g.close()
    return fields, (np.concatenate(forces) if forces else None)


def velocity_error(fields, o, levels):
    num = den = 0.0
    for l in range(levels):
        mask = o.types(l) == 1
        _, ug, vg = fields[l]
        _, uo, vo = o.fields(l)
        num += (((ug - uo) ** 2 + (vg - vo) ** 2)[mask]).sum()
        den += ((uo ** 2 + vo ** 2)[mask]).sum()
    return math.sqrt(num / den)


def check(err, storage, measured_bound, case):
    """the bound at the measured level always; the target as stated, or an
    expected failure that says by how much it is missed"""
    assert err <= measured_bound, f"{case} {NAME[storage]}: {err:.3e} above the measured level {measured_bound:.1e}"
    if err > TARGET[storage]:
        pytest.xfail(f"{case} {NAME[storage]}: velocity L2 {err:.2e} misses the target {TARGET[storage]:.0e}")


# --- the steady cylinder (Re = 40), 10,000 finest steps -----------------------

@pytest.fixture(scope="module")
def steady_oracle():
    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=40.0)
    o = init_oracle(oracle_from_spec(spec, openmp=True), spec)
    o.step(2500)  # 2500 coarse steps = 10,000 finest steps
    return spec, o


# measured on a GB300: FP32 1.2e-6, FP16 4.1e-4, BF16 2.3e-3 (16-bit storage
# holds the deviation from the free-stream equilibrium; with the deviation
# from w_q FP16 gave 1.1e-3 and BF16 2.0e-2)
@pytest.mark.parametrize("storage,measured", [(wl.F32, 1e-5), (wl.F16DEV, 1e-3), (wl.BF16DEV, 3e-3)])
def test_steady_cylinder_velocity_after_10k_finest_steps(steady_oracle, storage, measured):
    spec, o = steady_oracle
    fields, _ = gpu_run(wl.replace_storage(spec, storage), 2500)
    check(velocity_error(fields, o, 3), storage, measured, "cylinder Re 40")


# --- the Taylor-Green vortex at tau = 0.52, 10,000 steps ----------------------

@pytest.fixture(scope="module")
def tgv_oracle():
    spec = wl.tgv(n=128, tau=0.52, storage=wl.F64)
    o = init_oracle(oracle_from_spec(spec, openmp=True), spec)
    o.step(10000)
    return spec, o


# measured on a GB300: FP32 1.4e-6, FP16 9.1e-4, BF16 1.9e-2
@pytest.mark.parametrize("storage,measured", [(wl.F32, 1e-5), (wl.F16DEV, 2e-3), (wl.BF16DEV, 3e-2)])
def test_taylor_green_velocity_after_10k_steps(tgv_oracle, storage, measured):
    spec, o = tgv_oracle
    fields, _ = gpu_run(wl.replace_storage(spec, storage), 10000)
    check(velocity_error(fields, o, 1), storage, measured, "Taylor-Green tau 0.52")


# --- the shedding cylinder (Re = 100): mean coefficients ----------------------

PERIOD = 10.0 / (0.165 * 0.05)  # shedding period D / (St U) in finest steps, St = 0.165
PERIODS = 22                     # developed from about period 17 (measured)


def shedding_spec(storage):
    spec = wl.cylinder(D=10, levels=3, block=8, storage=storage, re=100.0)
    b = spec.body
    spec.body = type(b)(**{**b.__dict__, "x0": (b.x0[0], b.x0[1] + 0.3)})
    return spec


def coefficient_stats(spec, forces, periods=5):
    """Eq. 19 over the last `periods` whole shedding periods of the history:
    mean drag coefficient and the rms of the lift coefficient about its mean"""
    q = 0.5 * spec.rho0 * spec.body.u_ref ** 2 * spec.body.l_ref
    n = int(round(periods * PERIOD))
    f = forces[-n:]
    cl = f[:, 1] / q
    return float(f[:, 0].mean() / q), float(np.sqrt(np.mean((cl - cl.mean()) ** 2)))


@pytest.fixture(scope="module")
def shedding_oracle():
    spec = shedding_spec(wl.F64)
    steps = int(math.ceil(PERIODS * PERIOD / 4))
    o = init_oracle(oracle_from_spec(spec, openmp=True), spec)
    o.step(steps)
    return steps, coefficient_stats(spec, o.forces())  # the oracle keeps its whole history


# measured on a GB300 (5 periods): FP32 within 3e-6, FP16 0.29 %; BF16 2.6 %
# off (8 % with the deviation from w_q)
@pytest.mark.parametrize("storage,measured", [(wl.F32, 5e-4), (wl.F16DEV, 5e-3), (wl.BF16DEV, 0.04)])
def test_shedding_cylinder_mean_coefficients_within_half_percent(shedding_oracle, storage, measured):
    steps, (cd_o, cl_o) = shedding_oracle
    spec = shedding_spec(storage)
    _, forces = gpu_run(spec, steps, chunk=1000)
    cd, cl = coefficient_stats(spec, forces)
    assert cl_o > 0.2  # developed shedding (the lift rms of the developed wake is about 0.25)
    worst = max(abs(cd - cd_o) / abs(cd_o), abs(cl - cl_o) / abs(cl_o))
    assert worst <= measured, (NAME[storage], cd, cd_o, cl, cl_o)
    if worst > 5e-3:
        pytest.xfail(f"{NAME[storage]}: mean coefficients {100 * worst:.2f} % from the oracle's (target 0.5 %)")


# --- conservation of mass and momentum in FP32 -------------------------------

@pytest.mark.parametrize("drho", [0.0, 1e-4])
def test_periodic_flow_keeps_its_momentum_in_fp32(drho):
    """Eq. 6 conserves the mass and momentum of a periodic box exactly; in
    FP32 the collision must return them without a per-step bias.  Two
    roundings did not: the nearest floats to the weights exceed them by
    2^-27, which the equilibrium's momentum carried into every step (a gain of
    omega 2^-27 = 1.4e-8 per step at tau = 0.52, 1.4e-4 after 10,000 steps),
    and for rho = 1 + d the float reciprocal of rho is below 1 / rho by about
    d^2 (a loss of 1e-8 per step at d = 1e-4).  Evaluated as
    (1 - omega) f + omega f^eq, Eq. 6 also rounds two O(f) terms (7e-6 of
    the momentum in 10,000 steps); the residual form f^eq + (1 - omega)
    (f - f^eq) rounds the result alone.  The state is a mean flow with
    a small smooth seeded perturbation, so that its values spread over the
    rounding boundaries (a uniform state rounds the same way at every cell and
    stays at a fixed point of the rounded arithmetic)."""
    from paper_2402_04606_gb300.native import Domain

    spec = wl.tgv(n=64, tau=0.52, storage=wl.F32)
    g = Domain(spec)
    r, u, v = wl.random_fields(spec.nx0, spec.ny0, seed=7, amp_u=0.002, amp_rho=0.001)
    rho0, ux0, uy0 = r + drho, u + 0.05, v - 0.02
    g.set_fields(0, rho0, ux0, uy0)
    g.step(10000)
    rho, ux, uy = g.fields(0)
    g.close()
    m0, m = rho0.sum(), rho.sum()
    jx0, jy0 = (rho0 * ux0).sum(), (rho0 * uy0).sum()
    jx, jy = (rho * ux).sum(), (rho * uy).sum()
    assert abs(m - m0) / m0 <= 1e-7
    assert abs(jx - jx0) / abs(jx0) <= 3e-6, jx / jx0 - 1
    assert abs(jy - jy0) / abs(jy0) <= 3e-6, jy / jy0 - 1
