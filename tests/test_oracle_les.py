"""Pins of the oracle's LES collision (Smagorinsky; reading R16).

- a Smagorinsky constant of zero gives the BGK collision;
- the relaxation time the collision applies (read back from its output)
  satisfies the model's defining relation tau_e - tau = 3 C^2 |S| with the
  strain rate of the non-equilibrium stress at tau_e, |S| = 3 Q / (2 rho tau_e);
- mass is conserved and momentum gains F;
- a shear wave decays faster the larger the constant.
"""
import math

import numpy as np
import pytest

import oracle as orc

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _state(rng, amp=0.05):
    rho = 1.0 + 0.05 * rng.uniform(-1, 1)
    u = 0.05 * rng.uniform(-1, 1, 2)
    f = np.array([orc.feq(i, rho, u[0], u[1]) for i in range(9)])
    return f * (1.0 + amp * rng.uniform(-1, 1, 9))


def test_zero_constant_is_bgk():
    rng = np.random.default_rng(11)
    for _ in range(10):
        f = _state(rng)
        a = orc.collide_cell_les(f, 0.53, 0.0, 1e-3, -2e-3)
        b = orc.collide_cell(f, 0.53, 1e-3, -2e-3)
        assert np.abs(a - b).max() <= 1e-16


@pytest.mark.parametrize("cs", [0.1, 0.17, 0.3])
def test_relaxation_time_satisfies_the_model(cs):
    rng = np.random.default_rng(12)
    tau = 0.51
    for _ in range(10):
        f = _state(rng)
        g = orc.collide_cell_les(f, tau, cs)
        rho = f.sum()
        ux, uy = CX @ f / rho, CY @ f / rho
        feq = np.array([orc.feq(i, rho, ux, uy) for i in range(9)])
        ne = f - feq
        te = ne / (f - g)  # f* = f - (f - f^eq) / tau_e without force
        assert np.ptp(te) <= 1e-9 * te.mean()
        te = te.mean()
        pxx, pyy, pxy = (CX * CX) @ ne, (CY * CY) @ ne, (CX * CY) @ ne
        Q = math.sqrt(2 * (pxx * pxx + pyy * pyy + 2 * pxy * pxy))
        S = 3 * Q / (2 * rho * te)
        assert te > tau
        assert abs((te - tau) - 3 * cs * cs * S) <= 1e-9 * (te - tau)


def test_conservation():
    rng = np.random.default_rng(13)
    for _ in range(10):
        f = _state(rng)
        g = orc.collide_cell_les(f, 0.52, 0.17, 2e-3, 1e-3)
        assert abs(g.sum() - f.sum()) <= 1e-15
        assert abs(CX @ g - CX @ f - 2e-3) <= 1e-15
        assert abs(CY @ g - CY @ f - 1e-3) <= 1e-15


def test_eddy_viscosity_speeds_up_decay():
    ny, A, steps = 32, 0.02, 200
    amps = []
    for cs in (0.0, 0.1, 0.2):
        dom = orc.Domain(nx0=16, ny0=ny, levels=1, block=16, tau_finest=0.51, coll=2, mrt_s=(cs, 0.0, 0.0))
        o = orc.Oracle(dom)
        y = np.arange(ny)
        k = 2 * math.pi / ny
        o.set_fields(0, np.ones((ny, 16)), np.tile((A * np.sin(k * y))[:, None], (1, 16)), np.zeros((ny, 16)))
        o.finalize_init()
        o.step(steps)
        _, u1, _ = o.fields(0)
        amps.append(2 * np.mean(u1[:, 0] * np.sin(k * y)))
    assert amps[0] > amps[1] > amps[2] > 0
