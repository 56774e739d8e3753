"""Pins of the oracle's walls and solid obstacles (reading R15: half-way
and linearly interpolated bounce-back).

- plane Couette flow between a wall at rest and a moving wall is a steady
  solution with an exactly linear profile: half-way walls reproduce it at
  any tau, and so does the interpolated bounce-back from a flat solid whose
  surface cuts the links at fractions below, at and above one half;
- mass is conserved exactly in a closed cavity with a tangentially moving
  lid;
- the link fractions at a circle equal a bisection along the link.
"""

import numpy as np
import pytest

import oracle as orc

WALLS = (orc.BC_PERIODIC, orc.BC_PERIODIC, orc.BC_WALL, orc.BC_WALL)


def couette(tau, H=16, U=0.01, steps=20000, y0=None, nx=16):
    uw = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0, U, 0.0)
    solid = (0, 0.0, 0.0, 0.0) if y0 is None else (2, y0, 0.0, 0.0)
    dom = orc.Domain(nx0=nx, ny0=H, levels=1, block=16, bc=WALLS, tau_finest=tau, uwall=uw, solid=solid)
    o = orc.Oracle(dom)
    o.set_fields(0, np.ones((H, nx)), np.zeros((H, nx)), np.zeros((H, nx)))
    o.finalize_init()
    o.step(steps)
    _, u, v = o.fields(0)
    fluid = o.types(0)[:, 0] == orc.T_INT
    y = np.arange(H) + 0.5
    lo = 0.0 if y0 is None else y0
    exact = U * (y - lo) / (H - lo)
    return np.abs(u[fluid, 0] - exact[fluid]).max() / U, np.abs(v).max() / U


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_half_way_walls_give_exact_couette(tau):
    err_u, err_v = couette(tau)
    assert err_u <= 1e-9 and err_v <= 1e-11


@pytest.mark.parametrize("y0", [2.3, 3.0, 2.7])  # first fluid row cut at t = 0.2, 0.5, 0.8
@pytest.mark.parametrize("tau", [0.6, 1.2])
def test_interpolated_bounce_back_gives_exact_couette(y0, tau):
    err_u, err_v = couette(tau, y0=y0, steps=30000)
    assert err_u <= 1e-9 and err_v <= 1e-11


def test_lid_driven_cavity_conserves_mass():
    n = 32
    bc = (orc.BC_WALL,) * 4
    dom = orc.Domain(nx0=n, ny0=n, levels=1, block=16, bc=bc, tau_finest=0.6,
                     uwall=(0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.05, 0.0))
    o = orc.Oracle(dom)
    rng = np.random.default_rng(3)
    o.set_fields(0, 1.0 + 0.01 * rng.uniform(-1, 1, (n, n)), 0.01 * rng.uniform(-1, 1, (n, n)),
                 0.01 * rng.uniform(-1, 1, (n, n)))
    o.finalize_init()
    m0 = o.checksum()[0]
    o.step(2000)
    assert abs(o.checksum()[0] - m0) <= 1e-12 * m0


def test_circle_link_fractions_match_bisection():
    dom = orc.Domain(nx0=64, ny0=64, levels=1, block=16, solid=(1, 31.3, 30.8, 9.7))
    o = orc.Oracle(dom)
    dirs = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    checked = 0
    for yy in range(64):
        for xx in range(64):
            px, py = xx + 0.5, yy + 0.5
            if o.in_solid(px, py):
                continue
            for ex, ey in dirs:
                if not o.in_solid(px + ex, py + ey):
                    continue
                lo, hi = 0.0, 1.0
                for _ in range(60):
                    mid = 0.5 * (lo + hi)
                    if o.in_solid(px + mid * ex, py + mid * ey):
                        hi = mid
                    else:
                        lo = mid
                assert abs(o.wall_fraction(px, py, ex, ey) - 0.5 * (lo + hi)) <= 1e-12
                checked += 1
    assert checked > 100
    types = o.types(0)
    assert (types == orc.T_SOLID).sum() == sum(o.in_solid(x + 0.5, y + 0.5) for y in range(64) for x in range(64))
