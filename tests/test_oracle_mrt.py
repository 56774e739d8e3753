"""Pins of the oracle's MRT collision (the option of Sec. 2.1; reading R14).

- the moment basis: orthogonal rows with the squared norms of the D2Q9
  basis, full rank;
- with every relaxation rate equal to 1/tau the MRT collision equals the
  BGK collision of Eq. 6 with Eq. 3 (each pinned by its own moment
  identities), forcing included;
- conservation: mass unchanged and momentum gaining exactly F;
- the equilibrium moments M f^eq and the forcing moments M Fb against their
  closed forms (the expressions the GPU evaluates);
- a shear wave decays at the rate of the viscosity of Eq. 9 set by tau
  alone, whatever the other rates.
"""
import math

import numpy as np
import pytest

import oracle as orc


def _state(rng):
    rho = 1.0 + 0.05 * rng.uniform(-1, 1)
    u = 0.05 * rng.uniform(-1, 1, 2)
    f = np.array([orc.feq(i, rho, u[0], u[1]) for i in range(9)])
    return f * (1.0 + 0.02 * rng.uniform(-1, 1, 9))


def test_basis_orthogonal_with_known_norms():
    M = orc.mrt_matrix()
    G = M @ M.T
    assert np.array_equal(np.diag(np.diag(G)), G)
    assert np.array_equal(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])
    assert np.linalg.matrix_rank(M) == 9


@pytest.mark.parametrize("tau", [0.51, 0.6, 0.8, 1.3])
def test_equal_rates_reduce_to_bgk(tau):
    rng = np.random.default_rng(7)
    for _ in range(20):
        f = _state(rng)
        Fx, Fy = 1e-3 * rng.uniform(-1, 1, 2)
        a = orc.collide_cell_mrt(f, tau, [1 / tau] * 3, Fx, Fy)
        b = orc.collide_cell(f, tau, Fx, Fy)
        assert np.abs(a - b).max() <= 1e-14


def test_conservation_with_force():
    rng = np.random.default_rng(8)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    for _ in range(20):
        f = _state(rng)
        Fx, Fy = 1e-3 * rng.uniform(-1, 1, 2)
        g = orc.collide_cell_mrt(f, 0.56, [1.64, 1.54, 1.9], Fx, Fy)
        assert abs(g.sum() - f.sum()) <= 1e-15
        assert abs((cx * g).sum() - (cx * f).sum() - Fx) <= 1e-15
        assert abs((cy * g).sum() - (cy * f).sum() - Fy) <= 1e-15


def test_equilibrium_is_a_fixed_point():
    f = np.array([orc.feq(i, 1.02, 0.03, -0.04) for i in range(9)])
    g = orc.collide_cell_mrt(f, 0.53, [1.64, 1.54, 1.9])
    assert np.abs(g - f).max() <= 1e-15


def test_equilibrium_and_forcing_moments_closed_form():
    M = orc.mrt_matrix()
    rho, ux, uy = 1.03, 0.04, -0.025
    feq = np.array([orc.feq(i, rho, ux, uy) for i in range(9)])
    uu = ux * ux + uy * uy
    want = [rho, rho * (-2 + 3 * uu), rho * (1 - 3 * uu), rho * ux, -rho * ux, rho * uy, -rho * uy,
            rho * (ux * ux - uy * uy), rho * ux * uy]
    assert np.allclose(M @ feq, want, atol=1e-15, rtol=0)
    # every rate zero (tau -> infinity): f* - f is the forcing term Fb itself,
    # at the velocity of Eq. 8 (jx + F/2) / rho
    Fx, Fy = 2e-3, -1e-3
    f = feq.copy()
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    vx, vy = (cx @ f + Fx / 2) / f.sum(), (cy @ f + Fy / 2) / f.sum()
    dm = M @ (orc.collide_cell_mrt(f, 1e300, [0.0, 0.0, 0.0], Fx, Fy) - f)
    uF = vx * Fx + vy * Fy
    want = [0, 6 * uF, -6 * uF, Fx, -Fx, Fy, -Fy, 2 * (vx * Fx - vy * Fy), vx * Fy + vy * Fx]
    assert np.allclose(dm, want, atol=1e-15, rtol=0)  # f* - f cancels values of about 0.4


@pytest.mark.parametrize("rates", [(1.64, 1.54, 1.9), (1.1, 1.0, 1.2)])
def test_shear_wave_decays_at_the_bgk_viscosity(rates):
    """u_x = A sin(k y) on a periodic strip: the amplitude decays as
    exp(-nu k^2 t), nu = (tau - 1/2) / 3, independent of the other rates."""
    tau, ny, A, steps = 0.8, 64, 1e-3, 400
    dom = orc.Domain(nx0=16, ny0=ny, levels=1, block=16, tau_finest=tau, coll=1, mrt_s=rates)
    o = orc.Oracle(dom)
    y = np.arange(ny)
    k = 2 * math.pi / ny
    ux = np.tile((A * np.sin(k * y))[:, None], (1, 16))
    o.set_fields(0, np.ones((ny, 16)), ux, np.zeros((ny, 16)))
    o.finalize_init()
    o.step(steps)
    _, u1, _ = o.fields(0)
    amp = 2 * np.mean(u1[:, 0] * np.sin(k * y))
    nu = (tau - 0.5) / 3
    rate = -math.log(amp / A) / steps
    assert abs(rate / (nu * k * k) - 1) <= 5e-3
