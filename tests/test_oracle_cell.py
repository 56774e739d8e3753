"""Pins of the oracle's single-cell formulas (Sec. 2.1) against the moment
identities the paper states (Eqs. 4-5, Eq. 8) and the textbook moments of
the D2Q9 equilibrium.  Each pin fails for a dropped term, a wrong weight, a
wrong sign or a swapped component."""
import numpy as np
import pytest

import oracle as orc

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
CS2 = 1.0 / 3.0
rng = np.random.default_rng(1234)
CASES = [(1.0 + 0.1 * rng.uniform(-1, 1), 0.1 * rng.uniform(-1, 1), 0.1 * rng.uniform(-1, 1)) for _ in range(20)]


def feq_vec(rho, ux, uy):
    return np.array([orc.feq(i, rho, ux, uy) for i in range(9)])


def test_lattice_is_the_papers_d2q9():
    # Eq. 1 directions: the rest direction, 4 axis and 4 diagonal unit moves
    assert orc.feq(0, 1.0, 0.0, 0.0) == pytest.approx(4.0 / 9.0, abs=1e-16)
    for i in range(1, 5):
        assert orc.feq(i, 1.0, 0.0, 0.0) == pytest.approx(1.0 / 9.0, abs=1e-16)
    for i in range(5, 9):
        assert orc.feq(i, 1.0, 0.0, 0.0) == pytest.approx(1.0 / 36.0, abs=1e-16)


@pytest.mark.parametrize("rho,ux,uy", CASES)
def test_equilibrium_moments(rho, ux, uy):
    f = feq_vec(rho, ux, uy)
    assert f.sum() == pytest.approx(rho, rel=1e-15, abs=1e-15)
    assert (CX * f).sum() == pytest.approx(rho * ux, abs=1e-15)
    assert (CY * f).sum() == pytest.approx(rho * uy, abs=1e-15)
    # second moment: rho cs^2 delta + rho u u
    assert (CX * CX * f).sum() == pytest.approx(rho * CS2 + rho * ux * ux, abs=2e-15)
    assert (CY * CY * f).sum() == pytest.approx(rho * CS2 + rho * uy * uy, abs=2e-15)
    assert (CX * CY * f).sum() == pytest.approx(rho * ux * uy, abs=2e-15)


@pytest.mark.parametrize("rho,ux,uy", CASES[:10])
def test_guo_moment_conditions(rho, ux, uy):
    tau = 0.6 + 0.5 * rng.uniform()
    Fx, Fy = 1e-3 * rng.uniform(-1, 1), 1e-3 * rng.uniform(-1, 1)
    F = np.array([orc.guo(i, tau, ux, uy, Fx, Fy) for i in range(9)])
    # Eq. 4 and Eq. 5
    assert F.sum() == pytest.approx(0.0, abs=1e-18)
    assert (CX * F).sum() == pytest.approx((1 - 1 / (2 * tau)) * Fx, rel=1e-13, abs=1e-19)
    assert (CY * F).sum() == pytest.approx((1 - 1 / (2 * tau)) * Fy, rel=1e-13, abs=1e-19)
    # the second moment of Guo's term (Guo et al. 2002): (1 - 1/2tau)(u F + F u)
    assert (CX * CX * F).sum() == pytest.approx((1 - 1 / (2 * tau)) * 2 * ux * Fx, abs=1e-18)
    assert (CX * CY * F).sum() == pytest.approx((1 - 1 / (2 * tau)) * (ux * Fy + uy * Fx), abs=1e-18)


@pytest.mark.parametrize("rho,ux,uy", CASES[:10])
def test_collision_conserves_mass_and_adds_force(rho, ux, uy):
    f = feq_vec(rho, ux, uy) * (1 + 0.05 * rng.uniform(-1, 1, 9))
    tau = 0.55 + rng.uniform()
    Fx, Fy = 1e-3 * rng.uniform(-1, 1), 1e-3 * rng.uniform(-1, 1)
    fs = orc.collide_cell(f, tau, Fx, Fy)
    assert fs.sum() == pytest.approx(f.sum(), rel=1e-15)
    # Eq. 6 with Eq. 8: the momentum gained in one collision is exactly F
    assert (CX * fs).sum() - (CX * f).sum() == pytest.approx(Fx, abs=1e-15)
    assert (CY * fs).sum() - (CY * f).sum() == pytest.approx(Fy, abs=1e-15)


def test_collision_relaxes_towards_equilibrium():
    rho, ux, uy = 1.02, 0.03, -0.01
    fe = feq_vec(rho, ux, uy)
    neq = 1e-3 * rng.uniform(-1, 1, 9)
    # keep mass and momentum of the perturbation zero so f^eq is unchanged
    M = np.stack([np.ones(9), CX, CY])
    neq = neq - M.T @ np.linalg.solve(M @ M.T, M @ neq)
    f = fe + neq
    tau = 0.7
    fs = orc.collide_cell(f, tau)
    # BGK (Eq. 6, F = 0): f* - f^eq = (1 - 1/tau) (f - f^eq)
    np.testing.assert_allclose(fs - fe, (1 - 1 / tau) * neq, atol=1e-16)
    # and an equilibrium is a fixed point
    np.testing.assert_allclose(orc.collide_cell(fe, tau), fe, atol=1e-16)
