"""Pins of the oracle's immersed-boundary operator (Sec. 2.2, Eqs. 11-16).

* Eq. 14 closed-form values and Peskin's discrete moment identities;
* interpolation and spreading against a dense brute-force double loop over
  every cell and marker (no stencil indexing);
* Eq. 16: sum_x F_x dx^2 = sum_j F_j ds_b (partition of unity);
* the multi-direct-forcing contraction on a straight line of markers with unit
  spacing, which has a closed form: each iteration removes exactly 3/8 of the
  slip (sum_y phi^2 = 3/8 and sum_j phi(x - x_j) = 1).
"""
import math

import numpy as np
import pytest

import oracle as orc

rng = np.random.default_rng(7)


def test_phi_closed_form_values():
    # Eq. 14 at 0, 1/2, 1, 3/2, 2
    assert orc.phi(0.0) == pytest.approx(0.5, abs=1e-16)
    assert orc.phi(1.0) == pytest.approx(0.25, abs=1e-16)
    assert orc.phi(2.0) == pytest.approx(0.0, abs=1e-16)
    assert orc.phi(0.5) == pytest.approx((2 + math.sqrt(2)) / 8, abs=1e-16)
    assert orc.phi(1.5) == pytest.approx((2 - math.sqrt(2)) / 8, abs=1e-16)
    assert orc.phi(2.5) == 0.0
    for r in rng.uniform(-3, 3, 50):
        assert orc.phi(r) == orc.phi(-r)


@pytest.mark.parametrize("r", list(rng.uniform(0, 1, 25)))
def test_phi_discrete_moments(r):
    ks = np.arange(-4, 5)
    v = np.array([orc.phi(r - k) for k in ks])
    assert v.sum() == pytest.approx(1.0, abs=1e-15)  # partition of unity
    assert ((r - ks) * v).sum() == pytest.approx(0.0, abs=1e-15)  # first moment
    assert v[ks % 2 == 0].sum() == pytest.approx(0.5, abs=1e-15)  # even / odd
    assert (v * v).sum() == pytest.approx(3.0 / 8.0, abs=1e-15)  # sum phi^2 = 3/8


def brute_interp(field, rx, ry):
    ny, nx = field.shape
    out = np.zeros(len(rx))
    for j in range(len(rx)):
        s = 0.0
        for cy in range(ny):
            for cx in range(nx):
                w = orc.phi(cx + 0.5 - rx[j]) * orc.phi(cy + 0.5 - ry[j])
                s += field[cy, cx] * w
        out[j] = s
    return out


def brute_spread(nx, ny, Fj, rx, ry, ds):
    out = np.zeros((ny, nx))
    for cy in range(ny):
        for cx in range(nx):
            s = 0.0
            for j in range(len(rx)):
                s += Fj[j] * orc.phi(cx + 0.5 - rx[j]) * orc.phi(cy + 0.5 - ry[j]) * ds[j]
            out[cy, cx] = s
    return out


@pytest.mark.parametrize("nmark", [1, 2, 3])
def test_single_iteration_against_brute_force(nmark):
    nx, ny = 14, 12
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.03 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.03 * rng.uniform(-1, 1, (ny, nx))
    rx = rng.uniform(3.0, nx - 3.0, nmark)
    ry = rng.uniform(3.0, ny - 3.0, nmark)
    udx = 0.01 * rng.uniform(-1, 1, nmark)
    udy = 0.01 * rng.uniform(-1, 1, nmark)
    ds = rng.uniform(0.5, 1.2, nmark)
    ux1, uy1, Fx, Fy, Fjx, Fjy = orc.ibm_mdf(rho, ux, uy, rx, ry, udx, udy, ds, K=1)
    # Eq. 12 and Eq. 11 by brute force
    uj = brute_interp(ux, rx, ry)
    vj = brute_interp(uy, rx, ry)
    rj = brute_interp(rho, rx, ry)
    np.testing.assert_allclose(Fjx, 2 * rj * (udx - uj), rtol=1e-13, atol=1e-17)
    np.testing.assert_allclose(Fjy, 2 * rj * (udy - vj), rtol=1e-13, atol=1e-17)
    # Eq. 15 by brute force
    np.testing.assert_allclose(Fx, brute_spread(nx, ny, Fjx, rx, ry, ds), rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(Fy, brute_spread(nx, ny, Fjy, rx, ry, ds), rtol=1e-13, atol=1e-18)
    # velocity correction u += F / (2 rho) (half-force shift of Eq. 8)
    np.testing.assert_allclose(ux1, ux + Fx / (2 * rho), rtol=1e-14, atol=1e-18)
    np.testing.assert_allclose(uy1, uy + Fy / (2 * rho), rtol=1e-14, atol=1e-18)
    # Eq. 16: the two expressions of the body force agree
    assert Fx.sum() == pytest.approx((Fjx * ds).sum(), rel=1e-13, abs=1e-18)
    assert Fy.sum() == pytest.approx((Fjy * ds).sum(), rel=1e-13, abs=1e-18)


def test_several_iterations_against_brute_force():
    nx, ny, n, K = 16, 16, 3, 4
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.03 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.03 * rng.uniform(-1, 1, (ny, nx))
    rx = np.array([6.3, 7.1, 8.4])
    ry = np.array([7.7, 8.9, 7.2])
    udx, udy, ds = np.full(n, 0.01), np.full(n, -0.005), np.full(n, 0.9)
    uxk, uyk = ux.copy(), uy.copy()
    Fx, Fy, Fjx, Fjy = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros(n), np.zeros(n)
    for _ in range(K):  # reading R4, written out with the brute-force operators
        rj = brute_interp(rho, rx, ry)
        dfx = 2 * rj * (udx - brute_interp(uxk, rx, ry))
        dfy = 2 * rj * (udy - brute_interp(uyk, rx, ry))
        sx = brute_spread(nx, ny, dfx, rx, ry, ds)
        sy = brute_spread(nx, ny, dfy, rx, ry, ds)
        uxk, uyk = uxk + sx / (2 * rho), uyk + sy / (2 * rho)
        Fx, Fy, Fjx, Fjy = Fx + sx, Fy + sy, Fjx + dfx, Fjy + dfy
    o = orc.ibm_mdf(rho, ux, uy, rx, ry, udx, udy, ds, K)
    for got, want in zip(o, (uxk, uyk, Fx, Fy, Fjx, Fjy)):
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-17)


@pytest.mark.parametrize("y0", [20.0, 20.3, 20.5, 20.77])
def test_mdf_line_contraction_is_five_eighths(y0):
    nx, ny, n = 90, 40, 70
    rho = np.ones((ny, nx))
    ux, uy = np.zeros((ny, nx)), np.zeros((ny, nx))
    rx = 10.0 + np.arange(n) + 0.37
    ry = np.full(n, y0)
    ud = np.array([0.01, 0.004])
    mid = slice(30, 40)  # markers far from the line ends
    for K in range(1, 6):
        uxk, uyk, *_ = orc.ibm_mdf(rho, ux, uy, rx, ry, np.full(n, ud[0]), np.full(n, ud[1]), np.ones(n), K)
        slip_x = ud[0] - brute_interp(uxk[:, 35:60], rx[mid] - 35, ry[mid])
        slip_y = ud[1] - brute_interp(uyk[:, 35:60], rx[mid] - 35, ry[mid])
        np.testing.assert_allclose(slip_x, ud[0] * (5.0 / 8.0) ** K, rtol=1e-12)
        np.testing.assert_allclose(slip_y, ud[1] * (5.0 / 8.0) ** K, rtol=1e-12)


def test_marker_placement():
    # circle: uniform angles; ellipse: equal arc length, perimeter close to Ramanujan's formula
    qx, qy, P = orc.place_markers(20.0, 20.0, 126)
    assert P == pytest.approx(2 * math.pi * 20.0, rel=1e-15)
    np.testing.assert_allclose(np.hypot(qx, qy), 20.0, rtol=1e-15)
    a, b, n = 32.0, 3.84, 200
    qx, qy, P = orc.place_markers(a, b, n)
    h = ((a - b) / (a + b)) ** 2
    ram = math.pi * (a + b) * (1 + 3 * h / (10 + math.sqrt(4 - 3 * h)))
    assert P == pytest.approx(ram, rel=1e-5)
    np.testing.assert_allclose((qx / a) ** 2 + (qy / b) ** 2, 1.0, rtol=1e-12)
    # equal arc length: the arc between consecutive markers, measured on a much
    # finer polygon than the one used for placement, is P / n everywhere
    t = np.unwrap(np.arctan2(qy / b, qx / a))
    t = np.r_[t, t[0] + 2 * math.pi]
    arcs = []
    for k in range(n):
        tt = np.linspace(t[k], t[k + 1], 2001)
        arcs.append(np.hypot(np.diff(a * np.cos(tt)), np.diff(b * np.sin(tt))).sum())
    np.testing.assert_allclose(arcs, P / n, rtol=2e-4)
