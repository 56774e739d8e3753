"""Pins of the oracle's body shapes and prescribed motions (Sec. 3.4-3.6).

Each check comes from the mathematics of the formula, not from a second
transcription of it:
- the pitch-up ramp (Eqs. 20-21): its limits before and after the ramp, its
  point symmetry about the ramp's midpoint, and the slope there in closed
  form;
- the asymmetric triangular pitch (Eqs. 22-24): peak and trough values and
  times, periodicity, continuity of the angle and of its first two
  derivatives at all six corners, the slopes of the linear pieces (Eqs. 23-24)
  and, for xi = 1/2, antisymmetry over half a period;
- marker shapes: the rectangle's perimeter and equal spacing exactly; the
  NACA section's markers on the thickness curve, its perimeter against an
  independent quadrature and its enclosed area against the closed form of
  the thickness polynomial's integral;
- the pose of a body with these motions: fixed centre, rotation
  alpha_mean - alpha(t);
- sinusoidal pitch and pitch plus tilted-stroke heave (Sec. 3.6, Eqs. 25-27):
  pose and markers against the equations written out, plus what the
  equations fix however they are coded (the pitch's extremes at the quarter
  periods, the stroke's direction, its length A0 and peak speed pi A0 / T, a
  rigid body turning about its pivot); a second test plants a flipped pitch
  sign, sin for cos in the heave, A0 for A0 / 2 and rotation about the centre
  in copies of the oracle's outputs and checks that each is caught.
"""
import math

import numpy as np
import pytest

import oracle as orc

A, AS, KR, T1 = math.pi / 2, 11.0, 0.2, 1.0  # the paper's pitch-up parameters (Sec. 3.4)
T2 = T1 + A / (2 * KR)


def ramp(ts):
    return orc.ramp_alpha(A, AS, KR, T1, ts)


def test_ramp_limits():
    assert abs(ramp(-50.0)) <= 1e-15
    assert abs(ramp(0.0)) <= 1e-4 * A  # before t1 the plate barely moves (a_s (t1 - t) = 11)
    assert abs(ramp(T2 + 5.0) - A) <= 1e-15 * 10
    assert abs(ramp(1e4) - A) <= 1e-12  # no overflow long after the ramp


def test_ramp_point_symmetry_and_midpoint():
    tm = 0.5 * (T1 + T2)
    assert abs(ramp(tm) - A / 2) <= 1e-14
    for s in (0.1, 0.7, 1.3, 2.9, 6.0):
        assert abs(ramp(tm + s) + ramp(tm - s) - A) <= 1e-13


def test_ramp_midpoint_slope_closed_form():
    # dG/dt* = a_s [tanh(a_s (t - t1)) - tanh(a_s (t - t2))], so at the
    # midpoint d alpha / d t* = A tanh(a_s d) / (t2 - t1), d = (t2 - t1) / 2
    tm, h = 0.5 * (T1 + T2), 1e-5
    slope = (ramp(tm + h) - ramp(tm - h)) / (2 * h)
    d = 0.5 * (T2 - T1)
    assert abs(slope - A * math.tanh(AS * d) / (T2 - T1)) <= 1e-8
    assert abs(slope - 2 * KR) <= 1e-8  # = 2 K for a_s d >> 1


def test_ramp_monotone():
    ts = np.linspace(-2, 12, 2001)
    a = np.array([ramp(t) for t in ts])
    assert np.all(np.diff(a) >= -1e-15)


@pytest.mark.parametrize("xi,acc", [(0.5, 0.15), (0.3, 0.1), (0.7, 0.12)])
def test_triangle_peaks_period_and_slopes(xi, acc):
    a0, T = math.radians(64.0), 1000.0
    f = lambda t: orc.triangle_alpha(a0, xi, acc, T, t)
    ta = acc * T
    t2, t5 = 0.5 * xi * T, T - 0.5 * xi * T
    assert abs(f(0.0)) <= 1e-15
    assert abs(f(t2) - a0) <= 1e-14
    assert abs(f(t5) + a0) <= 1e-14
    ts = np.linspace(0, T, 4001)
    v = np.array([f(t) for t in ts])
    assert v.max() <= a0 + 1e-14 and v.min() >= -a0 - 1e-14
    for t in (13.7, 250.0, 611.1, 999.0):
        assert abs(f(t + T) - f(t)) <= 1e-12 and abs(f(t - 3 * T) - f(t)) <= 1e-12
    ad1 = 2 * a0 / (xi * T - ta)
    ad2 = -2 * a0 / ((1 - xi) * T - ta)
    h = 1e-3
    t_up = 0.5 * (t2 - ta)  # inside the first linear piece
    t_dn = 0.5 * (t2 + ta + t5 - ta)  # inside the downstroke's linear piece
    assert abs((f(t_up + h) - f(t_up - h)) / (2 * h) - ad1) <= 1e-9
    assert abs((f(t_dn + h) - f(t_dn - h)) / (2 * h) - ad2) <= 1e-9


@pytest.mark.parametrize("xi,acc", [(0.5, 0.15), (0.3, 0.1)])
def test_triangle_smooth_at_corners(xi, acc):
    """alpha, alpha' and alpha'' continuous at t1..t6: one-sided differences
    from each side agree (a wrong denominator or sign in any quartic piece
    breaks one of these)."""
    a0, T = 1.0, 1000.0
    f = lambda t: orc.triangle_alpha(a0, xi, acc, T, t)
    ta = acc * T
    t2, t5 = 0.5 * xi * T, T - 0.5 * xi * T
    h = 1e-2
    for tk in (t2 - ta, t2, t2 + ta, t5 - ta, t5, t5 + ta):
        left = [f(tk - i * h) for i in range(3)]
        right = [f(tk + i * h) for i in range(3)]
        assert abs(left[0] - right[0]) <= 1e-12
        dl = (left[0] - left[1]) / h
        dr = (right[1] - right[0]) / h
        assert abs(dl - dr) <= 1e-5 * max(1.0, abs(dl)) * 10
        d2l = (left[0] - 2 * left[1] + left[2]) / h ** 2
        d2r = (right[0] - 2 * right[1] + right[2]) / h ** 2
        scale = a0 / ta ** 2
        assert abs(d2l - d2r) <= 0.05 * scale


def test_triangle_symmetric_case_antisymmetric():
    a0, T = 0.7, 800.0
    for t in np.linspace(0, T, 37):
        assert abs(orc.triangle_alpha(a0, 0.5, 0.15, T, t + T / 2) + orc.triangle_alpha(a0, 0.5, 0.15, T, t)) <= 1e-13


def test_rectangle_markers_exact():
    a, b, n = 32.0, 0.736, 131
    qx, qy, P = orc.place_markers(a, b, n, kind=2)
    assert abs(P - 4 * (a + b)) <= 1e-12
    on = (np.isclose(np.abs(qx), a, atol=1e-12) & (np.abs(qy) <= b + 1e-12)) | (
        np.isclose(np.abs(qy), b, atol=1e-12) & (np.abs(qx) <= a + 1e-12))
    assert on.all()
    # arc length along the boundary from (a, 0), counter-clockwise
    def arc(x, y):
        if abs(x - a) < 1e-9 and y >= -1e-12:
            return y
        if abs(y - b) < 1e-9:
            return b + (a - x)
        if abs(x + a) < 1e-9:
            return b + 2 * a + (b - y)
        if abs(y + b) < 1e-9:
            return 3 * b + 2 * a + (x + a)
        return 3 * b + 4 * a + (y + b)
    s = np.array([arc(x, y) for x, y in zip(qx, qy)])
    assert np.allclose(s, P * np.arange(n) / n, atol=1e-11)


def _naca_yt(t, xc):
    return 5 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2 + 0.2843 * xc ** 3 - 0.1036 * xc ** 4)


def test_naca_markers_on_curve_perimeter_and_area():
    from scipy.integrate import quad

    a, t, n = 32.0, 0.18, 400
    b = t * a
    qx, qy, P = orc.place_markers(a, b, n, kind=3)
    c = 2 * a
    xc = (qx + a) / c
    assert xc.min() >= -1e-15 and xc.max() <= 1 + 1e-15
    # markers lie on polygon chords of the curve: within the chord sagitta
    err = np.abs(np.abs(qy) - c * _naca_yt(t, np.clip(xc, 0, 1)))
    assert err.max() <= 2e-3
    # the perimeter against arc-length quadrature of the smooth curve
    # (x = c u^2 removes the square-root singularity at the leading edge)
    def dsdu(u):
        x = u * u
        dyt = 5 * t * (0.2969 * 0.5 / u - 0.1260 - 2 * 0.3516 * x + 3 * 0.2843 * x ** 2 - 4 * 0.1036 * x ** 3) if u > 0 else 0.0
        # d/du of (c u^2, c yt(u^2)) = (2 c u, c yt'(x) 2u)
        return math.hypot(2 * c * u, c * dyt * 2 * u) if u > 0 else c * 5 * t * 0.2969
    half, _ = quad(dsdu, 0.0, 1.0, limit=200, epsabs=1e-12)
    assert abs(P - 2 * half) <= 1e-5 * P
    # enclosed area: 2 c^2 int_0^1 y_t = 10 t c^2 (0.2969 * 2/3 - 0.1260/2 - 0.3516/3 + 0.2843/4 - 0.1036/5)
    area = 0.5 * abs(np.dot(qx, np.roll(qy, -1)) - np.dot(qy, np.roll(qx, -1)))
    exact = 10 * t * c * c * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1036 / 5)
    assert abs(area - exact) <= 2e-3 * exact
    # equal arc length: consecutive chord lengths within the polygon's error
    d = np.hypot(np.diff(np.r_[qx, qx[0]]), np.diff(np.r_[qy, qy[0]]))
    assert np.allclose(d, P / n, rtol=2e-3)
    # the maximum half-thickness is about b (0.50007 t c at x = 0.3 c)
    assert abs(np.abs(qy).max() - b) <= 0.01 * b


def test_pose_of_pitch_motions():
    dom = orc.Domain(nx0=64, ny0=64, levels=1, block=16)
    body = orc.Body(a=20.0, b=1.0, n_markers=84, pivot=(-20.0, 0.0), motion=3, x0=(512.0, 512.0),
                    alpha_mean=0.3, alpha_amp=A, kind=2, ramp_as=AS, ramp_rate=KR, ramp_t1=T1, t_ref=400.0)
    o = orc.Oracle(dom, body)
    for t in (0.0, 800.0, 1185.0, 4000.0):
        cx, cy, th = o.pose(t)
        assert (cx, cy) == (512.0, 512.0)
        assert abs(th - (0.3 - ramp(t / 400.0))) <= 1e-15
    # the leading edge (the pivot) stays put while the plate turns
    rx0, ry0 = o.markers(0)
    rx1, ry1 = o.markers(3000)
    qx, qy, _ = orc.place_markers(20.0, 1.0, 84, kind=2)
    le = np.argmin(np.hypot(qx + 20.0, qy))  # the marker nearest the pivot, if any lies on it
    if abs(qx[le] + 20.0) < 1e-12 and abs(qy[le]) < 1e-12:
        assert abs(rx1[le] - rx0[le]) <= 1e-12 and abs(ry1[le] - ry0[le]) <= 1e-12
    body4 = orc.Body(a=20.0, b=3.6, n_markers=84, pivot=(-10.0, 0.0), motion=4, x0=(512.0, 512.0),
                     alpha_mean=0.0, alpha_amp=1.1, period=900.0, phase=0.0, kind=3, xi=0.5, acc=0.15)
    o4 = orc.Oracle(dom, body4)
    for t in (0.0, 100.0, 450.0, 1234.0):
        assert abs(o4.pose(t)[2] + orc.triangle_alpha(1.1, 0.5, 0.15, 900.0, t)) <= 1e-15


# ---------------------------------------------------------------------------
# Sinusoidal pitch (motion 1) and pitch plus tilted-stroke heave (motion 2),
# Sec. 3.6, Eqs. 25-27: alpha(t) = alpha_mean - alpha_amp sin(2 pi t / T + phi),
# centre x0 + (A0 / 2) cos(2 pi t / T) (cos beta, sin beta), body turned by
# alpha about its pivot.  The checks below hold the oracle to the equations
# written out here and to properties the equations fix whatever way they are
# coded (quarter-period values, the stroke's direction and length, the peak
# heave speed pi A0 / T, a rigid body turning about the pivot).
# ---------------------------------------------------------------------------
FLAP = dict(a=32.0, b=3.84, n_markers=200, pivot=(-8.0, 1.5), x0=(1600.0, 1500.0), alpha_mean=math.pi / 2,
            alpha_amp=math.radians(45.0), period=4000.0, phase=0.3, heave_amp=160.0, beta=math.radians(60.0))
TIMES = (0, 250, 1000, 1377, 2000, 3000, 3999, 8421)


def _closed_form(p, motion, t):
    """Eqs. 25-27 written out: centre x, y and the pitch angle at finest time t."""
    al = p["alpha_mean"] - p["alpha_amp"] * math.sin(2 * math.pi * t / p["period"] + p["phase"])
    h = 0.5 * p["heave_amp"] * math.cos(2 * math.pi * t / p["period"]) if motion == 2 else 0.0
    return p["x0"][0] + h * math.cos(p["beta"]), p["x0"][1] + h * math.sin(p["beta"]), al


def _marker_closed_form(p, pose, qx, qy):
    """a body-frame point (qx, qy) turned by the pose's angle about the pivot"""
    cx, cy, al = pose
    px, py = qx - p["pivot"][0], qy - p["pivot"][1]
    return (cx + p["pivot"][0] + math.cos(al) * px - math.sin(al) * py,
            cy + p["pivot"][1] + math.sin(al) * px + math.cos(al) * py)


def _flap_oracle(motion, **over):
    p = dict(FLAP, **over)
    dom = orc.Domain(nx0=400, ny0=400, levels=1, block=16)
    body = orc.Body(a=p["a"], b=p["b"], n_markers=p["n_markers"], pivot=p["pivot"], motion=motion, x0=p["x0"],
                    alpha_mean=p["alpha_mean"], alpha_amp=p["alpha_amp"], period=p["period"], phase=p["phase"],
                    heave_amp=p["heave_amp"], beta=p["beta"])
    return orc.Oracle(dom, body), p


def _check_flapping(pose, markers, p, motion, qx, qy):
    """Raises AssertionError unless pose(t) -> (cx, cy, alpha) and
    markers(t) -> (rx, ry) follow Eqs. 25-27 for `motion` (1 or 2)."""
    T, A0, beta = p["period"], p["heave_amp"], p["beta"]
    x0 = np.array(p["x0"])
    for t in TIMES:
        cx, cy, al = pose(t)
        ex, ey, eal = _closed_form(p, motion, t)
        assert abs(al - eal) <= 1e-15 * max(1.0, abs(eal)), (t, al, eal)
        assert abs(cx - ex) <= 4e-16 * abs(ex) and abs(cy - ey) <= 4e-16 * abs(ey), (t, cx, cy, ex, ey)
        rx, ry = markers(t)
        for j in (0, 57, len(qx) - 1):
            mx, my = _marker_closed_form(p, (ex, ey, eal), qx[j], qy[j])
            assert abs(rx[j] - mx) <= 1e-12 and abs(ry[j] - my) <= 1e-12, (t, j, rx[j], mx, ry[j], my)
    # quarter-period values with the phase removed from the pitch: at
    # 2 pi t / T + phi = pi / 2 the angle is alpha_mean - alpha_amp (the
    # pitch's sign), at 3 pi / 2 it is alpha_mean + alpha_amp
    t_q = (math.pi / 2 - p["phase"]) * T / (2 * math.pi)
    assert abs(pose(t_q)[2] - (p["alpha_mean"] - p["alpha_amp"])) <= 1e-14
    assert abs(pose(t_q + T / 2)[2] - (p["alpha_mean"] + p["alpha_amp"])) <= 1e-14
    # the stroke: at t = 0 the centre is A0 / 2 along (cos beta, sin beta)
    # from x0, at T / 2 as far the other way, at T / 4 on x0; the centre moves
    # only along the stroke line, A0 peak to peak; its peak speed is pi A0 / T
    ts = np.linspace(0.0, T, 4001)
    c = np.array([pose(t)[:2] for t in ts]) - x0
    d = np.array([math.cos(beta), math.sin(beta)])
    if motion == 2:
        assert np.allclose(pose(0.0)[:2] - x0, 0.5 * A0 * d, rtol=0, atol=1e-12)
        assert np.allclose(pose(T / 2)[:2] - x0, -0.5 * A0 * d, rtol=0, atol=1e-12)
        assert np.allclose(pose(T / 4)[:2] - x0, 0.0, rtol=0, atol=1e-11)
        assert np.max(np.abs(c[:, 0] * d[1] - c[:, 1] * d[0])) <= 1e-11  # on the stroke line
        s = c @ d
        assert abs((s.max() - s.min()) - A0) <= 1e-9 * A0
        v = np.abs(np.diff(s)) / (ts[1] - ts[0])
        assert abs(v.max() - math.pi * A0 / T) <= 1e-5 * math.pi * A0 / T
    else:
        assert np.max(np.abs(c)) == 0.0  # motion 1: no heave
    # a rigid body turning about its pivot: marker distances are kept, and a
    # body point at the pivot moves with the centre (the heave) only
    r0 = np.stack(markers(0))
    for t in (1000, 1377, 3000):
        r = np.stack(markers(t))
        for j, k in ((0, 100), (57, 143), (10, 11)):
            assert abs(np.hypot(*(r[:, j] - r[:, k])) - np.hypot(*(r0[:, j] - r0[:, k]))) <= 1e-11
        # the markers' position relative to the pivot point turns by alpha(t) - alpha(0)
        piv, piv0 = np.array(pose(t)[:2]) + p["pivot"], np.array(pose(0)[:2]) + p["pivot"]
        dal = pose(t)[2] - pose(0)[2]
        rot = np.array([[math.cos(dal), -math.sin(dal)], [math.sin(dal), math.cos(dal)]])
        assert np.allclose(r - piv[:, None], rot @ (r0 - piv0[:, None]), rtol=0, atol=1e-11)


@pytest.mark.parametrize("motion", [1, 2])
def test_pose_of_flapping_motions(motion):
    o, p = _flap_oracle(motion)
    qx, qy, _ = orc.place_markers(p["a"], p["b"], p["n_markers"])
    _check_flapping(o.pose, lambda t: o.markers(int(t)), p, motion, qx, qy)


@pytest.mark.parametrize("mutation", ["pitch_sign", "heave_sin_for_cos", "heave_full_A0", "turn_about_centre"])
def test_flapping_pins_reject_planted_mistakes(mutation):
    """The checks above fail for each plausible mistake in the motion:
    the pitch's sign flipped, sin in place of cos in the heave, A0 in place
    of A0 / 2, rotation about the centre in place of the pivot.  The mistakes
    are planted in copies of the oracle's own outputs, on the CPU."""
    o, p = _flap_oracle(2)
    qx, qy, _ = orc.place_markers(p["a"], p["b"], p["n_markers"])
    T, x0 = p["period"], np.array(p["x0"])
    d = np.array([math.cos(p["beta"]), math.sin(p["beta"])])

    def pose(t):
        cx, cy, al = o.pose(t)
        c = np.array([cx, cy])
        if mutation == "pitch_sign":
            al = 2 * p["alpha_mean"] - al
        if mutation == "heave_sin_for_cos":
            c = x0 + 0.5 * p["heave_amp"] * math.sin(2 * math.pi * t / T) * d
        if mutation == "heave_full_A0":
            c = x0 + 2.0 * (c - x0)
        return c[0], c[1], al

    def markers(t):
        if mutation == "turn_about_centre":
            cx, cy, al = o.pose(t)
            return (cx + math.cos(al) * qx - math.sin(al) * qy, cy + math.sin(al) * qx + math.cos(al) * qy)
        cx, cy, al = pose(t)
        rx, ry = _marker_closed_form(p, (cx, cy, al), qx, qy)
        return np.asarray(rx), np.asarray(ry)

    with pytest.raises(AssertionError):
        _check_flapping(pose, markers, p, 2, qx, qy)
