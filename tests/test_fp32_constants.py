"""Facts about FP32 rounding that the collision's arithmetic relies on
(host only).

The deviation-form collision in FP32 takes the D2Q9 weights of Eq. 7 as
two-term constants and forms u = a - a (drho / rho) rather than a * fl(1 / rho).
Both choices rest on properties of the nearest floats, checked here with
numpy's IEEE single precision:
- fl(4/9), fl(1/9) and fl(1/36) each exceed the exact weight by exactly 2^-27
  of itself (so plain products bias the equilibrium's mass and momentum the
  same way at every cell), and fl(1/6) exceeds 1/6 by 2^-25;
- hi + lo (hi the nearest float, lo the float nearest the remainder) gives
  the weight to double precision;
- for rho = 1 + k 2^-23 with small k the nearest float to 1 / rho lies below
  the exact reciprocal, by about (rho - 1)^2 of it: the rounding takes
  momentum out of every collision in the same direction.
"""
from fractions import Fraction

import numpy as np


def _exact(x: np.float32) -> Fraction:
    return Fraction(float(x))


def test_weights_round_up_by_the_same_relative_amount():
    for num, den in ((4, 9), (1, 9), (1, 36)):
        w = Fraction(num, den)
        hi = np.float32(num / den)
        assert _exact(hi) / w - 1 == Fraction(1, 2 ** 27)
    assert _exact(np.float32(1 / 6)) * 6 - 1 == Fraction(1, 2 ** 25)


def test_two_term_weights_recover_the_weight():
    for num, den in ((4, 9), (1, 9), (1, 36), (1, 6)):
        w = Fraction(num, den)
        hi = np.float32(num / den)
        lo = np.float32(float(w - _exact(hi)))
        err = abs(_exact(hi) + _exact(lo) - w) / w
        plain = abs(_exact(hi) - w) / w  # 2^-27, or 2^-25 for 1/6
        assert err <= Fraction(1, 2 ** 50)
        assert err <= plain / 2 ** 23


def test_reciprocal_of_rho_near_one_rounds_low():
    below = 0
    for k in range(1, 1448):
        rho = np.float32(1.0) + np.float32(k) * np.float32(2.0 ** -23)
        r = np.float32(1.0) / rho
        exact = 1 / _exact(rho)
        if _exact(r) < exact:
            below += 1
            d = _exact(rho) - 1
            assert abs((exact - _exact(r)) / exact - d * d) < Fraction(1, 2 ** 40)
    assert below == 1447
