"""Pins of the WENO smoothness indicators (Eqs. 24 and 29) and of the nonlinear weights.

The exactness, symmetry and face-interpolation pins of test_oracle_weno.py hold
for any convex weights.  These pin the weights themselves:

* Eqs. 24 and 29 are the Jiang-Shu measure of the candidate polynomial,
  IS = sum over l >= 1 of the integral over the zone of (d^l p / d xi^l)^2 (unit
  zone width).  The test integrates that definition exactly, with the Hermite
  polynomials of Eq. 9 typed in here, and compares it with the oracle's
  smoothness functions.
* On small hand-made stencils, the candidates, their Jiang-Shu IS and the
  weights gamma_s / IS_s^2 (normalised; EPS = 1e-12 is negligible next to IS of
  order one) were worked out in exact rational arithmetic.  The blended moments
  are written below as those exact fractions, and the oracle must reproduce them.
  A wrong coefficient in IS (13/3, 781/20, 1/10) or a wrong power in the weights
  changes every one of them.
"""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import weno

# Eq. 9, ascending monomial coefficients: P1 = x, P2 = x^2 - 1/12, P3 = x^3 - 3x/20
_P = {1: [F(0), F(1)], 2: [F(-1, 12), F(0), F(1)], 3: [F(0), F(-3, 20), F(0), F(1)]}


def _poly(b, c, d):
    out = [F(0)] * 4
    for k, co in ((1, b), (2, c), (3, d)):
        for i, v in enumerate(_P[k]):
            out[i] += co * v
    return out


def _jiang_shu(b, c, d):
    """Sum over derivative orders l >= 1 of the exact integral of (p^(l))^2 over [-1/2, 1/2]."""
    p = _poly(b, c, d)
    total = F(0)
    while len(p) > 1:
        p = [i * p[i] for i in range(1, len(p))]
        sq = [F(0)] * (2 * len(p) - 1)
        for i, x in enumerate(p):
            for j, y in enumerate(p):
                sq[i + j] += x * y
        total += sum(co * (F(1, 2) ** (k + 1) - F(-1, 2) ** (k + 1)) / (k + 1) for k, co in enumerate(sq))
    return total


def test_quadratic_smoothness_is_the_jiang_shu_integral():
    """Eq. 24: b^2 + 13 c^2 / 3 for the quadratic candidate a + b P1 + c P2."""
    rng = np.random.default_rng(24)
    for _ in range(20):
        b, c = (F(int(x), 7) for x in rng.integers(-40, 40, 2))
        want = float(_jiang_shu(b, c, F(0)))
        got = weno.smoothness_quadratic(float(b), float(c))
        assert got == pytest.approx(want, rel=1e-14, abs=1e-300)


def test_cubic_smoothness_is_the_jiang_shu_integral():
    """Eq. 29: (b + d/10)^2 + 13 c^2 / 3 + 781 d^2 / 20 for the cubic a + b P1 + c P2 + d P3."""
    rng = np.random.default_rng(29)
    for _ in range(20):
        b, c, d = (F(int(x), 9) for x in rng.integers(-40, 40, 3))
        want = float(_jiang_shu(b, c, d))
        got = weno.smoothness_cubic(float(b), float(c), float(d))
        assert got == pytest.approx(want, rel=1e-14, abs=1e-300)


def _line(values, d, n_other=2):
    """Zone averages along direction d (x, y or z), constant in the other two directions."""
    v = np.asarray(values, dtype=float)
    shape = [n_other, n_other, n_other]
    shape[2 - d] = len(v)
    a = np.empty(shape)
    idx = [None, None, None]
    idx[2 - d] = slice(None)
    a[...] = v[tuple(idx)]
    return a


def _at(a, d, i):
    sl = [0, 0, 0]
    sl[2 - d] = i
    return a[tuple(sl)]


@pytest.mark.parametrize("d", [0, 1, 2])
def test_weno3_blend_on_a_hand_computed_stencil(d):
    """Zone averages (0, 1, 1, 3, 0) around the centre zone (index 2).

    Candidates (b, c): left {i-2..i} (-1/2, -1/2), centre (1, 1), right (9/2, -5/2).
    Jiang-Shu IS: 4/3, 16/3, 142/3.  alpha = gamma / IS^2 with gamma = (1, 10, 1)/12:
    3/64, 15/512, 3/80656, i.e. omega = (120984, 75615, 96) / 196695.
    Blend: b = 15555/196695 = 1037/13113, c = 14883/196695 = 4961/65565.
    """
    a = _line([0, 1, 1, 3, 0], d)
    b, c = weno.weno3(a, d)
    assert _at(b, d, 2) == pytest.approx(float(F(1037, 13113)), rel=1e-11)
    assert _at(c, d, 2) == pytest.approx(float(F(4961, 65565)), rel=1e-11)
    # the slope rule of the cross moments (the b of the same blend)
    assert _at(weno.slope(a, d), d, 2) == pytest.approx(float(F(1037, 13113)), rel=1e-11)


def test_weno4_blend_on_a_hand_computed_stencil():
    """Zone averages (0, 0, 1, 2, 2, 5, 1) around the centre zone (index 3).

    Candidates (b, c, d) of the stencils {i-3..i} .. {i..i+3}: (41/60, -1/2, -1/6) twice,
    (-7/30, -1/2, 2/3), (-14/3, 13/2, -5/3).  Jiang-Shu IS: 209/80, 209/80, 277/15, 3779/12.
    With gamma = (1, 10, 10, 1)/22 and omega = (gamma / IS^2) normalised, the blend is the
    three fractions below.
    """
    a = _line([0, 0, 1, 2, 2, 5, 1], 0)
    b, c, e = weno.weno4(a, 0)
    want = (F(14286369718388611, 21421408121334138), F(-3569927558503151, 7140469373778046),
            F(-1625721383126890, 10710704060667069))
    for got, w in zip((b, c, e), want):
        assert _at(got, 0, 3) == pytest.approx(float(w), rel=1e-11)


def test_face_b_third_order_weights_on_hand_computed_faces():
    """Faces B(i-3/2), B(i-1/2), B(i+1/2), B(i+3/2) = 0, 1, 3, 7 (Eqs. 22-24).

    Candidates (b0, bx, bxx): Eq. 22 (23/12, 2, 1/2), Eq. 23 (22/12, 2, 1).  IS (Eq. 24, the
    Jiang-Shu integral): 61/12 and 25/3.  alpha = (1/2) / IS^2: 72/3721 and 9/1250, so
    omega = (90000, 33489) / 123489.  Blend: b0 = 2806758/1481868, bx = 2, bxx = 78489/123489.
    """
    Bf = _line([0, 0, 1, 3, 7, 0], 0)        # face i-1/2 of zone i at index i; centre zone 2
    b0, (bx, bxx) = weno.face_b_moments(Bf, 0, 3)
    assert _at(b0, 0, 2) == pytest.approx(float(F(2806758, 1481868)), rel=1e-11)
    assert _at(bx, 0, 2) == pytest.approx(2.0, rel=1e-14)
    assert _at(bxx, 0, 2) == pytest.approx(float(F(78489, 123489)), rel=1e-11)


def test_face_b_fourth_order_weights_on_hand_computed_faces():
    """Faces B(i-5/2) .. B(i+5/2) = 0, 1, 1, 2, 4, 3 (Eqs. 25-29).

    Candidates (b0, bx, bxx, bxxx): Eq. 26 (4/3, 29/30, 1, 1/3), Eq. 27 (17/12, 1, 1/2, 0),
    Eq. 28 (5/4, 16/15, 3/2, -2/3).  IS (Eq. 29, the Jiang-Shu integral): 1741/180, 25/12,
    5059/180.  omega = ((1/4, 1/2, 1/4) / IS^2) normalised; the blend is the fractions below.
    """
    Bf = _line([0, 0, 1, 1, 2, 4, 3, 0], 0)  # centre zone 3: its faces are indices 3 and 4
    b0, mom = weno.face_b_moments(Bf, 0, 4)
    want = (F(2701560094155049, 1910125883966064), F(318171207878719, 318354313994344),
            F(163628731794047, 318354313994344), F(915530578125, 159177156997172))
    for got, w in zip((b0,) + tuple(mom), want):
        assert _at(got, 0, 3) == pytest.approx(float(w), rel=1e-11)
