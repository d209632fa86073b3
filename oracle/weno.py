"""Zone-centred WENO reconstruction to Hermite modes (Sec. II.1) and the face-B WENO of Sec. III.

The paper defers the zone-centred scheme to its ref. [11] and gives only the
Hermite form of the smoothness measure (Eqs. 24 and 29) and, for the normal
magnetic field, the stencils of Eqs. 22-23 and 26-28.  The rest is a reading,
fixed here and used by both sides (the readings are the module constants):

* 1-D, per direction, on zone averages: order 3 (and order 2) blends the three
  3-zone stencils {i-2..i}, {i-1..i+1}, {i..i+2}; order 4 blends the four
  4-zone stencils {i-3..i} .. {i..i+3}.  Each candidate is the polynomial
  a + b P1 + c P2 (+ d P3) whose averages over the stencil zones equal the zone
  averages (a = the zone's own average).  Order 2 keeps only b ("r = 3 WENO
  slopes", Sec. VI).
* Smoothness: IS = b^2 + 13 c^2/3 (Eq. 24 form) or
  (b + d/10)^2 + 13 c^2/3 + 781 d^2/20 (Eq. 29 form).
* Weights: omega_s = gamma_s / (EPS + IS_s)^2, normalised.
* Cross moments: the WENO slope S_e (order-3 candidate set, b kept) of a
  moment field in a transverse direction e, symmetrised:
  w8 = (S_eta w2 + S_xi w3)/2, w9 = (S_zeta w3 + S_eta w4)/2,
  w10 = (S_zeta w2 + S_xi w4)/2; at order 4 also w14 = S_eta w5,
  w15 = S_zeta w5, w16 = S_xi w6, w17 = S_zeta w6, w18 = S_xi w7,
  w19 = S_eta w7 and w20 = (S_zeta w8 + S_xi w9 + S_eta w10)/3.

Arrays: a zone field has the grid on its last three axes (z, y, x); direction
0/1/2 = x/y/z.  Boundaries are periodic.
"""
from fractions import Fraction as Fr

import numpy as np

from . import basis

EPS = 1.0e-12
GAMMA_O3 = (1.0 / 12.0, 10.0 / 12.0, 1.0 / 12.0)            # stencils L, C, R
GAMMA_O4 = (1.0 / 22.0, 10.0 / 22.0, 10.0 / 22.0, 1.0 / 22.0)
STENCILS_O3 = ((-2, -1, 0), (-1, 0, 1), (0, 1, 2))
STENCILS_O4 = ((-3, -2, -1, 0), (-2, -1, 0, 1), (-1, 0, 1, 2), (0, 1, 2, 3))
# face-B WENO linear weights (Sec. III gives none)
GAMMA_B_O3 = (0.5, 0.5)
GAMMA_B_O4 = (0.25, 0.5, 0.25)


def axis_of(d):
    return -1 - d


def shift(a, d, k):
    """Value of zone i+k along direction d (periodic)."""
    return np.roll(a, -k, axis=axis_of(d))


def _candidate_map(offsets, deg):
    """Exact matrix M with (b, c, d)[:deg] = M @ (u_{i+k} - u_i for k in offsets, k != 0).

    Solves "cell average over zone k of a + b P1 + c P2 + d P3 equals u_{i+k}".
    """
    ks = [k for k in offsets if k != 0]
    A = [[basis.P_average(p, Fr(k) - Fr(1, 2), Fr(k) + Fr(1, 2)) for p in range(1, deg + 1)] for k in ks]
    n = len(ks)
    # Gauss-Jordan inverse with Fractions
    aug = [row[:] + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        pv = aug[col][col]
        aug[col] = [x / pv for x in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                fac = aug[r][col]
                aug[r] = [x - fac * y for x, y in zip(aug[r], aug[col])]
    inv = [row[n:] for row in aug]
    return ks, np.array([[float(x) for x in row] for row in inv])


_MAPS3 = [_candidate_map(s, 2) for s in STENCILS_O3]
_MAPS4 = [_candidate_map(s, 3) for s in STENCILS_O4]


def smoothness_quadratic(b, c):
    """Eq. 24: smoothness of the candidate a + b P1 + c P2 on its zone, b^2 + 13 c^2 / 3.

    This is the Jiang-Shu measure, the sum over l = 1, 2 of the integral over
    the zone of (d^l p / d xi^l)^2 (unit zone width).
    """
    return b * b + (13.0 / 3.0) * c * c


def smoothness_cubic(b, c, d):
    """Eq. 29: smoothness of a + b P1 + c P2 + d P3, (b + d/10)^2 + 13 c^2 / 3 + 781 d^2 / 20.

    The Jiang-Shu measure of the cubic (derivatives of order 1 to 3).
    """
    return (b + 0.1 * d) ** 2 + (13.0 / 3.0) * c * c + (781.0 / 20.0) * d * d


def _weights(IS, gam):
    """Nonlinear weights omega_s = gamma_s / (EPS + IS_s)^2, normalised to sum to one."""
    alpha = [g / (EPS + s) ** 2 for g, s in zip(gam, IS)]
    tot = sum(alpha)
    return [a / tot for a in alpha]


def weno3(a, d):
    """Order-3 1-D WENO along d: returns (b, c), the P1 and P2 moments."""
    cands = []
    for ks, M in _MAPS3:
        diff = [shift(a, d, k) - a for k in ks]
        b = M[0, 0] * diff[0] + M[0, 1] * diff[1]
        c = M[1, 0] * diff[0] + M[1, 1] * diff[1]
        cands.append((b, c))
    IS = [smoothness_quadratic(b, c) for b, c in cands]
    w = _weights(IS, GAMMA_O3)
    return (sum(wi * bc[0] for wi, bc in zip(w, cands)),
            sum(wi * bc[1] for wi, bc in zip(w, cands)))


def weno4(a, d):
    """Order-4 1-D WENO along d: returns (b, c, e), the P1, P2, P3 moments."""
    cands = []
    for ks, M in _MAPS4:
        diff = [shift(a, d, k) - a for k in ks]
        cands.append(tuple(sum(M[r, j] * diff[j] for j in range(3)) for r in range(3)))
    IS = [smoothness_cubic(b, c, e) for b, c, e in cands]
    w = _weights(IS, GAMMA_O4)
    return tuple(sum(wi * cand[r] for wi, cand in zip(w, cands)) for r in range(3))


def slope(a, d):
    """S_d: WENO slope from the order-3 candidate set (the b of weno3)."""
    return weno3(a, d)[0]


def reconstruct(ubar, order, moments1d=None):
    """Spatial modes w_1..w_LS (Eqs. 10-12) from zone averages; returns array (LS, *ubar.shape).

    `moments1d` optionally supplies, per direction, the 1-D moments to use
    instead of the zone WENO (the face-B WENO of Sec. III for the normal
    magnetic field).
    """
    moments1d = moments1d or {}
    W = np.zeros((basis.LS[order],) + ubar.shape)
    W[0] = ubar
    m = {}
    for d in range(3):
        if d in moments1d:
            m[d] = moments1d[d]
        elif order == 2:
            m[d] = (slope(ubar, d),)
        elif order == 3:
            m[d] = weno3(ubar, d)
        else:
            m[d] = weno4(ubar, d)
    W[1], W[2], W[3] = m[0][0], m[1][0], m[2][0]                # w2, w3, w4
    if order == 2:
        return W
    W[4], W[5], W[6] = m[0][1], m[1][1], m[2][1]                # w5, w6, w7
    W[7] = 0.5 * (slope(W[1], 1) + slope(W[2], 0))              # w8  (xi eta)
    W[8] = 0.5 * (slope(W[2], 2) + slope(W[3], 1))              # w9  (eta zeta)
    W[9] = 0.5 * (slope(W[1], 2) + slope(W[3], 0))              # w10 (xi zeta)
    if order == 3:
        return W
    W[10], W[11], W[12] = m[0][2], m[1][2], m[2][2]             # w11, w12, w13
    W[13] = slope(W[4], 1)                                      # w14 P2(xi)P1(eta)
    W[14] = slope(W[4], 2)                                      # w15 P2(xi)P1(zeta)
    W[15] = slope(W[5], 0)                                      # w16 P1(xi)P2(eta)
    W[16] = slope(W[5], 2)                                      # w17 P2(eta)P1(zeta)
    W[17] = slope(W[6], 0)                                      # w18 P1(xi)P2(zeta)
    W[18] = slope(W[6], 1)                                      # w19 P1(eta)P2(zeta)
    W[19] = (slope(W[7], 2) + slope(W[8], 0) + slope(W[9], 1)) / 3.0   # w20 xi eta zeta
    return W


# ----------------------------------------------------------------------------- Sec. III
def face_b_moments(Bf, d, order):
    """Zone-averaged normal field and its normal moments from face values (Sec. III).

    Bf holds the face-averaged normal component, Bf[..., i] = B at face i-1/2
    along direction d.  Returns (b0, (bx, bxx, bxxx)[:order-1]).
    Order 2: average and difference (Sec. III, opening).  Order 3: Eqs. 21-24.
    Order 4: Eqs. 25-29.
    """
    Bm = Bf                      # B_{i-1/2}
    Bp = shift(Bf, d, 1)         # B_{i+1/2}
    if order == 2:
        return 0.5 * (Bp + Bm), (Bp - Bm,)
    if order == 3:
        Bmm = shift(Bf, d, -1)   # B_{i-3/2}
        Bpp = shift(Bf, d, 2)    # B_{i+3/2}
        s1 = ((8.0 * Bm - Bmm + 5.0 * Bp) / 12.0, Bp - Bm, (Bp + Bmm - 2.0 * Bm) / 2.0)   # Eq. 22
        s2 = ((8.0 * Bp - Bpp + 5.0 * Bm) / 12.0, Bp - Bm, (Bm + Bpp - 2.0 * Bp) / 2.0)   # Eq. 23
        cands = (s1, s2)
        IS = [smoothness_quadratic(c[1], c[2]) for c in cands]                             # Eq. 24
        w = _weights(IS, GAMMA_B_O3)
        out = [sum(wi * c[r] for wi, c in zip(w, cands)) for r in range(3)]
        return out[0], (out[1], out[2])
    Bmm = shift(Bf, d, -1)
    Bmmm = shift(Bf, d, -2)      # B_{i-5/2}
    Bpp = shift(Bf, d, 2)
    Bppp = shift(Bf, d, 3)       # B_{i+5/2}
    s1 = ((9 * Bp + 19 * Bm - 5 * Bmm + Bmmm) / 24.0,
          (59 * Bp - 57 * Bm - 3 * Bmm + Bmmm) / 60.0,
          (3 * Bp - 7 * Bm + 5 * Bmm - Bmmm) / 4.0,
          (Bp - 3 * Bm + 3 * Bmm - Bmmm) / 6.0)                                         # Eq. 26
    s2 = ((-Bpp + 13 * Bp + 13 * Bm - Bmm) / 24.0,
          (-Bpp + 63 * Bp - 63 * Bm + Bmm) / 60.0,
          (Bpp - Bp - Bm + Bmm) / 4.0,
          (Bpp - 3 * Bp + 3 * Bm - Bmm) / 6.0)                                          # Eq. 27
    s3 = ((Bppp - 5 * Bpp + 19 * Bp + 9 * Bm) / 24.0,
          (-Bppp + 3 * Bpp + 57 * Bp - 59 * Bm) / 60.0,
          (-Bppp + 5 * Bpp - 7 * Bp + 3 * Bm) / 4.0,
          (Bppp - 3 * Bpp + 3 * Bp - Bm) / 6.0)                                         # Eq. 28
    cands = (s1, s2, s3)
    IS = [smoothness_cubic(c[1], c[2], c[3]) for c in cands]                            # Eq. 29
    w = _weights(IS, GAMMA_B_O4)
    out = [sum(wi * c[r] for wi, c in zip(w, cands)) for r in range(4)]
    return out[0], (out[1], out[2], out[3])
