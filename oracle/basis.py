"""Space-time modal bases of the ADER-CG scheme (Sec. II.1-II.2, Eqs. 9-16; App. D, Eqs. D.2, D.7, D.12).

Mode k (1-based, as in the paper) of order M is the product
``P_a(xi) P_b(eta) P_c(zeta) Q_d(tau)`` and is stored as the exponent tuple
``(a, b, c, d)`` at position k-1.  P_0..P_3 are the Hermite-type polynomials
of Eq. 9, Q_d(tau) = tau**d (Eq. 13).  The reference element is
(xi, eta, zeta, tau) in [-1/2, 1/2]^3 x [0, 1] (Sec. II, after Eq. 4).

Parity of this module is pinned in tests/test_oracle_basis.py against the
paper's printed transcriptions and closed forms.
"""
from fractions import Fraction as Fr

import numpy as np

# Eq. 9: P0 = 1, P1 = x, P2 = x^2 - 1/12, P3 = x^3 - (3/20) x   (ascending powers)
P_MONO = (
    (Fr(1),),
    (Fr(0), Fr(1)),
    (Fr(-1, 12), Fr(0), Fr(1)),
    (Fr(0), Fr(-3, 20), Fr(0), Fr(1)),
)

# Eq. 14 (order 2), Eq. 15 (order 3), Eq. 16 (order 4): exponent tuples (a,b,c,d)
_O2 = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1)]
_SPATIAL_O3 = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0),
               (2, 0, 0, 0), (0, 2, 0, 0), (0, 0, 2, 0),
               (1, 1, 0, 0), (0, 1, 1, 0), (1, 0, 1, 0)]          # Eq. 11: w8=xy, w9=yz, w10=xz
_O3 = _SPATIAL_O3 + [(0, 0, 0, 1), (0, 0, 0, 2),
                     (1, 0, 0, 1), (0, 1, 0, 1), (0, 0, 1, 1)]    # Eq. 15: u11..u15
_SPATIAL_O4 = _SPATIAL_O3 + [(3, 0, 0, 0), (0, 3, 0, 0), (0, 0, 3, 0),
                             (2, 1, 0, 0), (2, 0, 1, 0),
                             (1, 2, 0, 0), (0, 2, 1, 0),
                             (1, 0, 2, 0), (0, 1, 2, 0),
                             (1, 1, 1, 0)]                        # Eq. 12: w11..w20
_O4 = _SPATIAL_O4 + [(0, 0, 0, 1), (0, 0, 0, 2), (0, 0, 0, 3),
                     (1, 0, 0, 1), (0, 1, 0, 1), (0, 0, 1, 1),
                     (1, 0, 0, 2), (0, 1, 0, 2), (0, 0, 1, 2),
                     (2, 0, 0, 1), (0, 2, 0, 1), (0, 0, 2, 1),
                     (1, 1, 0, 1), (0, 1, 1, 1), (1, 0, 1, 1)]    # Eq. 16: u21..u35

MODES = {2: _O2, 3: _O3, 4: _O4}
LS = {2: 4, 3: 10, 4: 20}          # number of spatial modes (Sec. II.1)
L = {2: 5, 3: 15, 4: 35}           # number of space-time modes (Sec. II.2)

# Facial space-time bases in (t1, t2, tau) on an x-face (Eqs. D.2, D.7, D.12)
FACE_MODES = {
    2: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
    3: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (0, 2, 0), (1, 1, 0),
        (0, 0, 1), (0, 0, 2), (1, 0, 1), (0, 1, 1)],
    4: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (0, 2, 0), (1, 1, 0),
        (3, 0, 0), (0, 3, 0), (2, 1, 0), (1, 2, 0),
        (0, 0, 1), (0, 0, 2), (0, 0, 3), (1, 0, 1), (0, 1, 1),
        (1, 0, 2), (0, 1, 2), (2, 0, 1), (0, 2, 1), (1, 1, 1)],
}


def P(a, x):
    """Eq. 9 evaluated at x (array), by its monomial expansion."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for p, c in enumerate(P_MONO[a]):
        out = out + float(c) * x ** p
    return out


def Q(d, t):
    """Eq. 13: Q_d(tau) = tau^d."""
    return np.asarray(t, dtype=np.float64) ** d


def eval_basis(order, pts):
    """Matrix V[n, k] = phi_k(pts[n]) for the order-M space-time basis (Eqs. 14-16)."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 4)
    V = np.empty((pts.shape[0], L[order]))
    for k, (a, b, c, d) in enumerate(MODES[order]):
        V[:, k] = P(a, pts[:, 0]) * P(b, pts[:, 1]) * P(c, pts[:, 2]) * Q(d, pts[:, 3])
    return V


def eval_face_basis(order, pts):
    """Matrix W[n, k] = psi_k(pts[n]) for the facial basis (Eqs. D.2, D.7, D.12); pts are (t1, t2, tau)."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    W = np.empty((pts.shape[0], len(FACE_MODES[order])))
    for k, (a, b, d) in enumerate(FACE_MODES[order]):
        W[:, k] = P(a, pts[:, 0]) * P(b, pts[:, 1]) * Q(d, pts[:, 2])
    return W


# ---------------------------------------------------------------- exact 1-D algebra
def _poly_int(coefs, lo, hi):
    """Exact integral of an ascending-power polynomial with Fraction coefficients."""
    return sum(c * (Fr(hi) ** (p + 1) - Fr(lo) ** (p + 1)) / (p + 1) for p, c in enumerate(coefs))


def _deriv_in_P(a):
    """d/dx P_a expressed in the P basis: returns {a': coef} (exact)."""
    mono = [p * c for p, c in enumerate(P_MONO[a])][1:]   # derivative, ascending powers
    out = {}
    # peel off the top power with the P of that degree (P_n is monic of degree n)
    mono = list(mono)
    while mono and any(m != 0 for m in mono):
        deg = len(mono) - 1
        while deg >= 0 and mono[deg] == 0:
            deg -= 1
        if deg < 0:
            break
        c = mono[deg]
        out[deg] = out.get(deg, Fr(0)) + c
        for p, pc in enumerate(P_MONO[deg]):
            mono[p] -= c * pc
    return out


def P_average(a, lo=Fr(-1, 2), hi=Fr(1, 2)):
    """Exact average of P_a over [lo, hi]."""
    return _poly_int(P_MONO[a], lo, hi) / (Fr(hi) - Fr(lo))


def P_at(a, x):
    """Exact value of P_a at a rational point."""
    return sum(c * Fr(x) ** p for p, c in enumerate(P_MONO[a]))


def deriv_matrix(order, axis):
    """D[j, k]: coefficient of mode j in d(phi_k)/d(coordinate `axis`), axis 0..2 spatial (xi, eta, zeta)."""
    modes = MODES[order]
    idx = {m: i for i, m in enumerate(modes)}
    D = np.zeros((len(modes), len(modes)))
    for k, m in enumerate(modes):
        a = m[axis]
        if a == 0:
            continue
        for a2, c in _deriv_in_P(a).items():
            m2 = list(m)
            m2[axis] = a2
            D[idx[tuple(m2)], k] += float(c)
    return D


def evolutionary_map(order):
    """For each evolutionary mode k (d >= 1) the index j of the mode (a,b,c,d-1) and the factor d.

    d/dtau of P_a P_b P_c tau^d is d * P_a P_b P_c tau^(d-1) (Eq. 13), which is how
    the evolutionary modes of Eqs. 14-16 enter du/dtau.
    """
    modes = MODES[order]
    idx = {m: i for i, m in enumerate(modes)}
    out = []
    for k, (a, b, c, d) in enumerate(modes):
        if d >= 1:
            out.append((k, idx[(a, b, c, d - 1)], d))
    return out


def spacetime_integral_weights(order, fixed):
    """Weights w[k] such that the average of u over the free coordinates equals sum_k w[k] u_hat[k].

    `fixed` maps a coordinate index (0..3) to the rational value it is held at;
    the free spatial coordinates are averaged over [-1/2, 1/2] and tau over [0, 1].
    This is the plain definition of Eqs. 54, 55 and 57.
    """
    w = np.zeros(L[order])
    for k, m in enumerate(MODES[order]):
        val = Fr(1)
        for ax in range(4):
            e = m[ax]
            if ax in fixed:
                val *= P_at(e, fixed[ax]) if ax < 3 else Fr(fixed[ax]) ** e
            else:
                val *= P_average(e) if ax < 3 else Fr(1, e + 1)
        w[k] = float(val)
    return w


def face_integral_weights(order, fixed):
    """Same as spacetime_integral_weights for the facial basis (t1, t2, tau): Eqs. D.5, D.10, D.15."""
    modes = FACE_MODES[order]
    w = np.zeros(len(modes))
    for k, m in enumerate(modes):
        val = Fr(1)
        for ax in range(3):
            e = m[ax]
            if ax in fixed:
                val *= P_at(e, fixed[ax]) if ax < 2 else Fr(fixed[ax]) ** e
            else:
                val *= P_average(e) if ax < 2 else Fr(1, e + 1)
        w[k] = float(val)
    return w
