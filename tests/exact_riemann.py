"""Exact solution of the 1-D Euler Riemann problem (ideal gas), for the Sod pin.

Standard two-rarefaction/shock construction: Newton iteration on the star
pressure, then sampling of the self-similar solution at x/t.  Tests only.
"""
import numpy as np


def _fk(p, rho, P, a, g):
    if p > P:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * P
        f = (p - P) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (B + p)) * (1.0 - (p - P) / (2.0 * (B + p)))
    else:
        f = 2.0 * a / (g - 1.0) * ((p / P) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * a) * (p / P) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g):
    rL, uL, PL = left
    rR, uR, PR = right
    aL, aR = np.sqrt(g * PL / rL), np.sqrt(g * PR / rR)
    p = max(1e-8, 0.5 * (PL + PR))
    for _ in range(100):
        fL, dL = _fk(p, rL, PL, aL, g)
        fR, dR = _fk(p, rR, PR, aR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        p = max(1e-10, p - dp)
        if abs(dp) < 1e-14 * p:
            break
    fL, _ = _fk(p, rL, PL, aL, g)
    fR, _ = _fk(p, rR, PR, aR, g)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def sample(left, right, g, s):
    """(rho, u, P) at similarity coordinate s = x/t (array)."""
    rL, uL, PL = left
    rR, uR, PR = right
    aL, aR = np.sqrt(g * PL / rL), np.sqrt(g * PR / rR)
    ps, us = star_state(left, right, g)
    s = np.asarray(s, dtype=float)
    rho, u, P = np.empty_like(s), np.empty_like(s), np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for i, x in np.ndenumerate(s):
        if x <= us:        # left of contact
            if ps > PL:    # left shock
                SL = uL - aL * np.sqrt((g + 1) / (2 * g) * ps / PL + (g - 1) / (2 * g))
                st = (rL * (ps / PL + gm) / (gm * ps / PL + 1.0), us, ps) if x >= SL else (rL, uL, PL)
            else:          # left rarefaction
                head, tail = uL - aL, us - aL * (ps / PL) ** ((g - 1) / (2 * g))
                if x < head:
                    st = (rL, uL, PL)
                elif x > tail:
                    st = (rL * (ps / PL) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) + gm / aL * (uL - x)
                    st = (rL * c ** (2.0 / (g - 1)), 2.0 / (g + 1) * (aL + (g - 1) / 2 * uL + x),
                          PL * c ** (2.0 * g / (g - 1)))
        else:
            if ps > PR:
                SR = uR + aR * np.sqrt((g + 1) / (2 * g) * ps / PR + (g - 1) / (2 * g))
                st = (rR * (ps / PR + gm) / (gm * ps / PR + 1.0), us, ps) if x <= SR else (rR, uR, PR)
            else:
                head, tail = uR + aR, us + aR * (ps / PR) ** ((g - 1) / (2 * g))
                if x > head:
                    st = (rR, uR, PR)
                elif x < tail:
                    st = (rR * (ps / PR) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) - gm / aR * (uR - x)
                    st = (rR * c ** (2.0 / (g - 1)), 2.0 / (g + 1) * (-aR + (g - 1) / 2 * uR + x),
                          PR * c ** (2.0 * g / (g - 1)))
        rho[i], u[i], P[i] = st
    return rho, u, P
