"""Euler and ideal-MHD physics in Gaussian units (Sec. II, Eq. 3).

Conserved variables U = (rho, rho vx, rho vy, rho vz, eps[, Bx, By, Bz]) with
eps = rho v^2/2 + P/(gamma-1) + B^2/(8 pi).  Euler is the B = 0 case (5 vars).
Arrays carry the variable index on axis 0 and any number of trailing axes.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi
EIGHT_PI = 8.0 * np.pi


def pressure(U, gamma):
    """P from the total energy of Eq. 3."""
    rho = U[0]
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    me = 0.0
    if U.shape[0] == 8:
        me = (U[5] ** 2 + U[6] ** 2 + U[7] ** 2) / EIGHT_PI
    return (gamma - 1.0) * (U[4] - ke - me)


def flux(U, gamma, d):
    """Physical flux in direction d (0: F, 1: G, 2: H) of Eq. 3."""
    nv = U.shape[0]
    rho = U[0]
    v = [U[1] / rho, U[2] / rho, U[3] / rho]
    P = pressure(U, gamma)
    out = np.empty_like(U)
    if nv == 5:
        vn = v[d]
        out[0] = U[1 + d]
        for c in range(3):
            out[1 + c] = U[1 + c] * vn
        out[1 + d] = out[1 + d] + P
        out[4] = (U[4] + P) * vn
        return out
    B = [U[5], U[6], U[7]]
    B2 = B[0] ** 2 + B[1] ** 2 + B[2] ** 2
    vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2]
    Ptot = P + B2 / EIGHT_PI
    vn, Bn = v[d], B[d]
    out[0] = U[1 + d]
    for c in range(3):
        out[1 + c] = U[1 + c] * vn - Bn * B[c] / FOUR_PI
    out[1 + d] = out[1 + d] + Ptot
    out[4] = (U[4] + Ptot) * vn - Bn * vB / FOUR_PI
    # induction part: flux of B_c in direction d is v_d B_c - v_c B_d (zero for c = d)
    for c in range(3):
        out[5 + c] = vn * B[c] - v[c] * Bn
    return out


def sound_speed2(U, gamma):
    return gamma * pressure(U, gamma) / U[0]


def fast_speed(U, gamma, d):
    """Fast magnetosonic speed in direction d (sound speed for Euler)."""
    a2 = sound_speed2(U, gamma)
    if U.shape[0] == 5:
        return np.sqrt(a2)
    rho = U[0]
    B2 = (U[5] ** 2 + U[6] ** 2 + U[7] ** 2) / (FOUR_PI * rho)
    Bn2 = U[5 + d] ** 2 / (FOUR_PI * rho)
    s = a2 + B2
    disc = np.sqrt(np.maximum(s * s - 4.0 * a2 * Bn2, 0.0))
    return np.sqrt(0.5 * (s + disc))


def physical(U, gamma):
    """True where rho > 0 and P > 0."""
    return (U[0] > 0.0) & (pressure(U, gamma) > 0.0)


def jacobian(U, gamma, d):
    """A = dF_d/dU at one state U (1-D array), by complex-step differentiation of `flux`.

    The derivative of an analytic function by a complex step h has no
    cancellation error, so A is exact to round-off.  Used by the linearized
    Riemann solver and by the eigen-structure pins.
    """
    nv = U.shape[0]
    A = np.empty((nv, nv))
    step = 1e-30
    for j in range(nv):
        Uc = U.astype(np.complex128)
        Uc[j] += 1j * step
        A[:, j] = flux_complex(Uc, gamma, d).imag / step
    return A


def flux_complex(U, gamma, d):
    """`flux` for complex arrays (complex-step differentiation)."""
    nv = U.shape[0]
    rho = U[0]
    v = [U[1] / rho, U[2] / rho, U[3] / rho]
    ke = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
    out = np.empty_like(U)
    if nv == 5:
        P = (gamma - 1.0) * (U[4] - ke)
        out[0] = U[1 + d]
        for c in range(3):
            out[1 + c] = U[1 + c] * v[d]
        out[1 + d] = out[1 + d] + P
        out[4] = (U[4] + P) * v[d]
        return out
    B = [U[5], U[6], U[7]]
    B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
    P = (gamma - 1.0) * (U[4] - ke - B2 / EIGHT_PI)
    vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2]
    Ptot = P + B2 / EIGHT_PI
    out[0] = U[1 + d]
    for c in range(3):
        out[1 + c] = U[1 + c] * v[d] - B[d] * B[c] / FOUR_PI
    out[1 + d] = out[1 + d] + Ptot
    out[4] = (U[4] + Ptot) * v[d] - B[d] * vB / FOUR_PI
    for c in range(3):
        out[5 + c] = v[d] * B[c] - v[c] * B[d]
    return out


def prim_to_cons(rho, vx, vy, vz, P, gamma, B=None):
    ke = 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    if B is None:
        return np.stack([rho, rho * vx, rho * vy, rho * vz, P / (gamma - 1.0) + ke])
    Bx, By, Bz = B
    me = (Bx * Bx + By * By + Bz * Bz) / EIGHT_PI
    return np.stack([rho, rho * vx, rho * vy, rho * vz, P / (gamma - 1.0) + ke + me, Bx, By, Bz])
