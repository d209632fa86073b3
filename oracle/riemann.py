"""Space-time averaged numerical fluxes with the eigen-structure frozen at the face barycentre (Sec. II.3, Sec. V).

Inputs per face i+1/2 in direction d: the barycentre states u_bL = u_b+(i),
u_bR = u_b-(i+1) (Eq. 54), the averages <u>_L, <u>_R (Eq. 55) and the averaged
physical fluxes <F>_L, <F>_R (= dx/dt <f>, Eq. 56).

Readings (the paper is silent, G13):
* HLL wave speeds (Eq. 56): lambda_L = min(v_L - c_L, v_R - c_R, 0) and
  lambda_R = max(v_L + c_L, v_R + c_R, 0) with c the fast speed (sound speed
  for Euler) of each barycentre state (Sec. II.3 resets to <= 0 / >= 0).
* Linearized (Roe / Harten-Hyman form of ref. [29]):
  F = (<F>_L + <F>_R)/2 - |A| (<u>_R - <u>_L)/2, |A| = R |Lambda| R^-1 of
  the flux Jacobian at the arithmetic mean of the two barycentre states'
  primitive variables (rho, v, P[, B]).  For MHD the normal field is a
  parameter (its jump carries no wave): A is the 7x7 block without B_n.
* A barycentre state with rho <= 0 or P <= 0 is replaced by its zone's
  average state for the wave speeds / eigen-structure.
"""
import numpy as np

from . import physics


def _safe(ub, uzone, gamma):
    ok = physics.physical(ub, gamma)
    return np.where(ok[None], ub, uzone)


def hll(d, gamma, ubL, ubR, uL, uR, FL, FR, zL, zR):
    ubL = _safe(ubL, zL, gamma)
    ubR = _safe(ubR, zR, gamma)
    vL = ubL[1 + d] / ubL[0]
    vR = ubR[1 + d] / ubR[0]
    cL = physics.fast_speed(ubL, gamma, d)
    cR = physics.fast_speed(ubR, gamma, d)
    lamL = np.minimum(np.minimum(vL - cL, vR - cR), 0.0)
    lamR = np.maximum(np.maximum(vL + cL, vR + cR), 0.0)
    den = lamR - lamL
    return (lamR * FL - lamL * FR + lamR * lamL * (uR - uL)) / den     # Eq. 56


def _prim(U, gamma):
    rho = U[0]
    out = [rho, U[1] / rho, U[2] / rho, U[3] / rho, physics.pressure(U, gamma)]
    if U.shape[0] == 8:
        out += [U[5], U[6], U[7]]
    return out


def abs_jacobian(Ustar, gamma, d):
    """|A| = R|Lambda|R^-1 of dF_d/dU at the states Ustar (nvar, n); returns (n, m, m).

    m = 5 for Euler; m = 7 for MHD (rows/columns of B_d removed).  For Euler
    |A| is evaluated as the interpolating polynomial of |lambda| on the three
    distinct eigenvalues (exact for a diagonalisable A, and well conditioned
    when v_d = 0 makes the middle eigenvalue a triple one).
    """
    nv, n = Ustar.shape
    keep = list(range(nv)) if nv == 5 else [c for c in range(8) if c != 5 + d]
    m = len(keep)
    A = np.empty((n, nv, nv))
    step = 1e-30
    for j in range(nv):
        Uc = Ustar.astype(np.complex128)
        Uc[j] += 1j * step
        A[:, :, j] = (physics.flux_complex(Uc, gamma, d).imag / step).T
    A = A[:, keep][:, :, keep]
    if nv == 5:
        # Euler: A is diagonalisable with the three distinct eigenvalues v - a, v, v + a,
        # so |A| is the Lagrange-Sylvester polynomial p(A) with p(lambda_i) = |lambda_i|.
        v = Ustar[1 + d] / Ustar[0]
        a = np.sqrt(physics.sound_speed2(Ustar, gamma))
        lam = np.stack([v - a, v, v + a], axis=1)
        eye = np.eye(m)[None]
        absA = np.zeros_like(A)
        for i in range(3):
            P = np.broadcast_to(eye, A.shape).copy()
            for j in range(3):
                if j != i:
                    P = P @ ((A - lam[:, j, None, None] * eye) / (lam[:, i] - lam[:, j])[:, None, None])
            absA += np.abs(lam[:, i])[:, None, None] * P
        return absA, keep
    lam, R = np.linalg.eig(A)
    Rinv = np.linalg.inv(R)
    absA = np.einsum("nij,nj,njk->nik", R, np.abs(lam), Rinv)
    return absA.real, keep


def linearized(d, gamma, ubL, ubR, uL, uR, FL, FR, zL, zR):
    ubL = _safe(ubL, zL, gamma)
    ubR = _safe(ubR, zR, gamma)
    pL, pR = _prim(ubL, gamma), _prim(ubR, gamma)
    pm = [0.5 * (a + b) for a, b in zip(pL, pR)]
    B = None if ubL.shape[0] == 5 else (pm[5], pm[6], pm[7])
    Ustar = physics.prim_to_cons(pm[0], pm[1], pm[2], pm[3], pm[4], gamma, B)
    shape = Ustar.shape[1:]
    flat = Ustar.reshape(Ustar.shape[0], -1)
    absA, keep = abs_jacobian(flat, gamma, d)
    jump = (uR - uL).reshape(uR.shape[0], -1)[keep]                  # (m, n)
    diss = np.einsum("nij,jn->in", absA, jump)
    out = 0.5 * (FL + FR)
    D = np.zeros_like(out).reshape(out.shape[0], -1)
    D[keep] = diss
    return out - 0.5 * D.reshape(out.shape)


SOLVERS = {"hll": hll, "linearized": linearized}
