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


def transonic(vL, cL, vR, cR):
    """A face's Riemann problem is transonic when a fast wave speed changes sign between its two
    barycentre states, (v - c)_L (v - c)_R < 0 or (v + c)_L (v + c)_R < 0: a sonic point lies in the
    fan (the reading of Sec. II.3's "transonic", which the paper does not define)."""
    return ((vL - cL) * (vR - cR) < 0.0) | ((vL + cL) * (vR + cR) < 0.0)


def hll(d, gamma, ubL, ubR, uL, uR, FL, FR, zL, zR, double_transonic=False):
    """Eq. 56 (the HLL form of Eq. 17).  double_transonic: twice the third (dissipative) term at
    transonic faces, the option Sec. V gives for the electric fields."""
    ubL = _safe(ubL, zL, gamma)
    ubR = _safe(ubR, zR, gamma)
    vL = ubL[1 + d] / ubL[0]
    vR = ubR[1 + d] / ubR[0]
    cL = physics.fast_speed(ubL, gamma, d)
    cR = physics.fast_speed(ubR, gamma, d)
    lamL = np.minimum(np.minimum(vL - cL, vR - cR), 0.0)
    lamR = np.maximum(np.maximum(vL + cL, vR + cR), 0.0)
    den = lamR - lamL
    w = np.where(transonic(vL, cL, vR, cR), 2.0, 1.0) if double_transonic else 1.0
    return (lamR * FL - lamL * FR + w * lamR * lamL * (uR - uL)) / den     # Eq. 56


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
    return _mhd_abs_jacobian(Ustar, gamma, d, A, keep), keep


def _mhd_abs_jacobian(Ustar, gamma, d, A, keep):
    """|A| of the seven-wave MHD system (the row and column of B_d removed), by symmetrisation.

    In primitive variables W = (rho, v, P, B_t1, B_t2) the Jacobian is A_W = M^-1 A M with M = dU/dW.
    Replacing rho by s = P - a^2 rho separates the entropy wave (eigenvalue v_d); the remaining six rows
    (v, P, B_t) become symmetric under S = diag(rho, rho, rho, 1/(gamma P), 1/(4 pi), 1/(4 pi)).  So
    |A| = M T^-1 diag(|v_d|, S^-1/2 |S^1/2 A6 S^-1/2| S^1/2) T M^-1, with the absolute value of the symmetric
    matrix taken from its orthonormal eigen-decomposition (well conditioned also where wave speeds coincide).
    """
    n = Ustar.shape[1]
    rho = Ustar[0]
    v = [Ustar[1 + c] / rho for c in range(3)]
    P = physics.pressure(Ustar, gamma)
    B = [Ustar[5 + c] for c in range(3)]
    W = np.stack([rho, v[0], v[1], v[2], P, B[0], B[1], B[2]])          # (8, n)
    M = np.empty((n, 8, 8))
    step = 1e-30
    for j in range(8):
        Wc = W.astype(np.complex128)
        Wc[j] += 1j * step
        Uc = physics.prim_to_cons(Wc[0], Wc[1], Wc[2], Wc[3], Wc[4], gamma, (Wc[5], Wc[6], Wc[7]))
        M[:, :, j] = (Uc.imag / step).T
    M = M[:, keep][:, :, keep]
    AW = np.linalg.solve(M, A @ M)
    a2 = gamma * P / rho
    T = np.broadcast_to(np.eye(7), (n, 7, 7)).copy()
    T[:, 0, 0] = -a2
    T[:, 0, 4] = 1.0
    Ti = np.broadcast_to(np.eye(7), (n, 7, 7)).copy()
    Ti[:, 0, 0] = -1.0 / a2
    Ti[:, 0, 4] = 1.0 / a2
    Ap = T @ AW @ Ti
    sq = np.stack([np.sqrt(rho)] * 3 + [1.0 / np.sqrt(gamma * P)] + [np.full(n, 1.0 / np.sqrt(4.0 * np.pi))] * 2,
                  axis=1)                                               # S^1/2 of (v, P, B_t1, B_t2)
    X = sq[:, :, None] * Ap[:, 1:, 1:] / sq[:, None, :]
    X = 0.5 * (X + np.swapaxes(X, 1, 2))
    lam, Q = np.linalg.eigh(X)
    absX = np.einsum("nij,nj,nkj->nik", Q, np.abs(lam), Q)
    absAp = np.zeros((n, 7, 7))
    absAp[:, 0, 0] = np.abs(Ap[:, 0, 0])
    absAp[:, 1:, 1:] = absX / sq[:, :, None] * sq[:, None, :]
    return M @ (Ti @ absAp @ T) @ np.linalg.inv(M)


def linearized(d, gamma, ubL, ubR, uL, uR, FL, FR, zL, zR, double_transonic=False):
    """F = (F_L + F_R)/2 - |A| (u_R - u_L)/2 with |A| at the mean barycentre state (Sec. II.3).
    double_transonic: twice the dissipative term at transonic faces (see `transonic`)."""
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
    D = D.reshape(out.shape)
    if double_transonic:
        vL, vR = ubL[1 + d] / ubL[0], ubR[1 + d] / ubR[0]
        cL, cR = physics.fast_speed(ubL, gamma, d), physics.fast_speed(ubR, gamma, d)
        D = D * np.where(transonic(vL, cL, vR, cR), 2.0, 1.0)
    return out - 0.5 * D


SOLVERS = {"hll": hll, "linearized": linearized}
