"""One ADER-WENO time step, the CFL time step and the SSP-RK comparison (Sec. II, Eqs. 6, 8, 18-20).

State layout (same as the CUDA boundary): U has shape (5, nz, ny, nx) with
(rho, rho vx, rho vy, rho vz, eps) as zone averages; for MHD Bface has shape
(3, nz, ny, nx) where Bface[d][..., i_d] is the normal field on the face
i_d - 1/2 of direction d.  Periodic boundaries in every direction.

Readings (the paper is silent, G13):
* CFL time step: dt = cfl / max_zones sum_d (|v_d| + c_d) / dx_d with c_d the
  fast speed in direction d (the sound speed for Euler).
* SSP-RK face rule: the App. D facial quadrature applied to the reconstructed
  polynomial with every time mode zero.
"""
import numpy as np

from . import basis, faces, physics, predictor, riemann, weno


def _face_fluxes(Uhat, order, gamma, solver, zone_avg, mhd):
    """Numerical fluxes Fbar[d] on faces i+1/2 (stored at zone i) and, for MHD, edge data."""
    solve = riemann.SOLVERS[solver]
    F = []
    edge_data = []
    for d in range(3):
        up = faces.face_quantities(Uhat, order, gamma, d, +1, edges=mhd)
        um = faces.face_quantities(Uhat, order, gamma, d, -1, edges=mhd)
        # left state: zone i (its + face); right state: zone i+1 (its - face)
        R = [weno.shift(x, d, 1) for x in um[:3]]
        zR = weno.shift(zone_avg, d, 1)
        F.append(solve(d, gamma, up[0], R[0], up[1], R[1], up[2], R[2], zone_avg, zR))
        if mhd:
            edge_data.append((up, um))
    return F, edge_data


def zone_state(U, Bface, order):
    """Zone averages of all variables and the spatial modes W (LS, nvar, ...) (Sec. II.1, Sec. III)."""
    Wh = np.stack([weno.reconstruct(U[v], order) for v in range(5)], axis=1)
    if Bface is None:
        return U, Wh
    WB = []
    zB = []
    for d in range(3):
        b0, mom = weno.face_b_moments(Bface[d], d, order)
        zB.append(b0)
        WB.append(weno.reconstruct(b0, order, moments1d={d: mom}))
    Uz = np.concatenate([U, np.stack(zB)], axis=0)
    W = np.concatenate([Wh, np.stack(WB, axis=1)], axis=1)
    return Uz, W


def ader_step(U, dx, dt, order, form="nodal", solver="hll", gamma=1.4, Bface=None,
              n_iter=None, tol=None, guess=None, return_iters=False):
    """Ubar^{n+1} by Eq. 6 (and B_face^{n+1} by Eq. 8 for MHD) after one ADER step of size dt."""
    mhd = Bface is not None
    Uz, W = zone_state(U, Bface, order)
    Uhat, iters = predictor.predict(W, order, form, gamma, dt, dx, n_iter=n_iter, tol=tol, guess=guess)
    F, edge_data = _face_fluxes(Uhat, order, gamma, solver, Uz, mhd)
    Un = U.copy()
    for d in range(3):
        Un = Un - (dt / dx[d]) * (F[d][:5] - weno.shift(F[d][:5], d, -1))
    out = Un
    if mhd:
        Bn = ct_update(Bface, F, edge_data, Uz, order, gamma, solver, dt, dx)
        out = (Un, Bn)
    if return_iters:
        return out, iters
    return out


def max_dt(U, dx, cfl, gamma=1.4, Bface=None):
    """dt = cfl / max over zones of sum_d (|v_d| + c_d)/dx_d (reading of the CFL rule, Secs. II.d, VI)."""
    if Bface is not None:
        Uz, _ = zone_state(U, Bface, 2)
        Uz = Uz[:, ...]
        zb = [weno.face_b_moments(Bface[d], d, 2)[0] for d in range(3)]
        Uz = np.concatenate([U, np.stack(zb)], axis=0)
    else:
        Uz = U
    s = 0.0
    for d in range(3):
        s = s + (np.abs(Uz[1 + d] / Uz[0]) + physics.fast_speed(Uz, gamma, d)) / dx[d]
    return cfl / float(np.max(s))


# ----------------------------------------------------------------------------- constrained transport
def ct_update(Bface, F, edge_data, Uz, order, gamma, solver, dt, dx):
    raise NotImplementedError("MHD constrained transport")


# ----------------------------------------------------------------------------- SSP-RK, Sec. II.d
def rk_operator(U, dx, order, solver="hll", gamma=1.4):
    """L(U) = -sum_d (Fbar(i+1/2) - Fbar(i-1/2))/dx_d with the spatial-only face rule."""
    Uz, W = zone_state(U, None, order)
    LSn, Ln = basis.LS[order], basis.L[order]
    Uhat = np.zeros((Ln,) + W.shape[1:])
    Uhat[:LSn] = W
    F, _ = _face_fluxes(Uhat, order, gamma, solver, Uz, False)
    out = np.zeros_like(U)
    for d in range(3):
        out = out - (F[d][:5] - weno.shift(F[d][:5], d, -1)) / dx[d]
    return out


RK_STAGES = {
    # Eq. 18 (order 2), Eq. 19 (order 3) and Eq. 20 (order 4): each stage is
    # U(s) = sum_j a[s][j] U(j) + sum_j b[s][j] dt L(U(j)), j over U^n = U(0), U(1), ...
    2: ([[1.0], [0.5, 0.5]],
        [[1.0], [0.0, 0.5]]),
    3: ([[1.0], [0.75, 0.25], [1.0 / 3.0, 0.0, 2.0 / 3.0]],
        [[1.0], [0.0, 0.25], [0.0, 0.0, 2.0 / 3.0]]),
    4: ([[1.0],
         [0.44437049406734, 0.55562950593266],
         [0.62010185138540, 0.0, 0.37989814861460],
         [0.17807995410773, 0.0, 0.0, 0.82192004589227],
         [0.00683325884039, 0.0, 0.51723167208978, 0.12759831133288, 0.34833675773694]],
        [[0.39175222700392],
         [0.0, 0.36841059262959],
         [0.0, 0.0, 0.25189177424738],
         [0.0, 0.0, 0.0, 0.54497475021237],
         [0.0, 0.0, 0.0, 0.08460416338212, 0.22600748319395]]),
}


def rk_step(U, dx, dt, order, solver="hll", gamma=1.4):
    """One SSP-RK step of the order's scheme (Eq. 18, 19 or 20)."""
    A, B = RK_STAGES[order]
    states = [U]
    ops = []
    for s in range(len(A)):
        ops.append(rk_operator(states[-1], dx, order, solver, gamma))
        nxt = np.zeros_like(U)
        for j, a in enumerate(A[s]):
            if a != 0.0:
                nxt = nxt + a * states[j]
        for j, b in enumerate(B[s]):
            if b != 0.0:
                nxt = nxt + b * dt * ops[j]
        states.append(nxt)
    return states[-1]
