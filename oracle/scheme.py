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
              n_iter=None, tol=None, guess=None, return_iters=False, source=None, emf_transonic=False,
              positivity=False):
    """Ubar^{n+1} by Eq. 6 (and B_face^{n+1} by Eq. 8 for MHD) after one ADER step of size dt.

    `source`: a non-stiff source model of ``oracle.source`` (None: S = 0); it enters the predictor and
    the update through S-bar, the space-time average of the final iterate's source polynomial."""
    mhd = Bface is not None
    Uz, W = zone_state(U, Bface, order)
    res = predictor.predict(W, order, form, gamma, dt, dx, n_iter=n_iter, tol=tol, guess=guess, source=source)
    Uhat, iters = res[0], res[1]
    F, edge_data = _face_fluxes(Uhat, order, gamma, solver, Uz, mhd)
    Un = U.copy()
    for d in range(3):
        Un = Un - (dt / dx[d]) * (F[d][:5] - weno.shift(F[d][:5], d, -1))
    if source is not None:
        Un = Un + res[2][:5]
    out = Un
    if mhd:
        E = edge_emfs(edge_fluxes(edge_data, Uz, order, gamma, solver, emf_transonic))
        Bn = ct_from_emfs(Bface, E, dt, dx)
        if positivity:
            Un, Bn = positivity_fallback(U, Un, F, dx, dt, gamma, None if source is None else res[2][:5], Uz=Uz,
                                         Bnew=Bn, Bold=Bface, E=E)
        out = (Un, Bn)
    elif positivity:
        out = positivity_fallback(U, Un, F, dx, dt, gamma, None if source is None else res[2][:5])
    if return_iters:
        return out, iters
    return out


def positivity_fallback(U, Un, F, dx, dt, gamma, extra=None, passes=3, Uz=None, Bnew=None, Bold=None, E=None):
    """A posteriori positivity fallback (an option of this implementation; the paper names none).

    Zones whose updated average is non-physical (rho <= 0, P <= 0 or not finite) are marked; every face
    of a marked zone takes the first-order HLL flux of the two zone averages of step n (Eq. 56 with the
    zone averages as both the barycentre and the averaged states), and every zone is updated again from
    U^n with the modified fluxes, which its neighbour across each face shares (so the update stays
    conservative).  `passes` rounds, the marks accumulating.  `extra` is the source part (dt S-bar) of the
    update.

    MHD (Uz: the zone states of step n with the zone field of the face-B reconstruction; Bold: the face
    field of step n; E: the step's edge fields (Ex, Ey, Ez); Bnew: the face field after constrained
    transport): a zone's pressure is taken with the mean of its two new face values per direction, and
    the first-order flux is the MHD one, of which the five hydrodynamic components replace the stored
    fluxes.  Every edge that touches a marked zone takes the first-order electric field, Eq. 7's mean of
    the four adjacent faces' first-order fluxes (the edge averages of a piecewise-constant state are its
    zone averages), and the face field is advanced again from step n by Eq. 8 with those edges: low-beta
    zones, whose pressure is a small difference of energies, otherwise keep the high-order field's
    errors.  The discrete curl keeps div B for any edge fields.  Returns Un, or (Un, Bn) for MHD."""
    mark = np.zeros(U.shape[1:], dtype=bool)
    F = [f[:5].copy() for f in F]
    mhd = Bnew is not None
    W = U if Uz is None else Uz
    F1 = []
    for d in range(3):
        WR = weno.shift(W, d, 1)
        F1.append(riemann.hll(d, gamma, W, WR, W, WR, physics.flux(W, gamma, d), physics.flux(WR, gamma, d), W, WR))
    if mhd:
        E1 = edge_emfs([{(e, se): F1[d] for e in range(3) if e != d for se in (+1, -1)} for d in range(3)])
        sh = weno.shift
        # edge touching zones: x-edge (j+1/2, k+1/2) the zones (j..j+1, k..k+1), likewise for y and z
        around = ((1, 2), (0, 2), (0, 1))
    for _ in range(passes):
        if mhd:
            zB = np.stack([0.5 * (Bnew[d] + weno.shift(Bnew[d], d, 1)) for d in range(3)])
            state = np.concatenate([Un, zB])
        else:
            state = Un
        mark |= ~physics.physical(state, gamma)
        if not mark.any():
            break
        for d in range(3):
            face = mark | weno.shift(mark, d, 1)          # face i+1/2 is stored at zone i
            F[d] = np.where(face[None], F1[d][:5], F[d])
        Un = U.copy()
        for d in range(3):
            Un = Un - (dt / dx[d]) * (F[d] - weno.shift(F[d], d, -1))
        if extra is not None:
            Un = Un + extra
        if mhd:
            Em = []
            for c in range(3):
                a, b = around[c]
                touch = mark | sh(mark, a, 1) | sh(mark, b, 1) | sh(sh(mark, a, 1), b, 1)
                Em.append(np.where(touch, E1[c], E[c]))
            Bnew = ct_from_emfs(Bold, Em, dt, dx)
    return (Un, Bnew) if mhd else Un


def max_dt(U, dx, cfl, gamma=1.4, Bface=None):
    """dt = cfl / max over zones of sum_d (|v_d| + c_d)/dx_d (reading of the CFL rule, Secs. II.d, VI).

    For MHD c_d is the fast speed of the zone state whose field is the mean of
    the two face values (Sec. III, opening).
    """
    if Bface is not None:
        zb = [weno.face_b_moments(Bface[d], d, 2)[0] for d in range(3)]
        Uz = np.concatenate([U, np.stack(zb)], axis=0)
    else:
        Uz = U
    s = 0.0
    for d in range(3):
        s = s + (np.abs(Uz[1 + d] / Uz[0]) + physics.fast_speed(Uz, gamma, d)) / dx[d]
    return cfl / float(np.max(s))


# ----------------------------------------------------------------------------- constrained transport
def edge_fluxes(edge_data, Uz, order, gamma, solver, emf_transonic=False):
    """Numerical flux of each face evaluated with the face's edge averages (Sec. II.3, Eq. 57).

    The frozen wave speeds (or eigen-structure) are the face's own (barycentre
    states, Eq. 54); the averaged states and fluxes are the edge averages of
    Eq. 57 and of the facial flux polynomial (Eqs. D.5, D.10, D.15).  Returns
    Fe[d][(e, se)]: flux of the face i+1/2 of direction d at its edge on side se
    of direction e, stored at the face's lower zone.
    """
    solve = riemann.SOLVERS[solver]
    Fe = []
    for d in range(3):
        up, um = edge_data[d]
        ubR = weno.shift(um[0], d, 1)
        zR = weno.shift(Uz, d, 1)
        out = {}
        for key, (uL, FL) in up[3].items():
            uR, FR = um[3][key]
            out[key] = solve(d, gamma, up[0], ubR, uL, weno.shift(uR, d, 1), FL, weno.shift(FR, d, 1), Uz, zR,
                             double_transonic=emf_transonic)
        Fe.append(out)
    return Fe


def edge_emfs(Fe):
    """Edge-averaged electric fields as the mean of the four adjacent faces' edge fluxes (Sec. II.3, Eq. 7).

    Ez on the z-edge (i+1/2, j+1/2), Ey on the y-edge (i+1/2, k+1/2) and Ex on the
    x-edge (j+1/2, k+1/2), each stored at zone (k, j, i).  Eq. 7 identifies
    Ez = -F7 = G6, Ey = F8 = -H6, Ex = -G8 = H7 (0-based components 6, 7, 5 ...).
    """
    sh = weno.shift
    Ez = 0.25 * (-Fe[0][1, +1][6] - sh(Fe[0][1, -1][6], 1, 1) + Fe[1][0, +1][5] + sh(Fe[1][0, -1][5], 0, 1))
    Ey = 0.25 * (Fe[0][2, +1][7] + sh(Fe[0][2, -1][7], 2, 1) - Fe[2][0, +1][5] - sh(Fe[2][0, -1][5], 0, 1))
    Ex = 0.25 * (-Fe[1][2, +1][7] - sh(Fe[1][2, -1][7], 2, 1) + Fe[2][1, +1][6] + sh(Fe[2][1, -1][6], 1, 1))
    return Ex, Ey, Ez


def ct_update(Bface, F, edge_data, Uz, order, gamma, solver, dt, dx, emf_transonic=False):
    """Face-averaged B at t^{n+1} by the discrete Stokes theorem of Eq. 8.  emf_transonic: the electric
    fields take twice the dissipation at transonic faces (Sec. V's option for Eq. 17)."""
    return ct_from_emfs(Bface, edge_emfs(edge_fluxes(edge_data, Uz, order, gamma, solver, emf_transonic)), dt, dx)


def ct_from_emfs(Bface, E, dt, dx):
    """Eq. 8: B^{n+1} = B^n - dt curl E on every face, from the edge fields E = (Ex, Ey, Ez) of edge_emfs."""
    Ex, Ey, Ez = E
    sh = weno.shift
    # Bface[d][..., i_d] is the face i_d - 1/2: its edges are stored one zone lower along d
    Ez_x, Ey_x = sh(Ez, 0, -1), sh(Ey, 0, -1)
    Ex_y, Ez_y = sh(Ex, 1, -1), sh(Ez, 1, -1)
    Ey_z, Ex_z = sh(Ey, 2, -1), sh(Ex, 2, -1)
    Bx = Bface[0] - dt * ((Ez_x - sh(Ez_x, 1, -1)) / dx[1] - (Ey_x - sh(Ey_x, 2, -1)) / dx[2])
    By = Bface[1] - dt * ((Ex_y - sh(Ex_y, 2, -1)) / dx[2] - (Ez_y - sh(Ez_y, 0, -1)) / dx[0])
    Bz = Bface[2] - dt * ((Ey_z - sh(Ey_z, 0, -1)) / dx[0] - (Ex_z - sh(Ex_z, 1, -1)) / dx[1])
    return np.stack([Bx, By, Bz])


def div_b(Bface, dx):
    """Discrete divergence of the face field in every zone (what Eq. 8 preserves)."""
    return sum((weno.shift(Bface[d], d, 1) - Bface[d]) / dx[d] for d in range(3))


# ----------------------------------------------------------------------------- SSP-RK, Sec. II.d
def rk_operator(U, dx, order, solver="hll", gamma=1.4, Bface=None):
    """L(U) = -sum_d (Fbar(i+1/2) - Fbar(i-1/2))/dx_d with the spatial-only face rule.

    MHD (Bface given): also L(B) = -curl E of the face field, the rate whose Euler step is Eq. 8, with the
    edge fields of Eq. 7 from the same spatial-only face and edge data; returns (L(U), L(B)).
    """
    mhd = Bface is not None
    Uz, W = zone_state(U, Bface, order)
    LSn, Ln = basis.LS[order], basis.L[order]
    Uhat = np.zeros((Ln,) + W.shape[1:])
    Uhat[:LSn] = W
    F, edge_data = _face_fluxes(Uhat, order, gamma, solver, Uz, mhd)
    out = np.zeros_like(U)
    for d in range(3):
        out = out - (F[d][:5] - weno.shift(F[d][:5], d, -1)) / dx[d]
    if not mhd:
        return out
    return out, ct_update(np.zeros_like(Bface), F, edge_data, Uz, order, gamma, solver, 1.0, dx)


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


def rk_step(U, dx, dt, order, solver="hll", gamma=1.4, Bface=None):
    """One SSP-RK step of the order's scheme (Eq. 18, 19 or 20); MHD advances (U, Bface) together."""
    A, B = RK_STAGES[order]
    mhd = Bface is not None
    states = [(U, Bface) if mhd else (U,)]
    ops = []
    for s in range(len(A)):
        op = rk_operator(states[-1][0], dx, order, solver, gamma, states[-1][1] if mhd else None)
        ops.append(op if mhd else (op,))
        nxt = []
        for c in range(len(states[0])):
            x = np.zeros_like(states[0][c])
            for j, a in enumerate(A[s]):
                if a != 0.0:
                    x = x + a * states[j][c]
            for j, b in enumerate(B[s]):
                if b != 0.0:
                    x = x + b * dt * ops[j][c]
            nxt.append(x)
        states.append(tuple(nxt))
    return states[-1] if mhd else states[-1][0]
