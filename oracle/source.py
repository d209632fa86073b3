"""Non-stiff source terms S(U) of Eq. 4 in the ADER-CG predictor and in the update of Eq. 6.

Test infrastructure (the oracle): plain FP64 numpy, no blocking or fusion.

The paper carries a general source S through every formulation (Sec. II, Eq. 4;
Sec. IV: Eqs. 30/34-35, 36/43-44, 45/52-53; Apps. A-C: A.4/A.7, B.2-B.3/B.6,
C.2-C.3/C.6) but never names one.  Two source models are built here:

* ``("linear", k)``: S = -k U on the five hydrodynamic components (each
  decays at the rate k), whose uniform solution U(t) = U(0) exp(-k t) is a
  closed form;
* ``("gravity", (gx, gy, gz))``: a uniform gravitational acceleration,
  S = (0, rho g, rho v . g) (and zero for B), whose solution with a uniform
  velocity and pressure is the initial density profile carried along
  x - v0 t - g t^2 / 2 while v = v0 + g t (exact for Euler and MHD with a
  uniform field).

For MHD the field components get no source: the face field evolves by the
constrained transport of Eq. 8 alone.

How the source enters (the reading of the printed formulas, pinned against
them in tests/test_oracle_source.py):

* the predictor evaluates S at every node of the current iterate (scaled by
  dt, like the fluxes are scaled by dt/dx) and turns the node values into a
  source polynomial s: by the extraction rules with f -> s, g -> s, h -> s
  plus Eqs. 34 / 43 / 52 in modal space, by interpolation at the nodes in
  nodal space;
* the evolutionary modes solve du/dtau = -div f + s in the Galerkin sense
  with the evolutionary basis functions as test functions: the modal ones
  (tau-dependent modes of Eqs. 14-16) in modal space, the nodal ones (the
  Lagrange polynomials of the nodes with tau > 0) in nodal space.  For s = 0
  both reduce to the derivative matching of ``predictor.update_from_fluxes``;
  with s the paper's coefficients (e.g. -3/10 and 3/5 of s_12 in Eq. 36) are
  exactly these projections;
* S-bar of Eq. 6 is the space-time average of s over the reference element
  divided by dt (Eqs. 35, 44, 53, A.7, B.6).
"""
from fractions import Fraction as Fr

import numpy as np

from . import basis, extraction, nodes

KINDS = ("linear", "gravity")


def evaluate(U, model):
    """S(U) at states U (nvar, ...) for a source model ("linear", k) or ("gravity", (gx, gy, gz))."""
    kind, par = model
    if kind == "linear":
        out = np.zeros_like(U)
        out[:5] = -float(par) * U[:5]
        return out
    if kind == "gravity":
        g = [float(v) for v in par]
        out = np.zeros_like(U)
        for c in range(3):
            out[1 + c] = U[0] * g[c]
        out[4] = U[1] * g[0] + U[2] * g[1] + U[3] * g[2]
        return out
    raise ValueError("unknown source model %r" % (kind,))


# ----------------------------------------------------------------------------- source modes
def _remaining_modal(order, s, got):
    """The modes the flux extraction rules do not give (Eqs. 34, 43, 52); node n is s[n - 1]."""
    S = lambda n: s[n - 1]
    if order == 2:
        got[1] = (S(1) + S(2) + S(3) + S(4) + S(5) + S(6)) / 6.0
        got[5] = S(7) - got[1]
    elif order == 3:
        got[1] = S(1) + (got[5] + got[6] + got[7]) / 12.0
        got[11] = 2.0 * (S(14) + S(15) + S(16) + S(17) + S(18) + S(19) - 6.0 * got[1]) / 3.0 - S(20) + S(1)
        got[12] = S(20) - S(1) - got[11]
    else:
        got[1] = 0.125 * (S(14) + S(15) + S(16) + S(17) + S(18) + S(19) + S(20) + S(21)) - \
            (got[5] + got[6] + got[7]) / 6.0
        got[23] = 4.5 * (S(42) - S(1)) - 13.5 * (S(35) - S(22))
        got[22] = 2.25 * (S(1) - S(22) - S(35) + S(42)) - 1.5 * got[23]
        got[21] = S(42) - S(1) - got[22] - got[23] + (got[30] + got[31] + got[32]) / 12.0
    return got


def modal_modes(order, s):
    """All L source modes (L, nvar, ...) from the node values s (n_nodes, nvar, ...), modal rules."""
    fx, gy, hz = extraction.MODAL[order](s, s, s)
    got = {}
    for fam in (fx, gy, hz):
        for k, v in fam.items():
            got[k] = v
    got = _remaining_modal(order, s, got)
    L = basis.L[order]
    missing = [k for k in range(1, L + 1) if k not in got]
    if missing:
        raise AssertionError("modal source rules leave modes %s undetermined" % missing)
    return np.stack([got[k] for k in range(1, L + 1)])


def nodal_modes(order, s, Vinv):
    """All L source modes from the node values by interpolation at the nodal nodes."""
    return np.tensordot(Vinv, s, axes=(1, 0))


# ----------------------------------------------------------------------------- Galerkin projection
def _spatial_inner(m1, m2):
    """Exact integral over [-1/2, 1/2]^3 of the spatial parts of two modes."""
    val = Fr(1)
    for ax in range(3):
        a, b = m1[ax], m2[ax]
        coefs = [Fr(0)] * (len(basis.P_MONO[a]) + len(basis.P_MONO[b]) - 1)
        for i, ca in enumerate(basis.P_MONO[a]):
            for j, cb in enumerate(basis.P_MONO[b]):
                coefs[i + j] += ca * cb
        val *= basis._poly_int(coefs, Fr(-1, 2), Fr(1, 2))
    return val


def mass_matrix(order):
    """M[i, j] = integral over the reference element of phi_i phi_j (exact, as floats)."""
    modes = basis.MODES[order]
    n = len(modes)
    M = np.zeros((n, n))
    for i, mi in enumerate(modes):
        for j, mj in enumerate(modes):
            sp = _spatial_inner(mi, mj)
            if sp != 0:
                M[i, j] = float(sp * Fr(1, mi[3] + mj[3] + 1))
    return M


def dtau_matrix(order):
    """T[j, k]: coefficient of mode j in d(phi_k)/d(tau) (Eq. 13: d tau^d / d tau = d tau^(d-1))."""
    modes = basis.MODES[order]
    idx = {m: i for i, m in enumerate(modes)}
    T = np.zeros((len(modes), len(modes)))
    for k, (a, b, c, d) in enumerate(modes):
        if d >= 1:
            T[idx[(a, b, c, d - 1)], k] = d
    return T


_CACHE = {}


def galerkin(order, form):
    """(E, A, Bm): evolutionary mode indices E and matrices such that the evolutionary modes are
    u_E = A^-1 Bm r for a right-hand side r (all L modes) of du/dtau = r in the Galerkin sense.

    Test functions: the modal evolutionary modes (modal form) or the nodal Lagrange polynomials of
    the nodes with tau > 0 (nodal form)."""
    key = (order, form)
    if key in _CACHE:
        return _CACHE[key]
    modes = basis.MODES[order]
    E = [k for k, m in enumerate(modes) if m[3] >= 1]
    M = mass_matrix(order)
    T = dtau_matrix(order)
    if form == "modal":
        Psi = np.zeros((len(modes), len(E)))
        for col, k in enumerate(E):
            Psi[k, col] = 1.0
    else:
        pts = nodes.as_array(nodes.NODAL[order])
        Vinv = np.linalg.inv(basis.eval_basis(order, pts))
        evo_nodes = [n for n in range(pts.shape[0]) if pts[n, 3] > 0]
        Psi = Vinv[:, evo_nodes]                 # modal coefficients of the Lagrange polynomials
    A = Psi.T @ M @ T[:, E]
    Bm = Psi.T @ M
    _CACHE[key] = (E, A, Bm)
    return _CACHE[key]


def evolve(order, form, rhs):
    """Evolutionary modes (len(E), nvar, ...) from the full right-hand side modes rhs (L, nvar, ...)."""
    E, A, Bm = galerkin(order, form)
    b = np.tensordot(Bm, rhs, axes=(1, 0))
    return np.tensordot(np.linalg.solve(A, np.eye(len(E))), b, axes=(1, 0))


def average_weights(order):
    """w[k] = space-time average of mode k over the reference element (the S-bar of Eq. 6 times dt)."""
    return basis.spacetime_integral_weights(order, {})
