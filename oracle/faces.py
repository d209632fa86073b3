"""Face and edge space-time averages of one zone's predictor polynomial (Sec. V, App. D).

For the face of a zone whose outward normal is +-e_d:
* u_b   (Eq. 54): u at the face's space-time barycentre (xi_d = +-1/2, the
  transverse coordinates 0, tau = 1/2);
* <u>   (Eq. 55): average of u over the face and over tau in [0, 1];
* <u>_e (Eq. 57): average over the edge xi_d = +-1/2, xi_e = +-1/2 and tau;
* <F>, <F>_e: the same averages of the physical flux in direction d, taken
  from the facial flux polynomial of App. D.  Its modes come from the flux at
  the one-sided facial nodes (Eqs. D.1, D.6, D.11): by the paper's rule at
  orders 2 and 4 (Eqs. D.4, D.14), by interpolation at order 3 (ten nodes for
  ten modes; Eq. D.9 is that interpolation written out).

u_b, <u>, <u>_e and the facial node values are evaluated from the definition
(the basis expansion), the paper's closed forms Eqs. 58-66 and D.3, D.8, D.13
being the same numbers (pinned in tests/test_oracle_faces.py).

Transverse axes of a face normal to d are the other two directions in
increasing order (t1, t2); the facial node sets are symmetric in t1 <-> t2.
"""
from fractions import Fraction as Fr

import numpy as np

from . import basis, extraction, nodes, physics


def transverse(d):
    return [a for a in range(3) if a != d]


def _apply(w, X):
    return np.tensordot(w, X, axes=(0, 0))


class FaceTables:
    def __init__(self, order):
        self.order = order
        half = Fr(1, 2)
        self.ub, self.avg, self.edge, self.fnode_V = {}, {}, {}, {}
        fn = nodes.as_array(nodes.FACE[order])
        for d in range(3):
            t1, t2 = transverse(d)
            for s in (+1, -1):
                xs = s * half
                fixed = {d: xs, t1: 0, t2: 0, 3: half}
                self.ub[d, s] = basis.spacetime_integral_weights(order, fixed)
                self.avg[d, s] = basis.spacetime_integral_weights(order, {d: xs})
                for e in (t1, t2):
                    for se in (+1, -1):
                        self.edge[d, s, e, se] = basis.spacetime_integral_weights(order, {d: xs, e: se * half})
                pts = np.zeros((fn.shape[0], 4))
                pts[:, d] = float(xs)
                pts[:, t1] = fn[:, 0]
                pts[:, t2] = fn[:, 1]
                pts[:, 3] = fn[:, 2]
                self.fnode_V[d, s] = basis.eval_basis(order, pts)
        self.face_avg_w = basis.face_integral_weights(order, {})
        self.face_edge_w = {(0, +1): basis.face_integral_weights(order, {0: half}),
                            (0, -1): basis.face_integral_weights(order, {0: -half}),
                            (1, +1): basis.face_integral_weights(order, {1: half}),
                            (1, -1): basis.face_integral_weights(order, {1: -half})}
        if order == 3:
            self.Winv = np.linalg.inv(basis.eval_face_basis(3, fn))


_CACHE = {}


def tables(order):
    if order not in _CACHE:
        _CACHE[order] = FaceTables(order)
    return _CACHE[order]


def facial_flux_modes(fnodes, order):
    """Modes of the facial flux polynomial from its values at the facial nodes (App. D)."""
    if order == 2:
        m = extraction.face_o2(fnodes)
        return np.stack([m[k] for k in range(1, 5)])
    if order == 4:
        m = extraction.face_o4(fnodes)
        return np.stack([m[k] for k in range(1, 21)])
    return np.tensordot(tables(3).Winv, fnodes, axes=(1, 0))


def face_quantities(Uhat, order, gamma, d, s, edges=False):
    """(u_b, <u>, <F>[, edge dict]) for the face with outward normal s*e_d of every zone.

    The edge dict maps (e, se) -> (<u>_e, <F>_e) for the two transverse
    directions e and their two sides se.
    """
    T = tables(order)
    ub = _apply(T.ub[d, s], Uhat)
    uavg = _apply(T.avg[d, s], Uhat)
    un = np.tensordot(T.fnode_V[d, s], Uhat, axes=(1, 0))          # (n_fnodes, nvar, ...)
    fl = np.stack([physics.flux(un[n], gamma, d) for n in range(un.shape[0])])
    fm = facial_flux_modes(fl, order)
    favg = _apply(T.face_avg_w, fm)
    if not edges:
        return ub, uavg, favg
    t1, t2 = transverse(d)
    ed = {}
    for slot, e in ((0, t1), (1, t2)):
        for se in (+1, -1):
            ed[e, se] = (_apply(T.edge[d, s, e, se], Uhat), _apply(T.face_edge_w[slot, se], fm))
    return ub, uavg, favg, ed
