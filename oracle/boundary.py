"""Non-periodic box boundaries for the Euler step, by ghost zones (the paper's 2-D tests with walls and
open sides, Sec. VIII).

The paper runs problems with reflecting walls and open boundaries but does not say how its code treats
them; the reading here is the usual ghost-zone one (stated once, used by both sides):

* a face of the box is PERIODIC, OUTFLOW or REFLECTIVE (both faces of an axis periodic, or neither);
* before the step the state is extended by G ghost zones across every non-periodic face:
  OUTFLOW copies the nearest interior zone (zero gradient); REFLECTIVE copies the mirror-image interior
  zone (ghost zone -1 - k takes zone k) with the momentum normal to the face negated;
* the periodic step of ``scheme`` runs on the extended array and the interior is kept.  G is at least
  the reach of one step (the zones whose averages a zone's update reads): 3 zones at orders 2-3
  (three-zone WENO stencils plus the face) and 4 at order 4, so the wrap-around of the extended array
  never reaches the interior.

Axes: direction 0/1/2 = x/y/z, array axes (z, y, x) after the variable axis.
"""
import numpy as np

from . import scheme

PERIODIC, OUTFLOW, REFLECTIVE = 0, 1, 2


def ghost_width(order):
    """Zones of reach of one step along an axis (at least): 3 at orders 2 and 3, 4 at order 4."""
    return 4 if order == 4 else 3


def _check(bc):
    bc = tuple(bc)
    if len(bc) != 6 or any(b not in (PERIODIC, OUTFLOW, REFLECTIVE) for b in bc):
        raise ValueError("bc: six codes (x-, x+, y-, y+, z-, z+)")
    for d in range(3):
        if (bc[2 * d] == PERIODIC) != (bc[2 * d + 1] == PERIODIC):
            raise ValueError("an axis is periodic on both faces or on neither")
    return bc


def extend(U, bc, G):
    """The state with G ghost zones across every non-periodic face, filled by its rule."""
    bc = _check(bc)
    out = U
    for d in range(3):
        if bc[2 * d] == PERIODIC:
            continue
        ax = 3 - d                                  # array axis of direction d (variable axis first)
        n = out.shape[ax]
        idx = np.arange(-G, n + G)
        src = np.empty_like(idx)
        flip = np.zeros(idx.shape, dtype=bool)
        for side, sel in ((0, idx < 0), (1, idx >= n)):
            k = idx[sel]
            if bc[2 * d + side] == OUTFLOW:
                src[sel] = 0 if side == 0 else n - 1
            else:                                   # REFLECTIVE: ghost -1-k <- zone k, n+k <- n-1-k
                src[sel] = -1 - k if side == 0 else 2 * n - 1 - k
                flip[sel] = True
        inside = (idx >= 0) & (idx < n)
        src[inside] = idx[inside]
        if bc[2 * d] == REFLECTIVE or bc[2 * d + 1] == REFLECTIVE:
            if np.any((src < 0) | (src >= n)):
                raise ValueError("a reflective face needs at least G zones along its axis")
        ext = np.take(out, src, axis=ax)
        sign = np.where(flip, -1.0, 1.0)
        shape = [1] * ext.ndim
        shape[ax] = len(idx)
        ext[1 + d] = ext[1 + d] * sign.reshape(shape[1:])    # the normal momentum of mirrored ghosts
        out = ext
    return out


def interior(Ue, bc, G):
    """The zones of the original box inside an extended array."""
    sl = [slice(None)] * 4
    for d in range(3):
        if bc[2 * d] != PERIODIC:
            sl[3 - d] = slice(G, Ue.shape[3 - d] - G)
    return Ue[tuple(sl)]


def ader_step(U, dx, dt, order, form="modal", solver="hll", gamma=1.4, bc=(0,) * 6, G=None, **kw):
    """One ADER step of the Euler state U with the box boundaries bc (the periodic step on the extended
    state, interior kept)."""
    G = ghost_width(order) if G is None else G
    return interior(scheme.ader_step(extend(U, bc, G), dx, dt, order, form, solver, gamma, **kw), bc, G)


def max_dt(U, dx, cfl, gamma=1.4):
    """The CFL time step; ghost zones repeat interior speeds (a mirror only flips a velocity's sign)."""
    return scheme.max_dt(U, dx, cfl, gamma)
