"""ADER-CG local space-time predictor, modal (Sec. IV) and nodal (Apps. A-C).

Both forms compute a Picard iteration on the reference element (Eq. 5):
du/dtau = -(df/dxi + dg/deta + dh/dzeta) + s,  u(tau = 0) = w,
where f, g, h are the scaled fluxes f = dt F/dx etc. evaluated at the nodes
of the current iterate and turned back into polynomials:

* modal form: node values of u are the basis expansion evaluated at the
  nodes of Eq. 31 / 37 / 46; the needed flux modes come from the paper's
  extraction rules (Eqs. 33, 40-42, 49-51, ``oracle.extraction``);
* nodal form: node values at the nodes of Eq. A.1 / B.1 / C.1; the flux
  polynomial is their Lagrange interpolant (one node per mode).

The new evolutionary modes follow by matching du/dtau with -div(flux) mode
by mode (this is what Eqs. 30, 36, 45 and A.4, B.3, C.3 state for S = 0);
with a source s = dt S (``oracle.source``) they solve the Galerkin system
whose test functions are the evolutionary basis functions.
The iteration starts from zero evolutionary modes (the paper is silent) and
runs M-1 times (Secs. IV.1-IV.3), or - in converged mode - per zone until the
largest change of an evolutionary mode is below `tol` times (|w_1| + 1e-300),
capped at `max_iter`.
"""
import numpy as np

from . import basis, extraction, nodes, physics


class _Tables:
    def __init__(self, order, form):
        self.order = order
        self.form = form
        pts = nodes.as_array((nodes.MODAL if form == "modal" else nodes.NODAL)[order])
        self.V = basis.eval_basis(order, pts)
        if form == "nodal":
            self.Vinv = np.linalg.inv(self.V)
        self.D = [basis.deriv_matrix(order, a) for a in range(3)]
        self.evo = basis.evolutionary_map(order)


_CACHE = {}


def tables(order, form):
    key = (order, form)
    if key not in _CACHE:
        _CACHE[key] = _Tables(order, form)
    return _CACHE[key]


def _apply(M, X):
    """Contract a (m, n) matrix with the mode axis (axis 0) of X."""
    return np.tensordot(M, X, axes=(1, 0))


def flux_modes(Uhat, order, form, gamma, scale):
    """One pass: node values -> node fluxes -> flux modes (x, y, z) with all L modes (zeros where unused)."""
    T = tables(order, form)
    unodes = _apply(T.V, Uhat)                              # (n_nodes, nvar, ...)
    out = []
    fl = [np.stack([physics.flux(unodes[n], gamma, d) for n in range(unodes.shape[0])]) * scale[d]
          for d in range(3)]
    if form == "nodal":
        return [_apply(T.Vinv, fl[d]) for d in range(3)]
    ext = extraction.MODAL[order](*fl)
    for d in range(3):
        full = np.zeros_like(Uhat)
        for k in extraction.NEEDED[order][d]:
            full[k - 1] = ext[d][k]
        out.append(full)
    return out


def update_from_fluxes(Uhat, Fm, order):
    """Evolutionary modes from du/dtau = -div(flux), mode by mode (Eqs. 30, 36, 45 for S = 0)."""
    D = tables(order, "modal").D
    r = -(_apply(D[0], Fm[0]) + _apply(D[1], Fm[1]) + _apply(D[2], Fm[2]))
    new = Uhat.copy()
    for k, j, dd in basis.evolutionary_map(order):
        new[k] = r[j] / dd
    return new


def source_modes(Uhat, order, form, dt, model):
    """All L modes of the scaled source polynomial s (dt S at the nodes of the current iterate; modal
    extraction rules or nodal interpolation, see ``oracle.source``)."""
    from . import source
    T = tables(order, form)
    unodes = _apply(T.V, Uhat)                              # (n_nodes, nvar, ...)
    s = dt * np.stack([source.evaluate(unodes[n], model) for n in range(unodes.shape[0])])
    return source.modal_modes(order, s) if form == "modal" else _apply(T.Vinv, s)


def update_with_source(Uhat, Fm, Sm, order, form):
    """Evolutionary modes of du/dtau = -div(flux) + s in the Galerkin sense (Eqs. 30, 36, 45 and
    A.4, B.3, C.3 with S): test functions are the evolutionary basis functions of the form."""
    from . import source
    D = tables(order, "modal").D
    rhs = -(_apply(D[0], Fm[0]) + _apply(D[1], Fm[1]) + _apply(D[2], Fm[2])) + Sm
    E = [k for k, m in enumerate(basis.MODES[order]) if m[3] >= 1]
    new = Uhat.copy()
    new[E] = source.evolve(order, form, rhs)
    return new


def _step(Uhat, order, form, gamma, scale, dt, model):
    Fm = flux_modes(Uhat, order, form, gamma, scale)
    if model is None:
        return update_from_fluxes(Uhat, Fm, order)
    return update_with_source(Uhat, Fm, source_modes(Uhat, order, form, dt, model), order, form)


def predict(W, order, form, gamma, dt, dx, n_iter=None, tol=None, max_iter=50, guess=None, source=None):
    """Space-time modes u_hat (L, nvar, ...) from spatial modes W (LS, nvar, ...).

    dt/dx gives the reference-element scaling of Eq. 5.  Returns (Uhat, iterations)
    where iterations is an int (fixed count) or a per-zone integer array
    (converged mode).  `guess` optionally supplies initial evolutionary modes
    (L - LS, nvar, ...).  `source` is a source model of ``oracle.source``; with
    one, the result is (Uhat, iterations, Sdt) with Sdt (nvar, ...) the
    space-time average of the source polynomial of the final iterate (dt times
    the S-bar of Eq. 6).
    """
    LS, L = basis.LS[order], basis.L[order]
    Uhat = np.zeros((L,) + W.shape[1:])
    Uhat[:LS] = W
    if guess is not None:
        Uhat[LS:] = guess
    scale = [dt / dx[0], dt / dx[1], dt / dx[2]]
    if tol is None:
        n = order - 1 if n_iter is None else n_iter
        for _ in range(n):
            Uhat = _step(Uhat, order, form, gamma, scale, dt, source)
        iters = n
    else:
        grid = W.shape[2:]
        done = np.zeros(grid, dtype=bool)
        iters = np.zeros(grid, dtype=np.int64)
        ref = np.abs(W[0]).max(axis=0) + 1e-300
        for _ in range(max_iter):
            new = _step(Uhat, order, form, gamma, scale, dt, source)
            change = np.abs(new[LS:] - Uhat[LS:]).max(axis=(0, 1)) / ref
            act = ~done
            Uhat[:, :, act] = new[:, :, act]
            iters[act] += 1
            done |= change < tol
            if done.all():
                break
    if source is None:
        return Uhat, iters
    from . import source as src
    Sdt = _apply(src.average_weights(order)[None, :], source_modes(Uhat, order, form, dt, source))[0]
    return Uhat, iters, Sdt
