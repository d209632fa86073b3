"""Dense output inside one ADER step: the predictor's polynomial at an intermediate time (Sec. VII).

Test infrastructure (the oracle): plain FP64 numpy.  Only tests/, the smoke run and the bench's CPU legs
use it.

The paper notes that the space-time polynomial the predictor builds in each zone gives the solution at
any time inside the step, which is what an adaptive mesh needs to feed finer levels that take shorter
steps.  The polynomial is u(xi, eta, zeta, tau) = sum_k u_k P_a(xi) P_b(eta) P_c(zeta) tau^d on the
reference element (Eqs. 9, 13, 14-16), tau in [0, 1] spanning the step.  At a fixed tau it is a spatial
polynomial whose LS modes are

    w_s(tau) = sum over the modes k whose spatial part is s of u_k tau^(d_k).

w_1(tau) is the zone average at t^n + tau dt (every P_a with a >= 1 has zero mean on [-1/2, 1/2]).
"""
import numpy as np

from . import basis


def spatial_modes_at(order, Uhat, tau):
    """The LS spatial modes (LS, nvar, ...) of the space-time modes Uhat (L, nvar, ...) at time tau."""
    modes = basis.MODES[order]
    spatial = [m for m in modes if m[3] == 0]
    out = np.zeros((len(spatial),) + Uhat.shape[1:])
    for k, (a, b, c, d) in enumerate(modes):
        out[spatial.index((a, b, c, 0))] += Uhat[k] * float(tau) ** d
    return out


def dense_output(U, dx, dt, order, form, tau, gamma=1.4, Bface=None, tol=None, source=None):
    """Spatial modes (LS, nvar, ...) at t^n + tau dt of the predictor of the step of size dt from U."""
    from . import predictor, scheme
    _, W = scheme.zone_state(U, Bface, order)
    Uhat = predictor.predict(W, order, form, gamma, dt, dx, tol=tol, source=source)[0]
    return spatial_modes_at(order, Uhat, tau)
