"""The 2-D vortex states of Secs. VI.1-VI.2 (inputs.isentropic_vortex, inputs.magnetized_vortex).

Both are steady vortices carried by the mean flow v = (1, 1): the exact solution at t = h (one zone
width) is the initial state shifted by one zone in x and in y.  The oracle, run to t = h at 32^2, must
land within a few per cent of that shift's own change; a vortex whose pressure does not balance its
rotation and field (a wrong coefficient or sign in dT or dP) leaves 15-40 %.
"""
import numpy as np

from oracle import scheme
from paper_1006_2146_gb300 import inputs

N, L = 32, 10.0
H = L / N
DX = (H, H, inputs.slab_lengths(L)[2])


def _to_one_zone_shift(U, B, gamma):
    t = 0.0
    while t < H - 1e-13:
        dt = min(scheme.max_dt(U, DX, 0.45, gamma, Bface=B), H - t)
        r = scheme.ader_step(U, DX, dt, 3, "modal", "hll", gamma, Bface=B)
        U, B = (r, None) if B is None else r
        t += dt
    return U, B


def _rel(got, exact, start):
    num = np.abs(got - exact).reshape(got.shape[0], -1).mean(axis=1)
    den = np.abs(exact - start).reshape(got.shape[0], -1).mean(axis=1)
    live = den > 1e-12
    return (num[live] / den[live]).max()


def test_isentropic_vortex_translates():
    U0 = inputs.isentropic_vortex(N, L=L)
    assert U0.shape == (5, 1, N, N)
    # invariant under a quarter turn about the centre (rho and energy; momentum rotates with the mean flow)
    assert np.abs(np.rot90(U0[0, 0]) - U0[0, 0]).max() < 1e-14
    U1, _ = _to_one_zone_shift(U0, None, 1.4)
    assert _rel(U1, np.roll(U0, (1, 1), axis=(2, 3)), U0) < 0.06


def test_magnetized_vortex_translates_and_is_divergence_free():
    U0, B0 = inputs.magnetized_vortex(N, L=L)
    assert U0.shape == (5, 1, N, N) and B0.shape == (3, 1, N, N)
    div = (np.roll(B0[0], -1, axis=2) - B0[0]) / H + (np.roll(B0[1], -1, axis=1) - B0[1]) / H
    assert np.abs(div).max() < 1e-13 * np.abs(B0).max() / H
    assert abs(B0[0].sum()) < 1e-12 and abs(B0[1].sum()) < 1e-12       # no mean field
    assert np.all(U0[0] == 1.0)
    U1, B1 = _to_one_zone_shift(U0, B0, 5.0 / 3.0)
    assert _rel(U1, np.roll(U0, (1, 1), axis=(2, 3)), U0) < 0.06
    assert _rel(B1, np.roll(B0, (1, 1), axis=(2, 3)), B0) < 0.06
