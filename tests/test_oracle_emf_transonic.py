"""Pins of the oracle's transonic EMF option (twice the dissipative term of Eq. 17 in the electric fields
at transonic faces; Secs. II.3 and V).

* the transonic test fires exactly when a fast wave speed changes sign across the face;
* the option touches only the electric fields: the hydrodynamic update is bit for bit the plain one,
  and the face field stays divergence-free;
* without transonic faces (a slow smooth state) the step is bit for bit the plain one; with them (a
  supersonic magnetised state) the face field changes.
"""
import numpy as np
import pytest

from oracle import riemann, scheme
from paper_1006_2146_gb300 import inputs


def test_transonic_detects_a_sign_change_of_a_fast_speed():
    c = np.array([1.0, 1.0, 1.0, 1.0])
    vL = np.array([0.5, 1.2, -1.2, 0.5])
    vR = np.array([0.6, 0.8, -0.8, -0.6])
    got = riemann.transonic(vL, c, vR, c)
    # subsonic both sides; v - c from + to -; v + c from - to +; subsonic with opposite flow directions
    assert got.tolist() == [False, True, True, False]


def _state(n, transonic):
    if transonic:
        return inputs.random_magnetised(n, seed=512, amp=0.8, b_amp=1.0, B0=2.0, P0=0.2)
    return inputs.random_magnetised(n, seed=513, amp=0.05, b_amp=0.2)


@pytest.mark.parametrize("solver", ["hll", "linearized"])
def test_option_changes_only_the_field_and_only_at_transonic_faces(solver):
    n = 8
    dx = (1.0 / n,) * 3
    G = 5.0 / 3.0
    for transonic in (False, True):
        U, B = _state(n, transonic)
        dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
        U0, B0 = scheme.ader_step(U, dx, dt, 2, "modal", solver, G, Bface=B)
        U1, B1 = scheme.ader_step(U, dx, dt, 2, "modal", solver, G, Bface=B, emf_transonic=True)
        assert np.array_equal(U0, U1)
        d0 = scheme.div_b(B, dx)
        assert np.abs(scheme.div_b(B1, dx) - d0).max() <= 1e-12 * np.abs(B).max() / dx[0]
        if transonic:
            assert np.abs(B1 - B0).max() > 1e-8 * np.abs(B0).max()
        else:
            assert np.array_equal(B0, B1)
