"""Pins of the oracle's dense output (oracle/dense.py): the predictor's polynomial inside the step.

* at tau = 0 it is the reconstruction itself (the initial data of the local space-time problem);
* with the decay source S = -k U on a uniform state the exact solution is U e^{-k t}: the converged
  predictor's zone average at tau = 1/2 and 1 approaches it at the rate (k dt)^M of a degree M-1
  polynomial in time;
* on the translating density wave the zone averages at mid-step converge to the exact translated
  averages at (at least) the design order in the mesh width.
"""
import numpy as np
import pytest

from oracle import dense, scheme
from paper_1006_2146_gb300 import inputs


@pytest.mark.parametrize("order,form", [(2, "modal"), (3, "nodal"), (4, "modal")])
def test_tau_zero_is_the_reconstruction(order, form):
    U = inputs.random_smooth(6, seed=900 + order, amp=0.2)
    dx = (1 / 6,) * 3
    _, W = scheme.zone_state(U, None, order)
    w0 = dense.dense_output(U, dx, 0.5 * scheme.max_dt(U, dx, 0.4), order, form, 0.0)
    assert np.array_equal(w0, W)


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("form", ["modal", "nodal"])
def test_linear_decay_in_time(order, form):
    U = inputs.density_wave(4, amp=0.0)
    dx, dt = (0.25,) * 3, 0.01
    for tau in (0.5, 1.0):
        errs = []
        for kdt in (0.2, 0.1):
            w = dense.dense_output(U, dx, dt, order, form, tau, tol=1e-15, source=("linear", kdt / dt))
            exact = U * np.exp(-kdt * tau)
            errs.append((np.abs(w[0] - exact) / np.abs(exact)).max())
        assert errs[0] < 0.5 * 0.2 ** order
        assert np.log2(errs[0] / errs[1]) >= order - 0.3
        # the spatial slopes of a uniform state stay zero (to round-off of the nodal interpolation)
        w = dense.dense_output(U, dx, dt, order, form, tau, tol=1e-15, source=("linear", 10.0))
        assert np.abs(w[1:]).max() <= 1e-14 * np.abs(U).max()


@pytest.mark.parametrize("order", [2, 3, 4])
def test_translating_wave_mid_step(order):
    errs = []
    for n in (16, 32):
        U = inputs.density_wave(n)
        dx = (1 / n,) * 3
        dt = 0.4 * scheme.max_dt(U, dx, 0.4)
        w = dense.dense_output(U, dx, dt, order, "modal", 0.5)
        errs.append(np.abs(w[0, 0] - inputs.density_wave(n, t=0.5 * dt)[0]).mean())
    assert np.log2(errs[0] / errs[1]) >= order - 0.3
