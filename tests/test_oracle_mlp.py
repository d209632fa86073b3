"""Pins of the MLP oracle (learned predictor guess) against facts outside it."""
import math

import numpy as np
import pytest

from oracle import mlp, predictor, scheme
from paper_1006_2146_gb300 import inputs


def test_shape_counts():
    assert mlp.shape(False) == (52, 128, 25, 128 * 52 + 128 + 128 * 128 + 128 + 25 * 128 + 25)
    assert mlp.shape(True)[:3] == (82, 128, 40)


def test_gelu_against_exact_gelu():
    """The tanh form stays within 1e-3 of x Phi(x) (Phi by erf) and has the GELU limits."""
    x = np.linspace(-8, 8, 4001)
    exact = 0.5 * x * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in x]))
    assert np.abs(mlp.gelu(x) - exact).max() < 1e-3
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([30.0]))[0] == pytest.approx(30.0, rel=1e-15)
    assert abs(mlp.gelu(np.array([-30.0]))[0]) < 1e-15
    h = 1e-6
    xs = np.array([-2.0, -0.3, 0.0, 0.7, 3.0])
    fd = (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h)
    assert np.abs(mlp.gelu_prime(xs) - fd).max() < 1e-8


def test_forward_single_path_closed_form():
    """One nonzero weight per layer: y_o = b3_o + W3[o,i] g(b2_i + W2[i,j] g(b1_j + W1[j,k] x_k))."""
    n_in, H, n_out, npar = mlp.shape(False)
    P = np.zeros(npar)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(P, n_in, n_out)
    W1[7, 3] = 0.8
    b1[7] = -0.1
    W2[5, 7] = -1.3
    b2[5] = 0.2
    W3[11, 5] = 2.0
    b3[:] = np.arange(n_out) * 0.01
    x = np.zeros((2, n_in))
    x[0, 3] = 1.5
    x[1, 3] = -0.4
    y = mlp.forward(P, x, n_out)
    g = lambda v: 0.5 * v * (1 + math.tanh(math.sqrt(2 / math.pi) * (v + 0.044715 * v ** 3)))
    for r in range(2):
        inner = g(-0.1 + 0.8 * x[r, 3])
        want = b3.copy()
        want[11] += 2.0 * g(0.2 - 1.3 * inner)
        # every other hidden unit sees only its zero bias: g(0) = 0
        np.testing.assert_allclose(y[r], want, rtol=0, atol=1e-15)


def test_gradient_matches_finite_differences():
    """Backpropagation against central differences of the loss, on sampled parameters of every block."""
    n_in, H, n_out, npar = mlp.shape(False)
    P = mlp.init_params(n_in, n_out, seed=3)
    P += 0.05 * np.random.default_rng(4).standard_normal(npar)      # nonzero biases too
    rng = np.random.default_rng(5)
    X = rng.standard_normal((7, n_in))
    Y = rng.standard_normal((7, n_out))
    loss, g = mlp.loss_and_grad(P, X, Y)
    assert loss == pytest.approx(((mlp.forward(P, X, n_out) - Y) ** 2).mean(), rel=1e-14)
    bounds = np.cumsum([0, H * n_in, H, H * H, H, n_out * H, n_out])
    idx = np.concatenate([rng.integers(bounds[b], bounds[b + 1], 12) for b in range(6)])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (mlp.loss_and_grad(Pp, X, Y)[0] - mlp.loss_and_grad(Pm, X, Y)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-8)    # central-difference round-off ~ 1e-10


def test_features_of_uniform_state():
    """A uniform state at rest: slope magnitude 0, Courant features c dt/dx, no samples, zero guess."""
    shape = (4, 4, 4)
    U = np.zeros((5,) + shape)
    U[0] = 2.0
    U[4] = 5.0
    dx = (0.25, 0.25, 0.5)
    dt = 0.01
    _, W = scheme.zone_state(U, None, 3)
    X = mlp.features(W, dt, dx)
    c = math.sqrt(5.0 / 2.0)
    assert X.shape == (64, 52)
    np.testing.assert_allclose(X[:, :48], 0.0, atol=1e-15)     # 45 slopes and 3 Mach numbers at rest
    np.testing.assert_allclose(X[:, 48:51], np.tile([c * dt / 0.25, c * dt / 0.25, c * dt / 0.5], (64, 1)), rtol=1e-15)
    np.testing.assert_allclose(X[:, 51], 0.0, atol=0)
    assert not mlp.sample_mask(W).any()
    n_in, H, n_out, npar = mlp.shape(False)
    P = mlp.init_params(n_in, n_out, seed=1)
    P[-n_out:] = 1.0                                  # a network whose output is nonzero everywhere
    np.testing.assert_array_equal(mlp.guess_modes(P, W, dt, dx), 0.0)
    Uhat, _ = predictor.predict(W, 3, "modal", 1.4, dt, dx, tol=1e-13)
    np.testing.assert_allclose(Uhat[10:15], 0.0, atol=1e-15)     # the true evolution is zero as well


def test_features_are_scale_free():
    """Slopes over their magnitude: largest |x| is 1; adding a constant to rho and E changes the scales only
    through w1, and doubling every perturbation doubles g but keeps x[:48] (to first order in the amplitude)."""
    shape = (6, 6, 6)
    dx = (1.0 / 6,) * 3
    # amplitudes small enough for the state to be linear in them (to 1e-4), large enough for the WENO
    # smoothness indicators to dwarf their 1e-12 regulariser (scale-free weights)
    U = inputs.random_smooth(shape, seed=12, amp=1e-4)
    _, W = scheme.zone_state(U, None, 3)
    X = mlp.features(W, 1e-3, dx)
    np.testing.assert_allclose(np.abs(X[:, :45]).max(axis=1), 1.0, rtol=1e-15)
    assert (X[:, 51] > 0).all()
    U2 = inputs.random_smooth(shape, seed=12, amp=2e-4)
    _, W2 = scheme.zone_state(U2, None, 3)
    X2 = mlp.features(W2, 1e-3, dx)
    np.testing.assert_allclose(X2[:, 51], 2 * X[:, 51], rtol=2e-3)
    np.testing.assert_allclose(X2[:, :45], X[:, :45], atol=2e-3)
    np.testing.assert_allclose(X2[:, 45:48], 2 * X[:, 45:48], rtol=2e-3, atol=1e-12)   # Mach numbers ~ amp


def test_uniform_moving_flow_has_no_slopes():
    """A uniform flow in motion: g = 0, Mach-number features v/c, no samples; its evolution is zero."""
    shape = (4, 4, 4)
    U = np.zeros((5,) + shape)
    U[0] = 1.5
    U[1:4] = 1.5 * np.array([0.3, -0.2, 0.1])[:, None, None, None]
    U[4] = 4.0
    dx = (0.25,) * 3
    _, W = scheme.zone_state(U, None, 3)
    X = mlp.features(W, 0.01, dx)
    c = math.sqrt(4.0 / 1.5)
    np.testing.assert_allclose(X[:, :45], 0.0, atol=1e-15)
    np.testing.assert_allclose(X[:, 45:48], np.tile(np.array([0.3, -0.2, 0.1]) / c, (64, 1)), rtol=1e-14)
    assert (X[:, 51] == 0).all() and not mlp.sample_mask(W).any()
    Uhat, _ = predictor.predict(W, 3, "modal", 1.4, 0.01, dx, tol=1e-13)
    np.testing.assert_allclose(Uhat[10:15], 0.0, atol=1e-14)


def test_targets_roundtrip_through_guess_modes():
    """guess_modes undoes the target normalisation: a network that outputs the targets returns u_11..u_15."""
    shape = (4, 4, 4)
    U = inputs.random_smooth(shape, seed=9, amp=0.3)
    dx = (0.25, 0.25, 0.25)
    _, W = scheme.zone_state(U, None, 3)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    Uhat, _ = predictor.predict(W, 3, "modal", 1.4, dt, dx, tol=1e-13)
    T = mlp.targets(W, Uhat, dt, dx)
    assert mlp.sample_mask(W).all()
    n_in, H, n_out, npar = mlp.shape(False)
    P = np.zeros(npar)
    # constant network: b3 = the targets of zone 0, so guess_modes(zone 0) = u_11..u_15 of zone 0
    mlp.unpack(P, n_in, n_out)[5][:] = T[0]
    G = mlp.guess_modes(P, W, dt, dx).reshape(5, 5, -1)
    np.testing.assert_allclose(G[:, :, 0], Uhat[10:15].reshape(5, 5, -1)[:, :, 0], rtol=1e-13, atol=1e-15)
