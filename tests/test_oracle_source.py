"""Pins of the oracle's non-stiff source terms (oracle/source.py) against what the paper prints and what
the mathematics fixes.

* The Galerkin construction reproduces the printed source coefficients of the modal evolutionary
  equations (Eqs. 30, 36, 45), of the nodal ones (Eqs. A.4, B.2-B.3 and three rows of C.2) and the S-bar
  rules (Eqs. 35, 44, 53, A.7, B.6); the coefficients below are typed from those equations.
* The modal source rules return the exact modes of any polynomial in the span.
* The uniform decay u' = -k u: one second-order step is the Taylor polynomial 1 - x + x^2/2 (x = k dt),
  and every order's one-step error falls at order M + 1.
* Uniform gravity carries a density wave as x - v0 t - g t^2/2 with v = v0 + g t: the scheme converges
  at the design order to that exact solution.
"""
import numpy as np
import pytest

from oracle import basis, nodes, scheme, source
from paper_1006_2146_gb300 import inputs


def _coefs(order, form):
    E, A, Bm = source.galerkin(order, form)
    return E, np.linalg.solve(A, Bm)


# (evolutionary mode, {source mode: coefficient}) as printed; other entries are zero
PRINTED_MODAL = {
    2: {5: {1: 1.0, 5: 2.0 / 3.0}},                                                    # Eq. 30
    3: {11: {1: 1.0, 12: -0.3}, 12: {11: 0.5, 12: 0.6}, 13: {2: 1.0, 13: 2.0 / 3.0},    # Eq. 36
        14: {3: 1.0, 14: 2.0 / 3.0}, 15: {4: 1.0, 15: 2.0 / 3.0}},
    4: {21: {1: 1.0, 23: 8.0 / 70.0}, 22: {21: 0.5, 23: -3.0 / 7.0}, 23: {22: 1.0 / 3.0, 23: 4.0 / 7.0},  # Eq. 45
        24: {2: 1.0, 27: -0.3}, 25: {3: 1.0, 28: -0.3}, 26: {4: 1.0, 29: -0.3},
        27: {24: 0.5, 27: 0.6}, 28: {25: 0.5, 28: 0.6}, 29: {26: 0.5, 29: 0.6},
        30: {5: 1.0, 30: 2.0 / 3.0}, 31: {6: 1.0, 31: 2.0 / 3.0}},
}


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("form", ["modal", "nodal"])
def test_galerkin_reproduces_printed_modal_source_coefficients(order, form):
    E, C = _coefs(order, form)
    for k, row in PRINTED_MODAL[order].items():
        r = E.index(k - 1)
        want = np.zeros(basis.L[order])
        for j, c in row.items():
            want[j - 1] = c
        np.testing.assert_allclose(C[r], want, atol=1e-13, err_msg="u%d" % k)


def _nodal_source_only(order, s):
    """Node values at the tau > 0 nodes produced by sources alone (w = 0, no flux)."""
    pts = nodes.as_array(nodes.NODAL[order])
    V = basis.eval_basis(order, pts)
    E, C = _coefs(order, "nodal")
    uh = np.zeros(basis.L[order])
    uh[E] = C @ np.linalg.solve(V, s)
    return V @ uh


def test_nodal_second_order_matches_eq_A4_A7():
    s = np.random.default_rng(1).standard_normal(5)
    un = _nodal_source_only(2, s)
    assert un[4] == pytest.approx(s[0] / 3.0 + 2.0 * s[4] / 3.0, abs=1e-14)                 # Eq. A.4
    V = basis.eval_basis(2, nodes.as_array(nodes.NODAL[2]))
    assert source.average_weights(2) @ np.linalg.solve(V, s) == pytest.approx(0.5 * (s[0] + s[4]), abs=1e-14)  # A.7


def test_nodal_third_order_matches_eqs_B2_B3_B6():
    s = np.random.default_rng(2).standard_normal(15)
    S = lambda n: s[n - 1]
    q11 = (-9 * S(1) + 2 * (S(2) + S(3) + S(4) + S(5) + S(6) + S(7))) / 24.0
    q12 = (7 * S(1) - 8 * S(2) - 4 * S(3) + 2 * (S(4) + S(5) + S(6) + S(7))) / 24.0
    q13 = (7 * S(1) + 2 * (S(2) + S(3)) - 8 * S(4) - 4 * S(5) + 2 * (S(6) + S(7))) / 24.0
    q14 = (7 * S(1) + 2 * (S(2) + S(3) + S(4) + S(5)) - 8 * S(6) - 4 * S(7)) / 24.0
    q15 = (-27 * S(1) + 5 * (S(2) + S(3) + S(4) + S(5) + S(6) + S(7))) / 30.0
    q2 = (-4 * S(11) - 3 * S(15)) / 24.0
    want = [q11 + 0.125 * (4 * S(11) - S(15)), q12 + q2 + 2 * S(12) / 3, q13 + q2 + 2 * S(13) / 3,
            q14 + q2 + 2 * S(14) / 3, q15 + 0.1 * (8 * S(11) + S(15))]
    np.testing.assert_allclose(_nodal_source_only(3, s)[10:15], want, atol=1e-14)
    V = basis.eval_basis(3, nodes.as_array(nodes.NODAL[3]))
    sbar = source.average_weights(3) @ np.linalg.solve(V, s)
    assert sbar == pytest.approx((-5 * S(1) + S(2) + S(3) + S(4) + S(5) + S(6) + S(7) + 4 * S(11) + S(15)) / 6.0,
                                 abs=1e-14)                                                      # Eq. B.6


def test_nodal_fourth_order_matches_printed_rows_of_eq_C2():
    """The tau = 0 source terms of three printed rows of Eq. C.2 (q21, q34, q35), from the Galerkin
    solution with the tau > 0 sources set to zero (they enter only Eq. C.3)."""
    pts = nodes.as_array(nodes.NODAL[4])
    V = basis.eval_basis(4, pts)
    E, C = _coefs(4, "nodal")
    uh_of_s = np.zeros((35, 35))
    uh_of_s[E] = C @ np.linalg.inv(V)
    rows = V @ uh_of_s                                  # node values from node sources, w = 0
    printed = {
        21: ([-89091, 0] + [17955] * 6 + [0] * 12, 215460),
        34: ([413535, -114912, -138516, -11200, -163086, -32494, -343581, -156604, 171248, -11466, 159782,
              -1638, 122234, 13104, 35840, 35840, 29288, 29288, -119392, 110432], 323190),
        35: ([-29241, 0] + [5985] * 6 + [0] * 12, 71820),
    }
    for node, (num, den) in printed.items():
        np.testing.assert_allclose(rows[node - 1, :20], np.array(num, dtype=float) / den, atol=1e-13,
                                   err_msg="q%d" % node)


def test_modal_sbar_weights_match_eqs_35_44_53():
    for order, printed in ((2, {1: 1.0, 5: 0.5}), (3, {1: 1.0, 11: 0.5, 12: 1.0 / 3.0}),
                           (4, {1: 1.0, 21: 0.5, 22: 1.0 / 3.0, 23: 0.25})):
        want = np.zeros(basis.L[order])
        for k, c in printed.items():
            want[k - 1] = c
        np.testing.assert_allclose(source.average_weights(order), want, atol=1e-15)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_modal_source_rules_are_exact_on_the_span(order):
    """Eqs. 33-34, 40-43, 49-52 with f, g, h -> s recover every mode of a polynomial in the basis."""
    rng = np.random.default_rng(10 + order)
    modes = rng.standard_normal(basis.L[order])
    s_nodes = basis.eval_basis(order, nodes.as_array(nodes.MODAL[order])) @ modes
    np.testing.assert_allclose(source.modal_modes(order, s_nodes), modes, atol=1e-12)


def test_uniform_decay_second_order_is_the_taylor_polynomial():
    U = inputs.density_wave(4, amp=0.0, vel=(0.0, 0.0, 0.0))
    for form in ("modal", "nodal"):
        for k, dt in ((1.0, 0.2), (3.0, 0.05)):
            x = k * dt
            Un = scheme.ader_step(U, (0.25,) * 3, dt, 2, form, "hll", source=("linear", k))
            np.testing.assert_allclose(Un, U * (1.0 - x + 0.5 * x * x), rtol=1e-14)


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("form", ["modal", "nodal"])
def test_uniform_decay_one_step_error_order(order, form):
    U = inputs.density_wave(4, amp=0.0, vel=(0.2, 0.0, -0.1))
    errs = []
    for dt in (0.2, 0.1):
        Un = scheme.ader_step(U, (0.25,) * 3, dt, order, form, "hll", source=("linear", 1.0))
        errs.append(np.abs(Un - U * np.exp(-dt)).max())
    assert np.log2(errs[0] / errs[1]) == pytest.approx(order + 1, abs=0.1)


def test_zero_gravity_is_no_source():
    U = inputs.random_smooth((5, 6, 7), seed=4, amp=0.2)
    dx = (1 / 7, 1 / 6, 1 / 5)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    a = scheme.ader_step(U, dx, dt, 3, "nodal", "hll")
    b = scheme.ader_step(U, dx, dt, 3, "nodal", "hll", source=("gravity", (0.0, 0.0, 0.0)))
    np.testing.assert_allclose(b, a, rtol=1e-14, atol=1e-14)


V0 = np.array([0.4, -0.3, 0.2])
G = np.array([0.8, -0.5, 0.3])


def _accelerated_wave(n, t, amp=0.2, gamma=1.4, P=1.0):
    """Exact cell averages: rho = 1 + amp sin 2 pi (x + y + z - s(t)), v = v0 + g t, P uniform."""
    shift = V0.sum() * t + 0.5 * G.sum() * t * t
    rho = inputs.cell_average(lambda x, y, z: 1.0 + amp * np.sin(2 * np.pi * (x + y + z - shift)), n)
    v = V0 + G * t
    return np.stack([rho, rho * v[0], rho * v[1], rho * v[2], P / (gamma - 1.0) + 0.5 * rho * (v @ v)])


@pytest.mark.parametrize("order,form", [(2, "modal"), (2, "nodal"), (3, "modal"), (3, "nodal"), (4, "nodal")])
def test_gravity_accelerated_wave_converges_at_design_order(order, form):
    T = 0.05
    errs = []
    for n in (8, 16):
        U = _accelerated_wave(n, 0.0)
        dx = (1.0 / n,) * 3
        t = 0.0
        while t < T - 1e-14:
            dt = min(scheme.max_dt(U, dx, 0.4), T - t)
            U = scheme.ader_step(U, dx, dt, order, form, "hll", source=("gravity", tuple(G)))
            t += dt
        errs.append(np.abs(U - _accelerated_wave(n, T)).mean(axis=(1, 2, 3)).max())
    assert np.log2(errs[0] / errs[1]) >= order - 0.2
