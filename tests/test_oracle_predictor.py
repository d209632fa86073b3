"""Pins of the oracle's predictor: extraction exactness, the paper's nodal coefficients, linear-flux exactness."""
import json
import os

import numpy as np
import pytest

import paper_formulas as pf
from oracle import basis, extraction, faces, nodes, physics, predictor

RNG = np.random.default_rng(2146)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("order", [2, 3, 4])
def test_modal_extraction_exact_on_span(order):
    """Eqs. 33, 40-42, 49-51 return the exact modes of any flux polynomial in the span (P2)."""
    V = basis.eval_basis(order, nodes.as_array(nodes.MODAL[order]))
    for _ in range(5):
        c = RNG.normal(size=(3, basis.L[order]))
        out = extraction.MODAL[order](V @ c[0], V @ c[1], V @ c[2])
        for d in range(3):
            assert extraction.NEEDED[order][d] <= set(out[d])
            for k in extraction.NEEDED[order][d]:
                assert out[d][k] == pytest.approx(c[d][k - 1], abs=1e-12)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_needed_modes_are_exactly_the_direction_dependent_ones(order):
    for d in range(3):
        want = {k + 1 for k, m in enumerate(basis.MODES[order]) if m[d] > 0}
        assert extraction.NEEDED[order][d] == want


@pytest.mark.parametrize("order,fn", [(2, extraction.face_o2), (4, extraction.face_o4)])
def test_facial_extraction_exact_on_span(order, fn):
    """Eqs. D.4 and D.14 are exact for facial flux polynomials of Eqs. D.2 / D.12."""
    W = basis.eval_face_basis(order, nodes.as_array(nodes.FACE[order]))
    for _ in range(5):
        c = RNG.normal(size=W.shape[1])
        m = fn(W @ c)
        np.testing.assert_allclose([m[k] for k in range(1, W.shape[1] + 1)], c, atol=1e-12)


def test_facial_interpolation_matches_eqD9():
    """At third order the oracle interpolates through the ten nodes of Eq. D.6; Eq. D.9 is that interpolant."""
    for _ in range(5):
        f = RNG.normal(size=10)
        np.testing.assert_allclose(faces.facial_flux_modes(f[:, None], 3)[:, 0], pf.eqD9(f), atol=1e-12)


def _nodal_operator(order):
    T = predictor.tables(order, "nodal")
    n, L = T.V.shape
    C = np.zeros((3, n, n))
    for d in range(3):
        for j in range(n):
            fn = np.zeros((n, 1))
            fn[j, 0] = 1.0
            Fm = [np.zeros((L, 1)) for _ in range(3)]
            Fm[d] = T.Vinv @ fn
            new = predictor.update_from_fluxes(np.zeros((L, 1)), Fm, order)
            C[d, :, j] = (T.V @ new)[:, 0]
    return C


def test_nodal_update_reproduces_printed_coefficients():
    """Interpolation + du/dtau = -div f reproduces Eqs. A.4 (G8), B.2-B.3 and C.2-C.3 as printed."""
    rows = json.load(open(os.path.join(GOLDEN, "nodal_update_rows.json")))["rows"]
    ops = {}
    for row in rows:
        order = row["order"]
        C = ops.setdefault(order, _nodal_operator(order))
        for d, key in enumerate("fgh"):
            if key not in row:
                continue
            got = C[d, row["node"] - 1] * row["den"]
            want = np.zeros(C.shape[2])
            for j, v in row[key].items():
                want[int(j) - 1] = v
            np.testing.assert_allclose(got, want, atol=1e-6, err_msg=row["cite"] + " " + key)
    # the printed h part of Eq. A.4 uses node 3 (an eta node): not what the scheme needs (G8)
    a4 = rows[0]
    got = ops[2][2, 4] * a4["den"]
    assert got[2] == 0.0 and got[3] == -2


def _translated_modes(w, order, alpha):
    """Modes of u(x, tau) = w(x - alpha tau) by least squares on random points (exact for polynomials)."""
    pts = RNG.uniform(-0.5, 0.5, size=(400, 4))
    pts[:, 3] = RNG.uniform(0.0, 1.0, size=400)
    back = pts.copy()
    back[:, :3] -= np.outer(pts[:, 3], alpha)
    back[:, 3] = 0.0
    vals = basis.eval_basis(order, back) @ w
    coef, *_ = np.linalg.lstsq(basis.eval_basis(order, pts), vals, rcond=None)
    return coef


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("form", ["modal", "nodal"])
def test_linear_flux_predictor_is_exact(order, form, monkeypatch):
    """P3: with F_d = a_d u, M-1 Picard steps reproduce w(xi - a dt/dx tau) exactly (Eqs. 30, 36, 45; A-C)."""
    a = np.array([0.7, -1.3, 0.4])
    dx = (0.1, 0.2, 0.05)
    dt = 0.02
    monkeypatch.setattr(physics, "flux", lambda U, gamma, d: a[d] * U)
    w = RNG.normal(size=basis.L[order])
    w[basis.LS[order]:] = 0.0
    W = w[:basis.LS[order], None]
    Uhat, _ = predictor.predict(W, order, form, 1.4, dt, dx)
    alpha = a * dt / np.array(dx)
    np.testing.assert_allclose(Uhat[:, 0], _translated_modes(w, order, alpha), atol=1e-11)


@pytest.mark.parametrize("order", [3, 4])
def test_converged_mode_reaches_fixed_point(order):
    """Converged-tolerance mode: iterating past M-1 changes nothing for a linear flux, and stops early."""
    U = np.stack([1.0 + 0.1 * RNG.normal(size=(2, 2, 2)), 0.1 * RNG.normal(size=(2, 2, 2)),
                  0.1 * RNG.normal(size=(2, 2, 2)), 0.1 * RNG.normal(size=(2, 2, 2)), 2.5 + 0.1 * RNG.normal(size=(2, 2, 2))])
    W = np.zeros((basis.LS[order],) + U.shape)
    W[0] = U
    W[1:4] = 0.01 * RNG.normal(size=(3,) + U.shape)
    fixed, _ = predictor.predict(W, order, "modal", 1.4, 0.01, (0.1, 0.1, 0.1), n_iter=40)
    conv, iters = predictor.predict(W, order, "modal", 1.4, 0.01, (0.1, 0.1, 0.1), tol=1e-13)
    assert np.all(iters < 40) and np.all(iters >= 1)
    np.testing.assert_allclose(conv, fixed, atol=1e-12)
