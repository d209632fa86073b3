"""Pins of the oracle's bases, node sets and face/edge integrals against the paper's printed closed forms."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import paper_formulas as pf
from oracle import basis, faces, nodes

RNG = np.random.default_rng(1006)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_basis_is_complete_total_degree(order):
    """Eqs. 10-16 span exactly the polynomials of total degree <= M-1 (L = C(M+3, 4))."""
    modes = basis.MODES[order]
    assert len(modes) == basis.L[order] == len(set(modes))
    want = {(a, b, c, d) for a in range(order) for b in range(order) for c in range(order) for d in range(order)
            if a + b + c + d <= order - 1}
    assert set(modes) == want
    assert all(m[3] == 0 for m in modes[:basis.LS[order]])
    assert all(m[3] > 0 for m in modes[basis.LS[order]:])


def test_mode_index_conventions():
    """Eq. 11: w8 = xi eta, w9 = eta zeta, w10 = xi zeta; Eq. 16 time modes 21..35."""
    m = basis.MODES[4]
    assert m[7] == (1, 1, 0, 0) and m[8] == (0, 1, 1, 0) and m[9] == (1, 0, 1, 0)
    assert m[19] == (1, 1, 1, 0) and m[34] == (1, 0, 1, 1) and m[29] == (2, 0, 0, 1)


def test_hermite_polynomials_are_orthogonal():
    """Eq. 9: P0..P3 are mutually orthogonal on [-1/2, 1/2] (exact rational arithmetic)."""
    for a in range(4):
        for b in range(a + 1, 4):
            prod = [Fr(0)] * (len(basis.P_MONO[a]) + len(basis.P_MONO[b]) - 1)
            for i, x in enumerate(basis.P_MONO[a]):
                for j, y in enumerate(basis.P_MONO[b]):
                    prod[i + j] += x * y
            assert basis._poly_int(prod, Fr(-1, 2), Fr(1, 2)) == 0


@pytest.mark.parametrize("order,table,formula", [
    (2, nodes.MODAL_O2, pf.eq32), (3, nodes.MODAL_O3, pf.eq38_39), (4, nodes.MODAL_O4, pf.eq47_48)])
def test_modal_transcription_matches_basis(order, table, formula):
    """Eqs. 32, 38-39, 47-48 equal the basis expansion evaluated at the nodes of Eqs. 31, 37, 46."""
    for _ in range(5):
        w = RNG.normal(size=basis.L[order])
        np.testing.assert_allclose(formula(w), basis.eval_basis(order, nodes.as_array(table)) @ w, atol=1e-13)


@pytest.mark.parametrize("order,table,formula", [
    (2, nodes.NODAL_O2, pf.eqA5), (3, nodes.NODAL_O3, pf.eqB4), (4, nodes.NODAL_O4, pf.eqC4)])
def test_nodal_spatial_transcription(order, table, formula):
    """Eqs. A.5, B.4, C.4: the tau = 0 nodal values of Eqs. A.1, B.1, C.1 from the spatial modes."""
    for _ in range(5):
        w = RNG.normal(size=basis.L[order])
        w[basis.LS[order]:] = 0.0
        got = formula(w)
        np.testing.assert_allclose(got, (basis.eval_basis(order, nodes.as_array(table)) @ w)[:len(got)], atol=1e-13)


@pytest.mark.parametrize("order,formula", [(3, pf.eqB5), (4, pf.eqC5)])
def test_nodal_to_modal(order, formula):
    """Eqs. B.5, C.5: evolutionary modes from the nodal values (C.5 with garble G14 read)."""
    V = basis.eval_basis(order, nodes.as_array(nodes.NODAL[order]))
    for _ in range(5):
        w = RNG.normal(size=basis.L[order])
        np.testing.assert_allclose(formula(V @ w), w[basis.LS[order]:], atol=1e-12)


def test_eqC5_u35_as_printed_is_a_garble():
    """The printed last line of Eq. C.5 is off for generic data; with node 26 it is exact (G14)."""
    V = basis.eval_basis(4, nodes.as_array(nodes.NODAL[4]))
    w = RNG.normal(size=35)
    assert abs(pf.eqC5_u35_as_printed(V @ w) - w[34]) > 1e-3


@pytest.mark.parametrize("order,formula", [(2, pf.eq58_60), (3, pf.eq61_63), (4, pf.eq64_66)])
def test_face_and_edge_averages(order, formula):
    """Eqs. 58-66 equal the exact face/edge integrals of Eqs. 54, 55, 57."""
    T = faces.tables(order)
    for _ in range(5):
        w = RNG.normal(size=basis.L[order])
        o = formula(w)
        for s, sc in ((+1, "+"), (-1, "-")):
            assert o["ub" + sc] == pytest.approx(T.ub[0, s] @ w, abs=1e-13)
            assert o["avg" + sc] == pytest.approx(T.avg[0, s] @ w, abs=1e-13)
            for e, en in ((1, "y"), (2, "z")):
                for se, ses in ((+1, "+"), (-1, "-")):
                    assert o[en + ses + sc] == pytest.approx(T.edge[0, s, e, se] @ w, abs=1e-13)


def test_integral_weights_by_gauss_legendre():
    """The exact face integrals agree with 4-point Gauss-Legendre quadrature of the basis (independent route)."""
    x, wq = np.polynomial.legendre.leggauss(4)
    xs, ws = 0.5 * x, 0.5 * wq
    ts, wt = 0.5 * (x + 1), 0.5 * wq
    for order in (2, 3, 4):
        w = RNG.normal(size=basis.L[order])
        pts = np.array([(0.5, a, b, t) for a in xs for b in xs for t in ts])
        wts = np.array([wa * wb * wc for wa in ws for wb in ws for wc in wt])
        quad = wts @ (basis.eval_basis(order, pts) @ w)
        assert quad == pytest.approx(faces.tables(order).avg[0, +1] @ w, abs=1e-13)


@pytest.mark.parametrize("order,formula", [(2, pf.eqD3), (3, pf.eqD8), (4, pf.eqD13)])
def test_facial_node_transcription(order, formula):
    """Eqs. D.3, D.8, D.13 (D.13 with G6) equal the basis at the facial nodes of Eqs. D.1, D.6, D.11."""
    for _ in range(5):
        w = RNG.normal(size=basis.L[order])
        np.testing.assert_allclose(formula(w), faces.tables(order).fnode_V[0, +1] @ w, atol=1e-13)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_facial_flux_integrals(order):
    """Eqs. D.5, D.10, D.15 equal the exact integrals of the facial bases D.2, D.7, D.12."""
    T = faces.tables(order)
    for _ in range(5):
        m = RNG.normal(size=len(basis.FACE_MODES[order]))
        o = pf.eqD5_D10_D15(order, m)
        assert o["avg"] == pytest.approx(T.face_avg_w @ m, abs=1e-13)
        for slot, nm in ((0, "t1"), (1, "t2")):
            for se, ss in ((+1, "+"), (-1, "-")):
                assert o[nm + ss] == pytest.approx(T.face_edge_w[slot, se] @ m, abs=1e-13)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_nodal_node_sets_are_unisolvent(order):
    """Apps. A-C: one node per mode, so Lagrange interpolation is well posed."""
    V = basis.eval_basis(order, nodes.as_array(nodes.NODAL[order]))
    assert V.shape[0] == V.shape[1] and np.linalg.cond(V) < 1e4
