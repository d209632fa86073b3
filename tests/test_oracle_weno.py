"""Pins of the zone WENO and the face-B WENO of Sec. III."""
import numpy as np
import pytest

from oracle import basis, weno

RNG = np.random.default_rng(7)


def _poly_cell_averages(coef_fn, n):
    """Exact zone averages on an n^3 grid (h = 1) of sum_c coef * x^a y^b z^c, zone i centred at i."""
    terms = coef_fn
    idx = np.arange(n, dtype=float)

    def avg1(p):
        # average of x^p over [i - 1/2, i + 1/2]
        return ((idx + 0.5) ** (p + 1) - (idx - 0.5) ** (p + 1)) / (p + 1)
    out = np.zeros((n, n, n))
    for (a, b, c), v in terms.items():
        out += v * avg1(c)[:, None, None] * avg1(b)[None, :, None] * avg1(a)[None, None, :]
    return out


def _true_modes(terms, order, centre):
    """Modes (Eq. 10-12) of the polynomial about a zone centre (local coords = x - centre)."""
    pts = RNG.uniform(-0.5, 0.5, size=(300, 4))
    pts[:, 3] = 0.0
    X = pts[:, :3] + np.array(centre, dtype=float)
    vals = sum(v * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c for (a, b, c), v in terms.items())
    V = basis.eval_basis(order, pts)[:, :basis.LS[order]]
    return np.linalg.lstsq(V, vals, rcond=None)[0]


@pytest.mark.parametrize("order", [2, 3, 4])
def test_reconstruction_exact_for_polynomials(order):
    """Every candidate is exact on polynomials of its degree, so WENO is exact for total degree <= M-1."""
    n = 12
    terms = {(a, b, c): RNG.normal() for a in range(order) for b in range(order) for c in range(order)
             if a + b + c <= order - 1}
    # shift the polynomial so values stay O(1) on the grid
    ubar = _poly_cell_averages({k: v * 6.0 ** -(sum(k)) for k, v in terms.items()}, n)
    W = weno.reconstruct(ubar, order)
    scaled = {k: v * 6.0 ** -(sum(k)) for k, v in terms.items()}
    for zone in [(5, 5, 5), (6, 4, 7), (4, 7, 6)]:
        k, j, i = zone
        np.testing.assert_allclose(W[:, k, j, i], _true_modes(scaled, order, (i, j, k)), atol=1e-10)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_constant_state_has_no_slopes(order):
    W = weno.reconstruct(np.full((6, 6, 6), 3.7), order)
    assert np.all(W[0] == 3.7) and np.abs(W[1:]).max() == 0.0


@pytest.mark.parametrize("order", [2, 3, 4])
def test_reconstruction_mirror_and_permutation_symmetry(order):
    """Symmetric linear weights: reflecting or permuting the data reflects/permutes the modes."""
    a = RNG.normal(size=(8, 8, 8))
    W = weno.reconstruct(a, order)
    Wr = weno.reconstruct(a[:, :, ::-1], order)         # xi -> -xi
    for k, m in enumerate(basis.MODES[order][:basis.LS[order]]):
        np.testing.assert_allclose(Wr[k], (-1) ** m[0] * W[k][:, :, ::-1], atol=1e-12)
    Wp = weno.reconstruct(np.transpose(a, (0, 2, 1)), order)  # swap x and y
    idx = {m: k for k, m in enumerate(basis.MODES[order])}
    for k, m in enumerate(basis.MODES[order][:basis.LS[order]]):
        k2 = idx[(m[1], m[0], m[2], m[3])]
        np.testing.assert_allclose(Wp[k2], np.transpose(W[k], (0, 2, 1)), atol=1e-12)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_face_b_weno_matches_faces_for_any_data(order):
    """Sec. III: every stencil interpolates the two face values of its zone, hence so does the blend."""
    Bf = RNG.normal(size=(5, 5, 9))
    b0, mom = weno.face_b_moments(Bf, 0, order)
    P = lambda a, x: basis.P(a, x)
    val = lambda x: b0 + sum(m * P(a + 1, x) for a, m in enumerate(mom))
    np.testing.assert_allclose(val(0.5), np.roll(Bf, -1, axis=-1), atol=1e-12)
    np.testing.assert_allclose(val(-0.5), Bf, atol=1e-12)


def test_face_b_weno_second_order_is_average_and_difference():
    Bf = RNG.normal(size=(3, 3, 6))
    b0, (bx,) = weno.face_b_moments(Bf, 0, 2)
    np.testing.assert_allclose(b0, 0.5 * (Bf + np.roll(Bf, -1, -1)))
    np.testing.assert_allclose(bx, np.roll(Bf, -1, -1) - Bf)


@pytest.mark.parametrize("order", [3, 4])
def test_face_b_weno_zone_average_exact_for_polynomials(order):
    """b0 is the zone average of B_x when B_x is a polynomial of degree <= M-1 in x (face values exact)."""
    c = RNG.normal(size=order)
    x = np.arange(10) - 0.5                       # face i-1/2 at x = i - 1/2
    Bf = np.broadcast_to(sum(ci * x ** p for p, ci in enumerate(c)), (2, 2, 10)).copy()
    b0, _ = weno.face_b_moments(Bf, 0, order)
    i = np.arange(10)
    avg = sum(ci * ((i + 0.5) ** (p + 1) - (i - 0.5) ** (p + 1)) / (p + 1) for p, ci in enumerate(c))
    np.testing.assert_allclose(b0[0, 0, 3:7], avg[3:7], atol=1e-10)
