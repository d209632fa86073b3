"""Pins of the physics (Eq. 3) and of the Riemann solvers' frozen eigen-structure (Sec. II.3, Sec. V)."""
import numpy as np
import pytest

from oracle import physics, riemann

RNG = np.random.default_rng(11)


def _euler_state():
    rho, P = RNG.uniform(0.5, 2.0), RNG.uniform(0.5, 2.0)
    v = RNG.normal(size=3)
    return physics.prim_to_cons(np.array(rho), *[np.array(x) for x in v], np.array(P), 1.4)


def _mhd_state(g=5.0 / 3.0):
    rho, P = RNG.uniform(0.5, 2.0), RNG.uniform(0.5, 2.0)
    v = RNG.normal(size=3)
    B = RNG.normal(size=3) * 2.0
    return physics.prim_to_cons(np.array(rho), *[np.array(x) for x in v], np.array(P), g, B=tuple(np.array(b) for b in B))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_euler_jacobian_eigenvalues(d):
    """Eq. 3 with B = 0: the flux Jacobian has eigenvalues v_d - a, v_d (x3), v_d + a."""
    for _ in range(5):
        U = _euler_state()
        A = physics.jacobian(U, 1.4, d)
        lam = np.sort(np.linalg.eigvals(A).real)
        v = U[1 + d] / U[0]
        a = np.sqrt(physics.sound_speed2(U, 1.4))
        np.testing.assert_allclose(lam, [v - a, v, v, v, v + a], atol=1e-9)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_mhd_jacobian_eigenvalues(d):
    """Eq. 3: the 7x7 Jacobian without B_d has v +- c_f, v +- c_A, v +- c_s, v (Gaussian units)."""
    g = 5.0 / 3.0
    for _ in range(5):
        U = _mhd_state(g)
        keep = [c for c in range(8) if c != 5 + d]
        A = physics.jacobian(U, g, d)[np.ix_(keep, keep)]
        lam = np.sort(np.linalg.eigvals(A).real)
        rho = U[0]
        v = U[1 + d] / rho
        a2 = physics.sound_speed2(U, g)
        b2 = (U[5] ** 2 + U[6] ** 2 + U[7] ** 2) / (4 * np.pi * rho)
        bn2 = U[5 + d] ** 2 / (4 * np.pi * rho)
        disc = np.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)
        cf, cs, ca = np.sqrt(0.5 * (a2 + b2 + disc)), np.sqrt(max(0.5 * (a2 + b2 - disc), 0)), np.sqrt(bn2)
        np.testing.assert_allclose(lam, np.sort([v - cf, v - ca, v - cs, v, v + cs, v + ca, v + cf]), atol=1e-8)
        assert physics.fast_speed(U, g, d) == pytest.approx(cf)


def test_energy_definition():
    """eps = rho v^2/2 + P/(gamma-1) + B^2/8pi (Eq. 3) and pressure() inverts it."""
    U = _mhd_state()
    assert physics.pressure(U, 5.0 / 3.0) > 0
    P = physics.pressure(U, 5.0 / 3.0)
    rho = U[0]
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    me = (U[5] ** 2 + U[6] ** 2 + U[7] ** 2) / (8 * np.pi)
    assert U[4] == pytest.approx(P / (2.0 / 3.0) + ke + me)


def test_mhd_electric_field_identification():
    """Eq. 7: E = -v x B equals (-G8, F8, -F7) = (H7, -H6, G6)."""
    U = _mhd_state()
    v = U[1:4] / U[0]
    B = U[5:8]
    E = -np.cross(v, B)
    F, G, H = (physics.flux(U, 5.0 / 3.0, d) for d in range(3))
    np.testing.assert_allclose([-G[7], F[7], -F[6]], E, atol=1e-12)
    np.testing.assert_allclose([H[6], -H[5], G[5]], E, atol=1e-12)
    assert F[5] == 0 and G[6] == 0 and H[7] == 0


@pytest.mark.parametrize("solver", ["hll", "linearized"])
@pytest.mark.parametrize("mhd", [False, True])
def test_riemann_consistency(solver, mhd):
    """Equal states on both sides give the physical flux (F(U, U) = F(U))."""
    U = _mhd_state() if mhd else _euler_state()
    g = 5.0 / 3.0 if mhd else 1.4
    U2 = U[:, None]
    for d in range(3):
        F = physics.flux(U2, g, d)
        got = riemann.SOLVERS[solver](d, g, U2, U2, U2, U2, F, F, U2, U2)
        np.testing.assert_allclose(got, F, atol=1e-12)


@pytest.mark.parametrize("mhd", [False, True])
def test_absolute_jacobian(mhd):
    """|A| has the eigenvalues |lambda| of A and commutes with A; |A|^2 = A^2."""
    U = (_mhd_state() if mhd else _euler_state())[:, None]
    g = 5.0 / 3.0 if mhd else 1.4
    absA, keep = riemann.abs_jacobian(U, g, 0)
    A = physics.jacobian(U[:, 0], g, 0)[np.ix_(keep, keep)]
    np.testing.assert_allclose(absA[0] @ absA[0], A @ A, atol=1e-8 * np.abs(A @ A).max())
    np.testing.assert_allclose(absA[0] @ A, A @ absA[0], atol=1e-8 * np.abs(A @ A).max())
    np.testing.assert_allclose(np.sort(np.linalg.eigvals(absA[0]).real),
                               np.sort(np.abs(np.linalg.eigvals(A).real)), atol=1e-8)


@pytest.mark.parametrize("case", ["no_normal_field", "no_transverse_field", "triple_umbilic"])
def test_absolute_jacobian_degenerate_mhd_states(case):
    """Where MHD wave speeds coincide (B_n = 0: slow = Alfven = entropy; B_t = 0: Alfven = fast or slow;
    B_t = 0 and c_A = a: all three at one speed) |A| still satisfies |A|^2 = A^2, commutes with A and has
    the eigenvalues |lambda|."""
    g = 5.0 / 3.0
    rho, P = 1.3, 0.9
    B = {"no_normal_field": (0.0, 0.8, -0.5), "no_transverse_field": (1.7, 0.0, 0.0),
         "triple_umbilic": (np.sqrt(4 * np.pi * g * P), 0.0, 0.0)}[case]
    U = physics.prim_to_cons(np.array([rho]), np.array([0.4]), np.array([-0.3]), np.array([0.2]),
                             np.array([P]), g, tuple(np.array([b]) for b in B))
    absA, keep = riemann.abs_jacobian(U, g, 0)
    A = physics.jacobian(U[:, 0], g, 0)[np.ix_(keep, keep)]
    assert np.isfinite(absA).all()
    scale = np.abs(A @ A).max()
    np.testing.assert_allclose(absA[0] @ absA[0], A @ A, atol=1e-10 * scale)
    np.testing.assert_allclose(absA[0] @ A, A @ absA[0], atol=1e-10 * scale)
    np.testing.assert_allclose(np.sort(np.linalg.eigvals(absA[0]).real),
                               np.sort(np.abs(np.linalg.eigvals(A).real)), atol=1e-6)


def test_hll_upwinds_supersonic_flow():
    """Supersonic flow to the right: HLL returns the left averaged flux (lambda_L = 0 after the reset)."""
    U = physics.prim_to_cons(np.array([1.0]), np.array([5.0]), np.array([0.0]), np.array([0.0]), np.array([1.0]), 1.4)
    UR = physics.prim_to_cons(np.array([0.5]), np.array([4.0]), np.array([0.0]), np.array([0.0]), np.array([0.8]), 1.4)
    FL, FR = physics.flux(U, 1.4, 0), physics.flux(UR, 1.4, 0)
    got = riemann.hll(0, 1.4, U, UR, U, UR, FL, FR, U, UR)
    np.testing.assert_allclose(got, FL, atol=1e-12)
