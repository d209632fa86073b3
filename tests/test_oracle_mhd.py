"""Pins of the oracle's ideal-MHD step: constrained transport (Eq. 8), EMFs (Eq. 7), convergence."""
import numpy as np
import pytest

from oracle import physics, scheme, weno
from paper_1006_2146_gb300 import inputs

G = 5.0 / 3.0


def _run(U, B, dx, T, order, form="modal", solver="hll"):
    t = 0.0
    while t < T - 1e-14:
        dt = min(scheme.max_dt(U, dx, 0.4, G, Bface=B), T - t)
        U, B = scheme.ader_step(U, dx, dt, order, form, solver, G, Bface=B)
        t += dt
    return U, B


def test_initial_fields_are_divergence_free():
    for n in (8, 12):
        _, B = inputs.alfven_wave(n)
        assert np.abs(scheme.div_b(B, (1.0 / n,) * 3)).max() < 1e-12
        _, B = inputs.orszag_tang(n)
        assert np.abs(scheme.div_b(B, (1.0 / n,) * 3)).max() < 1e-12


@pytest.mark.parametrize("solver", ["hll", "linearized"])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_constrained_transport_keeps_div_b_and_conserves(order, solver):
    """Eq. 8 changes every zone's discrete div B by round-off only; hydro totals and face-B totals are conserved."""
    rng = np.random.default_rng(order)
    n = 8
    dx = (1.0 / n,) * 3
    U, B = inputs.alfven_wave(n, amp=0.3)
    U = U * (1.0 + 0.02 * rng.normal(size=U.shape))          # break the symmetry of the wave
    U[4] += 0.5
    d0 = scheme.div_b(B, dx)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    U1, B1 = scheme.ader_step(U, dx, dt, order, "nodal", solver, G, Bface=B)
    scale = np.abs(B).max() / dx[0]
    assert np.abs(scheme.div_b(B1, dx) - d0).max() <= 1e-13 * scale
    assert np.abs(B1 - B).max() > 1e-6
    np.testing.assert_allclose(B1.reshape(3, -1).sum(axis=1), B.reshape(3, -1).sum(axis=1), atol=1e-12 * np.abs(B).sum())
    np.testing.assert_allclose(U1.reshape(5, -1).sum(axis=1), U.reshape(5, -1).sum(axis=1), atol=1e-12 * np.abs(U).sum())


@pytest.mark.parametrize("solver", ["hll", "linearized"])
def test_uniform_magnetised_flow_is_unchanged(solver):
    n = 6
    dx = (1.0 / n,) * 3
    B = np.stack([np.full((n, n, n), b) for b in (0.7, -0.4, 1.1)])
    rho = np.ones((n, n, n))
    v = [0.3 * rho, -0.2 * rho, 0.1 * rho]
    U = physics.prim_to_cons(rho, *v, rho, G, B=(B[0], B[1], B[2]))[:5]
    U1, B1 = scheme.ader_step(U, dx, 0.01, 3, "modal", solver, G, Bface=B)
    np.testing.assert_allclose(U1, U, atol=1e-13)
    np.testing.assert_allclose(B1, B, atol=1e-13)


@pytest.mark.parametrize("order,solver", [(2, "hll"), (3, "hll"), (3, "linearized")])
def test_alfven_wave_convergence(order, solver):
    """Config 3: the circularly polarised Alfven wave translates exactly; L1 order within 0.2 of M."""
    errs = []
    for n in (8, 16):
        U, B = inputs.alfven_wave(n)
        dx = (1.0 / n,) * 3
        U, B = _run(U, B, dx, 0.05, order, solver=solver)
        Ue, Be = inputs.alfven_wave(n, t=0.05)
        errs.append(np.abs(B - Be).mean() + np.abs(U[1:4] - Ue[1:4]).mean())
    assert np.log2(errs[0] / errs[1]) >= order - 0.2


def test_emf_identification_on_uniform_state():
    """Eq. 7: with uniform v and B every edge EMF equals -v x B."""
    n = 4
    dx = (1.0 / n,) * 3
    Bv, vv = np.array([0.7, -0.4, 1.1]), np.array([0.3, -0.2, 0.1])
    B = np.stack([np.full((n, n, n), b) for b in Bv])
    rho = np.ones((n, n, n))
    U = physics.prim_to_cons(rho, *[c * rho for c in vv], rho, G, B=tuple(B))
    Uz, W = scheme.zone_state(U[:5], B, 3)
    from oracle import predictor
    Uhat, _ = predictor.predict(W, 3, "modal", G, 0.01, dx)
    _, ed = scheme._face_fluxes(Uhat, 3, G, "hll", Uz, True)
    Ex, Ey, Ez = scheme.edge_emfs(scheme.edge_fluxes(ed, Uz, 3, G, "hll"))
    E = -np.cross(vv, Bv)
    np.testing.assert_allclose(Ex, E[0], atol=1e-13)
    np.testing.assert_allclose(Ey, E[1], atol=1e-13)
    np.testing.assert_allclose(Ez, E[2], atol=1e-13)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ssprk_mhd_keeps_div_b_and_conserves(order):
    """SSP-RK with the spatial-only operator (Eqs. 18-20; L(B) = -curl E, the rate of Eq. 8): each stage is a
    combination of CT updates, so div B is unchanged to round-off and the totals are conserved."""
    rng = np.random.default_rng(10 + order)
    n = 8
    dx = (1.0 / n,) * 3
    U, B = inputs.alfven_wave(n, amp=0.3)
    U = U * (1.0 + 0.02 * rng.normal(size=U.shape))
    U[4] += 0.5
    d0 = scheme.div_b(B, dx)
    dt = 0.3 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    U1, B1 = scheme.rk_step(U, dx, dt, order, "hll", G, Bface=B)
    scale = np.abs(B).max() / dx[0]
    assert np.abs(scheme.div_b(B1, dx) - d0).max() <= 1e-13 * scale
    assert np.abs(B1 - B).max() > 1e-6
    np.testing.assert_allclose(B1.reshape(3, -1).sum(axis=1), B.reshape(3, -1).sum(axis=1), atol=1e-12 * np.abs(B).sum())
    np.testing.assert_allclose(U1.reshape(5, -1).sum(axis=1), U.reshape(5, -1).sum(axis=1), atol=1e-12 * np.abs(U).sum())


def test_ssprk_mhd_alfven_wave_convergence():
    """SSP-RK3 with the third-order spatial operator on the Alfven wave: L1 order within 0.2 of 3."""
    errs = []
    for n in (8, 16):
        U, B = inputs.alfven_wave(n)
        dx = (1.0 / n,) * 3
        t, T = 0.0, 0.05
        while t < T - 1e-14:
            dt = min(0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B), T - t)
            U, B = scheme.rk_step(U, dx, dt, 3, "hll", G, Bface=B)
            t += dt
        Ue, Be = inputs.alfven_wave(n, t=T)
        errs.append(np.abs(B - Be).mean() + np.abs(U[1:4] - Ue[1:4]).mean())
    assert np.log2(errs[0] / errs[1]) >= 3 - 0.2
