"""Global pins of the oracle step: conservation, convergence order, the exact Sod solution, symmetry."""
import numpy as np
import pytest

import exact_riemann
from oracle import scheme
from paper_1006_2146_gb300 import inputs

RNG = np.random.default_rng(5)


def _run(U, dx, T, cfl, step):
    t = 0.0
    while t < T - 1e-14:
        dt = min(scheme.max_dt(U, dx, cfl), T - t)
        U = step(U, dt)
        t += dt
    return U


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("form,solver", [("nodal", "hll"), ("modal", "linearized")])
def test_conservation_to_round_off(order, form, solver):
    """Eq. 6 telescopes on a periodic mesh: the totals of all five variables change only by round-off."""
    U = inputs.random_smooth((6, 8, 10), seed=3, amp=0.3)
    dx = (0.1, 0.125, 1.0 / 6.0)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    U1 = scheme.ader_step(U, dx, dt, order, form, solver)
    tot0, tot1 = U.sum(axis=(1, 2, 3)), U1.sum(axis=(1, 2, 3))
    scale = np.abs(U).sum(axis=(1, 2, 3)).max()
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)
    assert np.abs(U1 - U).max() > 1e-6         # something happened


@pytest.mark.parametrize("solver", ["hll", "linearized"])
def test_constant_state_is_preserved(solver):
    U = inputs.density_wave(6, amp=0.0, vel=(0.3, -0.2, 0.5))
    U1 = scheme.ader_step(U, (1 / 6,) * 3, 0.01, 3, "modal", solver)
    np.testing.assert_allclose(U1, U, atol=1e-14)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_density_wave_convergence_order(order):
    """Smooth advection along the diagonal (config-1 data): L1 order within 0.2 of M (cf. Table IV)."""
    errs = []
    for n in (8, 16):
        U = inputs.density_wave(n)
        dx = (1.0 / n,) * 3
        U = _run(U, dx, 0.05, 0.4, lambda U, dt: scheme.ader_step(U, dx, dt, order, "nodal", "hll"))
        errs.append(np.abs(U[0] - inputs.density_wave(n, t=0.05)[0]).mean())
    assert np.log2(errs[0] / errs[1]) >= order - 0.2


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ssp_rk_convergence_order(order):
    """Eqs. 18-20 with the spatial face rule converge at the design order on the same problem."""
    errs = []
    for n in (8, 16):
        U = inputs.density_wave(n)
        dx = (1.0 / n,) * 3
        U = _run(U, dx, 0.05, 0.2, lambda U, dt: scheme.rk_step(U, dx, dt, order))
        errs.append(np.abs(U[0] - inputs.density_wave(n, t=0.05)[0]).mean())
    assert np.log2(errs[0] / errs[1]) >= order - 0.2 - (0.3 if order == 4 else 0.0)


def _sod_error(n, order, solver, T=0.05):
    shape = (2, n, n)
    U = inputs.sod_planar(shape)
    dx = (1.0 / n, 1.0 / n, 0.5)
    U = _run(U, dx, T, 0.4, lambda U, dt: scheme.ader_step(U, dx, dt, order, "modal", solver))
    # exact: two Riemann problems along s = (x + y)/sqrt(2): sigma = x + y in [0, 2)
    c = (np.arange(n) + 0.5) / n
    sub = (np.arange(4) + 0.5) / 4 - 0.5
    exact = np.zeros((n, n))
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    for a in sub:
        for b in sub:
            sig = (c[None, :] + a / n) + (c[:, None] + b / n)
            frac = sig - np.floor(sig)
            # interface at sigma = 1/2 (left state below) and at sigma = 0 = 1 (left state above)
            s1 = (frac - 0.5) / np.sqrt(2.0) / T
            s2 = np.where(frac < 0.5, frac, frac - 1.0) / np.sqrt(2.0) / T
            r1, _, _ = exact_riemann.sample(L, R, 1.4, s1)
            r2, _, _ = exact_riemann.sample(R, L, 1.4, s2)
            exact += np.where(np.abs(frac - 0.5) < 0.25, r1, r2)
    exact /= 16
    return np.abs(U[0, 0] - exact).mean()


@pytest.mark.parametrize("solver", ["hll", "linearized"])
def test_sod_converges_to_exact_riemann_solution(solver):
    """Config-2 Sod tube along (1,1,0): L1 error against the exact solution falls with resolution."""
    e1, e2 = _sod_error(16, 3, solver), _sod_error(32, 3, solver)
    assert e2 < 0.75 * e1 and e2 < 0.03


@pytest.mark.parametrize("order", [2, 3])
def test_modal_blast_is_symmetric(order):
    """Sec. VIII.3: the modal scheme keeps a centred blast mirror- and permutation-symmetric to round-off."""
    n = 12
    U = inputs.blast(n, p_in=10.0, radius=0.2)
    dx = (1.0 / n,) * 3
    for _ in range(2):
        dt = scheme.max_dt(U, dx, 0.3)
        U = scheme.ader_step(U, dx, dt, order, "modal", "hll")
    scale = np.abs(U[0]).max()
    np.testing.assert_allclose(U[0], U[0][:, :, ::-1], atol=1e-13 * scale)
    np.testing.assert_allclose(U[1], -U[1][:, :, ::-1], atol=1e-13 * np.abs(U[4]).max())
    np.testing.assert_allclose(U[0], np.transpose(U[0], (0, 2, 1)), atol=1e-13 * scale)
    np.testing.assert_allclose(U[0], np.transpose(U[0], (2, 1, 0)), atol=1e-13 * scale)
    assert np.abs(U[1]).max() > 1e-3


def test_max_dt_definition():
    """dt = cfl / max sum_d (|v_d| + a)/dx_d."""
    U = inputs.density_wave(4, amp=0.0, vel=(1.0, -2.0, 0.5))
    a = np.sqrt(1.4)
    want = 0.4 / ((1.0 + a) * 4 + (2.0 + a) * 8 + (0.5 + a) * 2)
    assert scheme.max_dt(U, (0.25, 0.125, 0.5), 0.4) == pytest.approx(want)
