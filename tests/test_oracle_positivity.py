"""Pins of the oracle's a-posteriori positivity fallback (scheme.positivity_fallback; an option, the paper
names no safeguard).  Case: the double rarefaction (rho 1, P 0.4, v = -/+ 4 on the two halves of a
periodic line), whose near-vacuum centre drives the fourth-order step to a negative pressure in a few
steps.

* smooth data: the option changes nothing, bit for bit;
* the double rarefaction: with the option every step stays physical, and the totals are conserved;
* the fallback is local: zones farther than three zones from a non-physical one keep the plain update.
"""
import numpy as np

from oracle import physics, scheme
from paper_1006_2146_gb300 import inputs


def _double_rarefaction(n, v0=4.0, p0=0.4, gamma=1.4):
    x = (np.arange(n) + 0.5) / n
    vx = np.where(x < 0.5, -v0, v0)[None, None, :] * np.ones((1, 1, n))
    rho = np.ones((1, 1, n))
    z = np.zeros_like(rho)
    return np.stack([rho, rho * vx, z, z, p0 / (gamma - 1.0) * rho + 0.5 * rho * vx ** 2])


def test_no_change_on_smooth_data():
    U = inputs.random_smooth(8, seed=77, amp=0.3)
    dx = (1 / 8,) * 3
    dt = scheme.max_dt(U, dx, 0.4)
    assert np.array_equal(scheme.ader_step(U, dx, dt, 3, "modal", "hll"),
                          scheme.ader_step(U, dx, dt, 3, "modal", "hll", positivity=True))


def test_double_rarefaction_stays_physical_and_conservative():
    n = 32
    dx = (1 / n, 1.0, 1.0)
    U = _double_rarefaction(n)
    tot0 = U.sum(axis=(1, 2, 3))
    failed_plain = False
    for _ in range(20):
        dt = scheme.max_dt(U, dx, 0.3)
        plain = scheme.ader_step(U, dx, dt, 4, "modal", "hll")
        failed_plain |= not physics.physical(plain, 1.4).all()
        U = scheme.ader_step(U, dx, dt, 4, "modal", "hll", positivity=True)
        assert physics.physical(U, 1.4).all()
    assert failed_plain
    assert np.abs(U.sum(axis=(1, 2, 3)) - tot0).max() <= 1e-13 * np.abs(tot0).max()


def test_fallback_is_local():
    n = 32
    dx = (1 / n, 1.0, 1.0)
    U = _double_rarefaction(n)
    for _ in range(3):
        dt = scheme.max_dt(U, dx, 0.3)
        plain = scheme.ader_step(U, dx, dt, 4, "modal", "hll")
        bad = ~physics.physical(plain, 1.4)
        if bad.any():
            break
        U = plain
    assert bad.any()
    fixed = scheme.ader_step(U, dx, dt, 4, "modal", "hll", positivity=True)
    near = bad[0, 0].copy()
    for _ in range(3):
        near = near | np.roll(near, 1) | np.roll(near, -1)
    changed = np.any(fixed[:, 0, 0] != plain[:, 0, 0], axis=0)
    assert changed.any() and not (changed & ~near).any()


def _mhd_double_rarefaction(n, v0=4.0, by=5.0, p0=0.4, gamma=1.4):
    U = _double_rarefaction(n, v0, p0, gamma)
    U[4] += by ** 2 / (8.0 * np.pi)
    z = np.zeros((1, 1, n))
    return U, np.stack([z, by + z, z])


def _mhd_physical(U, B):
    zB = np.stack([0.5 * (B[d] + np.roll(B[d], -1, axis=2 - d)) for d in range(3)])
    return physics.physical(np.concatenate([U, zB]), 1.4)


def test_mhd_fallback_stays_physical_keeps_div_b_and_acts_locally():
    """MHD (transverse field 5, beta 0.4): where the plain fourth-order step leaves a non-physical zone, the
    fallback replaces the hydrodynamic fluxes around the marked zones and the electric fields of their
    edges by first-order ones.  The state stays physical, mass and energy are conserved, the face field
    changes only near the zones the plain step left non-physical (three passes, each widening the marks by
    a zone, plus the edges around them), and div B stays at round-off (Eq. 8's curl of any edge fields)."""
    n = 32
    dx = (1 / n, 1.0, 1.0)
    U, B = _mhd_double_rarefaction(n)
    tot0 = U.sum(axis=(1, 2, 3))
    failed_plain = False
    field_changed = False
    for _ in range(15):
        dt = scheme.max_dt(U, dx, 0.3, 1.4, Bface=B)
        pU, pB = scheme.ader_step(U, dx, dt, 4, "modal", "hll", 1.4, Bface=B)
        bad = ~_mhd_physical(pU, pB)
        failed_plain |= bad.any()
        U, B2 = scheme.ader_step(U, dx, dt, 4, "modal", "hll", 1.4, Bface=B, positivity=True)
        near = bad[0, 0].copy()
        for _ in range(4):
            near = near | np.roll(near, 1) | np.roll(near, -1)
        changed = np.any(B2[:, 0, 0] != pB[:, 0, 0], axis=0)
        assert not (changed & ~near).any()
        field_changed |= changed.any()
        assert np.abs(scheme.div_b(B2, dx)).max() <= 1e-12 * np.abs(B2).max() / dx[0]
        B = B2
        assert _mhd_physical(U, B).all()
    assert failed_plain and field_changed
    assert np.abs(U.sum(axis=(1, 2, 3)) - tot0).max() <= 1e-13 * np.abs(tot0).max()
