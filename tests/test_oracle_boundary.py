"""Pins of the ghost-zone box boundaries of the oracle (oracle.boundary).

* A reflecting wall is the mirror plane of a problem twice the size: the step of a box with reflecting
  faces on an axis equals the periodic step of the box followed by its mirror image (normal momentum
  negated), restricted to the original half.  This holds for every form, order and solver, whatever
  the symmetry of the scheme, because every interior zone then reads the same averages in both.
* Outflow (zero gradient) leaves a uniform flow unchanged, and equals periodic where the state near
  the boundary is uniform.
* A closed box (reflecting on all faces) conserves mass and energy to round-off with the modal form:
  its wall faces see mirror-image states, so their mass and energy fluxes vanish.
* The ghost width covers the reach of a step: a wider ghost layer changes nothing (beyond rounding), and
  a narrower one does.
"""
import numpy as np
import pytest

from oracle import boundary, scheme
from paper_1006_2146_gb300 import inputs


def _mirror_double(U, d):
    """The state followed by its mirror image along direction d, normal momentum negated."""
    ax = 3 - d
    M = np.flip(U, axis=ax).copy()
    M[1 + d] *= -1.0
    return np.concatenate([U, M], axis=ax)


def _dx(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


@pytest.mark.parametrize("order,form,solver", [(2, "modal", "hll"), (3, "nodal", "hll"), (3, "modal", "linearized"),
                                               (4, "nodal", "hll")])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_reflective_wall_is_the_mirror_plane(order, form, solver, d):
    shape = [3, 3, 3]
    shape[2 - d] = 8
    shape = tuple(shape)
    U = inputs.random_smooth(shape, seed=40 + d, amp=0.3)
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    bc = [0] * 6
    bc[2 * d] = bc[2 * d + 1] = boundary.REFLECTIVE
    got = boundary.ader_step(U, dx, dt, order, form, solver, bc=bc)
    big = scheme.ader_step(_mirror_double(U, d), dx, dt, order, form, solver)
    want = np.take(big, np.arange(shape[2 - d]), axis=3 - d)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(U).max())


def test_reflective_and_outflow_mixed_faces_match_the_mirror_plane():
    """x reflecting at both ends, y outflow, z periodic: the y boundaries see a uniform state there."""
    shape = (3, 8, 8)
    U = inputs.random_smooth(shape, seed=7, amp=0.3)
    U[:, :, :, :] = U[:, :, 3:4, :]                      # uniform along y: outflow equals periodic in y
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    bc = (boundary.REFLECTIVE, boundary.REFLECTIVE, boundary.OUTFLOW, boundary.OUTFLOW, 0, 0)
    got = boundary.ader_step(U, dx, dt, 3, "modal", "hll", bc=bc)
    want = scheme.ader_step(_mirror_double(U, 0), dx, dt, 3, "modal", "hll")[..., :8]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(U).max())


@pytest.mark.parametrize("order", [2, 3, 4])
def test_outflow_keeps_a_uniform_flow(order):
    shape = (5, 6, 7)
    U = np.empty((5,) + shape)
    rho, v, p = 1.3, (0.5, -0.3, 0.2), 0.9
    U[0] = rho
    for d in range(3):
        U[1 + d] = rho * v[d]
    U[4] = p / 0.4 + 0.5 * rho * sum(x * x for x in v)
    dx = _dx(shape)
    dt = scheme.max_dt(U, dx, 0.4)
    out = boundary.ader_step(U, dx, dt, order, "nodal", "hll", bc=(boundary.OUTFLOW,) * 6)
    np.testing.assert_allclose(out, U, rtol=1e-14, atol=0)


def test_outflow_equals_periodic_where_the_boundary_is_uniform():
    """A perturbation in the middle of x, uniform over the 10 zones next to each end (more than a ghost
    layer plus a step's reach): outflow in x gives the periodic step (to round-off)."""
    shape = (3, 4, 30)
    U = inputs.random_smooth(shape, seed=9, amp=0.3)
    U[..., :10] = U[..., 10:11]
    U[..., 20:] = U[..., 10:11]
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    got = boundary.ader_step(U, dx, dt, 3, "modal", "hll", bc=(boundary.OUTFLOW, boundary.OUTFLOW, 0, 0, 0, 0))
    want = scheme.ader_step(U, dx, dt, 3, "modal", "hll")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(U).max())


@pytest.mark.parametrize("order", [2, 3])
def test_closed_box_conserves_mass_and_energy(order):
    shape = (6, 6, 6)
    U = inputs.random_smooth(shape, seed=12, amp=0.3)
    dx = _dx(shape)
    tot0 = U.reshape(5, -1).sum(axis=1)
    for _ in range(3):
        dt = 0.7 * scheme.max_dt(U, dx, 0.4)
        U = boundary.ader_step(U, dx, dt, order, "modal", "hll", bc=(boundary.REFLECTIVE,) * 6)
    tot = U.reshape(5, -1).sum(axis=1)
    for v in (0, 4):
        assert abs(tot[v] - tot0[v]) <= 1e-13 * abs(tot0[v])
    # the walls push: momentum is not conserved
    assert np.abs(tot[1:4] - tot0[1:4]).max() > 1e-8


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ghost_width_covers_the_reach_of_a_step(order):
    shape = (4, 9, 9)
    U = inputs.random_smooth(shape, seed=20 + order, amp=0.3)
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    bc = (boundary.REFLECTIVE, boundary.OUTFLOW, boundary.OUTFLOW, boundary.REFLECTIVE, 0, 0)
    a = boundary.ader_step(U, dx, dt, order, "nodal", "hll", bc=bc)
    b = boundary.ader_step(U, dx, dt, order, "nodal", "hll", bc=bc, G=9)
    # equal up to the rounding of the oracle's array operations on arrays of other shapes; a ghost layer
    # narrower than the reach changes zones near the boundary at the size of the state's variation
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.abs(U).max())


def test_ghost_fill_rules():
    U = np.arange(5 * 2 * 2 * 6, dtype=float).reshape(5, 2, 2, 6) + 1.0
    E = boundary.extend(U, (boundary.OUTFLOW, boundary.REFLECTIVE, 0, 0, 0, 0), 3)
    assert E.shape == (5, 2, 2, 12)
    np.testing.assert_array_equal(E[..., :3], np.repeat(U[..., :1], 3, axis=-1))          # outflow: copies
    np.testing.assert_array_equal(E[[0, 2, 3, 4], ..., 9:], U[[0, 2, 3, 4], ..., ::-1][..., :3])   # mirror
    np.testing.assert_array_equal(E[1, ..., 9:], -U[1, ..., ::-1][..., :3])              # normal momentum flips
    with pytest.raises(ValueError):
        boundary.extend(U, (boundary.OUTFLOW, 0, 0, 0, 0, 0), 3)


def test_a_ghost_layer_narrower_than_the_reach_shows():
    """The check above can fail: one zone fewer than the reach of a third-order step changes the result."""
    shape = (4, 9, 9)
    U = inputs.random_smooth(shape, seed=23, amp=0.3)
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    bc = (boundary.REFLECTIVE, boundary.OUTFLOW, 0, 0, 0, 0)
    a = boundary.ader_step(U, dx, dt, 3, "nodal", "hll", bc=bc)
    b = boundary.ader_step(U, dx, dt, 3, "nodal", "hll", bc=bc, G=2)
    assert np.abs(a - b).max() > 1e-6
