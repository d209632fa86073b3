"""Non-periodic box faces on the GPU (ader_set_boundary, Euler) against the oracle's ghost-zone boundaries
(oracle.boundary, pinned in tests/test_oracle_boundary.py)."""
import itertools

import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import boundary, scheme
from paper_1006_2146_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

O, R = boundary.OUTFLOW, boundary.REFLECTIVE
PATTERNS = [(R, R, 0, 0, 0, 0), (O, O, R, R, 0, 0), (R, O, O, R, R, R), (O,) * 6]


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _dx(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


@pytest.mark.parametrize("order,form,solver", [(2, "modal", "hll"), (3, "nodal", "hll"), (3, "modal", "linearized"),
                                               (4, "nodal", "hll"), (4, "modal", "linearized")])
@pytest.mark.parametrize("bc", PATTERNS)
def test_boundary_step_parity_fp64(ader, order, form, solver, bc):
    shape = (6, 7, 9)
    U = inputs.random_smooth(shape, seed=60 + order, amp=0.3)
    dx = _dx(shape)
    dt = 0.7 * scheme.max_dt(U, dx, 0.4)
    want = boundary.ader_step(U, dx, dt, order, form, solver, bc=bc)
    s = ader.Solver(shape, order=order, form=form, solver=solver)
    s.set_boundary(bc)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    assert rel_l1(to_host(d), want) <= 1e-12
    s.close()


@pytest.mark.parametrize("order,tiled", list(itertools.product((2, 3, 4), (True, False))))
def test_boundary_step_parity_fp32(ader, order, tiled):
    shape = (5, 8, 40)
    U = inputs.random_smooth(shape, seed=70 + order, amp=0.3)
    dx = _dx(shape)
    dt = 0.7 * scheme.max_dt(U, dx, 0.4)
    bc = (R, O, O, R, 0, 0)
    want = boundary.ader_step(U, dx, dt, order, "nodal", "hll", bc=bc)
    s = ader.Solver(shape, order=order, form="nodal", solver="hll", fp32=True)
    s.set_tiled(tiled)
    s.set_boundary(bc)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    assert rel_l1(to_host(d), want) <= 1e-6
    s.close()


def test_sod_in_a_closed_box_each_step(ader):
    """A Sod tube between reflecting walls in x (outflow in y, periodic z): three steps, each against the
    oracle from the same input, and mass and energy kept to round-off (modal walls see mirror images)."""
    import torch
    shape = (4, 6, 24)
    x = (np.arange(24) + 0.5) / 24
    rho = np.where(x < 0.5, 1.0, 0.125)[None, None, :] * np.ones(shape)
    p = np.where(x < 0.5, 1.0, 0.1)[None, None, :] * np.ones(shape)
    U = np.stack([rho, 0 * rho, 0 * rho, 0 * rho, p / 0.4])
    dx = _dx(shape)
    bc = (R, R, O, O, 0, 0)
    s = ader.Solver(shape, order=3, form="modal", solver="hll")
    s.set_boundary(bc)
    d = to_dev(U)
    tot = torch.zeros(5, dtype=torch.float64, device="cuda")
    ader.ader_diagnostics(s.h, d, None, tot)
    t0 = tot.cpu().numpy().copy()
    for _ in range(3):
        Uk = to_host(d)
        dt = boundary.max_dt(Uk, dx, 0.4)
        want = boundary.ader_step(Uk, dx, dt, 3, "modal", "hll", bc=bc)
        s.step(d, dt)
        assert s.status() == 0
        assert rel_l1(to_host(d), want) <= 1e-12
    ader.ader_diagnostics(s.h, d, None, tot)
    t1 = tot.cpu().numpy()
    for v in (0, 4):
        assert abs(t1[v] - t0[v]) <= 1e-13 * abs(t0[v])
    s.close()


def test_boundary_with_source_converged_predictor_and_host_path(ader):
    shape = (5, 6, 10)
    U = inputs.random_smooth(shape, seed=80, amp=0.3)
    dx = _dx(shape)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    bc = (O, O, R, R, R, R)
    want = boundary.ader_step(U, dx, dt, 3, "nodal", "hll", bc=bc, source=("gravity", (0.0, 0.0, -1.0)))
    s = ader.Solver(shape, order=3, form="nodal")
    s.set_source("gravity", (0.0, 0.0, -1.0))
    s.set_boundary(bc)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    assert rel_l1(to_host(d), want) <= 1e-12
    s.close()
    # the host-memory path takes the same boundaries
    s = ader.Solver(shape, order=3, form="nodal")
    s.set_boundary(bc)
    host = U.copy()
    dt_used = ader.ader_step_host(s.h, host, None, 0.4)
    assert dt_used == pytest.approx(boundary.max_dt(U, dx, 0.4), rel=1e-14)
    assert rel_l1(host, boundary.ader_step(U, dx, dt_used, 3, "nodal", "hll", bc=bc)) <= 1e-12
    s.close()


def test_boundary_refusals(ader):
    shape = (6, 6, 6)
    s = ader.Solver(shape, order=3)
    with pytest.raises(_lib.AderError):
        s.set_boundary((R, 0, 0, 0, 0, 0))            # periodic on one face only
    with pytest.raises(_lib.AderError):
        s.set_boundary((7, 7, 0, 0, 0, 0))            # unknown code
    s.close()
    s = ader.Solver((6, 6, 2), order=3)
    with pytest.raises(_lib.AderError):
        s.set_boundary((R, R, 0, 0, 0, 0))            # two zones along a reflecting axis: fewer than the ghosts
    s.close()
    s = ader.Solver(shape, order=3)
    s.set_boundary((O,) * 6)
    with pytest.raises(_lib.AderError):
        s.rk_step(to_dev(inputs.random_smooth(shape, seed=1, amp=0.1)), 1e-3)
    s.set_boundary((0,) * 6)                           # back to periodic: SSP-RK runs again
    s.rk_step(to_dev(inputs.random_smooth(shape, seed=1, amp=0.1)), 1e-3)
    assert s.status() == 0
    s.close()
    s = ader.Solver(shape, order=3, mhd=True)
    with pytest.raises(_lib.AderError):
        s.set_boundary((O,) * 6)
    s.close()
