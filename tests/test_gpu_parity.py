"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the same seeded inputs.

Bars: FP64 <= 1e-12 relative L1 per step; FP32 bulk <= 1e-5 relative L1 after
10 steps (config 1); dt and totals to FP64 round-off.
"""
import itertools

import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import scheme
from paper_1006_2146_gb300 import inputs

pytestmark = pytest.mark.gpu

FORMS = ("modal", "nodal")
SOLVERS = ("hll", "linearized")


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


def _gpu_step(ader, U, shape, dt, order, form, solver, fp32=False):
    s = ader.Solver(shape, order=order, form=form, solver=solver, fp32=fp32)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    out = to_host(d)
    s.close()
    return out


@pytest.mark.parametrize("order,form,solver", list(itertools.product((2, 3, 4), FORMS, SOLVERS)))
def test_step_parity_fp64_ragged(ader, order, form, solver):
    """One step on a ragged 11x10x9 grid (several 128-zone blocks plus a tail), smooth random data."""
    shape = (9, 10, 11)
    U = inputs.random_smooth(shape, seed=100 + order, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, order, form, solver)
    got = _gpu_step(ader, U, shape, dt, order, form, solver)
    assert rel_l1(got, want) <= 1e-12


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("solver", SOLVERS)
def test_step_parity_fp64_sod_each_step(ader, order, solver):
    """Discontinuous data (Sod tube along (1,1,0)): three steps, parity checked from the same input each step."""
    shape = (4, 16, 16)
    U = inputs.sod_planar(shape)
    dx = _dx(shape)
    s = ader.Solver(shape, order=order, form="modal", solver=solver)
    d = to_dev(U)
    for _ in range(3):
        Uk = to_host(d)
        dt = scheme.max_dt(Uk, dx, 0.4)
        want = scheme.ader_step(Uk, dx, dt, order, "modal", solver)
        s.step(d, dt)
        assert rel_l1(to_host(d), want) <= 1e-12
    assert s.status() == 0


@pytest.mark.parametrize("shape", [(1, 12, 10), (10, 1, 1), (3, 5, 64)])
def test_degenerate_and_thin_grids(ader, shape):
    U = inputs.random_smooth(shape, seed=7, amp=0.2)
    dx = _dx(shape)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, 3, "nodal", "hll")
    assert rel_l1(_gpu_step(ader, U, shape, dt, 3, "nodal", "hll"), want) <= 1e-12


def test_config1_fp64_ten_steps(ader):
    """Config 1: 32^3 density wave, third-order nodal, HLL, CFL 0.4, 10 steps (same dt on both sides)."""
    n = 32
    U = inputs.density_wave(n)
    dx = (1.0 / n,) * 3
    s = ader.Solver((n, n, n), order=3, form="nodal", solver="hll")
    d = to_dev(U)
    Uo = U.copy()
    for _ in range(10):
        dt = scheme.max_dt(Uo, dx, 0.4)
        Uo = scheme.ader_step(Uo, dx, dt, 3, "nodal", "hll")
        s.step(d, dt)
    assert rel_l1(to_host(d), Uo) <= 1e-11


def test_config1_fp32_bulk_ten_steps(ader):
    """FP32 reconstruction/predictor/fluxes with FP64 update: <= 1e-5 relative L1 after 10 steps."""
    n = 32
    U = inputs.density_wave(n)
    dx = (1.0 / n,) * 3
    s = ader.Solver((n, n, n), order=3, form="nodal", solver="hll", fp32=True)
    d = to_dev(U)
    Uo = U.copy()
    for _ in range(10):
        dt = scheme.max_dt(Uo, dx, 0.4)
        Uo = scheme.ader_step(Uo, dx, dt, 3, "nodal", "hll")
        s.step(d, dt)
    err = rel_l1(to_host(d), Uo)
    assert err <= 1e-5
    print("fp32 bulk relative L1 after 10 steps:", err)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_fp32_bulk_all_orders_one_step(ader, order):
    shape = (8, 9, 10)
    U = inputs.random_smooth(shape, seed=3, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, order, "modal", "linearized")
    assert rel_l1(_gpu_step(ader, U, shape, dt, order, "modal", "linearized", fp32=True), want) <= 1e-6


@pytest.mark.parametrize("form", FORMS)
def test_fp32_tiled_cross_moments(ader, form):
    """FP32, third order, on a grid whose x and y sizes take the shared-memory tiles of the cross moments
    (x a multiple of 32, y of 8; z not a multiple of the 32-plane chunks): one step within the FP32 bar of
    the oracle."""
    shape = (10, 16, 64)
    U = inputs.random_smooth(shape, seed=21, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, 3, form, "hll")
    got = _gpu_step(ader, U, shape, dt, 3, form, "hll", fp32=True)
    assert rel_l1(got, want) <= 1e-6


def test_max_dt_parity(ader):
    import torch
    shape = (7, 9, 12)
    U = inputs.random_smooth(shape, seed=5, amp=0.4)
    dx = _dx(shape)
    s = ader.Solver(shape, order=3)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.max_dt(to_dev(U), 0.4, dt)
    torch.cuda.synchronize()
    assert float(dt.item()) == pytest.approx(scheme.max_dt(U, dx, 0.4), rel=1e-14)
    # the scratch resets itself: a second call gives the same value
    s.max_dt(to_dev(U), 0.4, dt)
    assert float(dt.item()) == pytest.approx(scheme.max_dt(U, dx, 0.4), rel=1e-14)


def test_conservation_on_gpu(ader):
    import torch
    shape = (16, 16, 16)
    U = inputs.sod_planar(shape)
    dx = _dx(shape)
    s = ader.Solver(shape, order=4, form="nodal", solver="linearized")
    d = to_dev(U)
    tot = torch.zeros(5, dtype=torch.float64, device="cuda")
    ader.ader_diagnostics(s.h, d, None, tot)
    t0 = tot.cpu().numpy().copy()
    np.testing.assert_allclose(t0, U.reshape(5, -1).sum(axis=1), rtol=1e-13)
    for _ in range(3):
        s.step(d, scheme.max_dt(to_host(d), dx, 0.4))
    ader.ader_diagnostics(s.h, d, None, tot)
    t1 = tot.cpu().numpy()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(U).reshape(5, -1).sum(axis=1).max())


@pytest.mark.parametrize("order", [2, 3, 4])
def test_rk_step_parity(ader, order):
    """SSP-RK (Eqs. 18-20) on the same GPU against the oracle's RK step."""
    shape = (8, 8, 10)
    U = inputs.random_smooth(shape, seed=9, amp=0.3)
    dx = _dx(shape)
    dt = 0.3 * scheme.max_dt(U, dx, 0.4)
    want = scheme.rk_step(U, dx, dt, order, "hll")
    s = ader.Solver(shape, order=order, solver="hll")
    d = to_dev(U)
    s.rk_step(d, dt)
    assert rel_l1(to_host(d), want) <= 1e-12


def test_host_path_equals_device_path(ader):
    import torch
    shape = (12, 12, 12)
    U = inputs.random_smooth(shape, seed=2, amp=0.3)
    s = ader.Solver(shape, order=3, form="nodal")
    host = U.copy()
    dt_used = ader.ader_step_host(s.h, host, None, 0.4)
    d = to_dev(U)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.max_dt(d, 0.4, dt)
    s.step_devdt(d, dt)
    assert dt_used == float(dt.item())
    assert np.array_equal(host, to_host(d))


def test_unphysical_state_is_reported(ader):
    import torch
    shape = (6, 6, 6)
    U = inputs.density_wave(6)
    U[0, 2, 3, 1] = -1.0
    s = ader.Solver(shape, order=2)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.max_dt(to_dev(U), 0.4, dt)
    assert s.status() == ader.AderError(-3, "").code
    assert s.status() == 0          # the flag is cleared by the read


def _patch(U, k, j, i, r):
    idx = [np.arange(c - r, c + r + 1) % n for c, n in zip((k, j, i), U.shape[1:])]
    return U[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]


@pytest.mark.parametrize("fp32", [False, True])
def test_full_size_sampled_parity(ader, fp32):
    """The bench workload (256^3 Sod tube, third-order nodal HLL, dt from ader_max_dt): sampled zones
    against the oracle evaluated on an 11^3 periodic patch around each sample (the update of a zone
    depends on zones at most 4 away)."""
    import torch
    n = 256
    U = inputs.sod_planar(n)
    s = ader.Solver((n, n, n), order=3, form="nodal", solver="hll", fp32=fp32)
    d = to_dev(U)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.max_dt(d, 0.4, dt)
    s.step_devdt(d, dt)
    got = to_host(d)
    dtv = float(dt.item())
    # FP32-bulk contexts compute the per-zone signal speeds in FP32 (reduction in FP64)
    assert dtv == pytest.approx(scheme.max_dt(U, (1.0 / n,) * 3, 0.4), rel=1e-6 if fp32 else 1e-14)
    rng = np.random.default_rng(42)
    samples = [(0, 0, 0), (255, 255, 255), (128, 64, 63)] + [tuple(rng.integers(0, n, 3)) for _ in range(9)]
    # include zones on the shock planes x + y = 1/2 and 1
    samples += [(10, 100, 27), (200, 3, 252)]
    tol = 1e-5 if fp32 else 1e-12
    for (k, j, i) in samples:
        P = _patch(U, k, j, i, 5)
        want = scheme.ader_step(P, (1.0 / n,) * 3, dtv, 3, "nodal", "hll")[:, 5, 5, 5]
        assert np.all(np.abs(got[:, k, j, i] - want) <= tol * np.abs(U[:, k, j, i]).max()), (k, j, i)
