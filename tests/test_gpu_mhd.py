"""GPU parity of the ideal-MHD path (face-B WENO, edge EMFs, constrained transport) against the oracle."""
import itertools

import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import scheme
from paper_1006_2146_gb300 import inputs

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _mhd_solver(ader, shape, order, form, fp32=False, solver="hll"):
    nz, ny, nx = shape
    h = ader.ader_create(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nz, order, G,
                         ader.ADER_LINEARIZED if solver == "linearized" else ader.ADER_HLL,
                         ader.ADER_MHD | (ader.ADER_NODAL if form == "nodal" else 0) | (ader.ADER_FP32_BULK if fp32 else 0))
    return h


def _perturbed_alfven(n, seed=1):
    U, B = inputs.alfven_wave(n, amp=0.3)
    rng = np.random.default_rng(seed)
    U = U * (1.0 + 0.02 * rng.normal(size=U.shape))
    U[4] += 0.3
    return U, B


def _divb_rel(B, dx):
    return np.abs(scheme.div_b(B, dx)).max() / (np.abs(B).max() / dx[0])


@pytest.mark.parametrize("order,form,solver",
                         list(itertools.product((2, 3, 4), ("modal", "nodal"), ("hll", "linearized"))))
def test_mhd_step_parity_fp64(ader, order, form, solver):
    n = 10
    U, B = _perturbed_alfven(n)
    dx = (1.0 / n,) * 3
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    Uo, Bo = scheme.ader_step(U, dx, dt, order, form, solver, G, Bface=B)
    h = _mhd_solver(ader, (n, n, n), order, form, solver=solver)
    dU, dB = to_dev(U), to_dev(B)
    ader.ader_step(h, dU, dB, dt)
    assert ader.ader_sync_status(h) == 0
    assert rel_l1(to_host(dU), Uo) <= 1e-12
    assert rel_l1(to_host(dB), Bo) <= 1e-12
    d0 = scheme.div_b(B, dx)
    assert np.abs(scheme.div_b(to_host(dB), dx) - d0).max() <= 1e-12 * np.abs(B).max() / dx[0]
    ader.ader_destroy(h)


def test_mhd_max_dt_parity(ader):
    import torch
    n = 12
    U, B = _perturbed_alfven(n, seed=4)
    h = _mhd_solver(ader, (n, n, n), 3, "modal")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    ader.ader_max_dt(h, to_dev(U), to_dev(B), 0.4, dt)
    assert float(dt.item()) == pytest.approx(scheme.max_dt(U, (1.0 / n,) * 3, 0.4, G, Bface=B), rel=1e-14)
    ader.ader_destroy(h)


@pytest.mark.parametrize("solver,n", [("hll", 24), ("linearized", 16)])
def test_orszag_tang_fp32_ten_steps(ader, solver, n):
    """Config 3 (Orszag-Tang-type vortex, third order, FP32 bulk; the config names the linearized solver):
    <= 1e-5 relative L1 after 10 steps, div B at round-off of FP32 (<= 1e-6 relative)."""
    import torch
    U, B = inputs.orszag_tang(n)
    dx = (1.0 / n,) * 3
    h = _mhd_solver(ader, (n, n, n), 3, "modal", fp32=True, solver=solver)
    dU, dB = to_dev(U), to_dev(B)
    Uo, Bo = U.copy(), B.copy()
    for _ in range(10):
        dt = scheme.max_dt(Uo, dx, 0.4, G, Bface=Bo)
        Uo, Bo = scheme.ader_step(Uo, dx, dt, 3, "modal", solver, G, Bface=Bo)
        ader.ader_step(h, dU, dB, dt)
    assert ader.ader_sync_status(h) == 0
    assert rel_l1(to_host(dU), Uo) <= 1e-5
    assert rel_l1(to_host(dB), Bo) <= 1e-5
    assert _divb_rel(to_host(dB), dx) <= 1e-6
    ader.ader_destroy(h)


def test_mhd_rejects_mismatched_arguments(ader):
    n = 6
    h = _mhd_solver(ader, (n, n, n), 2, "modal")
    U, B = _perturbed_alfven(n)
    with pytest.raises(ader.AderError):
        ader.ader_step(h, to_dev(U), None, 1e-3)
    ader.ader_destroy(h)


def test_mhd_diagnostics_totals_and_div_b(ader):
    """Nine diagnostics: zone totals, face-B totals and the relative max |div B|, against numpy sums of the
    same arrays; after a CT step the face totals are unchanged (periodic telescoping of Eq. 8)."""
    import torch
    n = 12
    U, B = _perturbed_alfven(n, seed=6)
    dx = (1.0 / n,) * 3
    B = B.copy()
    B[0] += 1e-3 * np.random.default_rng(2).standard_normal(B[0].shape)      # a field with nonzero div B
    h = _mhd_solver(ader, (n, n, n), 3, "modal")
    dU, dB = to_dev(U), to_dev(B)
    out = torch.zeros(9, dtype=torch.float64, device="cuda")
    ader.ader_diagnostics(h, dU, dB, out)
    got = out.cpu().numpy()
    want_tot = np.concatenate([U.reshape(5, -1).sum(axis=1), B.reshape(3, -1).sum(axis=1)])
    scale = np.maximum(np.abs(want_tot), np.abs(U).reshape(5, -1).sum(axis=1).max())
    assert np.all(np.abs(got[:8] - want_tot) <= 1e-13 * scale)
    assert got[8] == pytest.approx(_divb_rel(B, dx), rel=1e-12)
    assert got[8] > 1e-4
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    ader.ader_step(h, dU, dB, dt)
    out2 = torch.zeros(9, dtype=torch.float64, device="cuda")
    ader.ader_diagnostics(h, dU, dB, out2)
    assert ader.ader_sync_status(h) == 0
    got2 = out2.cpu().numpy()
    assert np.all(np.abs(got2[:8] - got[:8]) <= 1e-13 * scale)
    ader.ader_destroy(h)


@pytest.mark.parametrize("order,solver", [(2, "hll"), (3, "hll"), (3, "linearized"), (4, "hll")])
def test_mhd_ssprk_step_parity_fp64(ader, order, solver):
    """SSP-RK of the same order and solver for MHD (Eqs. 18-20 with the CT-rate operator) against the oracle;
    div B unchanged to round-off."""
    n = 10
    U, B = _perturbed_alfven(n, seed=8)
    dx = (1.0 / n,) * 3
    dt = 0.3 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    Uo, Bo = scheme.rk_step(U, dx, dt, order, solver, G, Bface=B)
    h = _mhd_solver(ader, (n, n, n), order, "modal", solver=solver)
    dU, dB = to_dev(U), to_dev(B)
    ader.ader_rk_step(h, dU, dB, dt)
    assert ader.ader_sync_status(h) == 0
    assert rel_l1(to_host(dU), Uo) <= 1e-12
    assert rel_l1(to_host(dB), Bo) <= 1e-12
    d0 = scheme.div_b(B, dx)
    assert np.abs(scheme.div_b(to_host(dB), dx) - d0).max() <= 1e-12 * np.abs(B).max() / dx[0]
    ader.ader_destroy(h)
