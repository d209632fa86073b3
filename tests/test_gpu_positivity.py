"""The a-posteriori positivity fallback (ADER_POSITIVITY_FALLBACK, FP64, Euler and MHD) on the GPU against the
oracle's (scheme.positivity_fallback, pinned in tests/test_oracle_positivity.py)."""
import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import physics, scheme
from paper_1006_2146_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _double_rarefaction(n, v0=4.0, p0=0.4, gamma=1.4):
    x = (np.arange(n) + 0.5) / n
    vx = np.where(x < 0.5, -v0, v0)[None, None, :] * np.ones((1, 1, n))
    rho = np.ones((1, 1, n))
    z = np.zeros_like(rho)
    return np.stack([rho, rho * vx, z, z, p0 / (gamma - 1.0) * rho + 0.5 * rho * vx ** 2])


@pytest.mark.parametrize("order,form", [(3, "modal"), (4, "modal"), (4, "nodal")])
def test_fallback_parity_on_the_double_rarefaction(ader, order, form):
    n = 32
    dx = (1 / n, 1.0, 1.0)
    U = _double_rarefaction(n)
    s = ader.Solver((1, 1, n), order=order, form=form, lengths=(1.0, 1.0, 1.0), positivity=True)
    d = to_dev(U)
    triggered = False
    for _ in range(20):
        Uh = to_host(d)
        dt = scheme.max_dt(Uh, (1 / n, 1.0, 1.0), 0.3)
        want = scheme.ader_step(Uh, dx, dt, order, form, "hll", positivity=True)
        triggered |= not physics.physical(scheme.ader_step(Uh, dx, dt, order, form, "hll"), 1.4).all()
        s.step(d, dt)
        assert s.status() == 0
        assert rel_l1(to_host(d), want) <= 1e-12
    s.close()
    assert triggered


def test_fallback_changes_nothing_on_smooth_data_and_checks_flags(ader):
    import torch
    shape = (8, 9, 10)
    U = inputs.random_smooth(shape, seed=78, amp=0.3)
    dt = 0.5 * scheme.max_dt(U, (1 / 10, 1 / 9, 1 / 8), 0.4)
    a, b = to_dev(U), to_dev(U)
    s0 = ader.Solver(shape, order=4, form="modal")
    s1 = ader.Solver(shape, order=4, form="modal", positivity=True)
    s0.step(a, dt)
    s1.step(b, dt)
    assert s0.status() == 0 and s1.status() == 0
    assert torch.equal(a, b)
    s0.close()
    s1.close()
    with pytest.raises(_lib.AderError):
        ader.Solver(shape, order=3, positivity=True, fp32=True)


def test_mhd_fallback_parity(ader):
    """Magnetised double rarefaction (transverse field 5): per-step parity with the oracle's MHD fallback."""
    n = 32
    dx = (1 / n, 1.0, 1.0)
    U = _double_rarefaction(n)
    U[4] += 25.0 / (8.0 * np.pi)
    z = np.zeros((1, 1, n))
    B = np.stack([z, 5.0 + z, z])
    s = ader.Solver((1, 1, n), order=4, form="modal", positivity=True, mhd=True)
    dU, dB = to_dev(U), to_dev(B)
    for _ in range(12):
        Uh, Bh = to_host(dU), to_host(dB)
        dt = scheme.max_dt(Uh, dx, 0.3, 1.4, Bface=Bh)
        wU, wB = scheme.ader_step(Uh, dx, dt, 4, "modal", "hll", 1.4, Bface=Bh, positivity=True)
        s.step(dU, dt, Bface=dB)
        assert s.status() == 0
        assert rel_l1(to_host(dU), wU) <= 1e-12
        assert np.abs(to_host(dB) - wB).max() <= 1e-12 * np.abs(wB).max()
    s.close()


def _mhd_physical(U, B):
    zB = np.stack([0.5 * (B[d] + np.roll(B[d], -1, axis=2 - d)) for d in range(3)])
    return physics.physical(np.concatenate([U, zB]), 1.4)


def test_mhd_fallback_fires_on_the_magnetised_double_rarefaction(ader):
    """The MHD parity case above is one where the fallback acts: the oracle's plain fourth-order MHD step
    leaves a non-physical zone in one of its steps, and the GPU fallback step stays physical."""
    n = 32
    dx = (1 / n, 1.0, 1.0)
    U = _double_rarefaction(n)
    U[4] += 25.0 / (8.0 * np.pi)
    z = np.zeros((1, 1, n))
    B = np.stack([z, 5.0 + z, z])
    s = ader.Solver((1, 1, n), order=4, form="modal", positivity=True, mhd=True)
    dU, dB = to_dev(U), to_dev(B)
    failed_plain = False
    for _ in range(12):
        Uh, Bh = to_host(dU), to_host(dB)
        dt = scheme.max_dt(Uh, dx, 0.3, 1.4, Bface=Bh)
        pU, pB = scheme.ader_step(Uh, dx, dt, 4, "modal", "hll", 1.4, Bface=Bh)
        failed_plain |= not _mhd_physical(pU, pB).all()
        s.step(dU, dt, Bface=dB)
        assert s.status() == 0
        assert _mhd_physical(to_host(dU), to_host(dB)).all()
    s.close()
    assert failed_plain


@pytest.mark.parametrize("mhd", [False, True])
def test_fallback_step_reports_a_non_finite_zone(ader, mhd):
    """A NaN planted on the host in one zone of U cannot be mended (the first-order fluxes take U^n): the
    step ends with ADER_ERR_NONFINITE, for Euler and MHD, and the context stays usable."""
    shape = (6, 7, 8)
    U = inputs.random_smooth(shape, seed=31, amp=0.2)
    B = np.ones((3,) + shape) * 0.5 if mhd else None
    if mhd:
        U[4] += 3 * 0.25 / (8.0 * np.pi)
    dx = (1 / 8, 1 / 7, 1 / 6)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, 1.4, Bface=B) if mhd else 0.5 * scheme.max_dt(U, dx, 0.4)
    bad = U.copy()
    bad[0, 3, 3, 3] = np.nan
    s = ader.Solver(shape, order=3, form="modal", positivity=True, mhd=mhd)
    dU = to_dev(bad)
    dB = to_dev(B) if mhd else None
    s.step(dU, dt, Bface=dB)
    assert s.status() == _lib.ADER_ERR_NONFINITE
    # the context stays usable: a clean step afterwards reports nothing
    dU = to_dev(U)
    dB = to_dev(B) if mhd else None
    s.step(dU, dt, Bface=dB)
    assert s.status() == 0
    s.close()


def test_fallback_step_reports_a_non_finite_face_field(ader):
    """MHD: a NaN planted on the host in the face field is reported by the step (ADER_ERR_NONFINITE)."""
    shape = (6, 7, 8)
    U = inputs.random_smooth(shape, seed=32, amp=0.2)
    U[4] += 3 * 0.25 / (8.0 * np.pi)
    B = np.ones((3,) + shape) * 0.5
    dx = (1 / 8, 1 / 7, 1 / 6)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, 1.4, Bface=B)
    B[1, 2, 2, 2] = np.nan
    s = ader.Solver(shape, order=3, form="modal", positivity=True, mhd=True)
    dU, dB = to_dev(U), to_dev(B)
    s.step(dU, dt, Bface=dB)
    assert s.status() == _lib.ADER_ERR_NONFINITE
    s.close()

