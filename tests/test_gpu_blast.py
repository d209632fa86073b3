"""Centred 3-D blasts (Secs. VIII.3 and IX.4) on the GPU: symmetry and robustness.

The paper finds the modal schemes keep the oppositely directed velocities of a centred blast equal to
round-off, and the nodal ones off by small amounts (0.0002-0.14 % at its sizes) because their node sets
are not symmetric.  Here, on small grids over a few dozen steps: modal stays point-symmetric to
round-off at every order, Euler and MHD; nodal departs from it by a small, non-zero amount; the low-beta
MHD blast (beta 0.00628 outside) keeps positive density and pressure and its field divergence-free.
"""
import numpy as np
import pytest

from gpu_util import ensure_built, to_dev, to_host
from paper_1006_2146_gb300 import inputs, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _asym(U):
    v = U[1:4] / U[0]
    return np.abs(v + v[:, ::-1, ::-1, ::-1]).max() / np.abs(v).max()


def _peak_asym(U):
    v = U[1:4] / U[0]
    return max(abs(v[d].max() - (-v[d]).max()) / np.abs(v[d]).max() for d in range(3))


def _run(ader, n, order, form, mhd, steps, solver="hll"):
    U, B = inputs.mhd_blast(n) if mhd else (inputs.blast(n), None)
    s = ader.Solver((n, n, n), order=order, form=form, solver=solver, gamma=1.4, mhd=mhd)
    dU = to_dev(U)
    dB = None if B is None else to_dev(B)
    run.advance(s, dU, 1.0, cfl=0.3, Bface=dB, max_steps=steps)
    s.close()
    return to_host(dU), (None if B is None else to_host(dB))


@pytest.mark.parametrize("order", [2, 3, 4])
def test_modal_hydro_blast_point_symmetric(ader, order):
    U, _ = _run(ader, 24, order, "modal", False, 30)
    assert _asym(U) <= 1e-11
    assert np.abs(U[1]).max() > 1.0


@pytest.mark.parametrize("order", [2, 3])
def test_modal_mhd_blast_point_symmetric_and_robust(ader, order):
    n = 25
    U, B = _run(ader, n, order, "modal", True, 30)
    assert _asym(U) <= 1e-11
    Bz = np.stack([0.5 * (B[d] + np.roll(B[d], -1, axis=2 - d)) for d in range(3)])
    P = 0.4 * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0] - (Bz ** 2).sum(axis=0) / (8 * np.pi))
    assert U[0].min() > 0 and P.min() > 0
    h = 1.0 / n
    div = sum((np.roll(B[d], -1, axis=2 - d) - B[d]) / h for d in range(3))
    assert np.abs(div).max() <= 1e-12 * np.abs(B).max() / h


@pytest.mark.parametrize("order", [2, 3, 4])
def test_nodal_blast_asymmetry_small_but_present(ader, order):
    U, _ = _run(ader, 24, order, "nodal", False, 30)
    print("nodal order %d: pointwise %.3e peak %.3e" % (order, _asym(U), _peak_asym(U)))
    assert _asym(U) > 1e-13
    assert _peak_asym(U) < 2e-2
