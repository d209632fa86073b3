"""The 2-D vortex problems of Secs. VI.1-VI.2 as one-zone z-slabs on the GPU.

* one-step parity with the oracle on slabs whose x-y extent is a multiple of the shared-memory tiles;
* the errors after one period of the mean flow against the paper's Tables I (density, isentropic vortex)
  and II (x-magnetic field, magnetised vortex), typed in tests/golden/vortex_tables.json: at 64^2 and
  128^2 no more than twice the printed value and not below a fifth of it, and close to the design order
  between them.  The paper's scheme differs from this one where it is silent (WENO weights, the HLLE
  speed estimate, the time-step rule), so the numbers are not expected to agree to more than that; on
  GB300 this path's errors are 0.3-1.3 times the printed ones (lower at third and fourth order).
"""
import itertools
import json
import os

import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import scheme
from paper_1006_2146_gb300 import inputs, run

pytestmark = pytest.mark.gpu

with open(os.path.join(os.path.dirname(__file__), "golden", "vortex_tables.json")) as _fh:
    TABLES = json.load(_fh)


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _problem(kind, order, n):
    """(U, Bface or None, gamma, L): the paper doubles the domain (and the end time) at fourth order."""
    L = 20.0 if order == 4 else 10.0
    if kind == "hydro":
        return inputs.isentropic_vortex(n, L=L), None, 1.4, L
    U, B = inputs.magnetized_vortex(n, L=L)
    return U, B, 5.0 / 3.0, L


def _solver(ader, kind, order, n, gamma, L):
    return ader.Solver((1, n, n), order=order, form="modal", solver="hll", gamma=gamma,
                       lengths=inputs.slab_lengths(L), mhd=(kind == "mhd"))


@pytest.mark.parametrize("kind,order", [("hydro", 2), ("hydro", 3), ("hydro", 4), ("mhd", 3)])
def test_vortex_slab_step_parity(ader, kind, order):
    n = 64 if kind == "hydro" else 32
    U, B, G, L = _problem(kind, order, n)
    dx = (L / n, L / n, inputs.slab_lengths(L)[2])
    dt = 0.9 * scheme.max_dt(U, dx, 0.45, G, Bface=B)
    want = scheme.ader_step(U, dx, dt, order, "modal", "hll", G, Bface=B)
    s = _solver(ader, kind, order, n, G, L)
    dU = to_dev(U)
    dB = None if B is None else to_dev(B)
    s.step(dU, dt, Bface=dB)
    assert s.status() == 0
    s.close()
    if B is None:
        assert rel_l1(to_host(dU), want) <= 1e-12
    else:
        assert rel_l1(to_host(dU), want[0]) <= 1e-12
        assert rel_l1(to_host(dB), want[1]) <= 1e-12
        h = L / n
        gB = to_host(dB)
        div = (np.roll(gB[0], -1, axis=2) - gB[0]) / h + (np.roll(gB[1], -1, axis=1) - gB[1]) / h
        assert np.abs(div).max() <= 1e-12 * np.abs(gB).max() / h


def vortex_error(ader, kind, order, n):
    """(L1, Linf) per zone after one period: density (hydro) or the x-face field (MHD)."""
    U, B, G, L = _problem(kind, order, n)
    s = _solver(ader, kind, order, n, G, L)
    dU = to_dev(U)
    dB = None if B is None else to_dev(B)
    t, _ = run.advance(s, dU, L, cfl=0.45, Bface=dB)
    s.close()
    assert abs(t - L) <= 1e-12 * L
    err = to_host(dU)[0] - U[0] if B is None else to_host(dB)[0] - B[0]
    return float(np.abs(err).mean()), float(np.abs(err).max())


@pytest.mark.parametrize("kind,order", list(itertools.product(("hydro", "mhd"), (2, 3, 4))))
def test_vortex_errors_against_paper_tables(ader, kind, order):
    table = TABLES["table_i" if kind == "hydro" else "table_ii"]["order%d" % order]
    errs = [vortex_error(ader, kind, order, n) for n in (64, 128)]
    for (l1, _), paper in zip(errs, table["l1"][:2]):
        assert 0.2 * paper <= l1 <= 2.0 * paper, (errs, table["l1"][:2])
    rate = np.log2(errs[0][0] / errs[1][0])
    assert rate >= order - 0.5, (rate, errs)
