"""Dense output inside a step (Sec. VII) on the GPU against the oracle (oracle/dense.py).

A step with ader_set_dense_output keeps every zone's space-time modes; ader_dense_output evaluates the
polynomial at t^n + tau dt.  The oracle's evaluation is pinned in tests/test_oracle_dense.py.
"""
import itertools

import numpy as np
import pytest

from gpu_util import ensure_built, to_dev, to_host
from oracle import dense, scheme
from paper_1006_2146_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

LS = {2: 4, 3: 10, 4: 20}


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _dense(ader, s, U, dt, order, taus, nv=5, Bface=None):
    import torch
    d = to_dev(U)
    dB = None if Bface is None else to_dev(Bface)
    s.set_dense_output(True)
    s.step(d, dt, Bface=dB)
    out = []
    for tau in taus:
        o = torch.empty((LS[order], nv) + tuple(U.shape[1:]), dtype=torch.float64, device="cuda")
        s.dense_output(tau, o)
        out.append(to_host(o))
    assert s.status() == 0
    return out, to_host(d)


@pytest.mark.parametrize("order,form", list(itertools.product((2, 3, 4), ("modal", "nodal"))))
def test_dense_output_parity_fp64(ader, order, form):
    shape = (9, 10, 11)
    U = inputs.random_smooth(shape, seed=300 + order, amp=0.3)
    dx = (1 / 11, 1 / 10, 1 / 9)
    dt = 0.7 * scheme.max_dt(U, dx, 0.4)
    taus = (0.0, 0.37, 1.0)
    s = ader.Solver(shape, order=order, form=form)
    got, _ = _dense(ader, s, U, dt, order, taus)
    s.close()
    for g, tau in zip(got, taus):
        want = dense.dense_output(U, dx, dt, order, form, tau)
        assert np.abs(g - want).max() <= 1e-12 * np.abs(want[0]).max()


def test_dense_output_mhd_and_source(ader):
    n = 10
    U, B = inputs.random_magnetised(n, seed=310, amp=0.2, b_amp=0.4)
    dx = (1.0 / n,) * 3
    G = 5.0 / 3.0
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    s = ader.Solver((n, n, n), order=3, form="modal", gamma=G, mhd=True)
    s.set_source("gravity", (0.8, -0.5, 0.3))
    got, _ = _dense(ader, s, U, dt, 3, (0.5,), nv=8, Bface=B)
    s.close()
    want = dense.dense_output(U, dx, dt, 3, "modal", 0.5, gamma=G, Bface=B, source=("gravity", (0.8, -0.5, 0.3)))
    assert np.abs(got[0] - want).max() <= 1e-12 * np.abs(want[0]).max()


def test_dense_output_fp32(ader):
    shape = (16, 16, 16)
    U = inputs.random_smooth(shape, seed=320, amp=0.3)
    dx = (1 / 16,) * 3
    dt = 0.7 * scheme.max_dt(U, dx, 0.4)
    s = ader.Solver(shape, order=3, form="nodal", fp32=True)
    got, _ = _dense(ader, s, U, dt, 3, (0.6,))
    s.close()
    want = dense.dense_output(U, dx, dt, 3, "nodal", 0.6)
    assert np.abs(got[0] - want).max() <= 1e-5 * np.abs(want[0]).max()


def test_dense_output_leaves_the_step_unchanged_and_checks_arguments(ader):
    import torch
    shape = (8, 8, 8)
    U = inputs.random_smooth(shape, seed=330, amp=0.2)
    dt = 0.5 * scheme.max_dt(U, (1 / 8,) * 3, 0.4)
    s = ader.Solver(shape, order=4, form="nodal")
    a = to_dev(U)
    s.step(a, dt)
    o = torch.empty((20, 5) + shape, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.AderError) as e:          # nothing kept yet
        s.dense_output(0.5, o)
    assert e.value.code == _lib.ADER_ERR_ARG
    _, b = _dense(ader, s, U, dt, 4, ())
    assert np.array_equal(to_host(a), b)
    with pytest.raises(_lib.AderError) as e:
        s.dense_output(1.5, o)
    assert e.value.code == _lib.ADER_ERR_ARG
    s.set_dense_output(False)
    with pytest.raises(_lib.AderError):
        s.dense_output(0.5, o)
    s.close()
