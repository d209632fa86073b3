"""The transonic EMF option (ADER_EMF_TRANSONIC: twice the dissipative term of Eq. 17 in the electric
fields at transonic faces, Secs. II.3 and V) on the GPU against the oracle, whose option is pinned in
tests/test_oracle_emf_transonic.py."""
import itertools

import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import scheme
from paper_1006_2146_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


@pytest.mark.parametrize("order,solver", list(itertools.product((2, 3, 4), ("hll", "linearized"))))
def test_emf_transonic_parity_fp64(ader, order, solver):
    n = 10
    U, B = inputs.random_magnetised(n, seed=512, amp=0.8, b_amp=1.0, B0=2.0, P0=0.2)
    dx = (1.0 / n,) * 3
    G = 5.0 / 3.0
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    wU, wB = scheme.ader_step(U, dx, dt, order, "modal", solver, G, Bface=B, emf_transonic=True)
    pU, pB = scheme.ader_step(U, dx, dt, order, "modal", solver, G, Bface=B)
    s = ader.Solver((n, n, n), order=order, form="modal", solver=solver, gamma=G, mhd=True, emf_transonic=True)
    dU, dB = to_dev(U), to_dev(B)
    s.step(dU, dt, Bface=dB)
    assert s.status() == 0
    s.close()
    gU, gB = to_host(dU), to_host(dB)
    assert rel_l1(gU, wU) <= 1e-12
    assert rel_l1(gB, wB) <= 1e-12
    assert rel_l1(wB, pB) > 1e-9            # the option did something on this state
    assert np.abs(scheme.div_b(gB, dx) - scheme.div_b(B, dx)).max() <= 1e-12 * np.abs(B).max() / dx[0]


def test_emf_transonic_fp32(ader):
    n = 12
    U, B = inputs.random_magnetised(n, seed=514, amp=0.8, b_amp=1.0, B0=2.0, P0=0.2)
    dx = (1.0 / n,) * 3
    G = 5.0 / 3.0
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    wU, wB = scheme.ader_step(U, dx, dt, 3, "nodal", "hll", G, Bface=B, emf_transonic=True)
    s = ader.Solver((n, n, n), order=3, form="nodal", gamma=G, mhd=True, fp32=True, emf_transonic=True)
    dU, dB = to_dev(U), to_dev(B)
    s.step(dU, dt, Bface=dB)
    assert s.status() == 0
    s.close()
    assert rel_l1(to_host(dU), wU) <= 1e-5
    assert rel_l1(to_host(dB), wB) <= 1e-5
