"""GPU: design-order convergence of the FP64 step on the config-1 density wave at sizes the CPU oracle cannot
reach in the test budget (the 3-D analogue of the paper's Table IV: orders 2-4, L1 error of rho)."""
import numpy as np
import pytest

from gpu_util import ensure_built, to_dev, to_host
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


def _l1_error(ader, n, order, form, T=0.05):
    import torch
    s = ader.Solver((n, n, n), order=order, form=form)
    d = to_dev(inputs.density_wave(n))
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = 0.0
    while t < T - 1e-14:
        s.max_dt(d, 0.4, dtv)
        dt = min(float(dtv.item()), T - t)
        s.step(d, dt)
        t += dt
    assert s.status() == 0
    s.close()
    return np.abs(to_host(d)[0] - inputs.density_wave(n, t=T)[0]).mean()


@pytest.mark.parametrize("order,form", [(2, "nodal"), (3, "nodal"), (3, "modal"), (4, "nodal"), (4, "modal")])
def test_density_wave_design_order(ader, order, form):
    e1, e2 = _l1_error(ader, 32, order, form), _l1_error(ader, 64, order, form)
    rate = np.log2(e1 / e2)
    print("order %d %s: L1 %.3e (32^3) %.3e (64^3), rate %.2f" % (order, form, e1, e2, rate))
    assert rate >= order - 0.2
