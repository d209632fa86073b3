"""GPU parity of the non-stiff source terms (orders 2-4, modal and nodal) against the oracle.

The oracle's source terms are pinned in tests/test_oracle_source.py (the printed coefficients of Eqs. 30,
36, A.4, B.2-B.3, the S-bar rules and design-order convergence to an exact gravity-accelerated wave).
"""
import itertools

import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import scheme
from paper_1006_2146_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

GRAV = ("gravity", (0.8, -0.5, 0.3))
LIN = ("linear", 2.0)


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


def _solver(ader, shape, order, form, src, solver="hll", fp32=False):
    s = ader.Solver(shape, order=order, form=form, solver=solver, fp32=fp32)
    s.set_source(src[0], src[1] if src[0] == "gravity" else (src[1],))
    return s


@pytest.mark.parametrize("order,form,src", list(itertools.product((2, 3, 4), ("modal", "nodal"), (GRAV, LIN))))
def test_source_step_parity_fp64_ragged(ader, order, form, src):
    shape = (9, 10, 11)
    U = inputs.random_smooth(shape, seed=200 + order, amp=0.3)
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, order, form, "hll", source=src)
    s = _solver(ader, shape, order, form, src)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    got = to_host(d)
    s.close()
    assert rel_l1(got, want) <= 1e-12
    # the source did something measurable
    assert rel_l1(want, scheme.ader_step(U, dx, dt, order, form, "hll")) > 1e-6


def test_source_with_linearized_solver_and_converged_predictor(ader):
    shape = (8, 9, 10)
    U = inputs.random_smooth(shape, seed=210, amp=0.3)
    dx = _dx(shape)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4)
    want, iters = scheme.ader_step(U, dx, dt, 3, "nodal", "linearized", source=GRAV, tol=1e-13, return_iters=True)
    s = _solver(ader, shape, 3, "nodal", GRAV, solver="linearized")
    s.set_predictor(1e-13, 50)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    total, largest, capped = s.predictor_stats()
    got = to_host(d)
    s.close()
    assert rel_l1(got, want) <= 1e-12
    assert capped == 0 and abs(largest - int(iters.max())) <= 1


def test_source_fp32_bulk_ten_steps(ader):
    """FP32 bulk with gravity: within 1e-5 relative L1 of the FP64 oracle after 10 steps."""
    shape = (16, 16, 16)
    dx = _dx(shape)
    U = inputs.random_smooth(shape, seed=220, amp=0.3)
    s = _solver(ader, shape, 3, "nodal", GRAV, fp32=True)
    d = to_dev(U)
    Uo = U.copy()
    for _ in range(10):
        dt = scheme.max_dt(Uo, dx, 0.4)
        Uo = scheme.ader_step(Uo, dx, dt, 3, "nodal", "hll", source=GRAV)
        s.step(d, dt)
    assert s.status() == 0
    got = to_host(d)
    s.close()
    assert rel_l1(got, Uo) <= 1e-5


@pytest.mark.parametrize("order", [2, 3])
def test_mhd_gravity_parity_and_div_b(ader, order):
    n = 10
    U, B = inputs.random_magnetised(n, seed=230, amp=0.2, b_amp=0.4)
    dx = (1.0 / n,) * 3
    G = 5.0 / 3.0
    dt = 0.5 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    wU, wB = scheme.ader_step(U, dx, dt, order, "modal", "hll", G, Bface=B, source=GRAV)
    s = ader.Solver((n, n, n), order=order, form="modal", gamma=G, mhd=True)
    s.set_source("gravity", GRAV[1])
    dU, dB = to_dev(U), to_dev(B)
    s.step(dU, dt, Bface=dB)
    assert s.status() == 0
    gU, gB = to_host(dU), to_host(dB)
    s.close()
    assert rel_l1(gU, wU) <= 1e-12
    assert rel_l1(gB, wB) <= 1e-12
    d0 = scheme.div_b(B, dx)
    assert np.abs(scheme.div_b(gB, dx) - d0).max() <= 1e-12 * np.abs(B).max() / dx[0]


def test_source_api_rules(ader):
    import torch
    shape = (6, 6, 6)
    U = inputs.random_smooth(shape, seed=240, amp=0.2)
    dx = _dx(shape)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    # removing the source gives the plain step bit for bit
    s = ader.Solver(shape, order=3, form="nodal")
    a = to_dev(U)
    s.step(a, dt)
    s.set_source("gravity", GRAV[1])
    s.set_source(None)
    b = to_dev(U)
    s.step(b, dt)
    assert torch.equal(a, b)
    # SSP-RK refuses a source; unknown kinds and non-finite parameters are argument errors
    s.set_source("linear", (1.0,))
    with pytest.raises(_lib.AderError) as e:
        s.rk_step(to_dev(U), dt)
    assert e.value.code == _lib.ADER_ERR_ARG
    with pytest.raises(_lib.AderError) as e:
        _lib.ader_set_source(s.h, 7, (1.0,))
    assert e.value.code == _lib.ADER_ERR_ARG
    with pytest.raises(_lib.AderError) as e:
        _lib.ader_set_source(s.h, _lib.ADER_SOURCE_GRAVITY, (1.0, float("nan"), 0.0))
    assert e.value.code == _lib.ADER_ERR_ARG
    with pytest.raises(_lib.AderError) as e:
        _lib.ader_set_source(s.h, _lib.ADER_SOURCE_LINEAR, None)
    assert e.value.code == _lib.ADER_ERR_ARG
    s.close()
