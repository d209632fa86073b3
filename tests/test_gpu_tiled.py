"""The per-tile launch layout of the Euler step (orders 2 and 3) against the per-zone layout.

ader_set_tiled(1) (the default) runs the predictor and the face solves of a 32 x 4 tile of columns in
one block that marches through z, solving each face once; ader_set_tiled(0) writes every zone's face
data to memory and solves the faces in a second pass.  The arithmetic of each face and of Eq. 6 is the
same, so the two must agree bit for bit in FP64 (in FP32 to FP32 rounding: the two kernels may contract
multiply-adds differently), on grids with ragged tiles, thin directions, several z chunks, with a source,
the converged predictor and SSP-RK.  Parity of the default layout with the oracle is the business of the
other GPU tests.
"""
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


def _both(ader, shape, U, dt, setup=None, rk=False, **kw):
    out = []
    for tiled in (True, False):
        s = ader.Solver(shape, **kw)
        s.set_tiled(tiled)
        if setup:
            setup(s)
        d = to_dev(U)
        (s.rk_step if rk else s.step)(d, dt)
        assert s.status() == 0
        out.append(to_host(d))
        s.close()
    return out


SHAPES = [(37, 9, 70), (1, 3, 5), (5, 4, 33), (20, 8, 64)]


@pytest.mark.parametrize("order,form,solver,fp32", list(itertools.product((2, 3), ("modal", "nodal"),
                                                                             ("hll", "linearized"), (False, True))))
def test_tiled_equals_per_zone_layout(ader, order, form, solver, fp32):
    for shape in SHAPES:
        nz, ny, nx = shape
        U = inputs.random_smooth(shape, seed=11 + order, amp=0.3)
        dt = 0.7 * scheme.max_dt(U, (1 / nx, 1 / ny, 1 / nz), 0.4)
        a, b = _both(ader, shape, U, dt, order=order, form=form, solver=solver, fp32=fp32)
        if fp32:
            # the shared FP32 predictor is compiled into two kernels whose multiply-add contractions may
            # differ: equal to FP32 rounding
            assert rel_l1(a, b) <= 1e-6, shape
        else:
            assert np.array_equal(a, b), shape


@pytest.mark.parametrize("fp32", [False, True])
def test_tiled_sod_many_chunks_matches_oracle(ader, fp32):
    """A Sod tube on a grid of several tiles and z chunks: the default layout against the oracle."""
    shape = (48, 12, 64)
    nz, ny, nx = shape
    U = inputs.sod_planar(shape)
    dx = (1 / nx, 1 / ny, 1 / nz)
    dt = scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, 3, "nodal", "hll")
    s = ader.Solver(shape, order=3, form="nodal", solver="hll", fp32=fp32)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    assert rel_l1(to_host(d), want) <= (1e-6 if fp32 else 1e-12)
    s.close()


def test_tiled_equals_per_zone_with_source_converged_and_rk(ader):
    shape = (9, 10, 40)
    nz, ny, nx = shape
    U = inputs.random_smooth(shape, seed=5, amp=0.3)
    dt = 0.6 * scheme.max_dt(U, (1 / nx, 1 / ny, 1 / nz), 0.4)
    for order in (2, 3):
        for fp32 in (False, True):
            same = (lambda a, b: rel_l1(a, b) <= 1e-6) if fp32 else np.array_equal
            a, b = _both(ader, shape, U, dt, setup=lambda s: s.set_source("gravity", (0.3, -0.2, 0.1)),
                         order=order, form="nodal", fp32=fp32)
            assert same(a, b)
            a, b = _both(ader, shape, U, dt, setup=lambda s: s.set_predictor(1e-6 if fp32 else 1e-13, 30),
                         order=order, form="modal", fp32=fp32)
            assert same(a, b)
            a, b = _both(ader, shape, U, dt, rk=True, order=order, form="modal", solver="linearized", fp32=fp32)
            assert same(a, b)


@pytest.mark.parametrize("form", ["modal", "nodal"])
@pytest.mark.parametrize("mhd", [False, True])
def test_tiled_cross_moments_on_full_tiles(ader, form, mhd):
    """Grids the cross-moment tiles cover (nx a multiple of 32, ny of 8; several tiles and z chunks), FP64,
    order 3: the tiled cross moments, whose per-position WENO terms are shared through shared memory, give
    the per-zone kernel's bits, and the step matches the oracle to 1e-12."""
    if mhd:
        shape, G = (32, 32, 32), 5.0 / 3.0
        U, B = inputs.random_magnetised(32, seed=3)
    else:
        shape, G = (20, 16, 64), 1.4
        U, B = inputs.random_smooth(shape, seed=5, amp=0.3), None
    nz, ny, nx = shape
    dx = (1 / nx, 1 / ny, 1 / nz)
    dt = 0.6 * scheme.max_dt(U, dx, 0.4, G, Bface=B)
    got = []
    for tiled in (True, False):
        s = ader.Solver(shape, order=3, form=form, solver="hll", gamma=G, mhd=mhd)
        s.set_tiled(tiled)
        dU = to_dev(U)
        dB = to_dev(B) if mhd else None
        s.step(dU, dt, Bface=dB)
        assert s.status() == 0
        got.append((to_host(dU), to_host(dB) if mhd else None))
        s.close()
    assert np.array_equal(got[0][0], got[1][0])
    if mhd:
        assert np.array_equal(got[0][1], got[1][1])
        Uo, Bo = scheme.ader_step(U, dx, dt, 3, form, "hll", G, Bface=B)
        assert rel_l1(got[0][1], Bo) <= 1e-12
    else:
        Uo = scheme.ader_step(U, dx, dt, 3, form, "hll", G)
    assert rel_l1(got[0][0], Uo) <= 1e-12
