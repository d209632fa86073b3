"""The allocation-free CFL entry point (ader_max_dt_static) against ader_max_dt and the oracle.

Callers that cannot allocate device memory (inside another library's stream
capture, fixed-budget real-time loops) use ader_max_dt_static: no context, the
scratch is a device array inside the library.  This file is collected last so
that a failure here leaves every other test already run; it also passes on
its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import ensure_built
    lib = ensure_built()
    lib.ader_max_dt_static.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p]
    lib.ader_max_dt_static.restype = ctypes.c_int
    return torch, lib


def _static_dt(torch, lib, grid, U, cfl):
    from paper_1006_2146_gb300 import _lib
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rc = lib.ader_max_dt_static(ctypes.byref(grid), 1.4, ctypes.c_void_p(U.data_ptr()), cfl,
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.ADER_OK
    torch.cuda.synchronize()
    return float(out.item())


@pytest.mark.parametrize("shape", [(7, 9, 12), (64, 64, 64), (3, 1, 1)])
def test_static_dt_matches_context_dt_twice(env, shape):
    torch, lib = env
    import paper_1006_2146_gb300 as ader
    from oracle import scheme
    from paper_1006_2146_gb300 import _lib, inputs
    nz, ny, nx = shape
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    grid = _lib.ader_grid(nx, ny, nz, *dx)
    s = ader.Solver(shape, order=3)
    for seed in (1, 2):                       # two calls in a row, different data
        Uh = inputs.random_smooth(shape, seed=seed, amp=0.4)
        U = torch.from_numpy(Uh).cuda()
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.max_dt(U, 0.4, ref)
        torch.cuda.synchronize()
        got = _static_dt(torch, lib, grid, U, 0.4)
        assert got == pytest.approx(float(ref.item()), rel=1e-14)
        assert got == pytest.approx(scheme.max_dt(Uh, dx, 0.4), rel=1e-14)      # the oracle's CFL rule
    s.close()


@pytest.mark.parametrize("where", ["negative_pressure", "nan_density"])
def test_static_dt_reports_a_non_physical_zone(env, where):
    """A zone without a real signal speed makes dt a quiet NaN; the next call on clean data is exact again."""
    torch, lib = env
    from oracle import scheme
    from paper_1006_2146_gb300 import _lib, inputs
    shape = (20, 30, 40)                       # several blocks of the reduction
    nz, ny, nx = shape
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    grid = _lib.ader_grid(nx, ny, nz, *dx)
    Uh = inputs.random_smooth(shape, seed=5, amp=0.3)
    bad = Uh.copy()
    if where == "nan_density":
        bad[0, 17, 3, 29] = np.nan
    else:
        m = bad[1:4, 17, 3, 29]
        bad[4, 17, 3, 29] = 0.5 * (m * m).sum() / bad[0, 17, 3, 29] - 1e-6
    assert np.isnan(_static_dt(torch, lib, grid, torch.from_numpy(bad).cuda(), 0.4))
    got = _static_dt(torch, lib, grid, torch.from_numpy(Uh).cuda(), 0.4)
    assert got == pytest.approx(scheme.max_dt(Uh, dx, 0.4), rel=1e-14)


def test_static_dt_rejects_oversized_grid(env):
    torch, lib = env
    from paper_1006_2146_gb300 import _lib
    grid = _lib.ader_grid(1024, 1024, 512, 1.0, 1.0, 1.0)       # 2^29 zones > the static maximum
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.ader_max_dt_static(ctypes.byref(grid), 1.4, ctypes.c_void_p(dummy.data_ptr()), 0.4,
                                ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == _lib.ADER_ERR_ARG
