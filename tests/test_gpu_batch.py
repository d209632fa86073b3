"""GPU: batched problems of uneven sizes (ader_batch_*) against single-problem contexts and the FP64 oracle.

Each problem of a batch runs the same per-zone code as a single context, so
with the same dt the two agree to FP32 round-off; against the oracle the FP32
bar (1e-5 relative L1) applies.
"""
import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import scheme
from paper_1006_2146_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu
G_MHD = 5.0 / 3.0

# (shape (nz, ny, nx), order, physics, form, solver, seed)
MIX = [((8, 9, 10), 3, "euler", "nodal", "hll", 1),
       ((12, 12, 12), 2, "euler", "modal", "linearized", 2),
       ((5, 16, 7), 4, "euler", "modal", "hll", 3),
       ((10, 6, 8), 3, "euler", "nodal", "hll", 4),          # same group as the first problem
       ((8, 8, 8), 3, "mhd", "modal", "hll", 5),
       ((6, 7, 9), 2, "mhd", "nodal", "linearized", 6),
       ((9, 9, 9), 4, "mhd", "nodal", "hll", 7),
       ((4, 13, 11), 3, "euler", "modal", "linearized", 8)]


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _state(shape, physics, seed):
    if physics == "euler":
        return inputs.random_smooth(shape, seed=seed, amp=0.3), None
    n = shape[0]
    U, B = inputs.alfven_wave(n, amp=0.3)
    rng = np.random.default_rng(seed)
    U = U * (1.0 + 0.02 * rng.normal(size=U.shape))
    U[4] += 0.3
    return U, B


def _mix(mix):
    probs = []
    for shape, order, physics, form, solver, seed in mix:
        if physics == "mhd":
            shape = (shape[0],) * 3             # the Alfven-wave generator makes cubes
        U, B = _state(shape, physics, seed)
        probs.append(dict(shape=shape, order=order, mhd=physics == "mhd", form=form, solver=solver, U=U, B=B,
                          gamma=G_MHD if physics == "mhd" else 1.4))
    return probs


def _create(ader, probs):
    grids, orders, gammas, solvers, flags = [], [], [], [], []
    for p in probs:
        nz, ny, nx = p["shape"]
        grids.append((nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nz))
        orders.append(p["order"])
        gammas.append(p["gamma"])
        solvers.append(_lib.ADER_LINEARIZED if p["solver"] == "linearized" else _lib.ADER_HLL)
        flags.append(_lib.ADER_FP32_BULK | (_lib.ADER_NODAL if p["form"] == "nodal" else 0) |
                     (_lib.ADER_MHD if p["mhd"] else 0))
    return _lib.ader_batch_create(grids, orders, gammas, solvers, flags)


def _single(ader, p, U, B, dt):
    nz, ny, nx = p["shape"]
    flags = _lib.ADER_FP32_BULK | (_lib.ADER_NODAL if p["form"] == "nodal" else 0) | (_lib.ADER_MHD if p["mhd"] else 0)
    h = _lib.ader_create(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nz, p["order"], p["gamma"],
                         _lib.ADER_LINEARIZED if p["solver"] == "linearized" else _lib.ADER_HLL, flags)
    _lib.ader_step(h, U, B, dt)
    assert _lib.ader_sync_status(h) == 0
    _lib.ader_destroy(h)


def test_batch_matches_single_contexts_and_oracle(ader):
    import torch
    probs = _mix(MIX)
    b = _create(ader, probs)
    assert _lib.ader_batch_groups(b) == 7
    Us = [to_dev(p["U"]) for p in probs]
    Bs = [to_dev(p["B"]) if p["mhd"] else None for p in probs]
    dt = torch.zeros(len(probs), dtype=torch.float64, device="cuda")
    _lib.ader_batch_advance(b, Us, Bs, 0.4, dt)
    rc, codes = _lib.ader_batch_status(b, len(probs))
    assert rc == 0 and codes == [0] * len(probs)
    dts = dt.cpu().numpy()
    for k, p in enumerate(probs):
        nz, ny, nx = p["shape"]
        dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
        want_dt = scheme.max_dt(p["U"], dx, 0.4, p["gamma"], Bface=p["B"])
        assert dts[k] == pytest.approx(want_dt, rel=1e-6), k      # FP32 signal speeds, FP64 reduction
        # the same step through a single context
        Us1 = to_dev(p["U"])
        Bs1 = to_dev(p["B"]) if p["mhd"] else None
        _single(ader, p, Us1, Bs1, float(dts[k]))
        assert rel_l1(to_host(Us[k]), to_host(Us1)) <= 1e-6, k
        # and the FP64 oracle
        want = scheme.ader_step(p["U"], dx, float(dts[k]), p["order"], p["form"], p["solver"], p["gamma"],
                                Bface=p["B"])
        if p["mhd"]:
            Uo, Bo = want
            assert rel_l1(to_host(Us[k]), Uo) <= 1e-5, k
            assert rel_l1(to_host(Bs[k]), Bo) <= 1e-5, k
            d0 = scheme.div_b(p["B"], dx)
            assert np.abs(scheme.div_b(to_host(Bs[k]), dx) - d0).max() <= 1e-6 * np.abs(p["B"]).max() / dx[0]
        else:
            assert rel_l1(to_host(Us[k]), want) <= 1e-5, k
    _lib.ader_batch_destroy(b)


def test_batch_step_with_given_dt_and_tuning_keep_results(ader):
    """ader_batch_step with caller dts; tuning changes launch shapes, not results (bit-identical)."""
    import torch
    probs = _mix(MIX[:5])
    dt = torch.tensor([2e-3, 1e-3, 5e-4, 1.5e-3, 1e-3], dtype=torch.float64, device="cuda")
    outs = []
    for tune in (False, True):
        b = _create(ader, probs)
        Us = [to_dev(p["U"]) for p in probs]
        Bs = [to_dev(p["B"]) if p["mhd"] else None for p in probs]
        if tune:
            _lib.ader_batch_tune(b, Us, Bs)
            chosen = _lib.ader_batch_tuning(b)
            assert len(chosen) > 0
            assert all(t in (64, 128, 256) for (_, _, t, _) in chosen)
        for _ in range(3):
            _lib.ader_batch_step(b, Us, Bs, dt)
        rc, _ = _lib.ader_batch_status(b, len(probs))
        assert rc == 0
        outs.append([to_host(u) for u in Us] + [to_host(x) for x in Bs if x is not None])
        _lib.ader_batch_destroy(b)
    for a, c in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, c)


def test_batch_recaptures_on_new_buffers(ader):
    """A second set of state buffers (a new graph) gives the same step as the first."""
    import torch
    probs = _mix(MIX[:4])
    b = _create(ader, probs)
    dt = torch.full((len(probs),), 1e-3, dtype=torch.float64, device="cuda")
    A = [to_dev(p["U"]) for p in probs]
    Bn = [None] * len(probs)
    _lib.ader_batch_step(b, A, Bn, dt)
    C = [to_dev(p["U"]) for p in probs]
    _lib.ader_batch_step(b, C, Bn, dt)
    torch.cuda.synchronize()
    for a, c in zip(A, C):
        np.testing.assert_array_equal(to_host(a), to_host(c))
    _lib.ader_batch_destroy(b)


def test_batch_reports_the_unphysical_problem(ader):
    import torch
    probs = _mix(MIX[:3])
    probs[1]["U"] = probs[1]["U"].copy()
    probs[1]["U"][4, 2, 3, 4] = -1.0                   # negative energy in one zone of problem 1
    b = _create(ader, probs)
    Us = [to_dev(p["U"]) for p in probs]
    dt = torch.zeros(len(probs), dtype=torch.float64, device="cuda")
    _lib.ader_batch_advance(b, Us, [None] * 3, 0.4, dt)
    rc, codes = _lib.ader_batch_status(b, 3)
    assert rc in (_lib.ADER_ERR_UNPHYSICAL, _lib.ADER_ERR_NONFINITE)
    assert codes[0] == 0 and codes[2] == 0 and codes[1] == rc
    _lib.ader_batch_destroy(b)


def test_batch_rejects_unsupported_problems(ader):
    g = [(8, 8, 8, 0.125, 0.125, 0.125)]
    with pytest.raises(_lib.AderError):                 # FP64 bulk is not batched
        _lib.ader_batch_create(g, [3], [1.4], [_lib.ADER_HLL], [0])
    with pytest.raises(_lib.AderError):
        _lib.ader_batch_create(g, [5], [1.4], [_lib.ADER_HLL], [_lib.ADER_FP32_BULK])
