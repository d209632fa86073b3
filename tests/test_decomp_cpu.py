"""The z-slab decomposition (paper_1006_2146_gb300.decomp) on the host, with the oracle as each part's step.

One halo exchange per step, dt the minimum over the parts, each part stepping its slab with G ghost planes:
the parts together must give the single-domain step.  The parts run in one process (LocalExchange) and as
two gloo ranks (DistExchange), on a Sod tube whose normal has a z component, over ten steps.  The oracle
works on arrays of other shapes in the two runs, so they agree to rounding (1e-14 relative), not bit for
bit; the GPU version of this test (test_gpu_decomp.py) compares bit for bit.
"""
import os
import socket

import numpy as np
import pytest

from oracle import scheme
from paper_1006_2146_gb300 import decomp, inputs

N, ORDER, STEPS, CFL = 24, 3, 10, 0.4
DX = (1.0 / N,) * 3


def _state():
    return inputs.sod_planar(N, normal=(1, 0, 1), sub=2)


def _oracle_fns(torch):
    def step_fn(slab, dt):
        U = slab.Upad.numpy()
        slab.Upad[:] = torch.from_numpy(scheme.ader_step(U, DX, dt, ORDER, "nodal", "hll"))

    def dt_fn(slab):
        return torch.tensor([scheme.max_dt(slab.Upad.numpy(), DX, CFL)], dtype=torch.float64)
    return step_fn, dt_fn


def _single_domain():
    U = _state()
    dts = []
    for _ in range(STEPS):
        dt = scheme.max_dt(U, DX, CFL)
        U = scheme.ader_step(U, DX, dt, ORDER, "nodal", "hll")
        dts.append(dt)
    return U, dts


@pytest.fixture(scope="module")
def reference():
    return _single_domain()


def test_split_and_offsets():
    assert decomp.split(24, 5) == [5, 5, 5, 5, 4]
    assert decomp.offsets([5, 5, 4]) == [0, 5, 10]
    assert decomp.ghost_planes(4) == 4


def test_local_exchange_three_parts_equals_single_domain(reference):
    torch = pytest.importorskip("torch")
    U0 = _state()
    counts = decomp.split(N, 3)
    offs = decomp.offsets(counts)
    parts = [torch.from_numpy(U0[:, o:o + c].copy()) for o, c in zip(offs, counts)]
    step_fn, dt_fn = _oracle_fns(torch)
    dd = decomp.Decomposed(parts, ORDER, decomp.LocalExchange(), step_fn=step_fn, dt_fn=dt_fn)
    dts = [dd.step() for _ in range(STEPS)]
    got = np.concatenate([s.interior.numpy() for s in dd.slabs], axis=1)
    want, want_dts = reference
    np.testing.assert_allclose(dts, want_dts, rtol=1e-14)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())


def test_a_part_thinner_than_the_ghost_width_is_refused():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        decomp.Slab(torch.zeros((5, 2, 4, 4), dtype=torch.float64), decomp.ghost_planes(3))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank)})
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        U0 = _state()
        counts = decomp.split(N, world)
        o = decomp.offsets(counts)[rank]
        part = torch.from_numpy(U0[:, o:o + counts[rank]].copy())
        step_fn, dt_fn = _oracle_fns(torch)
        dd = decomp.Decomposed([part], ORDER, decomp.DistExchange(), step_fn=step_fn, dt_fn=dt_fn)
        dts = [dd.step() for _ in range(STEPS)]
        out.put((rank, dd.slabs[0].interior.numpy().copy(), dts))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_equal_single_domain(reference):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=240) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want, want_dts = reference
    U = np.concatenate([g[1] for g in got], axis=1)
    for g in got:
        np.testing.assert_allclose(g[2], want_dts, rtol=1e-14)
    np.testing.assert_allclose(U, want, rtol=0, atol=1e-14 * np.abs(want).max())
