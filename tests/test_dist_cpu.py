"""The N > 1 launch path of bench.py on the host: two gloo ranks on the CPU.

Under torchrun every rank runs its own problem of the same size (weak scaling, no collective on the data
path); the only exchange is the max over ranks of the timed seconds.  These tests run that exchange, the
rank environment, the whole-job throughput and the rank-0-only reference arm without a GPU.
"""
import importlib.util
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, secs_by_rank, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    bench = _bench()
    w, r, loc = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        secs = bench.max_over_ranks(secs_by_rank[r], w, "cpu")
        value = bench.job_throughput(1000, 4, w, secs)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out.put((r, loc, w, secs, value))


@pytest.mark.timeout(120)
def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    secs_by_rank = [0.25, 0.75]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, secs_by_rank, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for r, (rank, local, world, secs, value) in enumerate(got):
        assert (rank, local, world) == (r, r, 2)
        # every rank sees the slowest rank's time, and the job counts both ranks' units
        assert secs == 0.75
        assert value == pytest.approx(1000 * 4 * 2 / 0.75, rel=1e-15)


def test_single_rank_needs_no_process_group():
    bench = _bench()
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5
    assert bench.job_throughput(10, 3, 1, 2.0) == 15.0


def test_cores_used():
    bench = _bench()
    assert bench.cores_used(10.0, 10.0) == 1
    assert bench.cores_used(0.2, 10.0) == 1
    assert bench.cores_used(31.0, 10.0) == 3
    assert bench.cores_used(1.0, 0.0) == 1


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
