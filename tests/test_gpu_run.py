"""GPU: a resumed run equals the uninterrupted one bit for bit; the step log records conserved totals."""
import json

import numpy as np
import pytest

from gpu_util import ensure_built, to_dev
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


def test_resume_equals_uninterrupted_run(ader, tmp_path):
    import torch
    from paper_1006_2146_gb300 import run
    n = 12
    U0 = inputs.random_smooth(n, seed=301, amp=0.3)
    s = ader.Solver((n, n, n), order=3, form="nodal")
    a = to_dev(U0)
    run.advance(s, a, 1.0, max_steps=4)
    b = to_dev(U0)
    path = str(tmp_path / "ck.pt")
    t, step = run.advance(s, b, 1.0, max_steps=2, checkpoint=path)
    ck = run.load_checkpoint(path)
    assert ck["step"] == 2 and ck["t"] == t
    c = ck["U"]
    run.advance(s, c, 1.0, t=ck["t"], step=ck["step"], max_steps=2)
    s.close()
    assert torch.equal(a, c)


def test_step_log_mhd(ader, tmp_path):
    from paper_1006_2146_gb300 import run
    n = 10
    U, B = inputs.random_magnetised(n, seed=302, amp=0.2, b_amp=0.4)
    s = ader.Solver((n, n, n), order=3, form="modal", gamma=5.0 / 3.0, mhd=True)
    s.set_predictor(1e-13, 50)
    dU, dB = to_dev(U), to_dev(B)
    path = str(tmp_path / "log.jsonl")
    log = run.StepLog(path, gamma=5.0 / 3.0)
    run.advance(s, dU, 1.0, Bface=dB, max_steps=3, log=log)
    s.close()
    recs = [json.loads(line) for line in open(path)]
    assert [r["step"] for r in recs] == [1, 2, 3]
    tot0 = U.sum(axis=(1, 2, 3))
    for r in recs:
        np.testing.assert_allclose(r["totals"], tot0, rtol=1e-12, atol=1e-14)
        assert r["rho_min"] > 0 and r["p_min"] > 0
        assert r["div_b_rel_max"] <= 1e-12
        assert r["predictor_iterations"] > 0 and r["predictor_capped"] == 0
