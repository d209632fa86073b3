"""The context's per-thread stack (ader_trim_local_memory): a fourth-order FP64 step needs a large stack
frame, the context keeps it for every later launch, and the trim hands it back (1 KB per thread) without
disturbing the context: the next step grows it again and gives the same result."""
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


def test_trim_after_a_large_frame(ader):
    import torch
    U = inputs.random_smooth(8, seed=1, amp=0.1)
    s = ader.Solver((8, 8, 8), order=4, form="modal")
    a, b = to_dev(U), to_dev(U)
    s.step(a, 1e-4)
    torch.cuda.synchronize()
    assert ader.ader_trim_local_memory() > 2048          # the predictor's frame was kept
    assert ader.ader_trim_local_memory() == 1024         # and is gone
    s.step(b, 1e-4)                                      # grows it again
    assert s.status() == 0
    assert np.array_equal(to_host(a), to_host(b))
    s.close()
