"""Checkpoint files on the host (no GPU): the state round-trips exactly and a write is atomic."""
import os

import pytest

torch = pytest.importorskip("torch")


def test_checkpoint_round_trip(tmp_path):
    from paper_1006_2146_gb300 import run
    U = torch.randn(5, 4, 5, 6, dtype=torch.float64)
    B = torch.randn(3, 4, 5, 6, dtype=torch.float64)
    P = torch.randn(100, dtype=torch.float32)
    path = str(tmp_path / "run.pt")
    run.save_checkpoint(path, U, B, t=0.125, step=7, guess=P, meta={"order": 3})
    assert not os.path.exists(path + ".tmp")
    got = run.load_checkpoint(path, device="cpu")
    assert got["t"] == 0.125 and got["step"] == 7 and got["meta"] == {"order": 3}
    assert torch.equal(got["U"], U) and torch.equal(got["Bface"], B) and torch.equal(got["guess"], P)
    run.save_checkpoint(path, U, None, t=0.25, step=8)
    got = run.load_checkpoint(path, device="cpu")
    assert got["Bface"] is None and got["guess"] is None and got["step"] == 8


def test_checkpoint_rejects_unknown_format(tmp_path):
    from paper_1006_2146_gb300 import run
    path = str(tmp_path / "bad.pt")
    torch.save({"format": 99}, path)
    with pytest.raises(ValueError):
        run.load_checkpoint(path, device="cpu")
