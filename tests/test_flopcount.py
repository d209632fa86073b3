"""flops.json (the per-zone FLOP counts the bench's roofline divides by) is the output of the host FLOP
counter over the kernels' current per-zone code: rebuilding and rerunning the counter reproduces it."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1006_2146_gb300", "csrc", "flopcount", "flopcount.cu")


def test_flops_json_matches_the_counter(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "flopcount")
    subprocess.run([nvcc, "-O0", "-Xcompiler", "-O0", "-std=c++17", "--expt-relaxed-constexpr",
                    "-gencode", "arch=compute_103a,code=sm_103a", SRC, "-o", exe], check=True,
                   capture_output=True, timeout=900)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=600).stdout
    with open(os.path.join(ROOT, "paper_1006_2146_gb300", "flops.json")) as fh:
        assert json.loads(out) == json.load(fh)
