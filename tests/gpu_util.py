"""Helpers for the GPU parity tests: build/load the library and move states between numpy and torch."""
import os

import numpy as np

_BUILT = False


def ensure_built():
    global _BUILT
    from paper_1006_2146_gb300 import _lib, build
    if not _BUILT:
        build.build()
        _BUILT = True
    return _lib.load()


def to_dev(U):
    import torch
    return torch.from_numpy(np.ascontiguousarray(U)).to("cuda")


def to_host(t):
    return t.detach().cpu().numpy()


def rel_l1(got, want):
    """max over variables of sum|got - want| / max(sum|want_v|, sum|rho|) (the parity measure)."""
    num = np.abs(got - want).reshape(want.shape[0], -1).sum(axis=1)
    den = np.maximum(np.abs(want).reshape(want.shape[0], -1).sum(axis=1), np.abs(want[0]).sum())
    return float((num / den).max())
