"""Training the learned initial guess of the third-order predictor, through the C ABI.

The library does the work: ``ader_guess_samples`` runs the converged FP64
predictor on every zone of a state and writes the network's features and
targets, and ``ader_mlp_train`` trains the MLP with the library's own GEMM,
GELU and Adam kernels.  This module only chooses the training states, moves
tensors and seeds the initial weights.

Training states (seeded, synthetic): Gaussian random fields of density and
velocity of several amplitudes, blasts of several pressure ratios, and planar
Sod-type shock tubes along lattice normals, each at Courant numbers 0.4 and
0.2 of the CFL rule, so that the Courant features span the range a run uses.
"""
import numpy as np

from . import _lib, inputs


def init_params(mhd=False, seed=0):
    """Seeded initial weights: N(0, 1/fan_in) matrices, zero biases (FP32, the packed layout of ader.h)."""
    n_in, H, n_out, n_par = _lib.ader_mlp_shape(mhd)
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((H, n_in)) / np.sqrt(n_in), np.zeros(H),
             rng.standard_normal((H, H)) / np.sqrt(H), np.zeros(H),
             rng.standard_normal((n_out, H)) / np.sqrt(H), np.zeros(n_out)]
    P = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    assert P.size == n_par
    return P


def training_states(n, seed=1006000):
    """Euler states (numpy, (5, n, n, n)) of the training mix."""
    rng = np.random.default_rng(seed)
    out = []
    for k, amp in enumerate((0.05, 0.2, 0.5)):
        out.append(inputs.random_smooth(n, seed=seed + 1 + k, amp=amp))
    for ratio in (10.0, 1e3):
        c = tuple(rng.uniform(0.3, 0.7, 3))
        out.append(inputs.blast(n, p_in=ratio * 0.1, p_out=0.1, radius=rng.uniform(0.05, 0.15), center=c))
    for normal, (rl, pl, rr, pr) in (((1, 1, 0), (1.0, 1.0, 0.125, 0.1)), ((1, 0, 0), (1.0, 5.0, 0.3, 0.5))):
        out.append(inputs.sod_planar(n, normal=normal, left=(rl, pl), right=(rr, pr)))
    return out


def make_samples(states, n, cfls=(0.4, 0.2), tol=1e-13):
    """Features X and targets Y (device, FP32) of every physical, converged zone of every state and CFL."""
    import torch
    n_in, _, n_out, _ = _lib.ader_mlp_shape(False)
    h = _lib.ader_create(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, 3, 1.4, _lib.ADER_HLL, 0)
    try:
        _lib.ader_set_predictor(h, tol, 50)
        zones = n ** 3
        X = torch.empty((zones, n_in), dtype=torch.float32, device="cuda")
        Y = torch.empty((zones, n_out), dtype=torch.float32, device="cuda")
        ok = torch.empty(zones, dtype=torch.int32, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        xs, ys = [], []
        for U in states:
            d = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
            _lib.ader_max_dt(h, d, None, 1.0, dt)
            dt1 = float(dt.item())
            for cfl in cfls:
                _lib.ader_guess_samples(h, d, None, cfl * dt1, X, Y, ok)
                keep = ok.bool()
                xs.append(X[keep].clone())
                ys.append(Y[keep].clone())
        torch.cuda.synchronize()
        return torch.cat(xs).contiguous(), torch.cat(ys).contiguous()
    finally:
        _lib.ader_destroy(h)


def train(X, Y, epochs=3, batch=8192, lr=1e-3, seed=0):
    """Trained parameters (device FP32) and the loss of the last minibatch of each epoch."""
    import torch
    P = torch.from_numpy(init_params(False, seed)).to("cuda")
    losses = _lib.ader_mlp_train(X, Y, X.shape[0], P, epochs, batch, lr, seed=seed)
    return P, losses
