"""Training the learned initial guess of the third-order predictor, through the C ABI.

The library does the work: ``ader_guess_samples`` runs the converged FP64
predictor on every zone of a state and writes the network's features and
targets, and ``ader_mlp_train`` trains the MLP with the library's own GEMM,
GELU and Adam kernels.  This module only chooses the training states, moves
tensors and seeds the initial weights.

Training states (seeded, synthetic), each at Courant numbers 0.4 and 0.2 of
the CFL rule, so that the Courant features span the range a run uses:
Euler: Gaussian random fields of density and velocity of several amplitudes,
blasts of several pressure ratios, and planar Sod-type shock tubes along
lattice normals.  MHD: the same random fields threaded by a uniform field and
a random periodic field from a vector potential, blasts in a uniform field,
and circularly polarised Alfven waves.  The Orszag-Tang-type vortex is kept
out of the MHD mix: it is the unseen evaluation state.
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


def training_states(n, seed=1006000, mhd=False):
    """States of the training mix: Euler U (numpy, (5, n, n, n)), or MHD pairs (U, Bface)."""
    if mhd:
        return mhd_training_states(n, seed)
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


def mhd_training_states(n, seed=1006100):
    """MHD pairs (U, Bface) of the training mix (gamma 5/3)."""
    rng = np.random.default_rng(seed)
    out = []
    for k, (amp, b_amp, B0, P0) in enumerate(((0.05, 0.2, 0.5, 1.0), (0.2, 0.5, 1.0, 1.0), (0.4, 1.0, 2.0, 1.0),
                                              (0.3, 0.3, 3.0, 1.0), (0.6, 0.6, 1.0, 0.3), (0.8, 1.0, 2.0, 0.2))):
        # the last two: transonic flow (Mach near 1) at plasma beta of a few
        out.append(inputs.random_magnetised(n, seed=seed + 1 + k, amp=amp, b_amp=b_amp, B0=B0, P0=P0))
    for ratio, B0 in ((10.0, 1.0), (100.0, 3.0)):
        c = tuple(rng.uniform(0.3, 0.7, 3))
        U = inputs.blast(n, gamma=5.0 / 3.0, p_in=ratio * 0.1, p_out=0.1, radius=rng.uniform(0.05, 0.15), center=c)
        out.append(inputs.with_field(U, inputs.uniform_field(n, B0, rng.normal(size=3))))
    for amp in (0.1, 0.3):
        out.append(inputs.alfven_wave(n, amp=amp))
    return out


def make_samples(states, n, cfls=(0.4, 0.2), tol=1e-13, mhd=False):
    """Features X and targets Y (device, FP32) of every physical, converged zone of every state and CFL.
    MHD states are (U, Bface) pairs."""
    import torch
    n_in, _, n_out, _ = _lib.ader_mlp_shape(mhd)
    h = _lib.ader_create(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, 3, 5.0 / 3.0 if mhd else 1.4, _lib.ADER_HLL,
                         _lib.ADER_MHD if mhd else 0)
    try:
        _lib.ader_set_predictor(h, tol, 50)
        zones = n ** 3
        X = torch.empty((zones, n_in), dtype=torch.float32, device="cuda")
        Y = torch.empty((zones, n_out), dtype=torch.float32, device="cuda")
        ok = torch.empty(zones, dtype=torch.int32, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        xs, ys = [], []
        for st in states:
            U, B = st if mhd else (st, None)
            d = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
            b = None if B is None else torch.from_numpy(np.ascontiguousarray(B)).to("cuda")
            _lib.ader_max_dt(h, d, b, 1.0, dt)
            dt1 = float(dt.item())
            for cfl in cfls:
                _lib.ader_guess_samples(h, d, b, cfl * dt1, X, Y, ok)
                keep = ok.bool()
                xs.append(X[keep].clone())
                ys.append(Y[keep].clone())
        torch.cuda.synchronize()
        return torch.cat(xs).contiguous(), torch.cat(ys).contiguous()
    finally:
        _lib.ader_destroy(h)


def train(X, Y, epochs=3, batch=8192, lr=1e-3, seed=0, mhd=False):
    """Trained parameters (device FP32) and the loss of the last minibatch of each epoch."""
    import torch
    P = torch.from_numpy(init_params(mhd, seed)).to("cuda")
    losses = _lib.ader_mlp_train(X, Y, X.shape[0], P, epochs, batch, lr, seed=seed, mhd=mhd)
    return P, losses
