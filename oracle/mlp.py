"""FP64 CPU oracle of the learned initial guess of the third-order predictor.

TEST INFRASTRUCTURE: only tests/, the smoke check and the CPU-baseline leg of
bench.py use this module; the product path never does.

The paper has no learned component.  What is defined here is a deployment
extension of its Picard predictor (Sec. IV.1, order 3): a small MLP maps a
zone's normalised spatial modes and Courant numbers to a first guess of the
evolutionary modes u_11..u_15, from which the iteration starts instead of
zero; the converged iteration decides the result.  This file restates, in
plain numpy FP64:

  * the network: y = W3 g(W2 g(W1 x + b1) + b2) + b3, hidden width 128, with
    g the tanh form of GELU, g(x) = x/2 (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3)));
  * the training loss (mean squared error over all outputs) and its gradient by
    backpropagation;
  * the features and targets of a zone (``features``, ``targets``):
      scales  s_rho = w1(rho), s_E = w1(E), c = sqrt(s_E / s_rho), s_m = s_rho c,
              s_B = sqrt(8 pi s_E) (Gaussian units, as in Sec. III);
      slopes  r = w2..w10 of every variable over its scale; magnitude g = max |r|;
      x       r / g (variable-major), then w1 of each momentum (and field)
              component over its scale, then c dt/dx, c dt/dy, c dt/dz, then g;
      y       u_{11+j} of variable v over (s_v sigma g), sigma = c (dt/dx + dt/dy + dt/dz),
              in the order j-major, variable-minor.
    A zone uniform to round-off (g <= MAG_MIN = 1e-12) has no time evolution to
    speak of: its guess is zero and it is no sample (``sample_mask``).

Parameters are one flat vector: W1 (H x IN, row-major), b1 (H), W2 (H x H),
b2 (H), W3 (OUT x H), b3 (OUT).

Pins (tests/test_oracle_mlp.py): the gradient against central finite
differences of the loss; the forward pass against a single-path network whose
output has a closed form; g against the exact (erf) GELU within the known
accuracy of the tanh form and its limits; the features of uniform states.
"""
import numpy as np

HIDDEN = 128
MAG_MIN = 1e-12


def shape(mhd=False):
    """(n_in, n_hidden, n_out, n_params)."""
    nv = 8 if mhd else 5
    n_in = 48 + (30 if mhd else 0) + 4
    n_out = 5 * nv
    H = HIDDEN
    return n_in, H, n_out, H * n_in + H + H * H + H + n_out * H + n_out


def unpack(P, n_in, n_out, H=HIDDEN):
    """Views (W1, b1, W2, b2, W3, b3) of the flat parameter vector."""
    sizes = [(H, n_in), (H,), (H, H), (H,), (n_out, H), (n_out,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(P[o:o + n].reshape(s))
        o += n
    assert o == P.size
    return out


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (x + 0.044715 * x ** 3)))


def gelu_prime(x):
    k = np.sqrt(2.0 / np.pi)
    t = np.tanh(k * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * k * (1.0 + 3 * 0.044715 * x * x)


def forward(P, X, n_out, H=HIDDEN):
    """Network outputs (n, n_out) for inputs X (n, n_in)."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(P, dtype=np.float64), X.shape[1], n_out, H)
    h1 = gelu(X @ W1.T + b1)
    h2 = gelu(h1 @ W2.T + b2)
    return h2 @ W3.T + b3


def loss_and_grad(P, X, Y, H=HIDDEN):
    """Mean squared error over all n x n_out outputs and its gradient (flat, like P)."""
    P = np.asarray(P, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n, n_out = Y.shape
    W1, b1, W2, b2, W3, b3 = unpack(P, X.shape[1], n_out, H)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    yp = h2 @ W3.T + b3
    d = yp - Y
    loss = float((d * d).sum() / d.size)
    dy = 2.0 * d / d.size
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_prime(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_prime(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def _scales(W, mhd):
    rho, E = W[0, 0], W[0, 4]
    c = np.sqrt(E / rho)
    s = [rho, rho * c, rho * c, rho * c, E]
    if mhd:
        sb = np.sqrt(8.0 * np.pi * E)
        s += [sb, sb, sb]
    return s, c


def _slopes(W):
    """Normalised slopes r (n_zones, 45 or 72): w2..w10 of each variable over its scale; their magnitude g."""
    nv = W.shape[1]
    Wf = W.reshape(W.shape[0], nv, -1)
    s, _ = _scales(Wf, nv == 8)
    cols = [Wf[k, v] / s[v] for v in range(nv) for k in range(1, 10)]
    r = np.stack(cols, axis=1)
    return r, np.abs(r).max(axis=1)


def _means(W):
    """Zone means of momentum (and field) over their scales (n_zones, 3 or 6)."""
    nv = W.shape[1]
    Wf = W.reshape(W.shape[0], nv, -1)
    s, _ = _scales(Wf, nv == 8)
    return np.stack([Wf[0, v] / s[v] for v in range(1, nv) if v != 4], axis=1)


def sample_mask(W):
    """Zones that are training samples: positive scales and a nonzero slope magnitude."""
    nv = W.shape[1]
    Wf = W.reshape(W.shape[0], nv, -1)
    _, g = _slopes(W)
    return (Wf[0, 0] > 0) & (Wf[0, 4] > 0) & (g > MAG_MIN)


def features(W, dt, dx):
    """Features (n_zones, n_in) from the third-order spatial modes W (10, nvar, *grid), modal order of Eq. 33.

    Rows of uniform zones (g = 0) keep r unscaled (all zero)."""
    nv = W.shape[1]
    Wf = W.reshape(W.shape[0], nv, -1)
    _, c = _scales(Wf, nv == 8)
    r, g = _slopes(W)
    inv = np.where(g > 0, 1.0 / np.where(g > 0, g, 1.0), 0.0)
    cols = [r * inv[:, None], _means(W)] + [(c * dt / dx[d])[:, None] for d in range(3)] + [g[:, None]]
    return np.concatenate(cols, axis=1)


def targets(W, Uhat, dt, dx):
    """Targets (n_zones, 5 nvar): the evolutionary modes u_11..u_15 of Uhat (15, nvar, *grid), normalised
    (rows of uniform zones are NaN: they are no samples)."""
    nv = W.shape[1]
    mhd = nv == 8
    Wf = W.reshape(W.shape[0], nv, -1)
    Uf = Uhat.reshape(Uhat.shape[0], nv, -1)
    s, c = _scales(Wf, mhd)
    _, g = _slopes(W)
    sigma = c * (dt / dx[0] + dt / dx[1] + dt / dx[2])
    cols = []
    with np.errstate(divide="ignore", invalid="ignore"):
        for j in range(5):
            for v in range(nv):
                cols.append(Uf[10 + j, v] / (s[v] * sigma * g))
    return np.stack(cols, axis=1)


def guess_modes(P, W, dt, dx):
    """The network's evolutionary modes (5, nvar, *grid) for spatial modes W, undoing the normalisation;
    zero for uniform zones."""
    nv = W.shape[1]
    mhd = nv == 8
    n_in, H, n_out, _ = shape(mhd)
    Wf = W.reshape(W.shape[0], nv, -1)
    s, c = _scales(Wf, mhd)
    _, g = _slopes(W)
    sigma = c * (dt / dx[0] + dt / dx[1] + dt / dx[2])
    y = forward(P, features(W, dt, dx), n_out, H)
    out = np.empty((5, nv, Wf.shape[2]))
    for j in range(5):
        for v in range(nv):
            out[j, v] = np.where(g > MAG_MIN, y[:, j * nv + v] * s[v] * sigma * g, 0.0)
    return out.reshape((5, nv) + W.shape[2:])


def init_params(n_in, n_out, seed, H=HIDDEN):
    """Seeded initial parameters: N(0, 1/fan_in) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((H, n_in)) / np.sqrt(n_in), np.zeros(H),
             rng.standard_normal((H, H)) / np.sqrt(H), np.zeros(H),
             rng.standard_normal((n_out, H)) / np.sqrt(H), np.zeros(n_out)]
    return np.concatenate([p.ravel() for p in parts])
