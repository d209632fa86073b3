"""GPU: the learned initial guess for ideal MHD (eight variables), through the C ABI, against the FP64 oracle.

The MHD network takes 82 features (72 normalised slopes of the eight variables, six normalised means, three
Courant numbers, the slope magnitude) and predicts 40 normalised evolutionary modes.  The samples, the
tensor-core guess and the gradient are checked against the oracle; a network trained on magnetised random
states must save predictor iterations on an unseen one without changing the converged result.
"""
import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import mlp as omlp
from oracle import predictor, scheme
from paper_1006_2146_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _solver(ader, n, **kw):
    return ader.Solver((n, n, n), order=3, gamma=GAMMA, mhd=True, **kw)


def _dt(U, B, n, frac=0.8):
    return frac * scheme.max_dt(U, (1.0 / n,) * 3, 0.4, gamma=GAMMA, Bface=B)


def test_mhd_guess_samples_match_oracle(ader):
    import torch
    n = 10
    U, B = inputs.random_magnetised(n, seed=81, amp=0.3, b_amp=0.5)
    dx = (1.0 / n,) * 3
    dt = _dt(U, B, n)
    n_in, _, n_out, _ = ader.ader_mlp_shape(True)
    assert (n_in, n_out) == (82, 40)
    N = n ** 3
    s = _solver(ader, n, form="modal")
    s.set_predictor(TOL, 50)
    X = torch.zeros((N, n_in), dtype=torch.float32, device="cuda")
    Y = torch.zeros((N, n_out), dtype=torch.float32, device="cuda")
    ok = torch.zeros(N, dtype=torch.int32, device="cuda")
    ader.ader_guess_samples(s.h, to_dev(U), to_dev(B), dt, X, Y, ok)
    torch.cuda.synchronize()
    s.close()
    _, W = scheme.zone_state(U, B, 3)
    Uhat, _ = predictor.predict(W, 3, "modal", GAMMA, dt, dx, tol=TOL)
    Xw = omlp.features(W, dt, dx)
    Yw = omlp.targets(W, Uhat, dt, dx)
    mask = omlp.sample_mask(W)
    assert mask.all()
    np.testing.assert_array_equal(ok.cpu().numpy() == 1, mask)
    np.testing.assert_allclose(X.cpu().numpy(), Xw, rtol=2e-7, atol=1e-7)
    np.testing.assert_allclose(Y.cpu().numpy(), Yw, rtol=2e-7, atol=2e-7 * np.abs(Yw).max())


def test_mhd_mlp_gradient_matches_oracle_backprop(ader):
    import torch
    n_in, _, n_out, npar = ader.ader_mlp_shape(True)
    P = omlp.init_params(n_in, n_out, seed=17)
    P += 0.02 * np.random.default_rng(18).standard_normal(npar)
    rng = np.random.default_rng(19)
    X = rng.standard_normal((257, n_in)).astype(np.float32)
    Y = rng.standard_normal((257, n_out)).astype(np.float32)
    P32 = P.astype(np.float32)
    grad = torch.zeros(npar, dtype=torch.float32, device="cuda")
    loss = ader.ader_mlp_grad(torch.from_numpy(P32).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(),
                              257, grad, mhd=True)
    want_loss, want = omlp.loss_and_grad(P32.astype(np.float64), X, Y)
    got = grad.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(want_loss, rel=1e-5)
    H = 128
    bounds = np.cumsum([0, H * n_in, H, H * H, H, n_out * H, n_out])
    for b in range(6):
        g, w = got[bounds[b]:bounds[b + 1]], want[bounds[b]:bounds[b + 1]]
        assert np.linalg.norm(g - w) <= 1e-4 * np.linalg.norm(w), b


@pytest.fixture(scope="module")
def trained_mhd_guess(ader):
    """MHD guess parameters trained on the samples of three seeded magnetised 20^3 states."""
    import torch
    n = 20
    n_in, _, n_out, _ = ader.ader_mlp_shape(True)
    N = n ** 3
    s = _solver(ader, n, form="modal")
    s.set_predictor(TOL, 50)
    Xs, Ys = [], []
    for seed, amp, b_amp in ((91, 0.3, 0.5), (92, 0.2, 0.3), (93, 0.35, 0.8)):
        U, B = inputs.random_magnetised(n, seed=seed, amp=amp, b_amp=b_amp)
        dt = _dt(U, B, n)
        X = torch.zeros((N, n_in), dtype=torch.float32, device="cuda")
        Y = torch.zeros((N, n_out), dtype=torch.float32, device="cuda")
        ok = torch.zeros(N, dtype=torch.int32, device="cuda")
        ader.ader_guess_samples(s.h, to_dev(U), to_dev(B), dt, X, Y, ok)
        keep = ok.bool()
        Xs.append(X[keep])
        Ys.append(Y[keep])
    s.close()
    X = torch.cat(Xs).contiguous()
    Y = torch.cat(Ys).contiguous()
    P = torch.from_numpy(omlp.init_params(n_in, n_out, seed=21).astype(np.float32)).cuda()
    losses = ader.ader_mlp_train(X, Y, X.shape[0], P, epochs=40, batch=512, lr=2e-3, seed=6, mhd=True)
    assert losses[-1] < 0.5 * losses[0]
    return P


@pytest.mark.parametrize("fp32", [False, True])
def test_mhd_tensor_core_guess_matches_oracle(ader, trained_mhd_guess, fp32):
    """The step's guess kernel for eight variables against the FP64 numpy network on the oracle's features."""
    import torch
    n = 12
    U, B = inputs.random_magnetised(n, seed=94, amp=0.3, b_amp=0.5)
    dx = (1.0 / n,) * 3
    dt = _dt(U, B, n)
    N = n ** 3
    s = _solver(ader, n, form="modal", fp32=fp32)
    s.set_guess(trained_mhd_guess)
    G = torch.full((40, N), 7.0, dtype=torch.float32, device="cuda")
    ader.ader_guess_eval(s.h, to_dev(U), to_dev(B), dt, G)
    assert s.status() == 0
    s.close()
    _, W = scheme.zone_state(U, B, 3)
    want = omlp.guess_modes(trained_mhd_guess.cpu().numpy().astype(np.float64), W, dt, dx)
    assert omlp.sample_mask(W).all()
    g = G.cpu().numpy()
    w = want.reshape(40, N)
    err = np.linalg.norm(g - w) / np.linalg.norm(w)
    print("MHD tensor-core guess relative L2 error vs FP64 network: %.3e" % err)
    assert err <= 2e-2


@pytest.mark.parametrize("form", ["modal", "nodal"])
def test_mhd_learned_guess_saves_iterations(ader, trained_mhd_guess, form):
    """An unseen magnetised state: the converged result equals the oracle's and the predictor needs fewer
    iterations from the learned guess than from zero."""
    n = 16
    U, B = inputs.random_magnetised(n, seed=95, amp=0.3, b_amp=0.5)
    dx = (1.0 / n,) * 3
    dt = _dt(U, B, n)
    want_U, want_B = scheme.ader_step(U, dx, dt, 3, form, "hll", gamma=GAMMA, Bface=B, tol=TOL)
    res = {}
    for use in (False, True):
        s = _solver(ader, n, form=form)
        s.set_predictor(TOL, 50)
        if use:
            s.set_guess(trained_mhd_guess)
        d, b = to_dev(U), to_dev(B)
        s.step(d, dt, Bface=b)
        assert s.status() == 0
        res[use] = (s.predictor_stats(), to_host(d), to_host(b))
        s.close()
    (tot0, _, cap0), U0, B0 = res[False]
    (tot1, _, cap1), U1, B1 = res[True]
    assert cap0 == cap1 == 0
    for Ug, Bg in ((U0, B0), (U1, B1)):
        assert rel_l1(Ug, want_U) <= 1e-12
        assert np.abs(Bg - want_B).sum() <= 1e-12 * np.abs(want_B).sum()
    print("MHD predictor iterations (%s): zero start %d, learned guess %d" % (form, tot0, tot1))
    assert tot1 < tot0, (tot0, tot1)
