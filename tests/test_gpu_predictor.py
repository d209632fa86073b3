"""GPU: the converged predictor and the learned initial guess, through the C ABI, against the FP64 oracle.

Converged mode iterates each zone until its change falls below tol times the
zone's largest mean; the result is the fixed point of the Picard iteration
(Sec. IV), so any start (zero or the MLP guess) gives the oracle's result to
round-off.  The MLP kernels are checked against the numpy oracle (loss and
gradient), and the trained guess must save iterations on unseen data.
"""
import numpy as np
import pytest

from gpu_util import ensure_built, rel_l1, to_dev, to_host
from oracle import mlp as omlp
from oracle import predictor, scheme
from paper_1006_2146_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def ader():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_1006_2146_gb300 as p
    return p


def _dx(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


@pytest.mark.parametrize("order,form", [(2, "modal"), (3, "modal"), (3, "nodal"), (4, "modal"), (4, "nodal")])
def test_converged_predictor_parity_and_counts(ader, order, form):
    shape = (9, 10, 11)
    U = inputs.random_smooth(shape, seed=300 + order, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    want, iters = scheme.ader_step(U, dx, dt, order, form, "hll", tol=TOL, return_iters=True)
    s = ader.Solver(shape, order=order, form=form)
    s.set_predictor(TOL, 50)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    total, largest, capped = s.predictor_stats()
    got = to_host(d)
    s.close()
    assert rel_l1(got, want) <= 1e-12
    assert capped == 0
    # per-zone stopping decisions sit on round-off only for zones whose change is within an ulp of tol
    assert abs(largest - int(iters.max())) <= 1
    assert abs(total - int(iters.sum())) <= max(2, iters.size // 100)


def test_converged_predictor_cap_reports_not_converged(ader):
    """tol below round-off with a cap of 2: every zone is capped; the state equals two fixed iterations."""
    shape = (9, 10, 11)
    U = inputs.random_smooth(shape, seed=41, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    want = scheme.ader_step(U, dx, dt, 3, "modal", "hll", n_iter=2)
    s = ader.Solver(shape, order=3, form="modal")
    s.set_predictor(1e-30, 2)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == _lib.ADER_ERR_NOT_CONVERGED
    total, largest, capped = s.predictor_stats()
    got = to_host(d)
    s.close()
    assert (total, largest, capped) == (2 * U[0].size, 2, U[0].size)
    assert rel_l1(got, want) <= 1e-12


def test_guess_samples_match_oracle_features_and_targets(ader):
    import torch
    shape = (8, 9, 10)
    U = inputs.random_smooth(shape, seed=51, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    n_in, _, n_out, _ = ader.ader_mlp_shape(False)
    n = U[0].size
    s = ader.Solver(shape, order=3, form="modal")
    s.set_predictor(TOL, 50)
    X = torch.zeros((n, n_in), dtype=torch.float32, device="cuda")
    Y = torch.zeros((n, n_out), dtype=torch.float32, device="cuda")
    ok = torch.zeros(n, dtype=torch.int32, device="cuda")
    ader.ader_guess_samples(s.h, to_dev(U), None, dt, X, Y, ok)
    torch.cuda.synchronize()
    s.close()
    _, W = scheme.zone_state(U, None, 3)
    Uhat, _ = predictor.predict(W, 3, "modal", 1.4, dt, dx, tol=TOL)
    Xw = omlp.features(W, dt, dx)
    Yw = omlp.targets(W, Uhat, dt, dx)
    mask = omlp.sample_mask(W)
    assert mask.all()
    np.testing.assert_array_equal(ok.cpu().numpy() == 1, mask)
    np.testing.assert_allclose(X.cpu().numpy(), Xw, rtol=2e-7, atol=1e-7)
    np.testing.assert_allclose(Y.cpu().numpy(), Yw, rtol=2e-7, atol=2e-7 * np.abs(Yw).max())


def test_guess_samples_skip_uniform_zones(ader):
    """A smooth field with a constant band: the zones whose whole stencil lies in the band are uniform to
    round-off and are no samples, the others are.  (A planar Sod tube is no test of this: its WENO slopes
    vanish in every zone.)"""
    import torch
    shape = (4, 5, 16)
    U = inputs.random_smooth(shape, seed=71, amp=0.3)
    U[:, :, :, 5:] = U[:, 0:1, 0:1, 5:6]
    dx = _dx(shape)
    dt = 0.5 * scheme.max_dt(U, dx, 0.4)
    n_in, _, n_out, _ = ader.ader_mlp_shape(False)
    n = U[0].size
    s = ader.Solver(shape, order=3, form="modal")
    X = torch.zeros((n, n_in), dtype=torch.float32, device="cuda")
    Y = torch.zeros((n, n_out), dtype=torch.float32, device="cuda")
    ok = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    ader.ader_guess_samples(s.h, to_dev(U), None, dt, X, Y, ok)
    torch.cuda.synchronize()
    s.close()
    _, W = scheme.zone_state(U, None, 3)
    mask = omlp.sample_mask(W)
    assert not mask.reshape(shape)[:, :, 7:14].any() and mask.reshape(shape)[:, :, :5].all()
    np.testing.assert_array_equal(ok.cpu().numpy(), mask.astype(np.int32))


def test_mlp_gradient_matches_oracle_backprop(ader):
    """Loss and gradient of the GPU MLP kernels (FP32) against the FP64 oracle, 300 rows (ragged tiles)."""
    import torch
    n_in, _, n_out, npar = ader.ader_mlp_shape(False)
    P = omlp.init_params(n_in, n_out, seed=7)
    P += 0.02 * np.random.default_rng(8).standard_normal(npar)
    rng = np.random.default_rng(9)
    X = rng.standard_normal((300, n_in)).astype(np.float32)
    Y = rng.standard_normal((300, n_out)).astype(np.float32)
    P32 = P.astype(np.float32)
    grad = torch.zeros(npar, dtype=torch.float32, device="cuda")
    loss = ader.ader_mlp_grad(torch.from_numpy(P32).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(),
                              300, grad)
    want_loss, want = omlp.loss_and_grad(P32.astype(np.float64), X, Y)
    got = grad.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(want_loss, rel=1e-5)
    H = 128
    bounds = np.cumsum([0, H * n_in, H, H * H, H, n_out * H, n_out])
    for b in range(6):
        g, w = got[bounds[b]:bounds[b + 1]], want[bounds[b]:bounds[b + 1]]
        assert np.linalg.norm(g - w) <= 1e-4 * np.linalg.norm(w), b


@pytest.fixture(scope="module")
def trained_guess(ader):
    """Guess parameters trained on the samples of three seeded 24^3 states (modal FP64 predictor data)."""
    import torch
    shape = (24, 24, 24)
    dx = _dx(shape)
    n_in, _, n_out, npar = ader.ader_mlp_shape(False)
    n = 24 ** 3
    s = ader.Solver(shape, order=3, form="modal")
    s.set_predictor(TOL, 50)
    Xs, Ys = [], []
    for seed, amp in ((61, 0.3), (62, 0.2), (63, 0.35)):
        U = inputs.random_smooth(shape, seed=seed, amp=amp)
        dt = 0.8 * scheme.max_dt(U, dx, 0.4)
        X = torch.zeros((n, n_in), dtype=torch.float32, device="cuda")
        Y = torch.zeros((n, n_out), dtype=torch.float32, device="cuda")
        ok = torch.zeros(n, dtype=torch.int32, device="cuda")
        ader.ader_guess_samples(s.h, to_dev(U), None, dt, X, Y, ok)
        keep = ok.bool()
        Xs.append(X[keep])
        Ys.append(Y[keep])
    s.close()
    X = torch.cat(Xs).contiguous()
    Y = torch.cat(Ys).contiguous()
    P = torch.from_numpy(omlp.init_params(n_in, n_out, seed=11).astype(np.float32)).cuda()
    losses = ader.ader_mlp_train(X, Y, X.shape[0], P, epochs=40, batch=512, lr=2e-3, seed=5)
    assert losses[-1] < 0.5 * losses[0]
    return P


@pytest.mark.parametrize("fp32", [False, True])
def test_tensor_core_guess_matches_oracle(ader, trained_guess, fp32):
    """The step's guess kernel (tcgen05, FP16 operands, FP32 accumulation) against the FP64 numpy network on the
    oracle's features: within FP16 operand rounding, and exactly zero for zones uniform to round-off."""
    import torch
    shape = (12, 11, 13)
    U = inputs.random_smooth(shape, seed=70, amp=0.3)
    U[:, :, :, 5:] = U[:, 0:1, 0:1, 5:6]              # a constant band: zones 7..10 see no slope at all
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    n = U[0].size
    s = ader.Solver(shape, order=3, form="modal", fp32=fp32)
    s.set_guess(trained_guess)
    G = torch.full((25, n), 7.0, dtype=torch.float32, device="cuda")
    ader.ader_guess_eval(s.h, to_dev(U), None, dt, G)
    assert s.status() == 0
    active = ader.ader_guess_count(s.h)
    s.close()
    got = G.cpu().numpy().reshape(5, 5, *shape)
    _, W = scheme.zone_state(U, None, 3)
    want = omlp.guess_modes(trained_guess.cpu().numpy().astype(np.float64), W, dt, dx)
    mask = omlp.sample_mask(W)
    assert 0 < mask.sum() < n
    g = got.reshape(25, n)
    w = want.reshape(25, n)
    if fp32:    # FP32 moments of uniform data keep round-off slopes: a guess of that size
        assert np.abs(g[:, ~mask]).max() <= 1e-5 * np.abs(w).max()
        assert mask.sum() <= active <= n
    else:
        np.testing.assert_array_equal(g[:, ~mask], 0.0)
        assert active == mask.sum()      # the network ran on the zones with slopes only
    err = np.linalg.norm(g[:, mask] - w[:, mask]) / np.linalg.norm(w[:, mask])
    print("tensor-core guess relative L2 error vs FP64 network: %.3e" % err)
    assert err <= 2e-2


@pytest.mark.parametrize("form", ["modal", "nodal"])
def test_learned_guess_saves_iterations(ader, trained_guess, form):
    """A fourth, unseen state: the converged result is unchanged and the predictor needs fewer iterations."""
    P = trained_guess
    shape2 = (16, 16, 16)
    U = inputs.random_smooth(shape2, seed=64, amp=0.3)
    dx2 = _dx(shape2)
    dt = 0.8 * scheme.max_dt(U, dx2, 0.4)
    want = scheme.ader_step(U, dx2, dt, 3, form, "hll", tol=TOL)
    res = {}
    for use in (False, True):
        s2 = ader.Solver(shape2, order=3, form=form)
        s2.set_predictor(TOL, 50)
        if use:
            s2.set_guess(P)
        d = to_dev(U)
        s2.step(d, dt)
        assert s2.status() == 0
        res[use] = (s2.predictor_stats(), to_host(d))
        s2.close()
    (tot0, _, cap0), got0 = res[False]
    (tot1, _, cap1), got1 = res[True]
    assert cap0 == cap1 == 0
    assert rel_l1(got0, want) <= 1e-12
    assert rel_l1(got1, want) <= 1e-12
    print("predictor iterations (%s): zero start %d, learned guess %d" % (form, tot0, tot1))
    assert tot1 < tot0, (tot0, tot1)


def test_fp32_learned_guess_ten_steps(ader, trained_guess):
    """FP32 bulk, converged predictor (tol 1e-6) started from the learned guess: within 1e-5 relative L1 of
    the FP64 converged oracle after 10 steps (nodal, third order, HLL)."""
    shape = (16, 16, 16)
    dx = _dx(shape)
    U = inputs.random_smooth(shape, seed=65, amp=0.3)
    s = ader.Solver(shape, order=3, form="nodal", fp32=True)
    s.set_predictor(1e-6, 50)
    s.set_guess(trained_guess)
    d = to_dev(U)
    Uo = U.copy()
    for _ in range(10):
        dt = scheme.max_dt(Uo, dx, 0.4)
        Uo = scheme.ader_step(Uo, dx, dt, 3, "nodal", "hll", tol=TOL)
        s.step(d, dt)
    assert s.status() == 0
    tot, mx, capped = s.predictor_stats()
    s.close()
    assert capped == 0
    assert rel_l1(to_host(d), Uo) <= 1e-5


@pytest.mark.parametrize("fp32", [False, True])
def test_bounded_tensor_core_wait_runs_out_and_the_context_recovers(ader, trained_guess, fp32):
    """Failure detection without a GPU fault: an armed guess launch issues no MMA for its first layer, so the
    barrier it waits on never completes; the bounded wait gives up, the step status is ADER_ERR_TIMEOUT, and
    the kernel freed its tensor memory: the next launches on the same context (the guess alone, then a
    converged step from the guess) run normally and match the oracle."""
    import torch
    from paper_1006_2146_gb300 import _lib
    shape = (12, 11, 13)
    U = inputs.random_smooth(shape, seed=71, amp=0.3)
    dx = _dx(shape)
    dt = 0.8 * scheme.max_dt(U, dx, 0.4)
    n = U[0].size
    s = ader.Solver(shape, order=3, form="modal", fp32=fp32)
    s.set_guess(trained_guess)
    G = torch.full((25, n), 7.0, dtype=torch.float32, device="cuda")
    ader.ader_test_bounded_wait(s.h)
    ader.ader_guess_eval(s.h, to_dev(U), None, dt, G)
    assert s.status() == _lib.ADER_ERR_TIMEOUT
    ader.ader_guess_eval(s.h, to_dev(U), None, dt, G)     # not armed any more
    assert s.status() == 0
    s.set_predictor(1e-6 if fp32 else TOL, 50)
    d = to_dev(U)
    s.step(d, dt)
    assert s.status() == 0
    s.close()
    want = scheme.ader_step(U, dx, dt, 3, "modal", "hll", tol=TOL)
    assert rel_l1(to_host(d), want) <= (1e-6 if fp32 else 1e-12)
