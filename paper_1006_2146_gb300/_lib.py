"""ctypes binding of libader_gb300.so (include/ader.h): argument marshalling only.

The functions keep the C names.  Device arrays are passed as torch CUDA
tensors (float64, contiguous, the layout of ader.h); streams as
torch.cuda.Stream or None (the current stream).  Every numerical step runs in
the library's CUDA kernels; there is no fallback: a missing library raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libader_gb300.so")

ADER_HLL, ADER_LINEARIZED = 0, 1
ADER_MHD, ADER_NODAL, ADER_FP32_BULK, ADER_CONVERGED_PREDICTOR, ADER_EMF_TRANSONIC = 1, 2, 4, 16, 32
ADER_POSITIVITY_FALLBACK = 64
ADER_OK, ADER_ERR_ARG, ADER_ERR_CUDA, ADER_ERR_UNPHYSICAL, ADER_ERR_NONFINITE, ADER_ERR_NOT_CONVERGED = 0, -1, -2, -3, -4, -5
ADER_ERR_TIMEOUT = -6
ADER_SOURCE_NONE, ADER_SOURCE_LINEAR, ADER_SOURCE_GRAVITY = 0, 1, 2
ADER_BC_PERIODIC, ADER_BC_OUTFLOW, ADER_BC_REFLECTIVE = 0, 1, 2

EXPORTS = ("ader_create", "ader_step", "ader_step_devdt", "ader_max_dt", "ader_rk_step", "ader_step_host",
           "ader_diagnostics", "ader_sync_status", "ader_launches_per_step", "ader_profile", "ader_profile_reset",
           "ader_profile_read", "ader_set_tiled", "ader_set_boundary", "ader_set_predictor", "ader_predictor_stats", "ader_set_source", "ader_set_dense_output", "ader_dense_output", "ader_set_guess",
           "ader_mlp_shape", "ader_guess_samples", "ader_guess_count", "ader_guess_eval", "ader_test_bounded_wait", "ader_trim_local_memory", "ader_mlp_train", "ader_mlp_grad", "ader_last_error", "ader_destroy",
           "ader_max_dt_static", "ader_batch_create", "ader_batch_tune", "ader_batch_step", "ader_batch_advance",
           "ader_batch_status", "ader_batch_tuning", "ader_batch_groups", "ader_batch_last_error",
           "ader_batch_destroy")


class AderError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ADER error %d: %s" % (code, msg))
        self.code = code


class ader_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


_LIB = None


def load(path=None):
    """Load the shared library (build it first with paper_1006_2146_gb300.build.build())."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libader_gb300.so not found at %s: run __graft_entry__.build() (nvcc, sm_103a)" % p)
    lib = ctypes.CDLL(p)
    vp, dbl, i32, u32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_uint
    lib.ader_create.argtypes = [ctypes.POINTER(ader_grid), i32, dbl, i32, u32, ctypes.POINTER(vp)]
    lib.ader_step.argtypes = [vp, vp, vp, dbl, vp]
    lib.ader_step_devdt.argtypes = [vp, vp, vp, vp, vp]
    lib.ader_max_dt.argtypes = [vp, vp, vp, dbl, vp, vp]
    lib.ader_rk_step.argtypes = [vp, vp, vp, dbl, vp]
    lib.ader_step_host.argtypes = [vp, vp, vp, dbl, ctypes.POINTER(dbl)]
    lib.ader_diagnostics.argtypes = [vp, vp, vp, vp, vp]
    lib.ader_sync_status.argtypes = [vp, vp]
    lib.ader_launches_per_step.argtypes = [vp]
    lib.ader_profile.argtypes = [vp, i32]
    lib.ader_profile_reset.argtypes = [vp]
    lib.ader_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32),
                                      ctypes.POINTER(dbl), i32]
    lib.ader_set_tiled.argtypes = [vp, i32]
    lib.ader_set_boundary.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.ader_set_predictor.argtypes = [vp, dbl, i32]
    lib.ader_predictor_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong), vp]
    lib.ader_set_guess.argtypes = [vp, vp]
    lib.ader_set_source.argtypes = [vp, ctypes.c_int, vp]
    lib.ader_set_dense_output.argtypes = [vp, ctypes.c_int]
    lib.ader_dense_output.argtypes = [vp, ctypes.c_double, vp, vp]
    lib.ader_guess_count.argtypes = [vp, vp, vp]
    lib.ader_mlp_shape.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(ctypes.c_longlong)]
    lib.ader_guess_samples.argtypes = [vp, vp, vp, dbl, vp, vp, vp, vp]
    lib.ader_guess_eval.argtypes = [vp, vp, vp, dbl, vp, vp]
    lib.ader_test_bounded_wait.argtypes = [vp]
    lib.ader_trim_local_memory.argtypes = [ctypes.POINTER(ctypes.c_size_t)]
    lib.ader_mlp_train.argtypes = [vp, vp, ctypes.c_longlong, i32, i32, i32, ctypes.c_float, ctypes.c_ulonglong,
                                   vp, ctypes.POINTER(dbl), vp]
    lib.ader_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_longlong, i32, vp, ctypes.POINTER(dbl), vp]
    lib.ader_last_error.argtypes = [vp]
    lib.ader_last_error.restype = ctypes.c_char_p
    lib.ader_destroy.argtypes = [vp]
    lib.ader_destroy.restype = None
    lib.ader_max_dt_static.argtypes = [ctypes.POINTER(ader_grid), dbl, vp, dbl, vp, vp]
    pp = ctypes.POINTER(vp)
    lib.ader_batch_create.argtypes = [i32, ctypes.POINTER(ader_grid), ctypes.POINTER(i32), ctypes.POINTER(dbl),
                                      ctypes.POINTER(i32), ctypes.POINTER(u32), ctypes.POINTER(vp)]
    lib.ader_batch_tune.argtypes = [vp, pp, pp, vp]
    lib.ader_batch_step.argtypes = [vp, pp, pp, vp, vp]
    lib.ader_batch_advance.argtypes = [vp, pp, pp, dbl, vp, vp]
    lib.ader_batch_status.argtypes = [vp, ctypes.POINTER(i32), vp]
    lib.ader_batch_tuning.argtypes = [vp, ctypes.POINTER(i32), i32]
    lib.ader_batch_groups.argtypes = [vp]
    lib.ader_batch_last_error.argtypes = [vp]
    lib.ader_batch_last_error.restype = ctypes.c_char_p
    lib.ader_batch_destroy.argtypes = [vp]
    lib.ader_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("ader_destroy", "ader_last_error", "ader_batch_destroy", "ader_batch_last_error"):
            getattr(lib, name).restype = i32
    if path is None:
        _LIB = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _stream(s):
    if s is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def _check(h, rc):
    if rc != ADER_OK:
        msg = load().ader_last_error(h).decode() if h else "invalid argument"
        raise AderError(rc, msg)
    return rc


def ader_create(nx, ny, nz, dx, dy, dz, order=3, gamma=1.4, solver=ADER_HLL, flags=0):
    g = ader_grid(nx, ny, nz, dx, dy, dz)
    h = ctypes.c_void_p()
    rc = load().ader_create(ctypes.byref(g), order, gamma, solver, flags, ctypes.byref(h))
    if rc != ADER_OK:
        raise AderError(rc, "ader_create failed (arguments or device memory)")
    return h


def ader_step(h, U, Bface, dt, stream=None):
    return _check(h, load().ader_step(h, _ptr(U), _ptr(Bface), float(dt), _stream(stream)))


def ader_step_devdt(h, U, Bface, dt_dev, stream=None):
    return _check(h, load().ader_step_devdt(h, _ptr(U), _ptr(Bface), _ptr(dt_dev), _stream(stream)))


def ader_max_dt(h, U, Bface, cfl, dt_dev, stream=None):
    return _check(h, load().ader_max_dt(h, _ptr(U), _ptr(Bface), float(cfl), _ptr(dt_dev), _stream(stream)))


def ader_rk_step(h, U, Bface, dt, stream=None):
    return _check(h, load().ader_rk_step(h, _ptr(U), _ptr(Bface), float(dt), _stream(stream)))


def ader_step_host(h, U_host, Bface_host, cfl):
    """Host-memory step (copies inside); returns the dt used."""
    dt = ctypes.c_double(0.0)
    _check(h, load().ader_step_host(h, _ptr(U_host), _ptr(Bface_host), float(cfl), ctypes.byref(dt)))
    return dt.value


def ader_diagnostics(h, U, Bface, totals_dev, stream=None):
    return _check(h, load().ader_diagnostics(h, _ptr(U), _ptr(Bface), _ptr(totals_dev), _stream(stream)))


def ader_sync_status(h, stream=None):
    """Returns the status code (does not raise on device flags)."""
    return load().ader_sync_status(h, _stream(stream))


def ader_launches_per_step(h):
    return load().ader_launches_per_step(h)


def ader_profile(h, enable=True):
    return _check(h, load().ader_profile(h, 1 if enable else 0))


def ader_profile_reset(h):
    return _check(h, load().ader_profile_reset(h))


def ader_profile_read(h):
    """{kernel name: (launches, total device ms)} of the traced launches so far."""
    cap = 32
    names = (ctypes.c_char_p * cap)()
    counts = (ctypes.c_int * cap)()
    ms = (ctypes.c_double * cap)()
    n = load().ader_profile_read(h, names, counts, ms, cap)
    if n < 0:
        _check(h, n)
    return {names[k].decode(): (counts[k], ms[k]) for k in range(min(n, cap))}


def ader_set_tiled(h, on):
    """Euler launch layout: 1 = per-tile predictor and face solves (default), 0 = face data through memory."""
    return _check(h, load().ader_set_tiled(h, 1 if on else 0))


def ader_set_boundary(h, bc):
    """Box faces (x-, x+, y-, y+, z-, z+), each ADER_BC_PERIODIC, ADER_BC_OUTFLOW or ADER_BC_REFLECTIVE."""
    arr = (ctypes.c_int * 6)(*[int(b) for b in bc])
    return _check(h, load().ader_set_boundary(h, arr))


def ader_set_predictor(h, tol, max_iter):
    """Converged predictor: iterate each zone until its change is below tol (tol 0: fixed count)."""
    return _check(h, load().ader_set_predictor(h, float(tol), int(max_iter)))


def ader_predictor_stats(h, stream=None):
    """(sum of iterations over zones and steps, largest count, zones capped) since the last read."""
    out = (ctypes.c_ulonglong * 3)()
    _check(h, load().ader_predictor_stats(h, out, _stream(stream)))
    return tuple(int(v) for v in out)


def ader_set_source(h, kind, params=None):
    """Non-stiff source of Eq. 4: ADER_SOURCE_LINEAR (params (k,)), ADER_SOURCE_GRAVITY ((gx, gy, gz)) or
    ADER_SOURCE_NONE; params are copied by the library."""
    arr = None
    if params is not None:
        vals = [float(v) for v in params]
        arr = (ctypes.c_double * len(vals))(*vals)
    return _check(h, load().ader_set_source(h, int(kind), arr))


def ader_set_dense_output(h, enable):
    """Keep (True) or drop (False) every later step's space-time modes for ader_dense_output."""
    return _check(h, load().ader_set_dense_output(h, 1 if enable else 0))


def ader_dense_output(h, tau, out, stream=None):
    """The LS spatial modes at t^n + tau dt of the last kept step into out (device FP64, (LS, nvar) + grid)."""
    return _check(h, load().ader_dense_output(h, float(tau), _ptr(out), _stream(stream)))


def ader_guess_count(h, stream=None):
    """Zones the network ran on in the last guess launch (synchronises the stream)."""
    out = ctypes.c_ulonglong()
    _check(h, load().ader_guess_count(h, ctypes.byref(out), _stream(stream)))
    return int(out.value)


def ader_set_guess(h, params):
    """Start the predictor from the MLP guess (FP32 device parameters, kept by pointer); None disables it."""
    return _check(h, load().ader_set_guess(h, _ptr(params)))


def ader_mlp_shape(mhd=False):
    """(n_in, n_hidden, n_out, n_params) of the guess MLP."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    d = ctypes.c_longlong()
    _check(None, load().ader_mlp_shape(1 if mhd else 0, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                       ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def ader_guess_samples(h, U, Bface, dt, X, Y, ok, stream=None):
    return _check(h, load().ader_guess_samples(h, _ptr(U), _ptr(Bface), float(dt), _ptr(X), _ptr(Y), _ptr(ok),
                                               _stream(stream)))


def ader_trim_local_memory():
    """Per-thread stack back to 1 KB; returns the size the context held before (bytes)."""
    kept = ctypes.c_size_t(0)
    rc = load().ader_trim_local_memory(ctypes.byref(kept))
    if rc != ADER_OK:
        raise AderError(rc, "the CUDA runtime refused the stack limit")
    return kept.value


def ader_test_bounded_wait(h):
    """Arm the next learned-guess launch to let its tensor-core barrier wait run out (ADER_ERR_TIMEOUT)."""
    return _check(h, load().ader_test_bounded_wait(h))


def ader_guess_eval(h, U, Bface, dt, G, stream=None):
    """Every zone's guessed evolutionary modes into G (device, 5*nvar x zones FP32) by the step's guess kernel."""
    return _check(h, load().ader_guess_eval(h, _ptr(U), _ptr(Bface), float(dt), _ptr(G), _stream(stream)))


def ader_mlp_train(X, Y, n, params, epochs, batch, lr, seed=0, mhd=False, stream=None):
    """Adam on the MSE in place on params; returns the last minibatch loss of each epoch."""
    losses = (ctypes.c_double * epochs)()
    _check(None, load().ader_mlp_train(_ptr(X), _ptr(Y), int(n), 1 if mhd else 0, int(epochs), int(batch),
                                       float(lr), int(seed), _ptr(params), losses, _stream(stream)))
    return list(losses)


def ader_mlp_grad(params, X, Y, n, grad, mhd=False, stream=None):
    """Mean-squared error of the MLP on (X, Y) and its gradient into grad (device); returns the loss."""
    loss = ctypes.c_double()
    _check(None, load().ader_mlp_grad(_ptr(params), _ptr(X), _ptr(Y), int(n), 1 if mhd else 0, _ptr(grad),
                                      ctypes.byref(loss), _stream(stream)))
    return loss.value


def ader_last_error(h):
    return load().ader_last_error(h).decode()


def ader_destroy(h):
    if h:
        load().ader_destroy(h)


# ----------------------------------------------------------------------------- batched problems
def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = None if t is None else t.data_ptr()
    return arr


def _bcheck(b, rc):
    if rc != ADER_OK:
        msg = load().ader_batch_last_error(b).decode() if b else "invalid argument"
        raise AderError(rc, msg)
    return rc


def ader_batch_create(grids, orders, gammas, solvers, flags):
    """grids: list of (nx, ny, nz, dx, dy, dz); the other arguments: one entry per problem."""
    n = len(grids)
    G = (ader_grid * n)(*[ader_grid(*g) for g in grids])
    O = (ctypes.c_int * n)(*orders)
    Gm = (ctypes.c_double * n)(*gammas)
    S = (ctypes.c_int * n)(*solvers)
    F = (ctypes.c_uint * n)(*flags)
    b = ctypes.c_void_p()
    rc = load().ader_batch_create(n, G, O, Gm, S, F, ctypes.byref(b))
    if rc != ADER_OK:
        raise AderError(rc, "ader_batch_create failed (arguments or device memory)")
    return b


def ader_batch_tune(b, Us, Bs, stream=None):
    return _bcheck(b, load().ader_batch_tune(b, _ptrs(Us), _ptrs(Bs), _stream(stream)))


def ader_batch_step(b, Us, Bs, dt_dev, stream=None):
    return _bcheck(b, load().ader_batch_step(b, _ptrs(Us), _ptrs(Bs), _ptr(dt_dev), _stream(stream)))


def ader_batch_advance(b, Us, Bs, cfl, dt_dev=None, stream=None):
    return _bcheck(b, load().ader_batch_advance(b, _ptrs(Us), _ptrs(Bs), float(cfl), _ptr(dt_dev), _stream(stream)))


def ader_batch_status(b, n, stream=None):
    """(worst code, per-problem codes); synchronises the stream."""
    codes = (ctypes.c_int * n)()
    rc = load().ader_batch_status(b, codes, _stream(stream))
    return rc, list(codes)


def ader_batch_tuning(b):
    """[(group, phase, threads, blocks)] chosen by ader_batch_tune (blocks 0: one block per `threads` zones)."""
    cap = 4 * 512
    out = (ctypes.c_int * cap)()
    k = load().ader_batch_tuning(b, out, cap)
    return [tuple(out[4 * i:4 * i + 4]) for i in range(min(k, cap // 4))]


def ader_batch_groups(b):
    return load().ader_batch_groups(b)


def ader_batch_destroy(b):
    if b:
        load().ader_batch_destroy(b)
