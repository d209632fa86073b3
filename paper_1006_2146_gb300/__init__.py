"""GB300-native (sm_103a) one-step ADER-WENO update on 3-D periodic meshes.

The operation is the time step of Balsara, Meyer, Dumbser, Du & Xu,
"Efficient implementation of ADER schemes for Euler and MHD flows on
structured meshes" (arXiv:1006.2146).  The compute runs in the CUDA library
built from csrc/ (C ABI: include/ader.h); this package is its ctypes binding
plus the seeded input generators (``inputs``).
"""
from . import inputs  # noqa: F401
from ._lib import (ADER_BC_OUTFLOW, ADER_BC_PERIODIC, ADER_BC_REFLECTIVE, ADER_CONVERGED_PREDICTOR, ADER_EMF_TRANSONIC, ADER_FP32_BULK, ADER_HLL,  # noqa: F401
                   ADER_LINEARIZED, ADER_MHD, ADER_NODAL, ADER_POSITIVITY_FALLBACK,
                   ADER_SOURCE_GRAVITY, ADER_SOURCE_LINEAR, ADER_SOURCE_NONE,
                   AderError, ader_create, ader_dense_output, ader_destroy, ader_diagnostics, ader_guess_count,
                   ader_guess_eval, ader_guess_samples, ader_last_error, ader_launches_per_step, ader_max_dt,
                   ader_mlp_grad, ader_mlp_shape, ader_mlp_train, ader_predictor_stats, ader_profile,
                   ader_profile_read, ader_profile_reset, ader_rk_step, ader_set_dense_output, ader_set_guess,
                   ader_set_boundary, ader_set_predictor, ader_set_source, ader_set_tiled, ader_step, ader_test_bounded_wait, ader_trim_local_memory, ader_step_devdt, ader_step_host,
                   ader_sync_status, load)


class Solver:
    """One ADER context on the current CUDA device (owns the library scratch).

    mhd=True makes an ideal-MHD context: every call then takes the face field Bface (device, (3, nz, ny, nx)
    FP64), which ader_step and ader_rk_step advance in place by constrained transport.  emf_transonic=True
    doubles the dissipative term of the electric fields at transonic faces (Secs. II.3, V).  positivity=True
    (FP64) re-solves the faces of zones a step leaves non-physical at first order."""

    def __init__(self, shape, order=3, form="modal", solver="hll", gamma=1.4, fp32=False, lengths=(1.0, 1.0, 1.0),
                 mhd=False, emf_transonic=False, positivity=False):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.mhd = mhd
        self.dx = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
        flags = (ADER_NODAL if form == "nodal" else 0) | (ADER_FP32_BULK if fp32 else 0) | (ADER_MHD if mhd else 0) | \
            (ADER_EMF_TRANSONIC if emf_transonic else 0) | (ADER_POSITIVITY_FALLBACK if positivity else 0)
        sol = ADER_HLL if solver == "hll" else ADER_LINEARIZED
        self.h = ader_create(nx, ny, nz, self.dx[0], self.dx[1], self.dx[2], order, gamma, sol, flags)

    def step(self, U, dt, stream=None, Bface=None):
        ader_step(self.h, U, Bface, dt, stream)

    def step_devdt(self, U, dt_dev, stream=None, Bface=None):
        ader_step_devdt(self.h, U, Bface, dt_dev, stream)

    def max_dt(self, U, cfl, dt_dev, stream=None, Bface=None):
        ader_max_dt(self.h, U, Bface, cfl, dt_dev, stream)

    def rk_step(self, U, dt, stream=None, Bface=None):
        ader_rk_step(self.h, U, Bface, dt, stream)

    def set_tiled(self, on):
        ader_set_tiled(self.h, on)

    def set_boundary(self, bc):
        """Box faces (x-, x+, y-, y+, z-, z+): "periodic", "outflow" or "reflective" (or the ADER_BC_* codes)."""
        names = {"periodic": ADER_BC_PERIODIC, "outflow": ADER_BC_OUTFLOW, "reflective": ADER_BC_REFLECTIVE}
        ader_set_boundary(self.h, [names.get(b, b) for b in bc])

    def set_predictor(self, tol, max_iter=50):
        ader_set_predictor(self.h, tol, max_iter)

    def predictor_stats(self, stream=None):
        return ader_predictor_stats(self.h, stream)

    def set_source(self, kind, params=None):
        """Non-stiff source: "linear" with params (k,), "gravity" with (gx, gy, gz), or None to remove it."""
        code = {None: ADER_SOURCE_NONE, "linear": ADER_SOURCE_LINEAR, "gravity": ADER_SOURCE_GRAVITY}[kind]
        ader_set_source(self.h, code, params)

    def set_dense_output(self, enable=True):
        """Keep each later step's space-time polynomial for dense_output (Sec. VII)."""
        ader_set_dense_output(self.h, enable)

    def dense_output(self, tau, out, stream=None):
        """Spatial modes (LS, nvar, nz, ny, nx) FP64 at t^n + tau dt of the last kept step, into out."""
        ader_dense_output(self.h, tau, out, stream)

    def set_guess(self, params):
        ader_set_guess(self.h, params)

    def status(self, stream=None):
        return ader_sync_status(self.h, stream)

    def close(self):
        if getattr(self, "h", None):
            ader_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
