"""Running a problem: checkpoint/resume and per-step metrics (JSON lines), over the C ABI.

The paper runs its tests from t = 0 to the end in one go and logs nothing; these are conveniences of the
library, with no arithmetic of the method in them:

* ``save_checkpoint`` / ``load_checkpoint``: the state of a run is (U, Bface, t, step) plus, when a learned
  guess is in use, its network parameters.  The file is a ``torch.save`` of CPU tensors; a resumed run
  that takes the same steps reproduces the uninterrupted run bit for bit (the step is deterministic:
  no atomics decide any value of U or Bface).
* ``StepLog``: one JSON object per logged step -- step, t, dt, the conservation totals (and, for MHD, the
  face-field totals and the largest relative div B) from ``ader_diagnostics``, the smallest density and
  pressure, and the converged predictor's iteration counts since the previous line.
* ``advance``: CFL-limited steps (``ader_max_dt`` on the device, then ``ader_step_devdt``) to a final time,
  logging and checkpointing on request.
"""
import json
import os

from . import _lib

FORMAT = 1


def save_checkpoint(path, U, Bface=None, t=0.0, step=0, guess=None, meta=None):
    """Write the run state to `path` (device tensors are copied to the host)."""
    import torch
    blob = {"format": FORMAT, "t": float(t), "step": int(step), "meta": dict(meta or {}),
            "U": U.detach().to("cpu").clone(),
            "Bface": None if Bface is None else Bface.detach().to("cpu").clone(),
            "guess": None if guess is None else guess.detach().to("cpu").clone()}
    tmp = path + ".tmp"
    torch.save(blob, tmp)
    os.replace(tmp, path)           # a crash mid-write leaves the previous checkpoint intact


def load_checkpoint(path, device="cuda"):
    """The run state written by save_checkpoint, its tensors on `device`."""
    import torch
    blob = torch.load(path, map_location="cpu", weights_only=False)
    if blob.get("format") != FORMAT:
        raise ValueError("%s: unknown checkpoint format %r" % (path, blob.get("format")))
    out = dict(blob)
    for k in ("U", "Bface", "guess"):
        if out[k] is not None:
            out[k] = out[k].to(device)
    return out


class StepLog:
    """Appends one JSON object per logged step to `path` (``None``: keep the records in ``records``)."""

    def __init__(self, path=None, gamma=1.4):
        self.path = path
        self.gamma = gamma
        self.records = []

    def log(self, solver, U, Bface, step, t, dt, stream=None):
        import torch
        nv = 9 if Bface is not None else 5
        tot = torch.zeros(nv, dtype=torch.float64, device=U.device)
        _lib.ader_diagnostics(solver.h, U, Bface, tot, stream)
        rho = U[0]
        ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
        me = 0.0
        if Bface is not None:       # zone field: the mean of the two faces of each direction
            bz = [0.5 * (Bface[d] + torch.roll(Bface[d], -1, dims=2 - d)) for d in range(3)]
            me = (bz[0] ** 2 + bz[1] ** 2 + bz[2] ** 2) / (8.0 * 3.141592653589793)
        P = (self.gamma - 1.0) * (U[4] - ke - me)
        stats = _lib.ader_predictor_stats(solver.h, stream)
        tl = tot.tolist()
        rec = {"step": int(step), "t": float(t), "dt": float(dt), "totals": tl[:5],
               "rho_min": float(rho.min()), "p_min": float(P.min()),
               "predictor_iterations": stats[0], "predictor_max": stats[1], "predictor_capped": stats[2]}
        if Bface is not None:
            rec["face_b_totals"] = tl[5:8]
            rec["div_b_rel_max"] = tl[8]
        self.records.append(rec)
        if self.path:
            with open(self.path, "a") as fh:
                fh.write(json.dumps(rec) + "\n")
        return rec


def advance(solver, U, t_end, cfl=0.4, Bface=None, t=0.0, step=0, max_steps=None, log=None, log_every=1,
            checkpoint=None, checkpoint_every=0, guess=None, stream=None):
    """CFL-limited ADER steps from t to t_end (the last step is shortened to land on t_end).

    Returns (t, step).  `log` is a StepLog; `checkpoint` a path written every `checkpoint_every` steps
    and at the end."""
    import torch
    dtv = torch.zeros(1, dtype=torch.float64, device=U.device)
    n = 0
    while t < t_end and (max_steps is None or n < max_steps):
        _lib.ader_max_dt(solver.h, U, Bface, cfl, dtv, stream)
        dt = min(float(dtv.item()), t_end - t)
        _lib.ader_step(solver.h, U, Bface, dt, stream)
        rc = _lib.ader_sync_status(solver.h, stream)
        if rc != _lib.ADER_OK:
            raise _lib.AderError(rc, _lib.ader_last_error(solver.h))
        t += dt
        step += 1
        n += 1
        if log is not None and step % log_every == 0:
            log.log(solver, U, Bface, step, t, dt, stream)
        if checkpoint and checkpoint_every and step % checkpoint_every == 0:
            save_checkpoint(checkpoint, U, Bface, t, step, guess)
    if checkpoint:
        save_checkpoint(checkpoint, U, Bface, t, step, guess)
    return t, step
