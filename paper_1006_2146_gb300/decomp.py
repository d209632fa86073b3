"""Domain decomposition of the Euler step along z: one halo exchange per step (Sec. II).

The one-step ADER scheme reads its neighbours' zone averages once per step: the reconstruction, the
local space-time predictor and the face fluxes of a step all start from U^n (an SSP-RK step of the same
order needs one exchange per stage).  A decomposed run gives each part a slab of z planes plus G ghost
planes below and above it, G being a step's reach (3 zones at orders 2-3, 4 at order 4):

* before a step every part receives the G planes next to its slab from its two neighbours (the global
  domain is periodic in z, so the first part's lower neighbour is the last part);
* dt is the smallest of the parts' CFL steps (an all-reduce MIN): each part takes its maximum signal speed
  over its padded slab, whose planes all belong to the global state, so the minimum is the single-domain
  dt exactly;
* every part steps its padded slab through the C ABI (the kernels treat it as periodic in z; the
  wrap-around stays inside the ghost planes) and keeps its interior planes.

z is the slowest axis of the (variable, z, y, x) layout, so a part's interior and the planes it sends are
contiguous blocks per variable.  This module holds no arithmetic of the method: it moves planes and
reduces two numbers; the steps, the CFL speeds and the totals run in the library's kernels.

Exchanges: ``LocalExchange`` for all parts in one process (one GPU, or the host), ``DistExchange`` for
one part per rank over ``torch.distributed`` (gloo on the host, NCCL between GPUs).
"""

GHOSTS = {2: 3, 3: 3, 4: 4}


def ghost_planes(order):
    """Planes of reach of one step along z."""
    return GHOSTS[order]


def split(nz, parts):
    """Plane counts of `parts` slabs of an nz-plane domain, as even as possible."""
    base, extra = divmod(nz, parts)
    return [base + (1 if r < extra else 0) for r in range(parts)]


def offsets(counts):
    out, k = [], 0
    for c in counts:
        out.append(k)
        k += c
    return out


class Slab:
    """One part: its padded state (5, nz_r + 2G, ny, nx) and the planes it owns."""

    def __init__(self, U_global_part, G):
        import torch
        nz_r = U_global_part.shape[1]
        if nz_r < G:
            raise ValueError("a part needs at least the ghost width of planes")
        shape = (U_global_part.shape[0], nz_r + 2 * G) + tuple(U_global_part.shape[2:])
        self.G, self.nz = G, nz_r
        self.Upad = torch.empty(shape, dtype=U_global_part.dtype, device=U_global_part.device)
        self.Upad[:, G:G + nz_r] = U_global_part

    @property
    def interior(self):
        return self.Upad[:, self.G:self.G + self.nz]

    def bottom(self):
        """The G lowest interior planes (the lower neighbour's upper ghosts)."""
        return self.Upad[:, self.G:2 * self.G].contiguous()

    def top(self):
        """The G highest interior planes (the upper neighbour's lower ghosts)."""
        return self.Upad[:, self.nz:self.nz + self.G].contiguous()

    def set_ghosts(self, lower, upper):
        self.Upad[:, :self.G] = lower
        self.Upad[:, self.G + self.nz:] = upper


class LocalExchange:
    """Every part in this process: the ghosts come straight from the neighbouring slabs."""

    def fill(self, slabs):
        tops = [s.top() for s in slabs]
        bottoms = [s.bottom() for s in slabs]
        n = len(slabs)
        for r, s in enumerate(slabs):
            s.set_ghosts(tops[(r - 1) % n], bottoms[(r + 1) % n])

    def min(self, x):
        return x

    def sum(self, x):
        return x


class DistExchange:
    """One part per rank of the default torch.distributed group (ranks in z order)."""

    TAG_UP, TAG_DOWN = 11, 12

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    def fill(self, slabs):
        (s,) = slabs
        dist = self.dist
        lo, hi = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        send_up, send_down = s.top(), s.bottom()
        from_lo = send_up.new_empty(send_up.shape)
        from_hi = send_down.new_empty(send_down.shape)
        reqs = [dist.isend(send_up, hi, tag=self.TAG_UP), dist.isend(send_down, lo, tag=self.TAG_DOWN),
                dist.irecv(from_lo, lo, tag=self.TAG_UP), dist.irecv(from_hi, hi, tag=self.TAG_DOWN)]
        for q in reqs:
            q.wait()
        s.set_ghosts(from_lo, from_hi)

    def min(self, x):
        t = x.clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
        return t

    def sum(self, x):
        t = x.clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t


class Decomposed:
    """The parts of one domain held by this process (all of them, or one per rank) and their steps.

    step_fn(slab, dt) advances slab.Upad in place by dt; dt_fn(slab) returns its CFL step as a one-element
    tensor (maximum signal speed over the padded slab); both default to the library's kernels (a context
    per part, for the padded shape).
    """

    def __init__(self, parts, order, exchange, step_fn=None, dt_fn=None, solver_kw=None, dx=None, cfl=0.4):
        self.slabs = [Slab(U, ghost_planes(order)) for U in parts]
        self.ex = exchange
        self.cfl = cfl
        self.solvers = None
        if step_fn is None or dt_fn is None:
            import torch

            from . import Solver
            kw = dict(solver_kw or {})
            self.solvers = []
            for s in self.slabs:
                shape = tuple(s.Upad.shape[1:])
                nzp, ny, nx = shape
                # the same zone widths as the global grid: lengths scale with the padded counts
                lengths = (dx[0] * nx, dx[1] * ny, dx[2] * nzp)
                self.solvers.append(Solver(shape, order=order, lengths=lengths, **kw))
            self._dt = torch.zeros(1, dtype=torch.float64, device=self.slabs[0].Upad.device)
        self.step_fn = step_fn or self._lib_step
        self.dt_fn = dt_fn or self._lib_dt

    def _lib_step(self, slab, dt):
        self.solvers[self.slabs.index(slab)].step(slab.Upad, float(dt))

    def _lib_dt(self, slab):
        out = self._dt.clone()
        self.solvers[self.slabs.index(slab)].max_dt(slab.Upad, self.cfl, out)
        return out

    def step(self):
        """One decomposed step (ghost exchange, global dt, the parts' steps); returns dt."""
        self.ex.fill(self.slabs)
        dts = [self.dt_fn(s) for s in self.slabs]
        dt = dts[0]
        for d in dts[1:]:
            dt = dt.minimum(d)
        dt = float(self.ex.min(dt).reshape(-1)[0])
        for s in self.slabs:
            self.step_fn(s, dt)
        return dt

    def status(self):
        """The library's status of every part (0 when all ran cleanly)."""
        return [s.status() for s in self.solvers] if self.solvers else []

    def close(self):
        for s in self.solvers or []:
            s.close()
