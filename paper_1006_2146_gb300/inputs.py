"""Seeded synthetic inputs (initial states) shared by the tests, the bench and the smoke run.

This module holds no arithmetic of the ADER-WENO method itself: it only
builds zone-averaged conserved states (numpy, FP64) of analytic or seeded
fields on a periodic unit cube, with the shapes of the paper's workloads.

Layout: U has shape (5, n, n, n) = (rho, rho vx, rho vy, rho vz, eps) with the
grid axes ordered (z, y, x); Bface has shape (3, n, n, n), Bface[d][..., i_d]
the face average of B_d on face i_d - 1/2 (x = i * dx for face i).
Units are Gaussian (B^2 / 8 pi in the energy), as in the paper's Eq. 3.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi


def _gauss(npts):
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * x, 0.5 * w          # nodes/weights on [-1/2, 1/2]


def grid_shape(n):
    """(nz, ny, nx) from an int n (cube) or a tuple (nz, ny, nx)."""
    return (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)


def _centres(shape):
    nz, ny, nx = shape
    return ((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx)


def cell_average(fn, n, npts=4):
    """Average of fn(x, y, z) over every zone of the periodic unit cube (tensor Gauss-Legendre)."""
    shape = grid_shape(n)
    xg, wg = _gauss(npts)
    cz, cy, cx = _centres(shape)
    out = 0.0
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            for e, we in zip(xg, wg):
                z = (cz + e / shape[0])[:, None, None]
                y = (cy + b / shape[1])[None, :, None]
                x = (cx + a / shape[2])[None, None, :]
                out = out + wa * wb * we * fn(x, y, z)
    return np.broadcast_to(out, shape).astype(np.float64).copy()


def subsample_average(fn, n, sub=8):
    """Average of a discontinuous fn by sub^3 mid-point samples per zone."""
    shape = grid_shape(n)
    s = (np.arange(sub) + 0.5) / sub - 0.5
    cz, cy, cx = _centres(shape)
    out = np.zeros(shape)
    for a in s:
        for b in s:
            for e in s:
                z = (cz + e / shape[0])[:, None, None]
                y = (cy + b / shape[1])[None, :, None]
                x = (cx + a / shape[2])[None, None, :]
                out += fn(x, y, z)
    return out / sub ** 3


def _cons(rho, v, P, gamma, B=None):
    ke = 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    me = 0.0 if B is None else (B[0] ** 2 + B[1] ** 2 + B[2] ** 2) / (2.0 * FOUR_PI)
    return np.stack([rho, rho * v[0], rho * v[1], rho * v[2], P / (gamma - 1.0) + ke + me])


def density_wave(n, t=0.0, amp=0.2, vel=(1.0, 1.0, 1.0), P=1.0, gamma=1.4, npts=4):
    """rho = 1 + amp sin(2 pi (x + y + z - (vx + vy + vz) t)), uniform v and P (exact translation)."""
    s = vel[0] + vel[1] + vel[2]
    rho = cell_average(lambda x, y, z: 1.0 + amp * np.sin(2 * np.pi * (x + y + z - s * t)), n, npts)
    one = np.ones_like(rho)
    return _cons(rho, [vel[0] * one, vel[1] * one, vel[2] * one], P * one, gamma)


def sod_planar(n, gamma=1.4, normal=(1, 1, 0), left=(1.0, 1.0), right=(0.125, 0.1), sub=8):
    """Planar Sod tube: (rho, P) = left where frac(n.x) < 1/2, else right; at rest.

    The integer normal keeps the problem periodic on the unit cube.
    """
    def ind(x, y, z):
        s = normal[0] * x + normal[1] * y + normal[2] * z
        return ((s - np.floor(s)) < 0.5).astype(np.float64)
    shape = grid_shape(n)
    if normal[2] == 0:
        # uniform in z: average over one z-layer and repeat it
        f = np.broadcast_to(subsample_average(ind, (1,) + shape[1:], sub), shape).copy()
    else:
        f = subsample_average(ind, shape, sub)
    rho = right[0] + (left[0] - right[0]) * f
    P = right[1] + (left[1] - right[1]) * f
    z = np.zeros_like(rho)
    return _cons(rho, [z, z, z], P, gamma)


def blast(n, gamma=1.4, p_in=1000.0, p_out=0.1, radius=0.1, center=(0.5, 0.5, 0.5), sub=4):
    """Hydrodynamic blast (Sec. VIII.3): rho = 1 at rest, P = p_in for r < radius else p_out."""
    def ind(x, y, z):
        r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2
        return (r2 < radius * radius).astype(np.float64)
    f = subsample_average(ind, n, sub)
    P = p_out + (p_in - p_out) * f
    rho = np.ones_like(P)
    z = np.zeros_like(P)
    return _cons(rho, [z, z, z], P, gamma)


def mhd_blast(n, B0=20.0, direction=(1.0, 1.0, 1.0), gamma=1.4, p_in=1000.0, p_out=0.1, radius=0.1, sub=4):
    """MHD blast (Sec. IX.4): the blast of Sec. VIII.3 threaded by the uniform field B0 along `direction`
    (the paper: |B| = 20 along the diagonal, plasma beta 0.00628 outside).  Returns (U, Bface)."""
    B = uniform_field(n, B0, direction)
    return with_field(blast(n, gamma, p_in, p_out, radius, sub=sub), B)


def random_smooth(n, seed, amp=0.1, kmax=None, gamma=1.4, P0=1.0):
    """Seeded Gaussian random fields for rho and v (|k|^-2 spectrum, |k| <= kmax), P = P0."""
    rng = np.random.default_rng(seed)
    shape = grid_shape(n)
    kmax = kmax or max(1, min(shape) // 4)
    kz, ky, kx = np.meshgrid(*(np.fft.fftfreq(m) * m for m in shape), indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    filt = np.where((kk > 0) & (kk <= kmax), 1.0 / np.maximum(kk, 1.0), 0.0)

    def field():
        ph = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        f = np.real(np.fft.ifftn(np.fft.fftn(ph.real) * filt))
        return f / (np.abs(f).max() + 1e-300)
    rho = 1.0 + amp * field()
    v = [amp * field() for _ in range(3)]
    P = P0 * np.ones_like(rho)
    return _cons(rho, v, P, gamma)


# ----------------------------------------------------------------------------- MHD
def _edge_line_average(A, n, npts, d):
    """Average of the component A_d along every edge parallel to direction d.

    Edge (i, j, k) of direction d starts at the grid node x = (i, j, k)/n and
    spans one zone along d.  Returns an (n, n, n) array indexed [k, j, i].
    """
    xg, wg = _gauss(npts)
    idx = np.arange(n) / n
    out = 0.0
    for s, w in zip(xg, wg):
        pos = [idx, idx, idx]
        pos = [p.copy() for p in pos]
        pos[d] = idx + (s + 0.5) / n
        z = pos[2][:, None, None]
        y = pos[1][None, :, None]
        x = pos[0][None, None, :]
        out = out + w * A(x, y, z)
    return np.broadcast_to(out, (n, n, n)).astype(np.float64).copy()


def face_field_from_potential(Acomp, n, npts=6):
    """Face-averaged B = curl A by Stokes' theorem over each face (divergence-free to round-off).

    Acomp = (Ax, Ay, Az) callables of (x, y, z).  Bface[d][k, j, i] is the
    average normal field on the face of direction d through the grid node (i, j, k).
    """
    h = 1.0 / n
    Ae = [_edge_line_average(Acomp[d], n, npts, d) for d in range(3)]   # line averages
    sh = lambda a, d: np.roll(a, -1, axis=2 - d)
    # Bx on x-face: (1/h^2) * circulation = (1/h)[(Az(j+1) - Az(j)) - (Ay(k+1) - Ay(k))]
    Bx = ((sh(Ae[2], 1) - Ae[2]) - (sh(Ae[1], 2) - Ae[1])) / h
    By = ((sh(Ae[0], 2) - Ae[0]) - (sh(Ae[2], 0) - Ae[2])) / h
    Bz = ((sh(Ae[1], 0) - Ae[1]) - (sh(Ae[0], 1) - Ae[0])) / h
    return np.stack([Bx, By, Bz])


def alfven_wave(n, t=0.0, B0=1.0, amp=0.1, rho0=1.0, P0=1.0, gamma=5.0 / 3.0, npts=4):
    """Circularly polarised Alfven wave along (1,1,1) (exact nonlinear solution, Gaussian units).

    Wave vector 2 pi (1,1,1) (wavelength 1/sqrt(3), periodic on the unit
    cube); B = B0 n + amp B0 (cos phi e1 + sin phi e2), v = -(B - B0 n)/sqrt(4 pi rho0),
    phase phi = k . x - |k| V_A t with V_A = B0 / sqrt(4 pi rho0).
    Returns (U, Bface); Bface comes from a vector potential.
    """
    nvec = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)
    e1 = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
    e2 = np.cross(nvec, e1)
    kmag = 2 * np.pi * np.sqrt(3.0)
    VA = B0 / np.sqrt(FOUR_PI * rho0)

    def phase(x, y, z):
        return 2 * np.pi * (x + y + z) - kmag * VA * t

    def Bvec(x, y, z, c):
        ph = phase(x, y, z)
        return B0 * nvec[c] + amp * B0 * (np.cos(ph) * e1[c] + np.sin(ph) * e2[c])

    # The wave part of B is curl(A_w) with A_w = -(amp B0 / |k|)(cos phi e1 + sin phi e2): since
    # curl A_w = |k| n x dA_w/dphi and n x e1 = e2, n x e2 = -e1, this is amp B0 (cos phi e1 + sin phi e2).
    # A_w is periodic; the uniform part B0 n is added to the face averages exactly.
    wave_A = [lambda x, y, z, c=c: -(amp * B0 / kmag) * (np.cos(phase(x, y, z)) * e1[c] + np.sin(phase(x, y, z)) * e2[c])
              for c in range(3)]
    Bw = face_field_from_potential(wave_A, n, npts=6)
    Bface = np.stack([Bw[c] + B0 * nvec[c] for c in range(3)])
    rho = rho0 * np.ones((n, n, n))
    vz = [cell_average(lambda x, y, z, c=c: -(Bvec(x, y, z, c) - B0 * nvec[c]) / np.sqrt(FOUR_PI * rho0), n, npts)
          for c in range(3)]
    # energy: cell average of P/(g-1) + rho v^2/2 + B^2/8pi (|v|, |B| constant for this wave)
    v2 = (amp * B0) ** 2 / (FOUR_PI * rho0)
    B2 = B0 ** 2 * (1.0 + amp ** 2)
    eps = (P0 / (gamma - 1.0) + 0.5 * rho0 * v2 + B2 / (2.0 * FOUR_PI)) * np.ones((n, n, n))
    U = np.stack([rho, rho0 * vz[0], rho0 * vz[1], rho0 * vz[2], eps])
    return U, Bface


def orszag_tang(n, gamma=5.0 / 3.0, rho0=25.0 / (36.0 * np.pi), P0=5.0 / (12.0 * np.pi), B0=None):
    """Orszag-Tang-type vortex, uniform in z (the standard 2-D fields; Gaussian units).

    v = (-sin 2 pi y, sin 2 pi x, 0) and B = B0 (-sin 2 pi y, sin 4 pi x, 0) = curl(A_z z) with
    A_z = B0 (cos 4 pi x / (4 pi) + cos 2 pi y / (2 pi)); B0 = 1 here is the usual Heaviside
    amplitude 1/sqrt(4 pi) converted to Gaussian units.  rho and P are uniform.
    """
    if B0 is None:
        B0 = 1.0          # equals the Heaviside-unit amplitude 1/sqrt(4 pi) times sqrt(4 pi)
    Az = lambda x, y, z: B0 * (np.cos(4 * np.pi * x) / (4 * np.pi) + np.cos(2 * np.pi * y) / (2 * np.pi)) + 0 * z
    zero = lambda x, y, z: 0.0 * (x + y + z)
    Bface = face_field_from_potential([zero, zero, Az], n, npts=6)
    rho = rho0 * np.ones((n, n, n))
    vx = cell_average(lambda x, y, z: -np.sin(2 * np.pi * y) + 0 * x * z, n)
    vy = cell_average(lambda x, y, z: np.sin(2 * np.pi * x) + 0 * y * z, n)
    Bx2 = cell_average(lambda x, y, z: (B0 * np.sin(2 * np.pi * y)) ** 2 + 0 * x * z, n)
    By2 = cell_average(lambda x, y, z: (B0 * np.sin(4 * np.pi * x)) ** 2 + 0 * y * z, n)
    v2 = cell_average(lambda x, y, z: np.sin(2 * np.pi * y) ** 2 + np.sin(2 * np.pi * x) ** 2 + 0 * z, n)
    eps = P0 / (gamma - 1.0) + 0.5 * rho0 * v2 + (Bx2 + By2) / (2.0 * FOUR_PI)
    U = np.stack([rho, rho0 * vx, rho0 * vy, np.zeros_like(rho), eps])
    return U, Bface


def _zone_field(Bface):
    """Zone-centred B: the mean of each component's two faces (for the magnetic energy of synthetic states)."""
    return np.stack([0.5 * (Bface[d] + np.roll(Bface[d], -1, axis=2 - d)) for d in range(3)])


def with_field(U, Bface):
    """Euler state U plus the magnetic energy of the face field Bface: the MHD state (U, Bface)."""
    Bz = _zone_field(Bface)
    U = U.copy()
    U[4] += (Bz ** 2).sum(axis=0) / (2.0 * FOUR_PI)
    return U, Bface


def random_magnetised(n, seed, amp=0.2, b_amp=0.3, B0=1.0, modes=6, kmax=2, gamma=5.0 / 3.0, P0=1.0):
    """Seeded magnetised random state: rho and v as random_smooth, and B = B0 e + b from a periodic vector
    potential.

    e is a random unit vector; b = curl A with A a sum of `modes` Fourier modes a_m cos(2 pi k_m . x + phi_m)
    (integer wave vectors, |k_m,i| <= kmax, a_m transverse to k_m), scaled so that the bound
    sum_m 2 pi |k_m| |a_m| on |b| equals b_amp B0.  Bface comes from A by Stokes' theorem (divergence-free
    to round-off).  Returns (U, Bface).
    """
    U = random_smooth(n, seed, amp=amp, gamma=gamma, P0=P0)
    rng = np.random.default_rng(seed + 7919)
    e = rng.normal(size=3)
    e /= np.linalg.norm(e)
    ks, amps, phases = [], [], []
    for _ in range(modes):
        k = np.zeros(3)
        while not k.any():
            k = rng.integers(-kmax, kmax + 1, 3).astype(np.float64)
        a = rng.normal(size=3)
        a -= k * (a @ k) / (k @ k)
        ks.append(k)
        amps.append(a)
        phases.append(rng.uniform(0.0, 2 * np.pi))
    bound = sum(2 * np.pi * np.linalg.norm(k) * np.linalg.norm(a) for k, a in zip(ks, amps))
    scale = b_amp * B0 / bound

    def comp(c):
        def A(x, y, z):
            out = 0.0 * (x + y + z)
            for k, a, ph in zip(ks, amps, phases):
                out = out + scale * a[c] * np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + ph)
            return out
        return A

    Bw = face_field_from_potential([comp(0), comp(1), comp(2)], n, npts=6)
    Bface = np.stack([Bw[c] + B0 * e[c] for c in range(3)])
    return with_field(U, Bface)


def uniform_field(n, B0, direction):
    """Face field of the uniform B = B0 direction / |direction| on an n^3 grid."""
    e = np.asarray(direction, dtype=np.float64)
    e = e / np.linalg.norm(e)
    return np.stack([np.full((n, n, n), B0 * e[c]) for c in range(3)])


def batch_problems(count=64, seed=1006, sizes=(32, 48, 64, 80, 96, 112, 128), mhd_fraction=0.5):
    """Seeded set of independent problems of uneven cubic sizes for the batched step.

    Each problem draws: its size from `sizes`; Euler or ideal MHD (probability mhd_fraction); its order
    uniformly from 2, 3, 4; modal or nodal; HLL or linearized (Euler only).  Euler problems are either
    Gaussian random fields (amplitude 0.1) or planar shock tubes along a lattice normal with density and
    pressure ratios drawn from [2, 10]; MHD problems are the Orszag-Tang-type vortex shifted by a random
    periodic offset.  Returns dicts with keys shape, order, mhd, form, solver, gamma, U, B (B None for Euler).
    """
    rng = np.random.default_rng(seed)
    out = []
    vortex = {}
    for k in range(count):
        n = int(rng.choice(sizes))
        mhd = bool(rng.random() < mhd_fraction)
        order = int(rng.integers(2, 5))
        form = "nodal" if rng.random() < 0.5 else "modal"
        if mhd:
            if n not in vortex:
                vortex[n] = orszag_tang(n)
            U, B = vortex[n]
            sh = tuple(int(v) for v in rng.integers(0, n, 3))
            U = np.roll(U, sh, axis=(1, 2, 3))
            B = np.roll(B, sh, axis=(1, 2, 3))
            out.append(dict(shape=(n, n, n), order=order, mhd=True, form=form, solver="hll", gamma=5.0 / 3.0,
                            U=np.ascontiguousarray(U), B=np.ascontiguousarray(B)))
            continue
        solver = "linearized" if rng.random() < 0.5 else "hll"
        if rng.random() < 0.5:
            U = random_smooth(n, seed=seed * 1000 + k, amp=0.1)
        else:
            normal = [(1, 0, 0), (1, 1, 0), (2, 1, 0)][int(rng.integers(0, 3))]
            rr, pr = rng.uniform(2.0, 10.0, 2)
            U = sod_planar(n, normal=normal, left=(1.0, 1.0), right=(1.0 / rr, 1.0 / pr))
        out.append(dict(shape=(n, n, n), order=order, mhd=False, form=form, solver=solver, gamma=1.4,
                        U=np.ascontiguousarray(U), B=None))
    return out


# ----------------------------------------------------------------------------- 2-D problems as z-slabs
SLAB_DEPTH = 2.0 ** 40
"""Depth of a z-slab in units of its zone width.  A 2-D problem runs as one zone in z (periodic, so every
z-difference is exactly zero); the large depth only takes the z signal speed out of the CFL time step,
which then has the 2-D form."""


def slab_lengths(L):
    """Domain lengths (Lx, Ly, Lz) of an n x n slab over [-L/2, L/2]^2 for Solver(..., lengths=)."""
    return (float(L), float(L), float(L) * SLAB_DEPTH)


def _slab_average(fn, n, L, npts):
    """Average of fn(x, y) over every zone of an n x n grid on [-L/2, L/2]^2, shape (1, n, n) [z, y, x]."""
    xg, wg = _gauss(npts)
    h = L / n
    c = -0.5 * L + (np.arange(n) + 0.5) * h
    out = 0.0
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            out = out + wa * wb * fn((c + a * h)[None, :], (c + b * h)[:, None])
    return np.broadcast_to(out, (n, n))[None].astype(np.float64).copy()


def isentropic_vortex(n, L=10.0, eps=5.0, gamma=1.4, npts=5):
    """Isentropic hydrodynamic vortex of Sec. VI.1 on [-L/2, L/2]^2, shape (5, 1, n, n).

    Mean flow rho = P = 1, v = (1, 1, 0); the vortex adds dv = eps/(2 pi) e^{(1 - r^2)/2} (-y, x) and
    dT = -(gamma - 1) eps^2 / (8 gamma pi^2) e^{1 - r^2} to T = P / rho at constant entropy P / rho^gamma = 1,
    so rho = T^{1/(gamma-1)} and P = rho T.  Zone averages of the conserved variables by npts^2 Gauss points.
    After t = L the mean flow has carried the vortex once across the periodic domain: the exact solution
    is the initial state again.
    """
    k = (gamma - 1.0) * eps ** 2 / (8.0 * gamma * np.pi ** 2)
    s = eps / (2.0 * np.pi)

    def prim(x, y):
        r2 = x * x + y * y
        T = 1.0 - k * np.exp(1.0 - r2)
        rho = T ** (1.0 / (gamma - 1.0))
        a = s * np.exp(0.5 * (1.0 - r2))
        return rho, 1.0 - a * y, 1.0 + a * x, rho * T

    def cons(c):
        def f(x, y):
            rho, vx, vy, P = prim(x, y)
            return [rho, rho * vx, rho * vy, 0.0 * rho, P / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)][c]
        return f

    return np.concatenate([_slab_average(cons(c), n, L, npts)[None] for c in range(5)])


def magnetized_vortex(n, L=10.0, kappa=1.0, mu=np.sqrt(FOUR_PI), gamma=5.0 / 3.0, npts=5):
    """Magnetised isodensity vortex of Sec. VI.2 on [-L/2, L/2]^2: (U (5, 1, n, n), Bface (3, 1, n, n)).

    rho = 1, mean v = (1, 1, 0), mean B = 0; with f = e^{(1 - r^2)/2} the vortex adds
    dv = kappa/(2 pi) f (-y, x), dB = mu/(2 pi) f (-y, x) and
    dP = (mu/(2 pi))^2 (1 - r^2) f^2 / (8 pi) - (kappa/(2 pi))^2 f^2 / 2 (Gaussian units: it balances the
    centrifugal, magnetic-pressure and tension forces).  The paper leaves kappa and mu to its ref. [8];
    kappa = 1 and mu = sqrt(4 pi) are the values of that vortex.  B = curl(A_z z) with
    A_z = mu/(2 pi) f, so the face averages are differences of A_z at the grid nodes (Stokes; divergence-free
    to round-off).  The exact solution at t = L is the initial state.
    """
    b = mu / (2.0 * np.pi)
    q = kappa / (2.0 * np.pi)

    def f(x, y):
        return np.exp(0.5 * (1.0 - x * x - y * y))

    def prim(x, y):
        r2 = x * x + y * y
        e = f(x, y)
        P = 1.0 + b * b * (1.0 - r2) * e * e / (2.0 * FOUR_PI) - 0.5 * q * q * e * e
        return 1.0 - q * e * y, 1.0 + q * e * x, -b * e * y, b * e * x, P

    def energy(x, y):
        vx, vy, Bx, By, P = prim(x, y)
        return P / (gamma - 1.0) + 0.5 * (vx * vx + vy * vy) + (Bx * Bx + By * By) / (2.0 * FOUR_PI)

    rho = np.ones((1, n, n))
    mx = _slab_average(lambda x, y: prim(x, y)[0], n, L, npts)
    my = _slab_average(lambda x, y: prim(x, y)[1], n, L, npts)
    U = np.stack([rho, mx, my, np.zeros_like(rho), _slab_average(energy, n, L, npts)])
    h = L / n
    xn = -0.5 * L + np.arange(n) * h
    Az = b * f(xn[None, :], xn[:, None])                 # [j, i] at the grid node (x_i, y_j)
    Bx = (np.roll(Az, -1, axis=0) - Az) / h               # face x_i - 1/2 of zone (i, j)
    By = -(np.roll(Az, -1, axis=1) - Az) / h
    Bface = np.stack([Bx[None], By[None], np.zeros((1, n, n))])
    return U, Bface
