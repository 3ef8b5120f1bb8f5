"""Seeded synthetic initial conditions.

This module only builds inputs: primitive fields are drawn or written from
closed forms, the face magnetic field comes from the discrete curl of an
edge-centred vector potential (so its face divergence is zero to round-off),
and the conserved state is filled from the definitions of the conserved
variables.  It holds none of the solver's arithmetic and is shared, as input
data only, by the CUDA library's callers and by the CPU oracle's tests.

Layout: ``U[8, nz, ny, nx]`` = (rho, mx, my, mz, Bx, By, Bz, E), x fastest;
``bx[k, j, i]`` on face (i-1/2, j, k), ``by`` on (i, j-1/2, k), ``bz`` on
(i, j, k-1/2); cell B is the two-face mean.  Units have the magnetic
permeability absorbed (magnetic pressure |B|^2/2).
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field

import numpy as np

GAMMA = 5.0 / 3.0


@dataclass
class State:
    U: np.ndarray                  # (8, nz, ny, nx) float64
    bx: np.ndarray                 # (nz, ny, nx)
    by: np.ndarray
    bz: np.ndarray
    dx: float
    dy: float
    dz: float
    gamma: float = GAMMA
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.bx.shape

    @property
    def dims(self):
        nz, ny, nx = self.bx.shape
        return nx, ny, nz

    def copy(self) -> "State":
        return State(self.U.copy(), self.bx.copy(), self.by.copy(), self.bz.copy(),
                     self.dx, self.dy, self.dz, self.gamma, dict(self.meta))


def assemble(rho, vx, vy, vz, p, bx, by, bz, dx, dy, dz, gamma=GAMMA, meta=None) -> State:
    """Conserved state from primitives and face fields (definitions only)."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = np.broadcast_shapes(rho.shape, np.shape(bx))
    f = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shape))
    rho, vx, vy, vz, p, bx, by, bz = map(f, (rho, vx, vy, vz, p, bx, by, bz))
    Bx = 0.5 * (bx + np.roll(bx, -1, axis=2))
    By = 0.5 * (by + np.roll(by, -1, axis=1))
    Bz = 0.5 * (bz + np.roll(bz, -1, axis=0))
    U = np.empty((8,) + shape)
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = Bx
    U[5] = By
    U[6] = Bz
    U[7] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) \
        + 0.5 * (Bx * Bx + By * By + Bz * Bz)
    return State(U, bx.copy(), by.copy(), bz.copy(), dx, dy, dz, gamma, meta or {})


def curl_faces(Ax, Ay, Az, dx, dy, dz):
    """Face field b = curl A from edge potentials.

    Ax[k,j,i] on edge (i, j-1/2, k-1/2), Ay on (i-1/2, j, k-1/2), Az on
    (i-1/2, j-1/2, k).  Periodic differences, so the face divergence of the
    result vanishes identically (up to round-off)."""
    r = lambda a, ax: np.roll(a, -1, axis=ax)
    bx = (r(Az, 1) - Az) / dy - (r(Ay, 0) - Ay) / dz
    by = (r(Ax, 0) - Ax) / dz - (r(Az, 2) - Az) / dx
    bz = (r(Ay, 2) - Ay) / dx - (r(Ax, 1) - Ax) / dy
    return bx, by, bz


def _centres(nx, ny, nz, dx, dy, dz):
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    z = (np.arange(nz) + 0.5) * dz
    return np.meshgrid(z, y, x, indexing="ij")[::-1]   # X, Y, Z with shape (nz,ny,nx)


# ------------------------------------------------------------------ states
def uniform(nx, ny, nz, rho=1.0, v=(0.3, -0.2, 0.1), p=0.7, B=(0.4, -0.3, 0.2),
            dx=None, dy=None, dz=None, gamma=GAMMA) -> State:
    dx = dx or 1.0 / nx
    dy = dy or 1.0 / ny
    dz = dz or 1.0 / nz
    shape = (nz, ny, nx)
    one = np.ones(shape)
    return assemble(rho * one, v[0] * one, v[1] * one, v[2] * one, p * one,
                    B[0] * one, B[1] * one, B[2] * one, dx, dy, dz, gamma,
                    {"kind": "uniform"})


def alfven_wave(nx, ny=4, nz=4, amp=0.1, rho=1.0, p=0.1, b_par=1.0, t=0.0,
                dx=None, gamma=GAMMA) -> State:
    """Circularly polarised Alfven wave along +x (exact travelling solution).

    B_perp = amp (sin 2 pi (x - t v_A), cos 2 pi (x - t v_A)), v_perp =
    -B_perp / sqrt(rho), v_A = b_par / sqrt(rho), uniform rho, p and B_par.
    Wavelength 1 = the box length in x; dy = dz = dx (cubic cells).  Values
    are point values at cell centres (face by/bz share the cell's x)."""
    dx = dx or 1.0 / nx
    X, _, _ = _centres(nx, ny, nz, dx, dx, dx)
    va = b_par / np.sqrt(rho)
    ph = 2.0 * np.pi * (X - va * t)
    By = amp * np.sin(ph)
    Bz = amp * np.cos(ph)
    vy = -By / np.sqrt(rho)
    vz = -Bz / np.sqrt(rho)
    shape = X.shape
    return assemble(np.full(shape, rho), np.zeros(shape), vy, vz, np.full(shape, p),
                    np.full(shape, b_par), By, Bz, dx, dx, dx, gamma,
                    {"kind": "alfven", "amp": amp, "t": t})


@functools.lru_cache(maxsize=None)
def _modes(kmin, kmax):
    """Integer wavevectors (kx, ky, kz) with kmin <= |k| <= kmax in the half
    space (kx > 0, or kx = 0 and ky > 0, or kx = ky = 0 and kz > 0), in a
    fixed order that does not depend on the grid."""
    K = int(np.floor(kmax))
    out = []
    for kx in range(0, K + 1):
        for ky in range(-K, K + 1):
            for kz in range(-K, K + 1):
                if kx == 0 and (ky < 0 or (ky == 0 and kz <= 0)):
                    continue
                k2 = kx * kx + ky * ky + kz * kz
                if kmin * kmin <= k2 <= kmax * kmax:
                    out.append((kx, ky, kz))
    out = np.array(out, dtype=np.int64).reshape(-1, 3)
    out.setflags(write=False)
    return out


def gaussian_field(shape, rng, kmin=1.0, kmax=8.0, slope=-11.0 / 3.0):
    """Unit-variance Gaussian random field on a periodic grid.

    A sum of Fourier modes with integer wavevector kmin <= |k| <= kmax (units
    of 2 pi / box), each with a complex Gaussian amplitude of variance
    |k|^slope (random phase), plus its conjugate.  The amplitudes are drawn
    per mode in a grid-independent order, so one seed gives the same
    continuous field at every resolution; it is evaluated on the cell grid
    by three separable partial sums (x, then y, then z as a matrix
    product) and scaled to zero mean and unit variance over the grid."""
    nz, ny, nx = shape
    ks = _modes(kmin, kmax)
    K = int(np.floor(kmax))
    a = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    a *= np.power(np.sqrt((ks * ks).sum(axis=1)).astype(float), slope / 2.0)
    C = np.zeros((2 * K + 1, 2 * K + 1, K + 1), dtype=complex)     # [kz, ky, kx]
    C[ks[:, 2] + K, ks[:, 1] + K, ks[:, 0]] = 2.0 * a               # mode plus conjugate
    ex = np.exp(2j * np.pi * np.outer(np.arange(K + 1), np.arange(nx)) / nx)          # [kx, x]
    ey = np.exp(2j * np.pi * np.outer(np.arange(ny), np.arange(-K, K + 1)) / ny)      # [y, ky]
    ez = np.exp(2j * np.pi * np.outer(np.arange(nz), np.arange(-K, K + 1)) / nz)      # [z, kz]
    T1 = C @ ex                                           # [kz, ky, x]
    T2 = np.matmul(ey[None], T1)                          # [kz, y, x]
    T2 = T2.reshape(2 * K + 1, ny * nx)
    f = ez.real @ T2.real - ez.imag @ T2.imag             # real part, [z, y*x]
    f = f.reshape(nz, ny, nx)
    f -= f.mean()
    s = f.std()
    return f / s if s > 0 else f


def turbulence(n, seed=1808, mach=0.5, sigma_rho=0.1, p=1.0, b0=0.1, eb_frac=0.1,
               kmin=1.0, kmax=8.0, gamma=GAMMA, dims=None, h=None) -> State:
    """Decaying-turbulence start state on a periodic unit box.

    Velocity: three independent Gaussian fields with per-mode variance
    |k|^-11/3 for 1 <= |k| <= 8, scaled to rms Mach `mach` at the mean sound
    speed sqrt(gamma p / 1).  Density: log-normal exp(sigma g - sigma^2/2).
    Pressure uniform.  Field: (b0, 0, 0) plus the discrete curl of a random
    edge potential with the same spectrum, scaled so that the mean magnetic
    energy of the fluctuation is `eb_frac` of the mean kinetic energy.
    With `h` given the cells are cubes of edge h (box nx*h by ny*h by nz*h),
    otherwise the box is the unit cube."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    shape = (nz, ny, nx)
    if h is not None:
        dx = dy = dz = float(h)
    else:
        dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    rng = np.random.default_rng(seed)
    v = [gaussian_field(shape, rng, kmin, kmax) for _ in range(3)]
    cs = np.sqrt(gamma * p / 1.0)
    vrms = np.sqrt(sum((c * c).mean() for c in v))
    v = [c * (mach * cs / vrms) for c in v]
    g = gaussian_field(shape, rng, kmin, kmax)
    rho = np.exp(sigma_rho * g - 0.5 * sigma_rho ** 2)
    A = [gaussian_field(shape, rng, kmin, kmax) for _ in range(3)]
    dbx, dby, dbz = curl_faces(A[0], A[1], A[2], dx, dy, dz)
    ekin = 0.5 * (rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)).mean()
    emag = 0.5 * (dbx * dbx + dby * dby + dbz * dbz).mean()
    s = np.sqrt(eb_frac * ekin / emag) if emag > 0 else 0.0
    bx, by, bz = b0 + s * dbx, s * dby, s * dbz
    return assemble(rho, v[0], v[1], v[2], np.full(shape, p), bx, by, bz, dx, dy, dz,
                    gamma, {"kind": "turbulence", "seed": seed, "n": (nx, ny, nz)})


def add_blasts(st: State, seed=1808, nblast=64, rmin=0.02, rmax=0.05, jump=100.0) -> State:
    """Multiply the pressure by `jump` inside `nblast` seeded spheres (periodic
    distance, uniform centres, radii uniform in [rmin, rmax]; overlaps keep one
    jump).  The kinetic and magnetic parts of E are unchanged.  Each sphere
    is marked inside the periodic box of cells that bounds it."""
    st = st.copy()
    nx, ny, nz = st.dims
    rng = np.random.default_rng(seed + 7919)
    h = (st.dx, st.dy, st.dz)
    L = (nx * st.dx, ny * st.dy, nz * st.dz)
    n = (nx, ny, nz)
    inside = np.zeros(st.shape, dtype=bool)
    for _ in range(nblast):
        c = rng.uniform(0.0, 1.0, 3) * L
        r = rng.uniform(rmin, rmax)
        idx, d2 = [], []
        for d in range(3):
            lo = int(np.floor((c[d] - r) / h[d] - 0.5)) - 1
            hi = int(np.ceil((c[d] + r) / h[d] - 0.5)) + 1
            cells = np.arange(lo, hi + 1)
            if len(cells) >= n[d]:
                cells = np.arange(n[d])
            x = (np.mod(cells, n[d]) + 0.5) * h[d]
            dd = np.abs(x - c[d])
            dd = np.minimum(dd, L[d] - dd)
            idx.append(np.mod(cells, n[d]))
            d2.append(dd * dd)
        ball = d2[2][:, None, None] + d2[1][None, :, None] + d2[0][None, None, :] < r * r
        sub = np.ix_(idx[2], idx[1], idx[0])
        inside[sub] |= ball
    U = st.U
    sel = np.nonzero(inside)
    Us = U[(slice(None),) + sel]
    kin = 0.5 * (Us[1] ** 2 + Us[2] ** 2 + Us[3] ** 2) / Us[0]
    mag = 0.5 * (Us[4] ** 2 + Us[5] ** 2 + Us[6] ** 2)
    pth = (Us[7] - kin - mag) * (st.gamma - 1.0)
    U[(7,) + sel] = pth * jump / (st.gamma - 1.0) + kin + mag
    st.meta = dict(st.meta, blasts=nblast, blast_cells=int(inside.sum()))
    return st


def brio_wu_patch(dims, rng, bn=0.75, gamma=GAMMA, h=None) -> State:
    """Rotated Brio-Wu tube on a periodic patch.

    Left (rho, p, B_t) = (1, 1, 1), right (0.125, 0.1, -1), B_n = bn, at rest.
    The phase phi = 2 pi sum_d m_d x_d / L_d uses a seeded integer vector m
    (entries in -1..1, not all zero), so the pattern is periodic on the patch
    and has no seam; the state follows the sign of sin(phi), the normal is
    grad phi / |grad phi|.  The tangential field is the curl of an edge
    potential A = (t x n) Phi(phi) with Phi a periodic triangle wave (face
    divergence zero), the normal field is uniform."""
    nx, ny, nz = dims
    h = h or 1.0 / max(dims)
    shape = (nz, ny, nx)
    L = np.array([nx, ny, nz], dtype=float) * h
    while True:
        m = rng.integers(-1, 2, 3)
        if np.any(m != 0):
            break
    kvec = 2.0 * np.pi * m / L
    K = np.linalg.norm(kvec)
    nvec = kvec / K
    tmp = np.array([1.0, 0.0, 0.0]) if abs(nvec[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    tvec = np.cross(nvec, tmp)
    tvec /= np.linalg.norm(tvec)
    mvec = np.cross(tvec, nvec)

    def phase(ox, oy, oz):
        x = (np.arange(nx) + ox) * h
        y = (np.arange(ny) + oy) * h
        z = (np.arange(nz) + oz) * h
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return kvec[0] * X + kvec[1] * Y + kvec[2] * Z

    def Phi(ph):
        # antiderivative in x of sign(sin phi): d/dphi of K*Phi is sign(sin phi)
        q = np.mod(ph, 2.0 * np.pi)
        return np.where(q < np.pi, q, 2.0 * np.pi - q) / K

    # edge positions: Ax (i, j-1/2, k-1/2), Ay (i-1/2, j, k-1/2), Az (i-1/2, j-1/2, k)
    Ax = mvec[0] * Phi(phase(0.5, 0.0, 0.0))
    Ay = mvec[1] * Phi(phase(0.0, 0.5, 0.0))
    Az = mvec[2] * Phi(phase(0.0, 0.0, 0.5))
    bx, by, bz = curl_faces(Ax, Ay, Az, h, h, h)
    bx = bx + bn * nvec[0]
    by = by + bn * nvec[1]
    bz = bz + bn * nvec[2]
    left = np.sin(phase(0.5, 0.5, 0.5)) >= 0.0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    zero = np.zeros(shape)
    return assemble(rho, zero, zero, zero, p, bx, by, bz, h, h, h, gamma,
                    {"kind": "brio_wu", "normal": nvec.tolist(), "m": m.tolist()})


def field_loop(n, amp=1e-3, radius=0.3, v=(1.0, 1.0), rho=1.0, p=1.0, gamma=GAMMA) -> State:
    """Advected weak field loop on the periodic unit square (n x n x 1).

    A_z = amp (R - r) inside the radius R around the box centre, zero
    outside; b = curl A (face divergence zero); uniform rho, p and velocity,
    so the loop returns to its start after t = 1 with v = (1, 1)."""
    h = 1.0 / n
    x = np.arange(n) * h                        # edge positions (i - 1/2) * h + h/2
    X, Y = np.meshgrid(x, x, indexing="xy")     # [j, i]
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
    Az = np.where(r < radius, amp * (radius - r), 0.0)[None, :, :]
    zero = np.zeros((1, n, n))
    bx, by, bz = curl_faces(zero, zero, Az, h, h, h)
    return assemble(np.full((1, n, n), rho), v[0], v[1], 0.0, p, bx, by, bz, h, h, h, gamma,
                    {"kind": "field_loop", "n": n, "amp": amp, "radius": radius})


def orszag_tang(n, gamma=GAMMA) -> State:
    """Orszag-Tang vortex on the periodic unit square (n x n x 1), in units
    with the permeability absorbed: rho = 25/(36 pi), p = 5/(12 pi),
    v = (-sin 2 pi y, sin 2 pi x), B = B0 (-sin 2 pi y, sin 4 pi x) with
    B0 = 1/sqrt(4 pi), the field from A_z = B0 (cos 4 pi x / (4 pi) +
    cos 2 pi y / (2 pi))."""
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    xe = np.arange(n) * h
    B0 = 1.0 / np.sqrt(4.0 * np.pi)
    Xe, Ye = np.meshgrid(xe, xe, indexing="xy")
    Az = (B0 * (np.cos(4.0 * np.pi * Xe) / (4.0 * np.pi) + np.cos(2.0 * np.pi * Ye) / (2.0 * np.pi)))[None]
    zero = np.zeros((1, n, n))
    bx, by, bz = curl_faces(zero, zero, Az, h, h, h)
    Xc, Yc = np.meshgrid(xc, xc, indexing="xy")
    vx = -np.sin(2.0 * np.pi * Yc)[None]
    vy = np.sin(2.0 * np.pi * Xc)[None]
    return assemble(np.full((1, n, n), 25.0 / (36.0 * np.pi)), vx, vy, 0.0, 5.0 / (12.0 * np.pi),
                    bx, by, bz, h, h, h, gamma, {"kind": "orszag_tang", "n": n})


def patch_dims(npatch, seed=1808, lo=16, hi=64, max_aspect=2.0):
    """Patch edges drawn independently log-uniform in [lo, hi]; a draw whose
    longest/shortest edge exceeds max_aspect is redrawn."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < npatch:
        e = np.exp(rng.uniform(np.log(lo), np.log(hi), 3))
        e = np.clip(np.rint(e).astype(int), lo, hi)
        if e.max() / e.min() <= max_aspect:
            out.append(tuple(int(v) for v in e))
    return out


def patch_batch(npatch, seed=1808, lo=16, hi=64, gamma=GAMMA):
    """Independent periodic patches: each a coin flip between a rotated
    Brio-Wu tube and a turbulence state of its own size.  Returns a list of
    State; every patch uses unit cell size h = 1/64."""
    dims = patch_dims(npatch, seed, lo, hi)
    rng = np.random.default_rng(seed + 1)
    out = []
    for p, d in enumerate(dims):
        if rng.uniform() < 0.5:
            st = brio_wu_patch(d, rng, gamma=gamma, h=1.0 / 64.0)
        else:
            st = turbulence(None, seed=seed + 1000 + p, gamma=gamma, dims=d, h=1.0 / 64.0)
        out.append(st)
    return out


def perturbed(nx, ny, nz, seed=0, amp=0.05, jump=False, gamma=GAMMA) -> State:
    """Smooth random state (low modes) for parity tests; with jump=True a
    pressure/density step is added so that the WENO weights leave the linear
    regime."""
    shape = (nz, ny, nx)
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    rng = np.random.default_rng(seed)
    g = lambda: gaussian_field(shape, rng, 1.0, 3.0)
    rho = 1.0 + amp * g()
    vx, vy, vz = (0.3 * g() for _ in range(3))
    p = 0.6 + amp * g()
    A = [0.05 * g() for _ in range(3)]
    bx, by, bz = curl_faces(A[0], A[1], A[2], dx, dy, dz)
    bx = bx + 0.3
    by = by - 0.2
    bz = bz + 0.1
    if jump:
        X, _, _ = _centres(nx, ny, nz, dx, dy, dz)
        step = (X > 0.3) & (X < 0.7)
        rho = np.where(step, rho * 0.3, rho)
        p = np.where(step, p * 0.2, p)
    return assemble(rho, vx, vy, vz, p, bx, by, bz, dx, dy, dz, gamma,
                    {"kind": "perturbed", "seed": seed, "jump": jump})
