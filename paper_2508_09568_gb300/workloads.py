"""Seeded synthetic workloads for the MHD bunch update: patch geometry and initial states.

This module is shared by the CUDA path and the FP64 oracle as the one source of inputs.
It only lays out patches and evaluates the analytic / seeded initial conditions of the
test problems (Sod shock tube, Orszag-Tang vortex, a 3D turbulence-like box, a ragged
box of mixed patch sizes, and the smooth adjoint rollout box).  It holds no part of the
update itself (no primitive recovery, slopes, Riemann solvers, EMFs, time step or guard
fill).

State layout (the same on every side): a bunch is a flat buffer of patches, patch ``p``
starting at element ``offsets[p]``; each patch is ``[8][Z][Y][X]`` with ``x`` fastest,
variables ``(rho, rho*u, rho*v, rho*w, E, Bx, By, Bz)``.  An active axis carries ``guard``
ghost cells on each side, a collapsed axis (domain extent 1) carries none.  ``Bx`` at
local index ``i`` is the x-face at the low side of cell ``i`` (staggered field of Sec. 2.1.3,
Fig. 2; the index offsets of Eqs. 8-12 put ``Bx(i)`` on the left face of cell ``i``); ``By`` and
``Bz`` likewise on the low y- and z-faces.  Guard cells of a freshly built state hold NaN.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

NVAR = 8
RHO, MX, MY, MZ, EN, BX, BY, BZ = range(8)
BC_PERIODIC, BC_OUTFLOW = 0, 1


@dataclass
class Geometry:
    """Patch decomposition of a box.

    patch_n  (P,3) int64  active cells per patch along (x, y, z)
    origin   (P,3) int64  global index of each patch's first active cell
    domain   (3,)  int64  cells of the whole box along (x, y, z)
    dx       (3,)  float64 cell size along (x, y, z)
    bc       (3,2) int32  boundary kind at the low/high end of each axis
    guard    int          ghost-cell width on active axes
    bunches  list of index arrays: how the patches are grouped into bunches (one group
             holding every patch when not given)
    """

    patch_n: np.ndarray
    origin: np.ndarray
    domain: np.ndarray
    dx: np.ndarray
    bc: np.ndarray
    guard: int = 3
    bunches: list = field(default_factory=list)

    def __post_init__(self):
        self.patch_n = np.asarray(self.patch_n, dtype=np.int64).reshape(-1, 3)
        self.origin = np.asarray(self.origin, dtype=np.int64).reshape(-1, 3)
        self.domain = np.asarray(self.domain, dtype=np.int64).reshape(3)
        self.dx = np.asarray(self.dx, dtype=np.float64).reshape(3)
        self.bc = np.asarray(self.bc, dtype=np.int32).reshape(3, 2)
        if not self.bunches:
            self.bunches = [np.arange(self.npatch, dtype=np.int64)]

    @property
    def npatch(self) -> int:
        return int(self.patch_n.shape[0])

    @property
    def active(self) -> np.ndarray:
        """Axes with more than one cell in the box."""
        return self.domain > 1

    @property
    def gvec(self) -> np.ndarray:
        """Ghost width per axis (0 on collapsed axes)."""
        return np.where(self.active, self.guard, 0).astype(np.int64)

    def padded(self, p: int) -> tuple:
        """(Z, Y, X) extent of patch p including ghost cells."""
        n = self.patch_n[p] + 2 * self.gvec
        return int(n[2]), int(n[1]), int(n[0])

    def patch_elems(self) -> np.ndarray:
        return np.array([NVAR * int(np.prod(self.padded(p))) for p in range(self.npatch)], dtype=np.int64)

    def offsets(self) -> np.ndarray:
        e = self.patch_elems()
        return np.concatenate([[0], np.cumsum(e)[:-1]]).astype(np.int64)

    def state_elems(self) -> int:
        return int(self.patch_elems().sum())

    def uniform(self) -> bool:
        return bool(np.all(self.patch_n == self.patch_n[0]))

    def interior_cells(self) -> int:
        return int(np.prod(self.patch_n, axis=1).sum())

    def interior_offsets(self) -> np.ndarray:
        """Element offset of each patch in the interior layout ([8][nz][ny][nx] per patch)."""
        e = NVAR * np.prod(self.patch_n, axis=1)
        return np.concatenate([[0], np.cumsum(e)[:-1]]).astype(np.int64)


def uniform_geometry(domain, patch, dx=None, bc=None, guard=3, order="xyz") -> Geometry:
    """Box of ``domain`` cells cut into equal patches of ``patch`` cells (x fastest in patch order)."""
    domain = np.asarray(domain, dtype=np.int64)
    patch = np.asarray(patch, dtype=np.int64)
    if np.any(domain % patch):
        raise ValueError("domain must be a multiple of the patch size")
    counts = domain // patch
    org = []
    for kz in range(counts[2]):
        for ky in range(counts[1]):
            for kx in range(counts[0]):
                org.append([kx * patch[0], ky * patch[1], kz * patch[2]])
    org = np.array(org, dtype=np.int64)
    if dx is None:
        dx = [1.0 / domain[0]] * 3
    if bc is None:
        bc = [[BC_PERIODIC, BC_PERIODIC]] * 3
    return Geometry(np.tile(patch, (len(org), 1)), org, domain, dx, bc, guard)


# ----------------------------------------------------------------------------------------
# global field <-> patch buffer
# ----------------------------------------------------------------------------------------

def _wrap_index(idx: np.ndarray, n: int, lo: int, hi: int) -> np.ndarray:
    """Map global cell indices outside [0,n) onto the box: periodic wrap or edge clamp.

    This only decides which global cell a ghost position mirrors; it is used to build
    inputs (padding a global field), never to advance the state.
    """
    out = idx.copy()
    below, above = idx < 0, idx >= n
    out[below] = (idx[below] % n) if lo == BC_PERIODIC else 0
    out[above] = (idx[above] % n) if hi == BC_PERIODIC else n - 1
    return out


def to_patches(fields, geom: Geometry, dtype=np.float64, fill_guards=False, out=None) -> np.ndarray:
    """Cut a global field into the flat patch buffer.

    ``fields`` is either an array (8, Nz, Ny, Nx) or a callable ``v -> (Nz, Ny, Nx)`` array
    (used for the large boxes, one variable at a time).  Ghost cells are NaN unless
    ``fill_guards`` (then they mirror the global cells the boundary kind names; used only by
    input checks).
    """
    offs = geom.offsets()
    if out is None:
        out = np.empty(geom.state_elems(), dtype=dtype)
    g = geom.gvec
    for v in range(NVAR):
        a = fields(v) if callable(fields) else fields[v]
        for p in range(geom.npatch):
            Z, Y, X = geom.padded(p)
            n = geom.patch_n[p]
            o = geom.origin[p]
            dst = out[offs[p] + v * X * Y * Z: offs[p] + (v + 1) * X * Y * Z].reshape(Z, Y, X)
            if fill_guards:
                ix = _wrap_index(np.arange(X) + o[0] - g[0], geom.domain[0], *geom.bc[0])
                iy = _wrap_index(np.arange(Y) + o[1] - g[1], geom.domain[1], *geom.bc[1])
                iz = _wrap_index(np.arange(Z) + o[2] - g[2], geom.domain[2], *geom.bc[2])
                dst[...] = a[np.ix_(iz, iy, ix)]
            else:
                dst[...] = np.nan
                dst[g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]] = \
                    a[o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]]
    return out


def from_patches(flat: np.ndarray, geom: Geometry, dtype=np.float64) -> np.ndarray:
    """Assemble the interiors of a flat patch buffer into a global (8, Nz, Ny, Nx) field."""
    offs = geom.offsets()
    N = geom.domain
    out = np.full((NVAR, N[2], N[1], N[0]), np.nan, dtype=dtype)
    g = geom.gvec
    for p in range(geom.npatch):
        Z, Y, X = geom.padded(p)
        n, o = geom.patch_n[p], geom.origin[p]
        blk = np.asarray(flat[offs[p]: offs[p] + NVAR * X * Y * Z]).reshape(NVAR, Z, Y, X)
        out[:, o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = \
            blk[:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
    return out


def to_interior(fields, geom: Geometry, dtype=np.float64, out=None) -> np.ndarray:
    """Cut a global field (array (8, Nz, Ny, Nx) or callable v -> (Nz, Ny, Nx)) into the
    interior layout: the owned cells of each patch, [8][nz][ny][nx], patches back to back."""
    offs = geom.interior_offsets()
    if out is None:
        out = np.empty(geom.interior_cells() * NVAR, dtype=dtype)
    for v in range(NVAR):
        a = fields(v) if callable(fields) else fields[v]
        for p in range(geom.npatch):
            n, o = geom.patch_n[p], geom.origin[p]
            cells = int(np.prod(n))
            dst = out[offs[p] + v * cells: offs[p] + (v + 1) * cells].reshape(n[2], n[1], n[0])
            dst[...] = a[o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]]
    return out


def from_interior(flat: np.ndarray, geom: Geometry, dtype=np.float64) -> np.ndarray:
    """Assemble an interior-layout buffer into a global (8, Nz, Ny, Nx) field."""
    offs = geom.interior_offsets()
    N = geom.domain
    out = np.full((NVAR, N[2], N[1], N[0]), np.nan, dtype=dtype)
    for p in range(geom.npatch):
        n, o = geom.patch_n[p], geom.origin[p]
        blk = np.asarray(flat[offs[p]: offs[p] + NVAR * int(np.prod(n))]).reshape(NVAR, n[2], n[1], n[0])
        out[:, o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = blk
    return out


def patch_view(flat: np.ndarray, geom: Geometry, p: int) -> np.ndarray:
    """(8, Z, Y, X) view of patch p inside a flat buffer."""
    offs = geom.offsets()
    Z, Y, X = geom.padded(p)
    return flat[offs[p]: offs[p] + NVAR * X * Y * Z].reshape(NVAR, Z, Y, X)


# ----------------------------------------------------------------------------------------
# initial conditions (global fields, float64; face B on the low faces)
# ----------------------------------------------------------------------------------------

def _centres(geom: Geometry):
    """Cell-centre and low-face coordinates along each axis."""
    c = [(np.arange(geom.domain[d]) + 0.5) * geom.dx[d] for d in range(3)]
    f = [np.arange(geom.domain[d]) * geom.dx[d] for d in range(3)]
    return c, f


def conserved_from_setup(rho, vel, p, bface, gamma) -> np.ndarray:
    """Conserved state of an initial condition given density, velocity, gas pressure and face B.

    The total energy uses the cell-centred field as the mean of the two faces of each cell;
    this is the set-up's own statement of its pressure (the adiabatic equation of state of
    Sec. 2.1 solved for E), done once when the input is made.
    """
    shape = np.broadcast_shapes(np.shape(rho), np.shape(vel[0]), np.shape(p),
                                np.shape(bface[0]), np.shape(bface[1]), np.shape(bface[2]))
    U = np.empty((NVAR,) + shape, dtype=np.float64)
    U[RHO] = rho
    for d in range(3):
        U[MX + d] = rho * vel[d]
        U[BX + d] = bface[d]
    bc = []
    for d in range(3):
        axis = 2 - d  # array axis of direction d in (z, y, x)
        bc.append(0.5 * (U[BX + d] + np.roll(U[BX + d], -1, axis=axis)))
    U[EN] = p / (gamma - 1.0) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2) \
        + 0.5 * (bc[0] ** 2 + bc[1] ** 2 + bc[2] ** 2)
    return U


def sod(ncell=256, npatch=16, gamma=1.4):
    """1D Sod shock tube on [0,1]: x-extent ``ncell`` split into ``npatch`` patches, outflow ends."""
    geom = uniform_geometry([ncell, 1, 1], [ncell // npatch, 1, 1], dx=[1.0 / ncell, 1.0, 1.0],
                            bc=[[BC_OUTFLOW, BC_OUTFLOW], [BC_PERIODIC] * 2, [BC_PERIODIC] * 2])
    (xc, _, _), _ = _centres(geom)
    left = xc < 0.5
    rho = np.where(left, 1.0, 0.125)[None, None, :]
    p = np.where(left, 1.0, 0.1)[None, None, :]
    z = np.zeros_like(rho)
    U = conserved_from_setup(rho, (z, z, z), p, (z, z, z), gamma)
    return geom, U, dict(gamma=gamma, t_end=0.2)


def orszag_tang(ncell=512, patch=32, gamma=5.0 / 3.0):
    """2D Orszag-Tang vortex on the periodic unit square (z collapsed)."""
    geom = uniform_geometry([ncell, ncell, 1], [patch, patch, 1],
                            dx=[1.0 / ncell, 1.0 / ncell, 1.0])
    (xc, yc, _), (xf, yf, _) = _centres(geom)
    U = _ot_fields(xc, yc, xf, yf, 1, gamma)
    return geom, U, dict(gamma=gamma, t_end=0.5)


def _ot_fields(xc, yc, xf, yf, nz, gamma):
    b0 = 1.0 / np.sqrt(4.0 * np.pi)
    X, Y = np.meshgrid(xc, yc, indexing="xy")          # (Ny, Nx)
    rho = np.full((nz,) + X.shape, 25.0 / (36.0 * np.pi))
    p = np.full_like(rho, 5.0 / (12.0 * np.pi))
    vx = np.broadcast_to(-np.sin(2 * np.pi * Y), rho.shape)
    vy = np.broadcast_to(np.sin(2 * np.pi * X), rho.shape)
    vz = np.zeros_like(rho)
    # Bx on x-faces (x_f, y_c) depends on y only; By on y-faces (x_c, y_f) on x only
    bx = np.broadcast_to(-b0 * np.sin(2 * np.pi * Y), rho.shape)
    by = np.broadcast_to(b0 * np.sin(4 * np.pi * X), rho.shape)
    bz = np.zeros_like(rho)
    return conserved_from_setup(rho, (vx, vy, vz), p, (bx, by, bz), gamma)


def _solenoidal_modes(rng, kmax, slope):
    """Random-phase solenoidal Fourier coefficients c_k (Hermitian) for 1 <= |k| <= kmax.

    Each mode of the half space gets a unit vector drawn from a normal triple, projected
    perpendicular to k, times |k|**slope and a uniform random phase; c_{-k} = conj(c_k).
    Returns an array (3, 2K+1, 2K+1, 2K+1) indexed [comp, kz+K, ky+K, kx+K].
    """
    K = kmax
    C = np.zeros((3, 2 * K + 1, 2 * K + 1, 2 * K + 1), dtype=np.complex128)
    for kz in range(-K, K + 1):
        for ky in range(-K, K + 1):
            for kx in range(-K, K + 1):
                k = np.array([kx, ky, kz], dtype=np.float64)
                kk = np.sqrt(k @ k)
                if kk < 1.0 or kk > kmax:
                    continue
                # half space: first non-zero component positive
                first = kx if kx != 0 else (ky if ky != 0 else kz)
                if first < 0:
                    continue
                g = rng.standard_normal(3)
                khat = k / kk
                g = g - (g @ khat) * khat
                g /= np.linalg.norm(g)
                ph = rng.uniform(0.0, 2.0 * np.pi)
                c = g * kk ** slope * np.exp(1j * ph)
                C[:, kz + K, ky + K, kx + K] = c
                C[:, -kz + K, -ky + K, -kx + K] = np.conj(c)
    return C


def _eval_modes(Ccomp, xc, yc, zc):
    """Real field sum_k C[k] exp(2 pi i k.x) on the tensor grid (z, y, x), by separable sums."""
    K = (Ccomp.shape[0] - 1) // 2
    ks = np.arange(-K, K + 1)
    Ex = np.exp(2j * np.pi * np.outer(ks, xc))   # (k, x)
    Ey = np.exp(2j * np.pi * np.outer(ks, yc))
    Ez = np.exp(2j * np.pi * np.outer(ks, zc))
    T1 = np.einsum("zyk,kx->zyx", Ccomp, Ex)                  # (kz, ky, x)
    T2 = np.einsum("ky,zkx->zyx", Ey, T1)                     # (kz, y, x)
    nz, ny, nx = len(zc), len(yc), len(xc)
    T2 = T2.reshape(2 * K + 1, ny * nx)
    out = (Ez.real.T @ T2.real - Ez.imag.T @ T2.imag)         # (z, y*x)
    return out.reshape(nz, ny, nx)


def turbulence_box(ncell=512, patch=32, gamma=5.0 / 3.0, seed=20250809, kmax=8):
    """3D periodic box: rho=1, p=1, B=(0.1,0,0), seeded solenoidal velocity, rms Mach 1.

    The velocity has energy spectrum E(k) ~ k^-2 over 1 <= |k| <= kmax (mode amplitude
    ~ |k|^-2), uniform random phases, and is scaled to rms speed sqrt(gamma p / rho).
    Returns (geom, fields) where fields(v) yields one global variable at a time.
    """
    geom = uniform_geometry([ncell] * 3, [patch] * 3, dx=[1.0 / ncell] * 3)
    rng = np.random.default_rng(seed)
    C = _solenoidal_modes(rng, kmax, -2.0)
    (xc, yc, zc), _ = _centres(geom)
    cache = {}

    def vel(d):
        if d not in cache:
            cache[d] = _eval_modes(C[d], xc, yc, zc)
        return cache[d]

    v2 = None
    for d in range(3):
        v2 = vel(d) ** 2 if v2 is None else v2 + vel(d) ** 2
    vrms = np.sqrt(v2.mean())
    scale = np.sqrt(gamma * 1.0 / 1.0) / vrms
    b0 = np.array([0.1, 0.0, 0.0])
    shape = (ncell, ncell, ncell)
    e_const = 1.0 / (gamma - 1.0) + 0.5 * float(b0 @ b0)

    def fields(v):
        if v == RHO:
            return np.ones(shape)
        if MX <= v <= MZ:
            return vel(v - MX) * scale
        if v == EN:
            return e_const + 0.5 * v2 * scale ** 2
        return np.full(shape, b0[v - BX])

    return geom, fields, dict(gamma=gamma, steps=100, vrms=float(np.sqrt(gamma)))


def ragged_box(seed=20250810, gamma=5.0 / 3.0):
    """Periodic 288 x 288 x 296 box of z-layers of 16^3, 24^3 and 32^3 patches.

    Two 16-cell layers (18 x 18 patches each), three 24-cell layers (12 x 12) and six
    32-cell layers (9 x 9), in a seeded layer order; 1566 patches, 24.55 M cells.
    Orszag-Tang fields in x-y, invariant along z.  Patches are listed in a seeded random
    order and cut into bunches of sizes drawn uniformly from 8..512.
    """
    rng = np.random.default_rng(seed)
    layers = [16] * 2 + [24] * 3 + [32] * 6
    order = rng.permutation(len(layers))
    layers = [layers[i] for i in order]
    nxy = 288
    sizes, origins = [], []
    z0 = 0
    for s in layers:
        for j in range(nxy // s):
            for i in range(nxy // s):
                sizes.append([s, s, s])
                origins.append([i * s, j * s, z0])
        z0 += s
    sizes = np.array(sizes)
    origins = np.array(origins)
    perm = rng.permutation(len(sizes))
    sizes, origins = sizes[perm], origins[perm]
    bunches = []
    start = 0
    while start < len(sizes):
        b = int(rng.integers(8, 513))
        bunches.append(np.arange(start, min(start + b, len(sizes)), dtype=np.int64))
        start += b
    dx = 1.0 / nxy
    geom = Geometry(sizes, origins, [nxy, nxy, z0], [dx, dx, dx],
                    [[BC_PERIODIC] * 2] * 3, 3, bunches)
    (xc, yc, _), (xf, yf, _) = _centres(geom)
    U2 = _ot_fields(xc, yc, xf, yf, 1, gamma)

    def fields(v):
        return np.broadcast_to(U2[v], (z0, nxy, nxy))

    return geom, fields, dict(gamma=gamma, steps=50)


def _three_mode_velocity(rng, amp, geom):
    (xc, yc, zc), _ = _centres(geom)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    v = [np.zeros(Z.shape) for _ in range(3)]
    for _ in range(3):
        while True:
            k = rng.integers(-2, 3, size=3)
            if np.any(k != 0):
                break
        kf = k.astype(np.float64)
        e = rng.standard_normal(3)
        e = e - (e @ kf) / (kf @ kf) * kf
        e /= np.linalg.norm(e)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        s = np.sin(2 * np.pi * (kf[0] * X + kf[1] * Y + kf[2] * Z) + ph)
        for d in range(3):
            v[d] += amp * e[d] * s
    return v


def adjoint_box(ncell=64, patch=32, gamma=5.0 / 3.0, seed=20250811, target_seed=20250812):
    """Smooth periodic box for the adjoint rollout.

    rho = 1 + 0.01 sin(2 pi x), p = 1, B = (0.1, 0.05, 0), velocity = sum of three seeded
    sinusoids of amplitude 0.1 (wavevectors in {-2..2}^3 minus 0, directions perpendicular
    to k, random phases).  The target run starts from the same state with the velocity
    perturbed by 1e-2 times a second seeded three-mode field.
    Returns (geom, make_state(v) -> global conserved field, v0, v_target, meta).
    """
    geom = uniform_geometry([ncell] * 3, [patch] * 3, dx=[1.0 / ncell] * 3)
    (xc, yc, zc), _ = _centres(geom)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    rho = 1.0 + 0.01 * np.sin(2 * np.pi * X)
    p = np.ones_like(rho)
    b = (np.full_like(rho, 0.1), np.full_like(rho, 0.05), np.zeros_like(rho))
    v0 = _three_mode_velocity(np.random.default_rng(seed), 0.1, geom)
    dv = _three_mode_velocity(np.random.default_rng(target_seed), 1.0, geom)
    vt = [v0[d] + 1e-2 * dv[d] for d in range(3)]

    def make_state(v):
        return conserved_from_setup(rho, v, p, b, gamma)

    return geom, make_state, np.stack(v0), np.stack(vt), dict(gamma=gamma, steps=200, ckpt=10,
                                                                 rho=rho, p=p, b=b)


def small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=7, gamma=5.0 / 3.0, amp=0.3, bamp=0.2):
    """Small seeded 3D periodic box with smooth random fields (for parity tests).

    Density and pressure stay well positive; velocity and face B are sums of a few random
    Fourier modes (face B is taken divergence-free by building it as the discrete curl of
    a random edge potential).
    """
    geom = uniform_geometry(list(ncell), list(patch), dx=[1.0 / ncell[0], 1.0 / ncell[1], 1.0 / ncell[2]])
    rng = np.random.default_rng(seed)
    (xc, yc, zc), _ = _centres(geom)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")

    def smooth(a):
        s = np.zeros_like(X)
        for _ in range(3):
            k = rng.integers(-2, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            s += a * rng.uniform(0.3, 1.0) * np.sin(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
        return s

    rho = 1.0 + 0.5 * np.abs(smooth(0.5)) + 0.2
    p = 1.0 + 0.3 * smooth(0.5) ** 2
    vel = (smooth(amp), smooth(amp), smooth(amp))
    # divergence-free face field from a random edge-centred vector potential A:
    # Bx(i) = (Az(j+1)-Az(j))/dy - (Ay(k+1)-Ay(k))/dz, cyclic.
    h = bamp * geom.dx[0] / (2 * np.pi)
    Ax, Ay, Az = smooth(h), smooth(h), smooth(h)
    dxv = geom.dx

    def fwd(a, axis):
        return np.roll(a, -1, axis=axis) - a

    bx = fwd(Az, 1) / dxv[1] - fwd(Ay, 0) / dxv[2] + 0.1
    by = fwd(Ax, 0) / dxv[2] - fwd(Az, 2) / dxv[0] + 0.05
    bz = fwd(Ay, 2) / dxv[0] - fwd(Ax, 1) / dxv[1]
    U = conserved_from_setup(rho, vel, p, (bx, by, bz), gamma)
    return geom, U, dict(gamma=gamma)


def ragged_small(seed=5, gamma=5.0 / 3.0):
    """A small periodic 48 x 48 x 36 box tiled by z-layers of 8^3, 12^3 and 16^3 patches (in
    a seeded layer and patch order) with smooth seeded fields: the ragged layout of the
    mixed-size box at a size the oracle follows in seconds."""
    rng = np.random.default_rng(seed)
    layers = [8, 12, 16]
    layers = [layers[i] for i in rng.permutation(3)]
    nxy = 48
    sizes, origins = [], []
    z0 = 0
    for s in layers:
        for j in range(nxy // s):
            for i in range(nxy // s):
                sizes.append([s, s, s])
                origins.append([i * s, j * s, z0])
        z0 += s
    perm = rng.permutation(len(sizes))
    sizes, origins = np.array(sizes)[perm], np.array(origins)[perm]
    dx = 1.0 / nxy
    geom = Geometry(sizes, origins, [nxy, nxy, z0], [dx, dx, dx], [[BC_PERIODIC] * 2] * 3, 3)
    g2, U, meta = small_box(ncell=(nxy, nxy, z0), patch=(nxy, nxy, z0), seed=seed + 1000, gamma=gamma)
    return geom, U, dict(gamma=gamma)
