"""Pins of the oracle's use of each axis's own cell size (Sec. 2.1: the CT update of Eq. 12
and the flux differences divide by the spacing of the axis they difference along).

* div B stays at roundoff and mass, momentum and energy are conserved in a 3D box whose
  three cell sizes all differ: CT keeps the discrete divergence only when every EMF
  difference is divided by its own axis's spacing, so a swapped or shared spacing breaks
  it;
* a smooth MHD wave along one axis of a thin 3D box gives the same profile whichever axis
  carries it (the fields rotated cyclically with it) and whatever the spacings of the two
  transverse axes, and the same as the purely 1D run: the transverse differences are
  exact zeros, so a flux, predictor or CT term divided by another axis's spacing changes
  the result.
"""
import numpy as np

from oracle import mhd
from paper_2508_09568_gb300 import workloads as W

G53 = 5.0 / 3.0


def _run(geom, U, gamma, **kw):
    B = mhd.Bunch(geom, gamma)
    P = B.split(W.to_patches(U, geom))
    P, t, k = B.run(P, **kw)
    return W.from_patches(B.join(P), geom)


def _divb(G, dx):
    return (np.roll(G[5], -1, 2) - G[5]) / dx[0] + (np.roll(G[6], -1, 1) - G[6]) / dx[1] \
        + (np.roll(G[7], -1, 0) - G[7]) / dx[2]


def test_divb_and_conservation_with_three_cell_sizes():
    geom, U, meta = W.small_box(ncell=(24, 16, 12), patch=(8, 8, 6), seed=17)
    assert len(set(float(d) for d in geom.dx)) == 3
    scale = float(np.max(np.abs(U[5:8])))
    assert np.max(np.abs(_divb(U, geom.dx))) * min(geom.dx) / scale < 1e-14
    Gs = _run(geom, U, meta["gamma"], nsteps=8)
    assert np.all(np.isfinite(Gs))
    for v in range(5):
        rel = abs(Gs[v].sum() - U[v].sum()) / np.abs(U[v]).sum()
        assert rel < 1e-13, (v, rel)
    assert np.max(np.abs(_divb(Gs, geom.dx))) * min(geom.dx) / scale < 1e-13


N = 32          # cells along the wave
T = 4           # cells across it (at least the guard width)


def _wave_1d(x):
    """(rho, vx, vy, vz, p, Bx, By, Bz) of a smooth wave along x; Bx constant (div B = 0)."""
    s = 2 * np.pi * x
    return (1.0 + 0.2 * np.sin(s), 0.1 * np.sin(s + 1.0), 0.05 * np.cos(s), 0.03 * np.sin(2 * s),
            1.0 + 0.1 * np.cos(s + 0.5), 0.3 + 0 * x, 0.2 * np.sin(s + 0.3), 0.1 * np.cos(s))


def _wave_box(axis, dx_t):
    """The wave along `axis` of a periodic box of N x T x T cells (the long side on `axis`),
    cell size 1/N along it and dx_t = (the next axis's, the one after's) across; vectors
    rotated cyclically with the axis.  Returns (geom, U, profile selector)."""
    ncell = [T, T, T]
    ncell[axis] = N
    patch = [T, T, T]
    patch[axis] = N // 2
    dx = [0.0, 0.0, 0.0]
    dx[axis] = 1.0 / N
    dx[(axis + 1) % 3], dx[(axis + 2) % 3] = dx_t
    geom = W.uniform_geometry(ncell, patch, dx=dx)
    x = (np.arange(N) + 0.5) / N
    xf = np.arange(N) / N                       # the low faces along the wave
    rho, vx, vy, vz, p, bx, by, bz = _wave_1d(x)
    _, _, _, _, _, bxf, _, _ = _wave_1d(xf)
    shape = [1, 1, 1]                           # (z, y, x) array axes: array axis 2 - axis
    shape[2 - axis] = N

    def field(a):
        return np.broadcast_to(np.reshape(a, shape), (ncell[2], ncell[1], ncell[0])).copy()

    vel = [None] * 3
    bf = [None] * 3
    for k, (v, b) in enumerate(((vx, bxf), (vy, by), (vz, bz))):
        vel[(axis + k) % 3] = field(v)
        bf[(axis + k) % 3] = field(b)
    U = W.conserved_from_setup(field(rho), tuple(vel), field(p), tuple(bf), G53)
    sel = [0, 0, 0]
    sel[2 - axis] = slice(None)

    def profile(G):
        """The eight variables along the wave, vectors rotated back to the wave's frame."""
        out = []
        for v in range(8):
            src = v
            if 1 <= v <= 3:
                src = 1 + (axis + v - 1) % 3
            elif v >= 5:
                src = 5 + (axis + v - 5) % 3
            out.append(G[src][tuple(sel)])
        return np.array(out)

    return geom, U, profile


def test_wave_along_each_axis_ignores_transverse_cell_sizes():
    dt, steps = 0.2 / N, 6                    # fixed dt (the CFL dt would see the transverse sizes)
    runs = []
    for axis, dx_t in ((0, (0.37, 0.23)), (1, (0.29, 0.41)), (2, (0.53, 0.19)), (0, (0.011, 0.7))):
        geom, U, profile = _wave_box(axis, dx_t)
        runs.append(profile(_run(geom, U, G53, nsteps=steps, dt_fixed=dt)))
    # the purely 1D run (transverse axes collapsed)
    geom = W.uniform_geometry([N, 1, 1], [N // 2, 1, 1], dx=[1.0 / N, 1.0, 1.0])
    x = (np.arange(N) + 0.5) / N
    rho, vx, vy, vz, p, bx, by, bz = _wave_1d(x)
    bxf = _wave_1d(np.arange(N) / N)[5]
    f = lambda a: np.reshape(a, (1, 1, N))
    U1 = W.conserved_from_setup(f(rho), (f(vx), f(vy), f(vz)), f(p), (f(bxf), f(by), f(bz)), G53)
    ref = _run(geom, U1, G53, nsteps=steps, dt_fixed=dt)[:, 0, 0, :]
    init = np.array([W.conserved_from_setup(f(rho), (f(vx), f(vy), f(vz)), f(p), (f(bxf), f(by), f(bz)),
                                            G53)[v, 0, 0] for v in range(8)])
    assert np.max(np.abs(ref - init)) > 1e-3          # the wave has moved
    for r in runs:
        assert np.max(np.abs(r - ref)) <= 1e-13 * np.max(np.abs(ref)), np.max(np.abs(r - ref))
