"""The seeded inputs against the recipes they state (host only).

* turbulence box: rho = 1, p = 1, B = (0.1, 0, 0) everywhere; the velocity is solenoidal
  (k . v(k) = 0 in every Fourier bin), band-limited to 1 <= |k| <= kmax with vector
  amplitude proportional to |k|^-2 in every populated bin, and has rms speed
  sqrt(gamma p / rho) (rms Mach 1); the same seed gives the same field, another seed
  another;
* ragged box: 1566 patches (648 of 16^3, 432 of 24^3, 486 of 32^3) tile the periodic
  288 x 288 x 296 box exactly once, and the bunches of 8..512 patches cover the list in
  order;
* adjoint box: rho = 1 + 0.01 sin(2 pi x), p = 1, B = (0.1, 0.05, 0); the starting
  velocity is three solenoidal Fourier modes of amplitude 0.1, and the target's velocity
  adds 1e-2 times three more of unit amplitude;
* Orszag-Tang: rho = 25/(36 pi), p = 5/(12 pi), v = (-sin 2 pi y, sin 2 pi x), and face
  B = B0 (-sin 2 pi y, sin 4 pi x) with B0 = 1/sqrt(4 pi) at the faces' own coordinates.
"""
import numpy as np

from paper_2508_09568_gb300 import workloads as W

G53 = 5.0 / 3.0


def _bins(v):
    """Fourier coefficients of the three components (z, y, x arrays) and the integer
    wavevector of every bin."""
    N = v[0].shape
    F = np.stack([np.fft.fftn(c) / c.size for c in v])
    kz, ky, kx = np.meshgrid(*(np.fft.fftfreq(n, 1.0 / n) for n in N), indexing="ij")
    return F, (kx, ky, kz)


def _pressure(U, gamma):
    """Gas pressure of a conserved field whose face B is uniform along its own axis."""
    rho = U[0]
    kin = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    mag = 0.5 * (U[5] ** 2 + U[6] ** 2 + U[7] ** 2)
    return (gamma - 1.0) * (U[4] - kin - mag)


def test_turbulence_box_recipe():
    kmax = 6
    geom, fields, meta = W.turbulence_box(ncell=32, patch=16, kmax=kmax)
    U = np.stack([np.asarray(fields(v), dtype=np.float64) for v in range(8)])
    assert np.all(U[0] == 1.0)
    assert np.all(U[5] == 0.1) and np.all(U[6] == 0.0) and np.all(U[7] == 0.0)
    assert np.max(np.abs(_pressure(U, G53) - 1.0)) < 1e-13
    v = [U[1 + d] / U[0] for d in range(3)]
    vrms = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    assert abs(vrms - np.sqrt(G53)) < 1e-13 * np.sqrt(G53)
    F, (kx, ky, kz) = _bins(v)
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    amp = np.sqrt(np.sum(np.abs(F) ** 2, axis=0))
    top = amp.max()
    assert np.max(np.abs(kx * F[0] + ky * F[1] + kz * F[2])) < 1e-12 * top           # solenoidal
    band = (kk >= 1.0) & (kk <= kmax)
    assert np.max(amp[~band]) < 1e-12 * top                                           # band-limited
    scaled = amp[band] * kk[band] ** 2                                                # |k|^-2 amplitude
    assert np.all(amp[band] > 1e-6 * top)
    assert np.max(np.abs(scaled / scaled.mean() - 1.0)) < 1e-10
    # seeded: the same seed the same field, another seed another
    _, f2, _ = W.turbulence_box(ncell=32, patch=16, kmax=kmax)
    _, f3, _ = W.turbulence_box(ncell=32, patch=16, kmax=kmax, seed=1)
    assert np.array_equal(np.asarray(f2(1)), U[1])
    assert not np.allclose(np.asarray(f3(1)), U[1])


def test_ragged_box_tiles_the_box_once():
    geom, fields, meta = W.ragged_box()
    sizes = geom.patch_n[:, 0]
    assert np.all(geom.patch_n == sizes[:, None])
    counts = {int(s): int(np.sum(sizes == s)) for s in np.unique(sizes)}
    assert counts == {16: 648, 24: 432, 32: 486}
    assert list(geom.domain) == [288, 288, 296]
    cover = np.zeros((296, 288, 288), dtype=np.int8)
    for o, n in zip(geom.origin, geom.patch_n):
        cover[o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] += 1
    assert np.all(cover == 1)
    assert geom.interior_cells() == 288 * 288 * 296 == 24_551_424
    flat = np.concatenate(geom.bunches)
    assert np.array_equal(flat, np.arange(geom.npatch))
    assert all(8 <= len(b) <= 512 for b in geom.bunches[:-1]) and 1 <= len(geom.bunches[-1]) <= 512


def test_adjoint_box_recipe():
    geom, make_state, v0, vt, meta = W.adjoint_box(ncell=32, patch=16)
    (xc, _, _), _ = W._centres(geom)
    U = make_state(v0)
    assert np.max(np.abs(U[0] - (1.0 + 0.01 * np.sin(2 * np.pi * xc))[None, None, :])) < 1e-15
    assert np.all(U[5] == 0.1) and np.all(U[6] == 0.05) and np.all(U[7] == 0.0)
    assert np.max(np.abs(_pressure(U, G53) - 1.0)) < 1e-13
    for v in (v0, vt):
        F, (kx, ky, kz) = _bins(list(v))
        amp = np.sqrt(np.sum(np.abs(F) ** 2, axis=0))
        assert np.max(np.abs(kx * F[0] + ky * F[1] + kz * F[2])) < 1e-12 * amp.max()
    for v, a in ((v0, 0.1), ((vt - v0) / 1e-2, 1.0)):
        F, _ = _bins(list(v))
        amp = np.sqrt(np.sum(np.abs(F) ** 2, axis=0))
        assert np.sum(amp > 1e-9 * amp.max()) <= 6        # three real modes: six bins at most
        assert np.max(np.abs(v)) <= 3 * a * (1 + 1e-12)    # three modes of amplitude a
        assert np.max(amp) <= 1.5 * a                     # a bin holds at most a/2 per mode


def test_orszag_tang_recipe():
    geom, U, meta = W.orszag_tang(ncell=64, patch=16)
    (xc, yc, _), _ = W._centres(geom)
    b0 = 1.0 / np.sqrt(4.0 * np.pi)
    assert np.all(U[0] == 25.0 / (36.0 * np.pi))
    assert np.max(np.abs(U[1] / U[0] + np.sin(2 * np.pi * yc)[None, :, None])) < 1e-15
    assert np.max(np.abs(U[2] / U[0] - np.sin(2 * np.pi * xc)[None, None, :])) < 1e-15
    # Bx at x-faces (x_f, y_c), By at y-faces (x_c, y_f)
    assert np.max(np.abs(U[5] + b0 * np.sin(2 * np.pi * yc)[None, :, None])) < 1e-15
    assert np.max(np.abs(U[6] - b0 * np.sin(4 * np.pi * xc)[None, None, :])) < 1e-15
    assert np.max(np.abs(_pressure(U, G53) - 5.0 / (12.0 * np.pi))) < 1e-13
