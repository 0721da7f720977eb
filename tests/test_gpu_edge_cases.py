"""Degenerate cases of the method on the GPU.

* a single periodic patch (its guard zone is its own interior, wrapped): one step against
  the oracle;
* dt = 0: the update adds exact zeros, so the interior is bitwise unchanged;
* a uniform state: every flux and EMF difference is exactly zero, so it stays bitwise
  uniform (and its CFL dt is the closed form C / sum_d (|u_d| + c_f,d) / dx_d).
"""
import math

import numpy as np
import pytest
import torch

from helpers import assert_parity, gpu_bunch, gpu_steps, interior_global, oracle_steps, rounded
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_single_periodic_patch(dtype):
    geom, U, meta = W.small_box(ncell=(8, 8, 8), patch=(8, 8, 8), seed=41)
    assert geom.npatch == 1
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    b.fill_guards()
    dt = b.cfl_dt()
    b.step(dt)
    got = interior_global(b.download(), geom)
    ref = interior_global(oracle_steps(geom, flat, meta["gamma"], [dt], dtype=dtype), geom)
    assert_parity(got, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_zero_dt_leaves_the_state_unchanged(dtype):
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=42)
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    got = interior_global(gpu_steps(b, [0.0, 0.0]), geom)
    assert np.array_equal(got, interior_global(flat, geom))


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_uniform_state_is_stationary(dtype):
    geom = W.uniform_geometry([16, 16, 16], [8, 8, 8], dx=[1 / 16] * 3)
    gamma = 5.0 / 3.0
    rho, vel, p, B = 1.3, (0.2, -0.1, 0.05), 0.8, (0.3, -0.2, 0.1)
    N = (16, 16, 16)
    one = np.ones(N)
    U = W.conserved_from_setup(rho * one, tuple(v * one for v in vel), p * one, tuple(c * one for c in B), gamma)
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, gamma, dtype)
    b.fill_guards()
    dt = b.cfl_dt()
    # closed form of the CFL dt of a uniform state (sum over the three axes)
    b2 = sum(c * c for c in B) / rho
    cs2 = gamma * p / rho
    rate = 0.0
    for d in range(3):
        cf = math.sqrt(0.5 * (cs2 + b2 + math.sqrt((cs2 + b2) ** 2 - 4 * cs2 * B[d] ** 2 / rho)))
        rate += (abs(vel[d]) + cf) * 16
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert abs(dt - 0.8 / rate) <= tol * dt
    got = interior_global(gpu_steps(b, [dt, dt]), geom)
    assert np.array_equal(got, interior_global(flat, geom))


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
@pytest.mark.parametrize("shape", [(4096, 8, 8), (8, 8, 4096)], ids=["x4096", "z4096"])
def test_largest_patch_extent(dtype, shape):
    """The largest patch extent the library accepts (4096 cells) along x (128 tiles of 32 in
    a row, 64-bit offsets across a 4,102-cell row) and along z (a tile marching 4,096
    planes): one periodic patch, one step against the oracle.  On the 4096 x 8 x 8 patch the
    seeded B_z is about 1e-3 of |B|, so the face field's relative L1 is taken as a vector
    (R21)."""
    geom, U, meta = W.small_box(ncell=shape, patch=shape, seed=43)
    assert geom.npatch == 1
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    b.fill_guards()
    dt = b.cfl_dt()
    b.step(dt)
    got = interior_global(b.download(), geom)
    ref = interior_global(oracle_steps(geom, flat, meta["gamma"], [dt], dtype=dtype), geom)
    assert_parity(got, ref, dtype, b_vector=True)
    code, msg = b.error()
    assert code == 0, msg
