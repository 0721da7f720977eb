"""The 2D Orszag-Tang vortex at its full size: 512^2 periodic cells as 256 patches of 32^2,
gamma = 5/3, run to t = 0.5 on the GPU.

* one step of the whole box from the initial state against the oracle (FP64 1e-12, FP32
  1e-5 relative L1 per variable);
* after the run to t = 0.5: the point symmetry of the vortex (rho(x) = rho(-x),
  u(x) = -u(-x), B(x) = -B(-x) about the box centre), mass and energy conserved, and
  div B within the rounding the CT update can add per step.  The symmetry bound is the oracle's own (1e-10) in FP64; FP32
  rounding breaks the mirror symmetry of the arithmetic, so there only conservation and
  div B are checked.
"""
import numpy as np
import pytest
import torch

from helpers import assert_parity, gpu_bunch, interior_global, oracle_steps, rounded
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _divb(G, dx):
    return (np.roll(G[5], -1, 2) - G[5]) / dx[0] + (np.roll(G[6], -1, 1) - G[6]) / dx[1]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_orszag_tang_full_size(dtype):
    geom, U, meta = W.orszag_tang(ncell=512, patch=32)
    gamma = meta["gamma"]
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, gamma, dtype)
    # one step from the initial state, whole box, against the oracle
    b.fill_guards()
    dt = b.cfl_dt()
    b.step(dt)
    got = interior_global(b.download(), geom)
    ref = interior_global(oracle_steps(geom, flat, gamma, [dt], dtype=dtype), geom)
    assert_parity(got, ref, dtype)
    # the run to t = 0.5 (last step clipped)
    b.upload(flat)
    t, k, t_end = 0.0, 0, meta["t_end"]
    while t < t_end:
        b.fill_guards()
        dt = min(b.cfl_dt(), t_end - t)
        b.step(dt)
        t += dt
        k += 1
    assert 200 < k < 5000
    G0 = interior_global(flat, geom)
    Gs = interior_global(b.download(), geom)
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    for v in (0, 4):
        assert abs(Gs[v].sum() - G0[v].sum()) <= tol * np.abs(G0[v]).sum(), v
    # div B: CT changes it per step only by the rounding of the four face updates of a
    # cell (at most about 4 ulp of max|B| in the working precision), so after k steps
    # |div B| dx <= k * 4 * eps * max|B| (FP64: within the conservation bound anyway)
    bmax = np.abs(Gs[5:7]).max()
    divb = np.max(np.abs(_divb(Gs, geom.dx))) * geom.dx[0] / bmax
    eps = np.finfo(np.float64 if dtype == torch.float64 else np.float32).eps / 2
    assert divb <= max(tol, k * 4 * eps), (divb, k)
    if dtype == torch.float64:
        r = Gs[0, 0]
        assert np.max(np.abs(r - r[::-1, ::-1])) / r.max() < 1e-10
        u = Gs[1, 0] / Gs[0, 0]
        assert np.max(np.abs(u + u[::-1, ::-1])) < 1e-10
        bx = Gs[5, 0]   # face x_{i-1/2} maps to face x_{N-i+1/2} = index N-i
        assert np.max(np.abs(bx + np.roll(bx[::-1, ::-1], 1, axis=1))) < 1e-10
    code, msg = b.error()
    assert code == 0, msg
