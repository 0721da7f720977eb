"""Trajectories against the oracle: many steps on both sides with the same dt sequence (the
oracle's own CFL steps, fed to the GPU), compared at the end, so that the growth of the
differences along a run is measured, not one step from a shared state.

* Orszag-Tang vortex, 512^2 as 256 patches of 32^2 (the vortex configuration), from the
  exact initial state: the FP64 GPU run after 200 steps and at t = 0.1 within 1e-10
  relative L1 per variable; the FP32 GPU run (from the FP32-rounded initial state) at
  t = 0.1 within 1e-3.
* The benchmark's turbulence field and patch geometry (32^3 patches, Mach 1, k <= 8) on a
  64^3 box of 8 patches, a size the oracle follows in seconds per step: FP64 after 100
  steps within 1e-10, FP32 within 1e-3.

The oracle runs once per workload in FP64; the FP32 GPU run is measured against it, so its
difference holds both the FP32 arithmetic and the rounding of the initial state.  Element
by element (max over cells of |a - b| over the variable's scale, momentum and field as
vectors): FP64 1e-12, FP32 1e-4.  Observed on a GB300: FP64 1.7e-15 relative L1 and 1.2e-14
element-wise on the vortex, 6e-16 / 1.8e-15 on the turbulence field; FP32 6.6e-7 / 4.6e-6
and 2.5e-7 / 6.9e-7, so the bounds leave margins of 20 or more while still failing a run
that went wrong in one region.
"""
import numpy as np
import pytest
import torch

from helpers import assert_parity, gpu_bunch, interior_global, oracle_bunch, rounded
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_run(geom, flat, gamma, keep, t_end=None, nsteps=None):
    """FP64 oracle run with its own CFL steps (the last clipped to t_end); returns the dt
    sequence and the interior state after each step count in keep (and at the end)."""
    ob = oracle_bunch(geom, gamma)
    P = ob.split(flat)
    dts, snaps, t = [], {}, 0.0
    while True:
        if nsteps is not None and len(dts) >= nsteps:
            break
        if t_end is not None and t >= t_end * (1 - 1e-14):
            break
        dt = ob.cfl_dt(ob.fill_guards(P))
        if t_end is not None and t + dt > t_end:
            dt = t_end - t
        P = ob.step(P, dt)
        t += dt
        dts.append(dt)
        if len(dts) in keep:
            snaps[len(dts)] = interior_global(ob.join(P), geom)
    snaps["end"] = interior_global(ob.join(P), geom)
    return dts, snaps


def _gpu_run(geom, flat, gamma, dtype, dts, keep):
    b = gpu_bunch(geom, rounded(flat, dtype), gamma, dtype)
    snaps = {}
    for k, dt in enumerate(dts, 1):
        b.fill_guards()
        b.step(dt)
        if k in keep:
            snaps[k] = interior_global(b.download(), geom)
    snaps["end"] = interior_global(b.download(), geom)
    code, msg = b.error()
    assert code == 0, msg
    b.close()
    return snaps


def test_orszag_tang_trajectory_fp64_200_steps_and_fp32_to_t01():
    geom, U, meta = W.orszag_tang(ncell=512, patch=32)
    gamma = meta["gamma"]
    flat = W.to_patches(U, geom)
    dts, ref = _oracle_run(geom, flat, gamma, keep={200}, t_end=0.1)
    assert len(dts) > 200
    got = _gpu_run(geom, flat, gamma, torch.float64, dts, keep={200})
    assert_parity(got[200], ref[200], torch.float64, l1=1e-10, mx=1e-12, what="f64 200 steps")
    assert_parity(got["end"], ref["end"], torch.float64, l1=1e-10, mx=1e-12, what="f64 t=0.1")
    got = _gpu_run(geom, flat, gamma, torch.float32, dts, keep=set())
    assert_parity(got["end"], ref["end"], torch.float32, l1=1e-3, mx=1e-4, what="f32 t=0.1")


def test_turbulence_field_64_cubed_100_steps():
    geom, fields, meta = W.turbulence_box(ncell=64, patch=32)
    gamma = meta["gamma"]
    flat = W.to_patches(fields, geom)
    dts, ref = _oracle_run(geom, flat, gamma, keep=set(), nsteps=100)
    for dtype, l1, mx in ((torch.float64, 1e-10, 1e-12), (torch.float32, 1e-3, 1e-4)):
        got = _gpu_run(geom, flat, gamma, dtype, dts, keep=set())
        assert_parity(got["end"], ref["end"], dtype, l1=l1, mx=mx, what=str(dtype))
