"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on the same inputs."""
from __future__ import annotations

import numpy as np
import torch

from oracle import mhd as O
from paper_2508_09568_gb300 import workloads as W

TOL_STEP = {torch.float64: 1e-12, torch.float32: 1e-5}
# element-wise bound per step: max |a - b| over the interior cells of a variable, divided
# by the largest magnitude of that quantity (max_rel).  FP32: one cell's value comes from
# flux differences of O(1) terms (|F| ~ the largest total pressure or energy flux) with
# dt/dx <= 0.8 and a few hundred rounded operations each, so its error is a few 1e-6 of
# the scale; 1e-4 leaves a margin of about 10 and still fails a single cell that is off by
# 0.01 % of the scale, far below what a wrong face, edge or ragged-tail cell would give.
# FP64: the same argument with 2^-53 gives ~1e-13; 1e-10 is the same margin as the L1
# bound of multi-step runs.  Observed per step on a GB300 (Sod, Orszag-Tang 64^2, 3D boxes
# with ragged tiles): FP32 at most 1.4e-7, FP64 at most 3.6e-16.
TOL_MAX = {torch.float64: 1e-10, torch.float32: 1e-4}


def interior_global(flat, geom):
    return W.from_patches(np.asarray(flat, dtype=np.float64), geom)


def rel_l1(a, b, floor=1e-300):
    """Per-variable relative L1 difference sum|a-b| / sum|b| over interior cells (8 values)."""
    out = []
    for v in range(8):
        den = np.abs(b[v]).sum()
        num = np.abs(a[v] - b[v]).sum()
        out.append(num / den if den > floor else num)
    return np.array(out)


# scale groups of max_rel: momentum and face field are taken as vectors, so that a
# component that is zero everywhere (the 1D and 2D boxes, the uniform-field boxes) is
# measured against the magnitude of its vector
_GROUPS = ((0,), (1, 2, 3), (1, 2, 3), (1, 2, 3), (4,), (5, 6, 7), (5, 6, 7), (5, 6, 7))


def max_rel(a, b):
    """Per-variable max |a - b| over interior cells divided by the largest magnitude of the
    variable (of the momentum or face-field vector for their components)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = []
    for v in range(8):
        g = _GROUPS[v]
        if len(g) == 1:
            scale = np.abs(b[v]).max()
        else:
            scale = np.sqrt(sum(b[c] ** 2 for c in g)).max()
        num = np.abs(a[v] - b[v]).max()
        out.append(num / scale if scale > 0 else num)
    return np.array(out)


def assert_parity(got, ref, dtype, l1=None, mx=None, what="", b_vector=False):
    """Relative L1 per variable (the tolerance of the scheme's parity) and the element-wise
    bound, on interior arrays (8, ...).  b_vector: the relative L1 of the face field is taken
    over the field vector (R21), for boxes where one component is orders of magnitude below
    the others and its own L1 measures the rounding of the large ones."""
    l1 = TOL_STEP[dtype] if l1 is None else l1
    mx = TOL_MAX[dtype] if mx is None else mx
    e1 = rel_l1(got, ref)
    if b_vector:
        a, b = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
        e1[5:8] = np.abs(a[5:8] - b[5:8]).sum() / np.abs(b[5:8]).sum()
    em = max_rel(got, ref)
    assert np.all(e1 <= l1), (what, "rel L1", e1)
    assert np.all(em <= mx), (what, "max", em)
    return e1, em


def rounded(flat, dtype):
    """Input as the precision under test sees it (FP32 rounding for float32 runs)."""
    if dtype == torch.float32:
        return np.asarray(flat, dtype=np.float32).astype(np.float64)
    return np.asarray(flat, dtype=np.float64)


def oracle_bunch(geom, gamma, courant=0.8, limiter=0, dtype=torch.float64, riemann=0):
    return O.Bunch(geom, gamma, courant=courant, limiter=limiter, eps=O.HLLD_EPS[4 if dtype == torch.float32 else 8],
                   riemann=riemann)


def oracle_steps(geom, flat, gamma, dts, limiter=0, dtype=torch.float64, riemann=0):
    """Oracle: fill + step for each dt in dts; returns the final flat buffer."""
    B = oracle_bunch(geom, gamma, limiter=limiter, dtype=dtype, riemann=riemann)
    P = B.split(flat)
    for dt in dts:
        P = B.step(P, dt)
    return B.join(P)


def gpu_bunch(geom, flat, gamma, dtype, courant=0.8, limiter=0, mode=None, config=-1, riemann=0):
    from paper_2508_09568_gb300.bunch import MHDBunch
    b = MHDBunch(geom, dtype=dtype, gamma=gamma, courant=courant, limiter=limiter, riemann=riemann)
    if mode is not None:
        b.set_mode(mode, config)
    b.upload(flat)
    return b


def gpu_steps(b, dts):
    for dt in dts:
        b.fill_guards()
        b.step(dt)
    return b.download()
