"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on the same inputs."""
from __future__ import annotations

import numpy as np
import torch

from oracle import mhd as O
from paper_2508_09568_gb300 import workloads as W

TOL_STEP = {torch.float64: 1e-12, torch.float32: 1e-5}


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
