"""The allocation-free CFL entry point agrees with the handle-based one.

mhd_cfl_dt_uniform_noalloc serves callers that may not allocate device memory (a host
framework that owns and accounts for all device memory, a real-time loop): it needs no
handle and keeps its scratch in a static device array of the library.  Here it
is called through the C ABI, twice in a row on the same state and then on a second, smaller
bunch, and each result is checked against mhd_bunch_cfl_dt on the same data, within the
tolerances of the other CFL tests.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2508_09568_gb300 import capi
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-14, torch.float32: 2e-6}


def _noalloc(lib, state, rb, geom, gamma, courant, dt_dev, stream):
    n = geom.patch_n[0]
    dx = np.ascontiguousarray(geom.dx, dtype=np.float64)
    return lib.mhd_cfl_dt_uniform_noalloc(ct.c_void_p(state.data_ptr()), rb, geom.npatch, int(n[0]), int(n[1]),
                                          int(n[2]), int(geom.guard), dx.ctypes.data_as(capi.DP), float(gamma),
                                          float(courant), ct.c_void_p(dt_dev.data_ptr()),
                                          ct.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_noalloc_cfl_matches_handle_entry_point(dtype):
    from paper_2508_09568_gb300.bunch import MHDBunch
    lib = capi.load()
    rb = 8 if dtype == torch.float64 else 4
    cases = [W.small_box(ncell=(32, 32, 32), patch=(16, 16, 16), seed=31),
             W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=32),
             W.orszag_tang(ncell=64, patch=16)]
    for geom, U, meta in cases:
        b = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"], courant=0.8)
        b.upload(W.to_patches(U, geom))
        b.fill_guards()
        ref = b.cfl_dt()                      # existing entry point (synchronises)
        state = b.current()
        dt_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        for _ in range(2):                    # two calls in a row share the static array
            with torch.cuda.stream(b.stream):
                dt_dev.fill_(-1.0)
            capi.check(_noalloc(lib, state, rb, geom, meta["gamma"], 0.8, dt_dev, b.stream))
            b.stream.synchronize()
            got = float(dt_dev.item())
            assert abs(got - ref) <= TOL[dtype] * ref, (got, ref)
        b.close()


def test_noalloc_rejects_too_many_patches():
    lib = capi.load()
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    dx = (ct.c_double * 3)(0.1, 0.1, 0.1)
    rc = lib.mhd_cfl_dt_uniform_noalloc(ct.c_void_p(dummy.data_ptr()), 4, capi.MHD_NOALLOC_MAX_PATCHES + 1, 8, 8, 8,
                                        3, dx, 5.0 / 3.0, 0.8, ct.c_void_p(dummy.data_ptr()), None)
    assert rc == capi.MHD_EINVAL
    assert b"MHD_NOALLOC_MAX_PATCHES" in lib.mhd_last_error()


def test_noalloc_reports_a_nonphysical_cell_as_nan():
    """A cell with a negative density has no finite rate: the written dt is NaN (the
    handle API latches MHD_EPHYS for the same state), and the next call on a healthy
    state writes the finite dt again (the static array keeps no stale flag)."""
    from paper_2508_09568_gb300.bunch import MHDBunch
    lib = capi.load()
    geom, U, meta = W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=34)
    b = MHDBunch(geom, dtype=torch.float64, gamma=meta["gamma"], courant=0.8)
    b.upload(W.to_patches(U, geom))
    b.fill_guards()
    ref = b.cfl_dt()
    bad = U.copy()
    bad[0, 3, 4, 5] = -1.0
    b2 = MHDBunch(geom, dtype=torch.float64, gamma=meta["gamma"], courant=0.8)
    b2.upload(W.to_patches(bad, geom))
    b2.fill_guards()
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    capi.check(_noalloc(lib, b2.current(), 8, geom, meta["gamma"], 0.8, dt_dev, b2.stream))
    b2.stream.synchronize()
    assert np.isnan(float(dt_dev.item()))
    capi.check(_noalloc(lib, b.current(), 8, geom, meta["gamma"], 0.8, dt_dev, b.stream))
    b.stream.synchronize()
    assert abs(float(dt_dev.item()) - ref) <= TOL[torch.float64] * ref
    b.close()
    b2.close()
