"""Asynchronous per-patch stepping (mhd_bunch_advance_async) against the oracle.

The GPU run records every round (the patches it updated and the dt each took).  The
oracle replays that schedule in FP64 and checks it: each round's patches are exactly the
ready ones by the rule (short of the target time, no neighbour earlier), each dt is the
patch's own CFL dt (clipped to the target time), every patch ends at the target time, and
the final states agree.
"""
import numpy as np
import pytest
import torch

from helpers import assert_parity, interior_global, rounded
from oracle import mhd as O
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(geom, U, gamma, dtype, spans=3.0):
    from paper_2508_09568_gb300.bunch import MHDBunch
    flat = rounded(W.to_patches(U, geom), dtype)
    ob = O.Bunch(geom, gamma)
    t_span = spans * ob.cfl_dt(ob.fill_guards(ob.split(flat)))
    b = MHDBunch(geom, dtype=dtype, gamma=gamma)
    b.upload(flat)
    rounds, updates = b.advance_async(t_span)
    log = b.async_rounds(rounds)
    code, msg = b.error()
    assert code == 0, msg
    ab = O.AsyncBunch(geom, gamma, eps=O.HLLD_EPS[4 if dtype == torch.float32 else 8])
    final, ready_sets, local_dts, t_cur = ab.replay(ob.split(flat), log, t_span)
    return b, flat, t_span, rounds, updates, log, final, ready_sets, local_dts, t_cur


@pytest.mark.parametrize("dtype,tol_dt,tol,tol_max", [(torch.float64, 1e-12, 1e-11, 1e-10),
                                                     (torch.float32, 2e-6, 5e-5, 5e-4)], ids=["f64", "f32"])
def test_async_schedule_and_states_match_oracle(dtype, tol_dt, tol, tol_max):
    # velocity amplitude large enough that the patches' own time steps differ
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=33, amp=0.9)
    b, flat, t_span, rounds, updates, log, final, ready_sets, local_dts, t_cur = _run(geom, U, meta["gamma"], dtype)
    P = geom.npatch
    assert all(t == t_span for t in t_cur)
    for (plist, dts), rs, ldt in zip(log, ready_sets, local_dts):
        assert list(plist) == rs
        assert np.allclose(dts, ldt, rtol=tol_dt, atol=0)
    assert updates == sum(len(p) for p, _ in log)
    assert any(len(p) < P for p, _ in log)          # genuinely asynchronous rounds
    ob = O.Bunch(geom, meta["gamma"])
    ref = interior_global(ob.join(final), geom)
    got = interior_global(b.download(), geom)
    assert_parity(got, ref, dtype, l1=tol, mx=tol_max)


def test_async_ragged_bunch_fp64():
    geom, U, meta = W.ragged_small()
    b, flat, t_span, rounds, updates, log, final, ready_sets, local_dts, t_cur = _run(geom, U, meta["gamma"],
                                                                                      torch.float64, spans=2.0)
    assert all(t == t_span for t in t_cur)
    for (plist, dts), rs, ldt in zip(log, ready_sets, local_dts):
        assert list(plist) == rs
        assert np.allclose(dts, ldt, rtol=1e-12, atol=0)
    ob = O.Bunch(geom, meta["gamma"])
    assert_parity(interior_global(b.download(), geom), interior_global(ob.join(final), geom), torch.float64,
                  l1=1e-11, mx=1e-10)


def test_async_many_rounds_and_max_rounds_cut():
    """More rounds than the device scheduler enqueues between two reads of its record (32):
    the schedule still replays on the oracle across the batch boundaries.  A second run cut
    short by max_rounds reports MHD_ESTATE and records exactly the first max_rounds rounds
    of the full run, bitwise."""
    from paper_2508_09568_gb300 import capi
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=33, amp=0.9)
    b, flat, t_span, rounds, updates, log, final, ready_sets, local_dts, t_cur = _run(geom, U, meta["gamma"],
                                                                                      torch.float64, spans=12.0)
    assert rounds > 40
    assert all(t == t_span for t in t_cur)
    for (plist, dts), rs, ldt in zip(log, ready_sets, local_dts):
        assert list(plist) == rs
        assert np.allclose(dts, ldt, rtol=1e-12, atol=0)
    ob = O.Bunch(geom, meta["gamma"])
    assert_parity(interior_global(b.download(), geom), interior_global(ob.join(final), geom), torch.float64,
                  l1=1e-11, mx=1e-10)
    cut = rounds - 5
    b2 = MHDBunch(geom, dtype=torch.float64, gamma=meta["gamma"])
    b2.upload(flat)
    with pytest.raises(capi.MHDError) as ei:
        b2.advance_async(t_span, max_rounds=cut)
    assert ei.value.code == capi.MHD_ESTATE
    log2 = b2.async_rounds(cut)
    for (p1, d1), (p2, d2) in zip(log[:cut], log2):
        assert np.array_equal(p1, p2)
        assert np.array_equal(d1, d2)


def test_async_nonphysical_state_is_reported():
    """Failure detection without a GPU fault: a patch whose every density is negative has no
    finite CFL rate, so its dt is not finite; the device scheduler sets that dt to 0 and
    schedules no further round, and the call returns MHD_EPHYS after one round."""
    from paper_2508_09568_gb300 import capi
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, U, meta = W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=1)
    U = U.copy()
    U[0, 0:8, 0:8, 0:8] = -1.0        # every cell of the patch at the origin
    b = MHDBunch(geom, dtype=torch.float64, gamma=meta["gamma"])
    b.upload(W.to_patches(U, geom))
    with pytest.raises(capi.MHDError) as ei:
        b.advance_async(1e-2)
    assert ei.value.code == capi.MHD_EPHYS
    assert len(b.async_rounds(1)[0][0]) == geom.npatch   # round 0: every patch (all at t = 0)
    with pytest.raises(capi.MHDError):                     # and no round after it
        b.async_rounds(2)
    code, msg = b.error()
    assert code == 0, msg          # the error word was read (and cleared) by the call
