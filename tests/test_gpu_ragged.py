"""Ragged bunches (patches of several sizes in one launch) against the oracle.

* a small box of 8^3 / 12^3 / 16^3 patches: per-step parity (FP64 1e-12, FP32 1e-5), bit-exact
  guard fill, and bitwise identical results from every launch mode and tile configuration;
* the full ragged box (288 x 288 x 296 cells, 1566 patches of 16^3 / 24^3 / 32^3, OT fields):
  one FP32 step of the whole bunch in one persistent launch, compared patch by patch with the
  oracle on a sample of patches of each size, and conservation / div B over 50 steps.
"""
import numpy as np
import pytest
import torch

from helpers import assert_parity, gpu_bunch, gpu_steps, interior_global, oracle_bunch, oracle_steps, rounded
from oracle import mhd as O
from paper_2508_09568_gb300 import capi
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_ragged_small_per_step_parity(dtype):
    geom, U, meta = W.ragged_small()
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    for _ in range(2):
        ob = oracle_bunch(geom, meta["gamma"], dtype=dtype)
        dt = ob.cfl_dt(ob.fill_guards(ob.split(flat)))
        ref = oracle_steps(geom, flat, meta["gamma"], [dt], dtype=dtype)
        b.upload(flat)
        got = gpu_steps(b, [dt])
        assert_parity(interior_global(got, geom), interior_global(ref, geom), dtype)
        flat = rounded(got, dtype)


def test_ragged_small_fill_and_modes():
    geom, U, meta = W.ragged_small()
    flat = W.to_patches(U, geom)
    b = gpu_bunch(geom, flat, meta["gamma"], torch.float64)
    b.fill_guards()
    ob = oracle_bunch(geom, meta["gamma"])
    assert np.array_equal(b.download(), ob.join(ob.fill_guards(ob.split(flat))))
    outs = []
    for mode in (capi.MHD_MODE_PER_PATCH, capi.MHD_MODE_BUNCHED, capi.MHD_MODE_PERSISTENT):
        for cfg in range(b.num_configs()):
            b.set_mode(mode, cfg)
            b.upload(flat)
            outs.append(interior_global(gpu_steps(b, [2e-3]), geom))
    # per-class configurations (one persistent launch per configuration in use), before
    # and after the autotuner assigned them; the autotuner leaves the state as it was
    b.set_mode(capi.MHD_MODE_MIXED, -1)
    b.upload(flat)
    outs.append(interior_global(gpu_steps(b, [2e-3]), geom))
    b.upload(flat)
    b.autotune(None)
    assert np.array_equal(interior_global(b.download(), geom), interior_global(flat, geom))
    n0 = b.launch_count()
    outs.append(interior_global(gpu_steps(b, [2e-3]), geom))
    assert 2 <= b.launch_count() - n0 <= 1 + b.num_configs()   # fill + one launch per configuration in use
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_bunch_lists_equal_one_launch():
    """MHD_MODE_BUNCH_LISTS (one persistent launch per bunch, the paper's bunches of
    patches) gives bitwise the state of the single persistent launch, with one launch per
    bunch; bad lists are rejected and change nothing."""
    geom, U, meta = W.ragged_small()
    flat = W.to_patches(U, geom)
    rng = np.random.default_rng(11)
    perm = rng.permutation(geom.npatch)
    cuts = np.sort(rng.choice(np.arange(1, geom.npatch), 3, replace=False))
    bunches = np.split(perm, cuts)
    for dtype in (torch.float64, torch.float32):
        b = gpu_bunch(geom, flat, meta["gamma"], dtype)
        b.set_mode(capi.MHD_MODE_PERSISTENT, 0)
        ref = interior_global(gpu_steps(b, [2e-3, 2e-3]), geom)
        with pytest.raises(capi.MHDError):
            b.set_bunches([perm[:-1]])                 # a patch missing
        with pytest.raises(capi.MHDError):
            b.set_bunches([perm, perm[:1]])            # a patch twice
        b.set_mode(capi.MHD_MODE_BUNCH_LISTS, 0)
        with pytest.raises(capi.MHDError) as ei:       # no bunches yet
            gpu_steps(b, [2e-3])
        assert ei.value.code == capi.MHD_ESTATE
        b.set_bunches(bunches)
        b.upload(flat)
        n0 = b.launch_count()
        got = interior_global(gpu_steps(b, [2e-3, 2e-3]), geom)
        assert b.launch_count() - n0 == 2 * (1 + len(bunches))   # fill + one launch per bunch, per step
        assert np.array_equal(got, ref)
        b.close()


def test_ragged_box_full_size_sampled_and_invariants():
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, fields, meta = W.ragged_box()
    gamma = meta["gamma"]
    flat = W.to_patches(fields, geom, dtype=np.float32)
    b = MHDBunch(geom, dtype=torch.float32, gamma=gamma)
    b.set_mode(capi.MHD_MODE_PERSISTENT, b.autotune(None))
    b.upload(flat)
    dt = 0.05 * geom.dx[0]           # a fixed step well inside the CFL limit, shared by both sides
    b.fill_guards()
    b.step(dt)
    got = b.download()
    # oracle on a sample of patches of each size, from the same FP32-rounded input
    G = torch.tensor(np.stack([fields(v) for v in range(8)]).astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(4)
    offs = geom.offsets()
    for size in (16, 24, 32):
        idx = np.where(geom.patch_n[:, 0] == size)[0]
        for p in rng.choice(idx, 2, replace=False):
            Up = O.window(G, geom.origin[p], geom.patch_n[p], geom.gvec, geom.domain, geom.bc)
            out = O.step(Up[None], dt, geom.active, geom.dx, gamma, eps=O.HLLD_EPS[4], gvec=geom.gvec,
                         n=geom.patch_n[p])[0].numpy()
            Z, Y, X = geom.padded(p)
            gp = got[offs[p]: offs[p] + 8 * X * Y * Z].reshape(8, Z, Y, X).astype(np.float64)
            sl = (slice(None),) + tuple(slice(3, 3 + size) for _ in range(3))
            assert_parity(gp[sl], out[sl], torch.float32, what=(size, int(p)))
    # 50 steps of the whole box: conservation and div B
    G0 = W.from_patches(flat, geom)
    b.upload(flat)
    for _ in range(50):
        b.fill_guards()
        b.step(b.cfl_dt())
    Gn = W.from_patches(b.download().astype(np.float64), geom)
    for v in (0, 1, 2, 4):
        ref = np.abs(G0[v]).sum()
        assert abs(Gn[v].sum() - G0[v].sum()) <= 1e-5 * ref, v
    dx = geom.dx
    d = (np.roll(Gn[5], -1, 2) - Gn[5]) / dx[0] + (np.roll(Gn[6], -1, 1) - Gn[6]) / dx[1] + \
        (np.roll(Gn[7], -1, 0) - Gn[7]) / dx[2]
    assert np.max(np.abs(d)) * dx[0] / np.sqrt((Gn[5:8] ** 2).mean()) < 1e-5
    code, msg = b.error()
    assert code == 0, msg
