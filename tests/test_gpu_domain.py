"""Slab handles (mhd_bunch_set_slab) and the split-box driver (domain.py) on one GPU.

A box cut into z-layer slabs, each held by its own slab handle with two halo layers, steps
exactly as the undivided box: every guard value, the global dt (the minimum of the slabs'
dts) and every updated cell bitwise equal, for one, two and three slabs, periodic and
outflow z boundaries, FP64 and FP32.  The slabs exchange their layers through device
copies (step_local) or, as one rank of a process group of one, through exchange_halos
(step_distributed, its own neighbour); the exchange between GPUs is the same
exchange_halos over NCCL (its message pattern is checked with gloo in
tests/test_domain_split.py).
"""
import numpy as np
import pytest
import torch

from helpers import rounded
from paper_2508_09568_gb300 import capi
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _box(bcz):
    g0, U, meta = W.small_box(ncell=(32, 32, 96), patch=(16, 16, 16), seed=53)
    bc = [[W.BC_PERIODIC, W.BC_PERIODIC], [W.BC_PERIODIC, W.BC_PERIODIC], [bcz, bcz]]
    return W.uniform_geometry([32, 32, 96], [16, 16, 16], dx=g0.dx, bc=bc), U, meta


def _reference(geom, flat, gamma, dtype, nsteps):
    from paper_2508_09568_gb300.bunch import MHDBunch
    b = MHDBunch(geom, dtype=dtype, gamma=gamma)
    b.upload(flat)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dts = []
    for _ in range(nsteps):
        b.fill_cfl_device(dt)
        b.step_device_dt(dt)
        b.stream.synchronize()
        dts.append(float(dt.item()))
    out = b.download()
    b.close()
    return out, dts


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("bcz", ["periodic", "outflow"])
def test_slabs_step_as_the_undivided_box(dtype, bcz):
    from paper_2508_09568_gb300.domain import SlabDomain, partition, step_distributed, step_local
    geom, U, meta = _box(W.BC_PERIODIC if bcz == "periodic" else W.BC_OUTFLOW)
    flat = rounded(W.to_patches(U, geom), dtype)
    want, want_dts = _reference(geom, flat, meta["gamma"], dtype, 3)
    want_i = W.from_patches(want.astype(np.float64), geom)
    nl = int(geom.domain[2] // geom.patch_n[0][2])
    for nslab in (1, 2, 3):
        doms = [SlabDomain(geom, z0, z1, dtype=dtype, gamma=meta["gamma"]) for z0, z1 in partition(nl, nslab)]
        for d in doms:
            d.load(flat)
        dts = [step_local(doms) for _ in range(3)]
        got = np.full(flat.shape, np.nan)
        for d in doms:
            d.store(got)
            code, msg = d.b.error()
            assert code == 0, msg
            d.close()
        assert dts == want_dts, nslab
        assert np.array_equal(W.from_patches(got, geom), want_i), nslab
    # one rank of a process group of one: exchange_halos with itself
    dom = SlabDomain(geom, 0, nl, dtype=dtype, gamma=meta["gamma"])
    dom.load(flat)
    dts = [step_distributed(dom, 0, 1) for _ in range(3)]
    got = np.full(flat.shape, np.nan)
    dom.store(got)
    dom.close()
    assert dts == want_dts
    assert np.array_equal(W.from_patches(got, geom), want_i)


def test_slab_rules():
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, U, meta = _box(W.BC_PERIODIC)
    b = MHDBunch(geom, dtype=torch.float32, gamma=meta["gamma"], slab=(1, 3))
    nl, ppl, lb = b.slab_info()
    assert (nl, ppl, lb) == (2, 4, 4 * 8 * 16 ** 3 * 4)
    assert b.nbytes == (2 + 2) * 4 * 8 * 22 ** 3 * 4           # owned layers + two halo layers
    host = torch.zeros(b.nbytes // 4, dtype=torch.float32).pin_memory()
    with pytest.raises(capi.MHDError) as ei:                   # the streamed paths are not for slabs
        b.advance_streamed(host, 1, 1)
    assert ei.value.code == capi.MHD_EINVAL
    assert b.lib.mhd_bunch_set_slab(b.h, 0, 1) == capi.MHD_ESTATE   # a slab's layers are fixed
    b.close()
    with pytest.raises(capi.MHDError):                         # ragged tilings have no layers
        g2, U2, m2 = W.ragged_small()
        MHDBunch(g2, dtype=torch.float32, gamma=m2["gamma"], slab=(0, 1))
    with pytest.raises(capi.MHDError):                         # layer range out of the box
        MHDBunch(geom, dtype=torch.float32, gamma=meta["gamma"], slab=(2, 7))
