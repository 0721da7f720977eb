"""Host-resident state streamed through the GPU every step (mhd_bunch_advance_streamed):
chunked copies overlapped with the update must give bitwise the state and simulated time
of the same steps run on the device-resident state."""
import numpy as np
import pytest
import torch

from helpers import interior_global, rounded
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", ["box", "ragged"])
def test_streamed_equals_device_resident(dtype, case):
    from paper_2508_09568_gb300.bunch import MHDBunch
    if case == "box":
        geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=31)
    else:
        geom, U, meta = W.ragged_small()
    flat = rounded(W.to_patches(U, geom), dtype)
    npd = np.float64 if dtype == torch.float64 else np.float32
    b = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"])
    ref = torch.tensor(flat.astype(npd)).pin_memory()
    t_ref = b.advance_host(ref, 3)
    want = interior_global(ref.numpy(), geom)
    for nchunks in (1, 3, 5, 64):
        host = torch.tensor(flat.astype(npd)).pin_memory()
        t = b.advance_streamed(host, 3, nchunks)
        assert t == t_ref
        assert np.array_equal(interior_global(host.numpy(), geom), want), nchunks
        # the device copy holds the final state as well
        assert np.array_equal(interior_global(b.download(), geom), want)
    code, msg = b.error()
    assert code == 0, msg


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", ["box", "ragged"])
def test_streamed_interior_equals_state_layout(dtype, case):
    """The interior-layout stream (owned cells only cross the link) gives bitwise the
    interior, the device state and the simulated time of the state-layout path."""
    from paper_2508_09568_gb300.bunch import MHDBunch
    if case == "box":
        geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=32)
    else:
        geom, U, meta = W.ragged_small()
    npd = np.float64 if dtype == torch.float64 else np.float32
    flat = rounded(W.to_patches(U, geom), dtype)
    b = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"])
    nbytes, offs = b.interior_size()
    assert np.array_equal(offs, geom.interior_offsets())
    assert nbytes == geom.interior_cells() * 8 * b.rb
    ref = torch.tensor(flat.astype(npd)).pin_memory()
    t_ref = b.advance_host(ref, 3)
    want = interior_global(ref.numpy(), geom)
    for nchunks in (1, 4, 64):
        host = torch.tensor(W.to_interior(U, geom, dtype=npd)).pin_memory()
        t = b.advance_streamed_interior(host, 3, nchunks)
        assert t == t_ref
        assert np.array_equal(W.from_interior(host.numpy().astype(np.float64), geom), want), nchunks
        assert np.array_equal(interior_global(b.download(), geom), want)
    code, msg = b.error()
    assert code == 0, msg


def test_streamed_chunks_cut_at_whole_waves():
    """A bunch of 512 one-tile patches: two requested chunks of 256 tiles each hold a wave
    of the persistent update, so the runs are cut at whole waves; the results stay bitwise
    those of the device-resident steps, in both host layouts."""
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, U, meta = W.small_box(ncell=(64, 64, 64), patch=(8, 8, 8), seed=34)
    flat = rounded(W.to_patches(U, geom), torch.float32)
    b = MHDBunch(geom, dtype=torch.float32, gamma=meta["gamma"])
    ref = torch.tensor(flat.astype(np.float32)).pin_memory()
    t_ref = b.advance_host(ref, 2)
    want = interior_global(ref.numpy(), geom)
    for nchunks in (2, 3, 4):
        host = torch.tensor(flat.astype(np.float32)).pin_memory()
        assert b.advance_streamed(host, 2, nchunks) == t_ref
        assert np.array_equal(interior_global(host.numpy(), geom), want)
        hi = torch.tensor(W.to_interior(U, geom, dtype=np.float32)).pin_memory()
        assert b.advance_streamed_interior(hi, 2, nchunks) == t_ref
        assert np.array_equal(W.from_interior(hi.numpy().astype(np.float64), geom), want)
    code, msg = b.error()
    assert code == 0, msg


def _tall_box(bcz):
    """A 32 x 32 x 512 box of sixteen 32^3 patches stacked along z (one patch per layer),
    seeded smooth fields; z boundaries periodic or outflow."""
    g0, U, meta = W.small_box(ncell=(32, 32, 512), patch=(32, 32, 32), seed=47)
    bc = [[W.BC_PERIODIC, W.BC_PERIODIC], [W.BC_PERIODIC, W.BC_PERIODIC], [bcz, bcz]]
    return W.uniform_geometry([32, 32, 512], [32, 32, 32], dx=g0.dx, bc=bc), U, meta


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("bcz", ["periodic", "outflow"])
def test_out_of_core_equals_device_resident(dtype, bcz):
    """mhd_bunch_advance_out_of_core on a handle with no device state, its working set
    capped below the size of the host state (so that the state cannot be held on the device
    at once): three steps equal, bitwise, the same steps run on the device-resident state
    (fused guard fill + CFL dt, then the update), interior and simulated time; likewise with
    budgets that take three layers per chunk (the last chunk shorter) and the whole box."""
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, U, meta = _tall_box(W.BC_PERIODIC if bcz == "periodic" else W.BC_OUTFLOW)
    npd = np.float64 if dtype == torch.float64 else np.float32
    flat = rounded(W.to_patches(U, geom), dtype)
    ref = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"])
    ref.upload(flat)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    t_ref = 0.0
    for _ in range(3):
        ref.fill_cfl_device(dt_dev)
        ref.step_device_dt(dt_dev)
        ref.stream.synchronize()
        t_ref += float(dt_dev.item())
    want = W.from_patches(ref.download().astype(np.float64), geom)
    code, msg = ref.error()
    assert code == 0, msg
    ref.close()
    ooc = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"], bind=False)
    host_bytes = ooc.interior_size()[0]
    rb = 8 if dtype == torch.float64 else 4
    layer_padded = 8 * 38 ** 3 * rb
    for budget in (host_bytes - 1, 2 * 5 * layer_padded + 8 * 32 ** 3 * 8 * rb + (2 << 20), 1 << 34):
        host = torch.tensor(W.to_interior(rounded(W.from_patches(flat, geom), dtype), geom, dtype=npd)).pin_memory()
        scratch = torch.empty_like(host).pin_memory()
        t = ooc.advance_out_of_core(host, scratch, 3, budget)
        assert t == t_ref, budget
        got = W.from_interior(host.numpy().astype(np.float64), geom)
        assert np.array_equal(got, want), budget
        # every step downloads the state once; with the whole box on the device (one
        # chunk) it uploads the 16 layers and the two wrapped halos once (the update pass
        # reuses the CFL pass's window)
        assert ooc.io_bytes[1] == 3 * host_bytes
        if budget == 1 << 34:
            layers = 16 + (2 if bcz == "periodic" else 0)
            assert ooc.io_bytes[0] == 3 * layers * host_bytes // 16
    ooc.close()


def test_out_of_core_rejects_a_budget_below_one_layer():
    from paper_2508_09568_gb300 import capi
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, U, meta = _tall_box(W.BC_PERIODIC)
    ooc = MHDBunch(geom, dtype=torch.float32, gamma=meta["gamma"], bind=False)
    host = torch.zeros(ooc.interior_size()[0] // 4, dtype=torch.float32).pin_memory()
    with pytest.raises(capi.MHDError) as ei:
        ooc.advance_out_of_core(host, host.clone(), 1, 1 << 20)
    assert ei.value.code == capi.MHD_ENOMEM
    ooc.close()
