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
