"""Host-side layouts of the bunch state: the state layout (ghost cells included) and the
interior layout (owned cells only) hold the same interior values at the same places."""
import numpy as np

from paper_2508_09568_gb300 import workloads as W


def _cases():
    yield W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=3)
    yield W.ragged_small()


def test_interior_layout_round_trip_and_offsets():
    for geom, U, meta in _cases():
        inter = W.to_interior(U, geom)
        assert inter.size == 8 * geom.interior_cells()
        assert np.array_equal(W.from_interior(inter, geom), U)
        offs = geom.interior_offsets()
        sizes = 8 * np.prod(geom.patch_n, axis=1)
        assert offs[0] == 0 and np.array_equal(np.diff(offs), sizes[:-1])


def test_interior_layout_matches_state_layout():
    for geom, U, meta in _cases():
        flat = W.to_patches(U, geom)
        inter = W.to_interior(U, geom)
        g = geom.gvec
        io = geom.interior_offsets()
        for p in range(geom.npatch):
            n = geom.patch_n[p]
            blk = W.patch_view(flat, geom, p)[:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
            got = inter[io[p]: io[p] + blk.size].reshape(blk.shape)
            assert np.array_equal(got, blk)
        # a callable field gives the same buffer
        assert np.array_equal(W.to_interior(lambda v: U[v], geom), inter)
