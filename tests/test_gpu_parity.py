"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Tolerances (relative L1 per variable over interior cells, per step): FP64 1e-12, FP32
1e-5 (FP32 run from the FP32-rounded input, oracle in FP64 on the same rounded input);
and element by element, max |a - b| of every variable over its largest magnitude (of the
momentum or field vector for their components): FP64 1e-10, FP32 1e-4 (helpers.TOL_MAX).
Integer/byte work (the guard fill) must be bit exact.
"""
import numpy as np
import pytest
import torch

from helpers import assert_parity, gpu_bunch, gpu_steps, interior_global, oracle_bunch, oracle_steps, rounded
from paper_2508_09568_gb300 import capi
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]


def _cases():
    return {
        "sod": lambda: W.sod(ncell=256, npatch=16),
        "ot_small": lambda: W.orszag_tang(ncell=64, patch=16),
        "box_8": lambda: W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=3),
        "box_ragged_tiles": lambda: W.small_box(ncell=(40, 24, 20), patch=(20, 24, 10), seed=4),
    }


@pytest.mark.parametrize("case", list(_cases()))
@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_one_step_matches_oracle(case, dtype):
    geom, U, meta = _cases()[case]()
    flat = rounded(W.to_patches(U, geom), dtype)
    ob = oracle_bunch(geom, meta["gamma"], dtype=dtype)
    dt = ob.cfl_dt(ob.fill_guards(ob.split(flat)))
    ref = interior_global(oracle_steps(geom, flat, meta["gamma"], [dt], dtype=dtype), geom)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    got = interior_global(gpu_steps(b, [dt]), geom)
    assert_parity(got, ref, dtype, what=case)
    code, msg = b.error()
    assert code == 0, msg


@pytest.mark.parametrize("case", list(_cases()))
@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_one_step_hll_matches_oracle(case, dtype):
    """The HLL face-flux variant (the paper's mockup solver) against the oracle's HLL step."""
    geom, U, meta = _cases()[case]()
    flat = rounded(W.to_patches(U, geom), dtype)
    ob = oracle_bunch(geom, meta["gamma"], dtype=dtype)
    dt = ob.cfl_dt(ob.fill_guards(ob.split(flat)))
    ref = interior_global(oracle_steps(geom, flat, meta["gamma"], [dt], dtype=dtype, riemann=capi.MHD_RIEMANN_HLL),
                          geom)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype, riemann=capi.MHD_RIEMANN_HLL)
    got = interior_global(gpu_steps(b, [dt]), geom)
    assert_parity(got, ref, dtype, what=case)
    # and it is a different scheme: HLLD's result differs
    b2 = gpu_bunch(geom, flat, meta["gamma"], dtype)
    assert not np.array_equal(interior_global(gpu_steps(b2, [dt]), geom), got)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_several_steps_per_step_tolerance(dtype):
    """Five steps, each compared from the same starting state on both sides."""
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 16), seed=9)
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    for _ in range(5):
        ob = oracle_bunch(geom, meta["gamma"], dtype=dtype)
        dt = ob.cfl_dt(ob.fill_guards(ob.split(flat)))
        ref_flat = oracle_steps(geom, flat, meta["gamma"], [dt], dtype=dtype)
        b.upload(flat)
        got_flat = gpu_steps(b, [dt])
        assert_parity(interior_global(got_flat, geom), interior_global(ref_flat, geom), dtype)
        flat = rounded(got_flat, dtype)


def test_guard_fill_bit_exact():
    geom, U, meta = W.small_box(ncell=(16, 24, 8), patch=(8, 8, 8), seed=5)
    flat = W.to_patches(U, geom)
    b = gpu_bunch(geom, flat, meta["gamma"], torch.float64)
    b.fill_guards()
    got = b.download()
    ob = oracle_bunch(geom, meta["gamma"])
    ref = ob.join(ob.fill_guards(ob.split(flat)))
    assert np.array_equal(got, ref)


def test_guard_fill_outflow_bit_exact():
    geom, U, meta = W.sod(ncell=64, npatch=8)
    flat = W.to_patches(U, geom)
    b = gpu_bunch(geom, flat, meta["gamma"], torch.float32)
    b.fill_guards()
    got = b.download()
    ob = oracle_bunch(geom, meta["gamma"])
    ref = ob.join(ob.fill_guards(ob.split(rounded(flat, torch.float32))))
    assert np.array_equal(got.astype(np.float64), ref)


def test_guard_fill_every_boundary_combination_bit_exact():
    """Equal patches on a regular grid use the neighbour-table fill: bit exact against the
    oracle's fill for all 64 periodic / outflow choices of the six box faces (a box with a
    single patch along y, so its neighbours there are itself)."""
    import itertools
    g0, U, meta = W.small_box(ncell=(16, 8, 16), patch=(8, 8, 8), seed=13)
    for bcx in itertools.product((W.BC_PERIODIC, W.BC_OUTFLOW), repeat=6):
        geom = W.uniform_geometry([16, 8, 16], [8, 8, 8], dx=g0.dx,
                                  bc=[[bcx[0], bcx[1]], [bcx[2], bcx[3]], [bcx[4], bcx[5]]])
        flat = W.to_patches(U, geom)
        b = gpu_bunch(geom, flat, meta["gamma"], torch.float64)
        b.fill_guards()
        ob = oracle_bunch(geom, meta["gamma"])
        assert np.array_equal(b.download(), ob.join(ob.fill_guards(ob.split(flat)))), bcx
        b.close()


def _outflow_box():
    g0, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=22)
    bc = [[W.BC_OUTFLOW, W.BC_OUTFLOW], [W.BC_PERIODIC, W.BC_OUTFLOW], [W.BC_OUTFLOW, W.BC_PERIODIC]]
    return W.uniform_geometry([24, 16, 16], [8, 8, 8], dx=g0.dx, bc=bc), U, meta


@pytest.mark.parametrize("case", ["box", "outflow", "ot", "sod", "odd"])
@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_fused_fill_cfl_equals_separate_passes(case, dtype):
    """mhd_bunch_fill_cfl_device (one pass on regular grids) writes the ghost cells of the
    guard fill and, bitwise, the dt of the separate CFL pass.  "odd": 5x7x6 patches, whose
    padded planes (11x13 reals) are not a multiple of 16 bytes, so their rows come in by
    element copies instead of bulk copies."""
    geom, U, meta = {"box": lambda: W.small_box(ncell=(16, 24, 16), patch=(8, 8, 8), seed=25),
                     "odd": lambda: W.small_box(ncell=(10, 14, 12), patch=(5, 7, 6), seed=26),
                     "outflow": _outflow_box,
                     "ot": lambda: W.orszag_tang(ncell=64, patch=16),
                     "sod": lambda: W.sod(ncell=64, npatch=8)}[case]()
    flat = rounded(W.to_patches(U, geom), dtype)
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    b.fill_cfl_device(dt_dev)
    b.stream.synchronize()
    fused, dt_fused = b.download(), float(dt_dev.item())
    b.upload(flat)
    b.fill_guards()
    dt_sep = b.cfl_dt()
    assert np.array_equal(b.download(), fused)
    assert dt_fused == dt_sep


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-14), (torch.float32, 2e-6)], ids=["f64", "f32"])
def test_cfl_dt_matches_oracle(dtype, tol):
    for geom, U, meta in (W.small_box(seed=2), W.orszag_tang(ncell=64, patch=16), W.sod(64, 4)):
        flat = rounded(W.to_patches(U, geom), dtype)
        b = gpu_bunch(geom, flat, meta["gamma"], dtype)
        b.fill_guards()
        got = b.cfl_dt()
        ob = oracle_bunch(geom, meta["gamma"])
        ref = ob.cfl_dt(ob.fill_guards(ob.split(flat)))
        assert abs(got - ref) <= tol * ref, (got, ref)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_launch_modes_and_tiles_bitwise_identical(dtype):
    geom, U, meta = W.small_box(ncell=(48, 32, 16), patch=(24, 16, 16), seed=6)
    flat = rounded(W.to_patches(U, geom), dtype)
    outs = []
    b = gpu_bunch(geom, flat, meta["gamma"], dtype)
    for mode in (capi.MHD_MODE_PER_PATCH, capi.MHD_MODE_BUNCHED, capi.MHD_MODE_PERSISTENT):
        for cfg in range(b.num_configs()):
            b.set_mode(mode, cfg)
            b.upload(flat)
            outs.append(gpu_steps(b, [1e-3, 1e-3]))
    for o in outs[1:]:
        assert np.array_equal(interior_global(o, geom), interior_global(outs[0], geom))


def test_graph_replay_matches_eager():
    geom, U, meta = W.small_box(ncell=(32, 32, 32), patch=(16, 16, 16), seed=8)
    flat = rounded(W.to_patches(U, geom), torch.float32)
    b = gpu_bunch(geom, flat, meta["gamma"], torch.float32)
    eager_dts = []
    for _ in range(4):
        b.fill_guards()
        dt = b.cfl_dt()
        eager_dts.append(dt)
        b.step(dt)
    eager = interior_global(b.download(), geom)
    b2 = gpu_bunch(geom, flat, meta["gamma"], torch.float32)
    dts = torch.zeros(4, dtype=torch.float64, device="cuda")
    b2.graph_capture(4, dts)
    b2.graph_launch()
    torch.cuda.synchronize()
    assert np.array_equal(dts.cpu().numpy(), np.array(eager_dts))
    assert np.array_equal(interior_global(b2.download(), geom), eager)


def test_invariants_many_steps_fp64():
    geom, U, meta = W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=12)
    flat = W.to_patches(U, geom)
    b = gpu_bunch(geom, flat, meta["gamma"], torch.float64)
    G0 = interior_global(flat, geom)
    for _ in range(40):
        b.fill_guards()
        b.step(b.cfl_dt())
    G = interior_global(b.download(), geom)
    for v in range(5):
        assert abs(G[v].sum() - G0[v].sum()) <= 1e-13 * np.abs(G0[v]).sum()
    d = (np.roll(G[5], -1, 2) - G[5]) / geom.dx[0] + (np.roll(G[6], -1, 1) - G[6]) / geom.dx[1] + \
        (np.roll(G[7], -1, 0) - G[7]) / geom.dx[2]
    assert np.max(np.abs(d)) * geom.dx[0] / np.sqrt((G[5:8] ** 2).mean()) < 1e-13


def test_sod_to_t_end_fp64_matches_oracle_run():
    """The whole Sod run (GPU dt from its own CFL kernel) against the oracle's run."""
    geom, U, meta = W.sod(ncell=256, npatch=16)
    flat = W.to_patches(U, geom)
    ob = oracle_bunch(geom, 1.4)
    P, t, k = ob.run(ob.split(flat), t_end=0.2)
    ref = interior_global(ob.join(P), geom)
    b = gpu_bunch(geom, flat, 1.4, torch.float64)
    t = 0.0
    steps = 0
    while t < 0.2 * (1 - 1e-14):
        b.fill_guards()
        dt = min(b.cfl_dt(), 0.2 - t)
        b.step(dt)
        t += dt
        steps += 1
    assert steps == k
    got = interior_global(b.download(), geom)
    # 140 steps through a shock: rel L1 1e-10, and no cell further than 1e-8 of the scale
    assert_parity(got, ref, torch.float64, l1=1e-10, mx=1e-8)


def test_nonphysical_state_is_reported():
    """Failure detection without a GPU fault: a negative density is latched in the error word."""
    geom, U, meta = W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=1)
    U = U.copy()
    U[0, 5, 5, 5] = -1.0
    flat = W.to_patches(U, geom)
    b = gpu_bunch(geom, flat, meta["gamma"], torch.float64)
    b.fill_guards()
    with pytest.raises(capi.MHDError) as ei:
        b.cfl_dt()
    assert ei.value.code in (capi.MHD_EPHYS,)
    b.step(1e-3)
    code, msg = b.error()
    assert code == capi.MHD_EPHYS, msg
    code, msg = b.error()
    assert code == 0
