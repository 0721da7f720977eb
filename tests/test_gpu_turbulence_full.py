"""The benchmark workload at its full size: the 512^3 periodic turbulence box as 4096
patches of 32^3, in the launch configuration the benchmark times (persistent launch with
the autotuned tile, fill -> CFL dt -> step replayed from a CUDA graph).

* one step of the whole box compared patch by patch with the oracle on a seeded sample of
  patches (the oracle advances each sampled patch from its window of the same
  FP32-rounded global field, with the dt the graph computed): relative L1 per
  hydrodynamic variable, and of the face field B as one vector (its y and z components
  start at exactly zero, so each alone has no scale);
* the graph's dt is no larger than courant / (maximum CFL rate) of any sampled patch
  (the global dt is the minimum over all patches);
* ten more steps: mass, momentum and energy conserved, div B at rounding level.

FP32 (the benchmark's precision) and an FP64 check run (default tile, one step).
"""
import numpy as np
import pytest
import torch

from helpers import TOL_MAX, TOL_STEP, max_rel, rel_l1
from oracle import mhd as O
from paper_2508_09568_gb300 import capi
from paper_2508_09568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NCELL, PATCH = 512, 32


def _interior_sums(U, geom, absolute=False, chunk=256):
    """Sum (of |values| with absolute) over the interior cells of every variable, in
    float64, on the device, a chunk of patches at a time."""
    Z, Y, X = geom.padded(0)
    g = int(geom.gvec[0])
    n = PATCH
    P = geom.npatch
    V = U.view(P, 8, Z, Y, X)
    tot = torch.zeros(8, dtype=torch.float64, device=U.device)
    for p0 in range(0, P, chunk):
        blk = V[p0:p0 + chunk, :, g:g + n, g:g + n, g:g + n].double()
        tot += (blk.abs() if absolute else blk).sum(dim=(0, 2, 3, 4))
    return tot.cpu().numpy()


def _max_divb(U, geom, chunk=256):
    """max |div B| dx / rms |B| over the interior (ghost faces filled beforehand)."""
    Z, Y, X = geom.padded(0)
    g = int(geom.gvec[0])
    n = PATCH
    V = U.view(geom.npatch, 8, Z, Y, X)
    dmax = 0.0
    b2 = 0.0
    for p0 in range(0, geom.npatch, chunk):
        blk = V[p0:p0 + chunk].double()
        s = slice(g, g + n)
        s1 = slice(g + 1, g + n + 1)
        d = (blk[:, 5, s, s, s1] - blk[:, 5, s, s, s]) + (blk[:, 6, s, s1, s] - blk[:, 6, s, s, s]) + \
            (blk[:, 7, s1, s, s] - blk[:, 7, s, s, s])
        dmax = max(dmax, float(d.abs().max()))
        b2 += float((blk[:, 5:8, s, s, s] ** 2).sum())
    rms = np.sqrt(b2 / (geom.interior_cells() * 3))
    return dmax / rms


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_turbulence_box_full_size_sampled_and_invariants(dtype):
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, fields, meta = W.turbulence_box(ncell=NCELL, patch=PATCH)
    gamma = meta["gamma"]
    npd = np.float32 if dtype == torch.float32 else np.float64
    b = MHDBunch(geom, dtype=dtype, gamma=gamma)
    host = torch.empty(geom.state_elems(), dtype=dtype).pin_memory()
    W.to_patches(fields, geom, dtype=npd, out=host.numpy())
    with torch.cuda.stream(b.stream):
        b.current().copy_(host, non_blocking=True)
    b.stream.synchronize()
    del host
    if dtype == torch.float32:
        b.set_mode(capi.MHD_MODE_PERSISTENT, b.autotune(None))
    else:
        b.set_mode(capi.MHD_MODE_PERSISTENT, -1)
    U0 = b.current()
    if dtype == torch.float32:
        sums0 = _interior_sums(U0, geom)
        absref = _interior_sums(U0, geom, absolute=True)
    dts = torch.zeros(1, dtype=torch.float64, device=U0.device)
    b.graph_capture(1, dts)
    b.graph_launch()
    b.stream.synchronize()
    dt = float(dts[0].cpu())
    assert dt > 0
    # the oracle on a sample of patches, each from its window of the same global input
    rng = np.random.default_rng(9)
    sample = rng.choice(geom.npatch, 6, replace=False)
    win = {int(p): [] for p in sample}
    for v in range(8):
        a = torch.tensor(np.asarray(fields(v)).astype(npd).astype(np.float64))[None]
        for p in sample:
            win[int(p)].append(O.window(a, geom.origin[p], geom.patch_n[p], geom.gvec, geom.domain, geom.bc))
        del a
    cur = b.current()
    offs = geom.offsets()
    Z, Y, X = geom.padded(0)
    g = int(geom.gvec[0])
    sl = (slice(None),) + tuple(slice(g, g + PATCH) for _ in range(3))
    eps = O.HLLD_EPS[4 if dtype == torch.float32 else 8]
    for p in sample:
        Up = torch.cat(win[int(p)], 0)
        # global dt <= this patch's own CFL dt (courant 0.8 over its interior rates)
        r = O.cfl_rate(Up[None], geom.active, geom.dx, gamma)[0][sl[1:]]
        assert dt <= 0.8 / float(r.max()) * (1 + 1e-6)
        out = O.step(Up[None], dt, geom.active, geom.dx, gamma, eps=eps, gvec=geom.gvec,
                     n=geom.patch_n[p])[0].numpy()
        gp = cur[int(offs[p]): int(offs[p]) + 8 * X * Y * Z].view(8, Z, Y, X).cpu().numpy().astype(np.float64)
        a, r = gp[sl], out[sl]
        # hydrodynamic variables: relative L1 per variable; the face field as one vector
        # (By and Bz start at exactly zero in this box, so each alone has no scale of its own)
        err = rel_l1(a, r)[:5]
        errb = np.abs(a[5:8] - r[5:8]).sum() / np.abs(r[5:8]).sum()
        assert np.all(err <= TOL_STEP[dtype]) and errb <= TOL_STEP[dtype], (int(p), err, errb)
        # element by element (momentum and field measured against their vectors' scale)
        em = max_rel(a, r)
        assert np.all(em <= TOL_MAX[dtype]), (int(p), em)
    if dtype == torch.float64:
        code, msg = b.error()
        assert code == 0, msg
        return
    # ten more steps: conservation and div B
    b.graph_capture(10, None)
    b.graph_launch()
    b.fill_guards()
    b.stream.synchronize()
    Un = b.current()
    sums = _interior_sums(Un, geom)
    for v in (0, 1, 2, 3, 4):
        assert abs(sums[v] - sums0[v]) <= 1e-5 * absref[v], (v, sums[v], sums0[v])
    assert _max_divb(Un, geom) < 1e-5
    code, msg = b.error()
    assert code == 0, msg
