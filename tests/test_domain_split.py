"""A box split over ranks by z-layers of patches (paper_2508_09568_gb300.domain), on CPU.

Two and three gloo ranks each own a run of patch layers of a periodic 16 x 16 x 48 box of 8^3
patches, exchange their bottom and top layers with exchange_halos every step (the same
function that moves the layers between GPUs over NCCL), take the global dt as the minimum
over ranks (all_reduce), and advance their own patches.  The oracle is each rank's
arithmetic here (this machine has no GPU): its guard zones are cut from an array holding
only the rank's own layers and the two received halo layers.  Three steps of the split box
equal the undivided box's three oracle steps bitwise, so the partition, the direction of
every message and the placement of the halos are right; the GPU side of the same sequence
(slab handles) is checked against the undivided box in tests/test_gpu_domain.py.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NSTEPS = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _box():
    from paper_2508_09568_gb300 import workloads as W
    return W.small_box(ncell=(16, 16, 48), patch=(8, 8, 8), seed=51)


def _rank_steps(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    torch.set_num_threads(2)
    import torch.distributed as dist

    from oracle import mhd as O
    from paper_2508_09568_gb300.domain import exchange_halos, partition
    dist.init_process_group("gloo", rank=rank, world_size=world)
    geom, U, meta = _box()
    gamma = meta["gamma"]
    nz = int(geom.patch_n[0][2])
    NL = int(geom.domain[2]) // nz
    z0, z1 = partition(NL, world)[rank]
    ppl = geom.npatch // NL
    mine = list(range(z0 * ppl, z1 * ppl))
    own = torch.tensor(U[:, z0 * nz:z1 * nz]).clone()          # only this rank's layers
    g = geom.gvec
    for _ in range(NSTEPS):
        bottom = own[:, :nz].contiguous()
        top = own[:, -nz:].contiguous()
        below, above = exchange_halos(bottom, top, rank, world)
        A = torch.full((8,) + tuple(int(v) for v in geom.domain[::-1]), float("nan"), dtype=torch.float64)
        A[:, z0 * nz:z1 * nz] = own
        lb, la = (z0 - 1) % NL, z1 % NL
        A[:, lb * nz:(lb + 1) * nz] = below
        A[:, la * nz:(la + 1) * nz] = above
        P = [O.window(A, geom.origin[p], geom.patch_n[p], geom.gvec, geom.domain, geom.bc) for p in mine]
        rmax = torch.zeros((), dtype=torch.float64)
        for Up, p in zip(P, mine):
            n = geom.patch_n[p]
            r = O.cfl_rate(Up[None], geom.active, geom.dx, gamma)[0][g[2]:g[2] + n[2], g[1]:g[1] + n[1],
                                                                      g[0]:g[0] + n[0]]
            rmax = torch.maximum(rmax, r.max())
        dist.all_reduce(rmax, op=dist.ReduceOp.MAX)
        dt = 0.8 / rmax
        new = O.step(torch.stack(P), float(dt), geom.active, geom.dx, gamma, gvec=geom.gvec, n=geom.patch_n[0])
        for k, p in enumerate(mine):
            o, n = geom.origin[p], geom.patch_n[p]
            own[:, o[2] - z0 * nz:o[2] - z0 * nz + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = \
                new[k][:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
    out[rank] = (z0, z1, own.numpy())
    dist.destroy_process_group()


def test_partition_covers_the_layers_once():
    from paper_2508_09568_gb300.domain import partition
    for nl in (1, 5, 16, 17):
        for parts in range(1, nl + 1):
            r = partition(nl, parts)
            assert r[0][0] == 0 and r[-1][1] == nl
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition(3, 4)


@pytest.mark.parametrize("world", [2, 3])
def test_split_box_gloo_ranks_equal_undivided_box(world):
    from oracle import mhd as O
    from paper_2508_09568_gb300 import workloads as W
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_steps, args=(world, port, out), nprocs=world, join=True)
    geom, U, meta = _box()
    ob = O.Bunch(geom, meta["gamma"])
    P, t, k = ob.run(ob.split(W.to_patches(U, geom)), nsteps=NSTEPS)
    want = W.from_patches(ob.join(P), geom)
    got = np.full_like(want, np.nan)
    nz = int(geom.patch_n[0][2])
    for rank, (z0, z1, own) in dict(out).items():
        got[:, z0 * nz:z1 * nz] = own
    assert np.array_equal(got, want)
