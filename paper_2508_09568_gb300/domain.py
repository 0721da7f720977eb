"""A box split over several GPUs by z-layers of patches (slabs), one rank per GPU.

Patches are independent given their guard zones (Secs. 2.2 and 4 of the paper), so the box
decomposes by whole patches: rank r owns a contiguous run of the patch layers along z
(partition), holds them in a slab handle (mhd_bunch_set_slab) together with two halo
layers, and per step
  1. copies the interiors of its bottom and top layers out of its state (slab_pack),
  2. sends its top layer to the rank above and its bottom layer to the rank below, and
     receives the layer below its slab and the layer above it (exchange_halos: point-to-
     point over torch.distributed -- NCCL between GPUs, gloo between CPU processes), into
     its own memory,
  3. writes them into its halo slots (slab_unpack), fills its guard zones and takes the
     CFL dt of its patches on the device (one pass),
  4. takes the minimum dt over all ranks (all_reduce MIN, the one collective), and
  5. updates its patches.
The layers wrap periodically across the box (rank 0's layer below is the last rank's top
layer); across an outflow box face the halo is sent but never read.  Every step is that of
the undivided box, bitwise: the same guard values, the same global dt, the same update.

step_local runs several slabs of one box in one process (on one GPU), exchanging through
device copies instead of messages: the same sequence without a process group.
"""
from __future__ import annotations

import numpy as np
import torch

from . import workloads as W
from .bunch import MHDBunch


def partition(nlayers: int, nparts: int):
    """Contiguous layer ranges [z0, z1) of nparts ranks, sizes differing by at most one."""
    if nparts < 1 or nlayers < nparts:
        raise ValueError("need 1 <= nparts <= nlayers")
    cuts = [nlayers * r // nparts for r in range(nparts + 1)]
    return [(cuts[r], cuts[r + 1]) for r in range(nparts)]


def exchange_halos(bottom: torch.Tensor, top: torch.Tensor, rank: int, world: int, group=None):
    """Send `top` to the rank above and `bottom` to the rank below (periodic in rank);
    return (below, above): the top layer of the rank below and the bottom layer of the rank
    above, received into new tensors on the same device.  world == 1: the slab is its own
    neighbour (copies of its own layers)."""
    if world == 1:
        return top.clone(), bottom.clone()
    import torch.distributed as dist
    up, down = (rank + 1) % world, (rank - 1) % world
    below = torch.empty_like(top)
    above = torch.empty_like(bottom)
    # the same posting order on every rank: with two ranks (up == down) the two messages
    # between a pair are matched in order, top -> the other's below, bottom -> its above
    ops = [dist.P2POp(dist.isend, top, up, group, tag=1), dist.P2POp(dist.irecv, below, down, group, tag=1),
           dist.P2POp(dist.isend, bottom, down, group, tag=2), dist.P2POp(dist.irecv, above, up, group, tag=2)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return below, above


class SlabDomain:
    """One rank's slab: patch layers [z0, z1) of the box geom (equal patches on a grid, x
    fastest, then y, then z) on one GPU."""

    def __init__(self, geom: W.Geometry, z0: int, z1: int, dtype=torch.float32, gamma=5.0 / 3.0, courant=0.8,
                 limiter=0, riemann=0, device="cuda:0"):
        self.geom = geom
        self.z0, self.z1 = int(z0), int(z1)
        self.b = MHDBunch(geom, dtype=dtype, gamma=gamma, courant=courant, limiter=limiter, device=device,
                          riemann=riemann, slab=(self.z0, self.z1))
        self.layers, self.ppl, self.layer_bytes = self.b.slab_info()
        n = self.layer_bytes // self.b.rb
        dev = self.b.device
        self.bottom = torch.empty(n, dtype=dtype, device=dev)
        self.top = torch.empty(n, dtype=dtype, device=dev)
        self.dt = torch.zeros(1, dtype=torch.float64, device=dev)

    def owned(self) -> range:
        """Global indices of the owned patches, in slab order."""
        return range(self.z0 * self.ppl, self.z1 * self.ppl)

    def load(self, global_flat: np.ndarray):
        """The owned patches of a whole-box buffer in the state layout (halo slots zeroed)."""
        offs = self.geom.offsets()
        pe = int(np.prod(self.geom.padded(0))) * 8
        flat = np.zeros(self.b.nbytes // self.b.rb, dtype=np.float64)
        for k, p in enumerate(self.owned()):
            flat[k * pe:(k + 1) * pe] = global_flat[offs[p]:offs[p] + pe]
        self.b.upload(flat)

    def store(self, global_flat: np.ndarray):
        """The owned patches of the current state into a whole-box buffer (state layout)."""
        offs = self.geom.offsets()
        pe = int(np.prod(self.geom.padded(0))) * 8
        mine = self.b.download()
        for k, p in enumerate(self.owned()):
            global_flat[offs[p]:offs[p] + pe] = mine[k * pe:(k + 1) * pe]

    def pack(self):
        """(bottom, top): the interiors of the bottom and top owned layers, ready to send."""
        self.b.slab_pack(self.bottom, self.top)
        self.b.stream.synchronize()
        return self.bottom, self.top

    def unpack(self, below: torch.Tensor, above: torch.Tensor):
        # the received layers are ordered on the caller's stream
        self.b.stream.wait_stream(torch.cuda.current_stream(self.b.device))
        self.b.slab_unpack(below, above)

    def local_dt(self):
        """Guard fill + CFL dt of the slab's patches (one pass) into self.dt."""
        self.b.fill_cfl_device(self.dt)
        self.b.stream.synchronize()
        return self.dt

    def advance(self):
        """The update of the owned patches with self.dt (the global dt by now)."""
        self.b.stream.wait_stream(torch.cuda.current_stream(self.b.device))
        self.b.step_device_dt(self.dt)

    def close(self):
        self.b.close()


def step_distributed(dom: SlabDomain, rank: int, world: int, group=None) -> float:
    """One step of the split box on this rank (see the module text); returns the dt."""
    bottom, top = dom.pack()
    below, above = exchange_halos(bottom, top, rank, world, group)
    dom.unpack(below, above)
    dt = dom.local_dt()
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(dt, op=dist.ReduceOp.MIN, group=group)
    dom.advance()
    return float(dt.item())


def step_local(doms) -> float:
    """One step of several slabs of one box held in this process; returns the dt."""
    packs = [d.pack() for d in doms]
    n = len(doms)
    for r, d in enumerate(doms):
        d.unpack(packs[(r - 1) % n][1], packs[(r + 1) % n][0])
    dts = [d.local_dt() for d in doms]
    dt = torch.min(torch.cat([x.to(dts[0].device) for x in dts]))
    for d in doms:
        d.dt.copy_(dt.reshape(1))
        d.advance()
    return float(dt.item())
