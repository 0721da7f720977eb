#!/usr/bin/env python
"""Benchmark of the MHD bunch update on GB300.

Workload (the 3D headline configuration): a 512^3 periodic MHD turbulence-like box as
4096 patches of 32^3 cells (guard 3), rho = 1, p = 1, gamma = 5/3, B = (0.1, 0, 0),
seeded solenoidal velocity with E(k) ~ k^-2 over 1 <= |k| <= 8 and rms Mach 1, FP32.
One step = guard fill + CFL dt on the device (one pass) + fused update (persistent
kernel), the sequence captured in a CUDA graph.  Metric: 3D MHD cell-updates per second.

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) the box is repeated N times along z
and split into one slab of patch layers per GPU (domain.SlabDomain): per step one patch
layer goes each way between neighbouring ranks (NCCL send/recv) and the dt is the minimum
over ranks (all_reduce); per-GPU work is that of N = 1 (weak scaling) and value counts the
cells of all slabs.  The other legs (per-kernel times, end to end, plain path) run on each
rank's own copy of the N = 1 box.  --impl reference times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D MHD cell-updates/s per GB300"
UNIT = "cell-updates/s"
# Algorithmic arithmetic of one cell-update: add/sub + mul + div + sqrt counted once per
# output element of the scheme's stages (python -m oracle.flops, 32^3 patch): 1395 add,
# 1464 mul, 282 div, 114 sqrt (plus 327 compares/selects, not counted as flops).
FLOPS_PER_CELL = 3255.0
BYTES_PER_CELL = {4: 64.0, 8: 128.0}       # read 8 values + write 8 values per cell-update
SMS, FP32_LANES = 152, 128                 # GB300: SMs, FP32 lanes per SM
E2E_CHUNKS = 32                            # chunks of the host-streamed end-to-end leg
OOC_BUDGET = 4 << 30                       # device budget of the out-of-core leg, FP32 (bytes; x2 for FP64)
# DRAM bytes (read + write) per cell-update of the fused step kernel, FP32, 32^3 patches,
# per tile configuration (the two the autotuner picks between on this machine):
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of a 192^3 box of the
# same patches and tiles (7,077,888 cells; 32 x 8: 451.83 MB + 232.93 MB, 16 x 16:
# 453.35 MB + 235.50 MB).  Traffic scales with the number of patches, so a launch on the
# full box moves this many bytes per cell.  Valid for this kernel version only.
STEP_DRAM_BYTES_PER_CELL = {(4, 32, (32, 8, 512)): (451.825920e6 + 232.927744e6) / 7077888,
                            (4, 32, (16, 16, 512)): (453.351168e6 + 235.501568e6) / 7077888}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks / throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f if l.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, ws):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(ncell=512, patch=32):
    from paper_2508_09568_gb300 import workloads as W
    geom, fields, meta = W.turbulence_box(ncell=ncell, patch=patch)
    return geom, fields, meta


# the oracle's bounded sample of the benchmark box: a seeded choice of its patches
CPU_SAMPLE_SEED = 20250813
CPU_SAMPLE_PATCHES = 512     # one step of an eighth of the 512^3 box's 4096 patches
CPU_CHUNK = 8                # patches the oracle advances per call


def cpu_sample_patches(geom, count):
    """A seeded choice of `count` patch indices of the box, ascending."""
    rng = np.random.default_rng(CPU_SAMPLE_SEED)
    return np.sort(rng.choice(geom.npatch, min(count, geom.npatch), replace=False))


def oracle_sample_step(geom, gamma, field_of, sample, courant=0.8):
    """The oracle's work on sampled patches of a box, timed: each patch's guard fill (its
    padded window of the global field, variable by variable), the CFL rates of their
    interiors, dt = courant / their maximum, and one oracle step of the sampled patches,
    CPU_CHUNK at a time.  field_of(v) gives global variable v as an FP64 tensor
    (1, Nz, Ny, Nx); producing it is not timed.  Returns the seconds of timed work."""
    from oracle import mhd as O
    wins = [[] for _ in sample]
    el = 0.0
    for v in range(8):
        a = field_of(v)
        t0 = time.perf_counter()
        for i, p in enumerate(sample):
            wins[i].append(O.window(a, geom.origin[p], geom.patch_n[p], geom.gvec, geom.domain, geom.bc))
        el += time.perf_counter() - t0
        del a
    t0 = time.perf_counter()
    g, n = geom.gvec, geom.patch_n[0]
    inner = (slice(None),) + tuple(slice(int(g[d]), int(g[d]) + int(n[d])) for d in (2, 1, 0))
    batches = []
    rmax = 0.0
    for k in range(0, len(sample), CPU_CHUNK):
        B = torch.stack([torch.cat(wins[i], 0) for i in range(k, min(k + CPU_CHUNK, len(sample)))])
        for i in range(k, min(k + CPU_CHUNK, len(sample))):
            wins[i] = None
        rmax = max(rmax, float(O.cfl_rate(B, geom.active, geom.dx, gamma)[inner].max()))
        batches.append(B)
    dt = courant / rmax
    for k in range(len(batches)):
        O.step(batches[k], dt, geom.active, geom.dx, gamma, gvec=geom.gvec, n=geom.patch_n[0])
        batches[k] = None
    return el + time.perf_counter() - t0


def cpu_baseline(npatches=CPU_SAMPLE_PATCHES, box=None, ncell=512, patch=32):
    """The oracle as it stands on the host cores, on a bounded sample of the benchmark box:
    one step (guard fill, CFL dt, update) of `npatches` seeded patches of it.  box =
    (geom, fields, meta) of the box when already generated."""
    from paper_2508_09568_gb300 import workloads as W
    geom, fields, meta = box if box is not None else W.turbulence_box(ncell=ncell, patch=patch)
    sample = cpu_sample_patches(geom, npatches)
    el = oracle_sample_step(geom, meta["gamma"], lambda v: torch.from_numpy(np.asarray(fields(v), np.float64))[None],
                            sample)
    cells = int(sum(int(np.prod(geom.patch_n[p])) for p in sample))
    N = int(geom.domain[0])
    return {"value": cells / el, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"one step of {len(sample)} of the {geom.npatch} patches of the {N}^3 box (seeded choice; "
                      f"guard zones from the global field, CFL dt over the sample, the update {CPU_CHUNK} "
                      f"patches per call), FP64, {el:.2f} s"}


def cpu_baseline_configs():
    """The oracle on host cores on the 1D and 2D configurations: the whole Sod run (256
    cells, to t = 0.2) and two steps of the 512^2 Orszag-Tang box, in cell-updates/s."""
    from oracle import mhd as O
    from paper_2508_09568_gb300 import workloads as W
    out = {}
    geom, U, meta = W.sod(ncell=256, npatch=16)
    ob = O.Bunch(geom, meta["gamma"])
    P = ob.split(W.to_patches(U, geom))
    t0 = time.perf_counter()
    P, t, k = ob.run(P, t_end=0.2)
    el = time.perf_counter() - t0
    out["sod_256"] = {"value": 256 * k / el, "unit": UNIT, "steps": k, "s": el}
    geom, U, meta = W.orszag_tang(ncell=512, patch=32)
    ob = O.Bunch(geom, meta["gamma"])
    P = ob.split(W.to_patches(U, geom))
    dt = float(ob.cfl_dt(ob.fill_guards(P)))
    t0 = time.perf_counter()
    for _ in range(2):
        P = ob.step(P, dt)
    el = time.perf_counter() - t0
    out["orszag_tang_512"] = {"value": 512 * 512 * 2 / el, "unit": UNIT, "steps": 2, "s": el}
    return out


def _time_ms(stream, fn, n):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / n


def split_leg(args, b, host, geom, ws, rank, local, cfg):
    """N > 1: the box repeated N times along z (512 x 512 x 512N for the default workload)
    split into one slab of patch layers per GPU (domain.SlabDomain): per step each rank
    sends its bottom and top patch layers to its neighbours (NCCL send/recv, into the
    receiver's memory), fills its guard zones, takes its CFL dt, joins the minimum over
    ranks (all_reduce) and updates its patches.  Each rank holds the state of the N = 1 box
    (the field is periodic, so the repeated box is continuous), so per-GPU work stays that
    of N = 1.  Returns (ms of args.steps steps on this rank, launches, clock sampler)."""
    from paper_2508_09568_gb300 import workloads as W
    from paper_2508_09568_gb300.domain import SlabDomain, step_distributed
    nl = int(geom.domain[2] // geom.patch_n[0][2])
    gg = W.uniform_geometry([int(geom.domain[0]), int(geom.domain[1]), int(geom.domain[2]) * ws],
                            [int(v) for v in geom.patch_n[0]], dx=geom.dx)
    dom = SlabDomain(gg, rank * nl, (rank + 1) * nl, dtype=b.dtype, gamma=b._params["gamma"],
                     courant=b._params["courant"], device=str(b.device))
    dom.b.set_mode(2, cfg)
    with torch.cuda.stream(dom.b.stream):
        dom.b.current().zero_()
        dom.b.current()[:host.numel()].copy_(host, non_blocking=True)
    dom.b.stream.synchronize()
    for _ in range(args.warmup):
        step_distributed(dom, rank, ws)
    torch.cuda.synchronize()
    barrier(ws)
    l0 = dom.b.launch_count()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(cur)
        for _ in range(args.steps):
            step_distributed(dom, rank, ws)
        cur.wait_stream(dom.b.stream)
        e1.record(cur)
        torch.cuda.synchronize()
    barrier(ws)
    launches = dom.b.launch_count() - l0
    code, msg = dom.b.error()
    dom.close()
    if code != 0:
        raise RuntimeError(f"device error in the split-domain steps: {msg}")
    return e0.elapsed_time(e1), launches, clk


def ragged_leg(dev, steps):
    """The ragged box: 1566 patches of 16^3 / 24^3 / 32^3 (24.55 M cells), FP32, the step in a
    CUDA graph with one persistent launch per tile configuration, configurations chosen per
    patch-size class by the autotuner; beside it one configuration for the whole bunch and
    the one-launch-per-patch path and the workload's own bunches (one launch per bunch)."""
    from paper_2508_09568_gb300 import capi
    from paper_2508_09568_gb300 import workloads as W
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, fields, meta = W.ragged_box()
    flat = W.to_patches(fields, geom, dtype=np.float32)
    b = MHDBunch(geom, dtype=torch.float32, gamma=meta["gamma"], device=str(dev))
    b.upload(flat)
    dts = torch.zeros(1, dtype=torch.float64, device=dev)

    def graph_ms():
        b.graph_capture(1, dts)
        for _ in range(3):
            b.graph_launch()
        return _time_ms(b.stream, b.graph_launch, steps)

    # one configuration for the whole bunch (autotuned), then one per patch-size class
    b.set_mode(capi.MHD_MODE_PERSISTENT, -1)
    cfg = b.autotune(None)
    ms_single = graph_ms()
    b.set_mode(capi.MHD_MODE_MIXED, -1)
    b.autotune(None)
    ms = graph_ms()
    cells = geom.interior_cells()
    # the workload's own bunches (sizes U{8..512}): one persistent launch per bunch
    b.set_bunches(geom.bunches)
    b.set_mode(capi.MHD_MODE_BUNCH_LISTS, cfg)
    ms_lists = graph_ms()
    b.set_mode(capi.MHD_MODE_PER_PATCH, cfg)
    dt_dev = torch.zeros(1, dtype=torch.float64, device=dev)

    def plain():
        b.fill_guards()
        b.cfl_dt_device(dt_dev)
        b.step_device_dt(dt_dev)

    plain()
    ms_plain = _time_ms(b.stream, plain, 2)
    code, msg = b.error()
    b.close()
    if code != 0:
        raise RuntimeError(msg)
    return {"workload": "ragged periodic box 288x288x296, 1566 patches of 16^3/24^3/32^3, OT fields, FP32",
            "cells": cells, "value": cells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "mode": "one persistent launch per tile configuration, configurations chosen per patch-size class",
            "single_configuration": {"value": cells / (ms_single * 1e-3), "ms_per_step": ms_single,
                                     "config_index": cfg},
            "bunch_lists": {"value": cells / (ms_lists * 1e-3), "ms_per_step": ms_lists, "config_index": cfg,
                            "bunches": len(geom.bunches), "launches_per_step": len(geom.bunches) + 1,
                            "mode": "one persistent launch per bunch of the workload (sizes drawn from 8..512)"},
            "plain_per_patch": {"value": cells / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                                "launches_per_step": geom.npatch + 2}}


def async_leg(b, host, geom, spans=4):
    """Asynchronous per-patch stepping against synchronous stepping over the same time span
    (spans global CFL steps of the starting state), both from the same state: patch updates,
    wall time, and the cell-update rate of the asynchronous run."""
    def load():
        with torch.cuda.stream(b.stream):
            b.current().copy_(host, non_blocking=True)
        b.stream.synchronize()
    load()
    b.fill_guards()
    t_span = spans * b.cfl_dt()
    # synchronous: fill -> dt -> step until t_span, the last step clipped
    t, n = 0.0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while t < t_span:
        b.fill_guards()
        dt = min(b.cfl_dt(), t_span - t)
        b.step(dt)
        t += dt
        n += 1
    b.stream.synchronize()
    ts = time.perf_counter() - t0
    # an untimed asynchronous run first: neighbour lists and scheduler arrays are built on
    # the first call
    load()
    b.advance_async(t_span)
    load()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rounds, updates = b.advance_async(t_span)
    ta = time.perf_counter() - t0
    pc = int(np.prod(geom.patch_n[0]))
    return {"workload": f"the bench box advanced by {spans} global CFL steps of its starting state",
            "sync": {"steps": n, "patch_updates": n * geom.npatch, "s": ts},
            "async": {"rounds": rounds, "patch_updates": updates, "s": ta,
                      "cell_updates_per_s": updates * pc / ta},
            "update_ratio_async_over_sync": updates / (n * geom.npatch),
            "time_ratio_async_over_sync": ta / ts}


def e2e_leg(b, host, host_int, cells, ws, ke):
    """End to end through the C ABI on host buffers: the host-resident state streamed
    through the GPU every step (mhd_bunch_advance_streamed_interior: the owned cells of at
    most E2E_CHUNKS chunks uploaded, updated and downloaded, overlapped; every step copies
    the whole interior state to the device and back), beside the state-layout stream and
    one serial call per step (copy in, fill, dt, step, copy out)."""
    ibytes = b.interior_size()[0]

    def timed(call, k):
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        call(k)
        return allmax(time.perf_counter() - t0, ws)

    b.advance_streamed_interior(host_int, 1, E2E_CHUNKS)
    te = timed(lambda k: b.advance_streamed_interior(host_int, k, E2E_CHUNKS), ke)
    b.advance_streamed(host, 1, E2E_CHUNKS)
    tp = timed(lambda k: b.advance_streamed(host, k, E2E_CHUNKS), ke)
    ks = 2
    ts = timed(lambda k: [b.advance_host(host, 1) for _ in range(k)], ks)
    # the out-of-core leg measures one GPU's capped working set (N = 1 runs only: every rank
    # would pin two more host copies of its state)
    ooc = out_of_core_leg(b, host_int, cells, ws, max(2, min(ke, 6))) if ws == 1 else None
    return {"value": cells * ke * ws / te, "unit": UNIT, "h2d_bytes_per_step": ibytes,
            "d2h_bytes_per_step": ibytes, "steps": ke, "out_of_core": ooc,
            "path": f"mhd_bunch_advance_streamed_interior, at most {E2E_CHUNKS} chunks cut at whole waves of "
                    "the update, pinned host state (owned cells only; ghost cells rebuilt on the device)",
            "state_layout": {"value": cells * ke * ws / tp, "steps": ke, "h2d_bytes_per_step": b.nbytes,
                             "path": f"mhd_bunch_advance_streamed, {E2E_CHUNKS} chunks (ghost cells included)"},
            "serial": {"value": cells * ks * ws / ts, "steps": ks,
                       "path": "mhd_bunch_advance_host one step per call: H2D, fill, dt, step, D2H"}}


def out_of_core_leg(b, host_int, cells, ws, k):
    """The box stepped with a device working set capped below its own size
    (mhd_bunch_advance_out_of_core on a handle that holds no device state): the interior
    state and a scratch buffer of the same size in pinned host memory, z-layers of patches
    streamed through a ring on the device, a CFL pass and an update pass per step."""
    from paper_2508_09568_gb300.bunch import MHDBunch
    h = MHDBunch(b.geom, dtype=b.dtype, gamma=b._params["gamma"], courant=b._params["courant"],
                 device=str(b.device), bind=False)
    state = host_int.clone().pin_memory()
    scratch = torch.empty_like(state).pin_memory()
    ibytes = h.interior_size()[0]
    budget = OOC_BUDGET * (b.rb // 4)
    h.advance_out_of_core(state, scratch, 1, budget)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    h.advance_out_of_core(state, scratch, k, budget)
    t = allmax(time.perf_counter() - t0, ws)
    up, down = h.io_bytes
    h.close()
    return {"value": cells * k * ws / t, "unit": UNIT, "steps": k, "device_budget_bytes": budget,
            "state_bytes": b.nbytes, "host_interior_bytes": ibytes,
            "h2d_bytes_per_step": up // k, "d2h_bytes_per_step": down // k,
            "path": "mhd_bunch_advance_out_of_core: working set capped at device_budget_bytes (below the size of "
                    "one state buffer and of the host state), per step a CFL pass and an update pass over "
                    "z-layers of patches"}


def adjoint_leg(dev, dtype, rollout_steps=200, ckpt=10, reps=5):
    """Adjoint / forward time on the adjoint workload (64^3 = 8 x 32^3, fixed dt): one step
    (fill + update) against one adjoint step, and a checkpointed rollout's backward against
    its forward."""
    from paper_2508_09568_gb300 import workloads as W
    from paper_2508_09568_gb300.autograd import rollout
    from paper_2508_09568_gb300.bunch import MHDBunch
    geom, make_state, v0, vt, meta = W.adjoint_box()
    flat = W.to_patches(make_state(v0), geom)
    b = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"], device=str(dev))
    b.upload(flat)
    b.fill_guards()
    dt = 0.5 * b.cfl_dt()
    U = b.current().clone()
    lam_next = torch.randn_like(U)
    lam = torch.empty_like(U)

    def fwd():
        b.fill_guards()
        b.step(dt)

    def adj():
        b.step_adjoint(dt, U, lam_next, lam)

    with torch.cuda.stream(b.stream):
        fwd()
        adj()
    t_f = _time_ms(b.stream, fwd, reps)
    t_a = _time_ms(b.stream, adj, reps)
    # checkpointed rollout (the autograd path); an untimed two-segment rollout first
    # creates the twin handle that recomputes segments beside the adjoint sweep
    Uw = U.clone().requires_grad_(True)
    rollout(Uw, b, dt, 2 * ckpt, ckpt).backward(torch.ones_like(Uw))
    U0 = U.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    UT = rollout(U0, b, dt, rollout_steps, ckpt)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    UT.backward(torch.randn_like(UT))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    b.close()
    return {"forward_ms": t_f, "adjoint_ms": t_a, "ratio": t_a / t_f,
            "rollout": {"steps": rollout_steps, "ckpt": ckpt, "forward_s": t1 - t0, "backward_s": t2 - t1,
                        "ratio": (t2 - t1) / (t1 - t0),
                        "backward": "segment k-1 recomputed on a twin stream while the adjoint sweeps segment k"}}


def workload_name(args, npatch):
    return (f"3D periodic MHD turbulence box {args.ncell}^3 as {npatch} patches of {args.patch}^3 (guard 3), "
            f"seeded solenoidal v, rms Mach 1, {args.dtype}; step = fill + CFL dt + persistent fused update "
            "in a CUDA graph")


def run_reference(args, ws, rank):
    """The oracle on the host cores: each step one call of the oracle on 32 seeded patches
    of the benchmark box (their guard fill from the global field, CFL dt, update), the
    patches of successive steps taken in turn from a seeded sample."""
    if rank != 0:
        return
    from paper_2508_09568_gb300 import workloads as W
    steps, warm = args.steps, args.warmup
    per_step = 4 * CPU_CHUNK
    geom, fields, meta = W.turbulence_box(ncell=args.ncell, patch=args.patch)
    G = [torch.from_numpy(np.asarray(fields(v), np.float64))[None] for v in range(8)]
    del fields
    sample = cpu_sample_patches(geom, per_step * (steps + warm))
    chunks = [sample[k:k + per_step] for k in range(0, len(sample), per_step)]

    def one(i):
        part = chunks[i % len(chunks)]
        el = oracle_sample_step(geom, meta["gamma"], lambda v: G[v], part)
        return el, int(sum(int(np.prod(geom.patch_n[p])) for p in part))

    for i in range(warm):
        one(i)
    tot, cells = 0.0, 0
    for i in range(warm, warm + steps):
        el, c = one(i)
        tot += el
        cells += c
    v = cells / tot
    sample_txt = (f"each step: one oracle step of {per_step} of the {geom.npatch} patches of the {args.ncell}^3 box "
                  f"(seeded choice, new patches every step; guard zones from the global field, CFL dt over them, "
                  f"the update {CPU_CHUNK} patches per call), FP64")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": warm, "ms_per_step": 1e3 * tot / max(steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, geom.npatch) if ws == 1 else
                      f"the {workload_name(args, geom.npatch)} repeated {ws} times along z, split into one slab of "
                      f"{int(geom.domain[2] // geom.patch_n[0][2])} patch layers per GPU", "sample": sample_txt},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample_txt},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, local):
    from paper_2508_09568_gb300 import capi
    from paper_2508_09568_gb300 import workloads as W
    from paper_2508_09568_gb300.bunch import MHDBunch, fma_rate

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.leg in ("ragged", "adjoint"):
        # one secondary leg alone (profiling); the adjoint leg in the --dtype precision
        if rank == 0:
            if args.leg == "ragged":
                res = ragged_leg(dev, max(3, min(args.steps, 10)))
            else:
                res = {args.dtype: adjoint_leg(dev, torch.float32 if args.dtype == "f32" else torch.float64)}
            print(json.dumps({"leg": args.leg, **res}), flush=True)
        return
    hbm_gbs, sm_max_mhz, peak_src = peaks()
    t_gen = time.perf_counter()
    geom, fields, meta = workload(args.ncell, args.patch)
    dtype = torch.float32 if args.dtype == "f32" else torch.float64
    rb = 4 if dtype == torch.float32 else 8
    host = torch.empty(geom.state_elems(), dtype=dtype).pin_memory()
    W.to_patches(fields, geom, dtype=np.float32 if rb == 4 else np.float64, out=host.numpy())
    host_int = None
    if not args.no_e2e and args.leg in (None, "e2e"):
        # the same state in the interior layout (owned cells only) for the end-to-end leg
        host_int = torch.empty(geom.interior_cells() * 8, dtype=dtype).pin_memory()
        W.to_interior(fields, geom, dtype=np.float32 if rb == 4 else np.float64, out=host_int.numpy())
    del fields
    t_gen = time.perf_counter() - t_gen
    cells = geom.interior_cells()

    b = MHDBunch(geom, dtype=dtype, gamma=meta["gamma"], courant=0.8, device=str(dev))
    with torch.cuda.stream(b.stream):
        b.current().copy_(host, non_blocking=True)
    b.stream.synchronize()
    if args.leg == "async":
        if rank == 0:
            print(json.dumps({"leg": "async", **async_leg(b, host, geom)}), flush=True)
        b.close()
        return
    if args.leg == "e2e":
        rec = e2e_leg(b, host, host_int, geom.interior_cells(), ws, max(2, min(args.steps, 20)))
        if rank == 0:
            print(json.dumps({"leg": "e2e", **rec}), flush=True)
        b.close()
        return
    if args.config >= 0:
        cfg = args.config
        b.set_mode(capi.MHD_MODE_PERSISTENT, cfg)
    else:
        b.set_mode(capi.MHD_MODE_PERSISTENT, -1)
        cfg = b.autotune(None)
    tile = b.config_info(cfg)

    if ws == 1:
        # ---- timed region: graph replay of (fill -> CFL dt -> step), K steps
        dts = torch.zeros(1, dtype=torch.float64, device=dev)
        b.graph_capture(1, dts)
        for _ in range(args.warmup):
            b.graph_launch()
        b.stream.synchronize()
        l0 = b.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            e0.record(b.stream)
            for _ in range(args.steps):
                b.graph_launch()
            e1.record(b.stream)
            torch.cuda.synchronize()
        barrier(ws)
        launches = b.launch_count() - l0
        ms = e0.elapsed_time(e1)
    else:
        ms, launches, clk = split_leg(args, b, host, geom, ws, rank, local, cfg)
    ms_max = allmax(ms, ws)
    value = cells * args.steps * ws / (ms_max * 1e-3)
    clocks = clk.summary()

    # ---- per-kernel times (eager, events on the bunch stream), the graph's sequence
    # (guard fill + CFL dt in one pass, then the step), then the fill and the CFL pass alone
    dt_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(b.stream)
        b.fill_cfl_device(dt_dev)
        ev[k][1].record(b.stream)
        b.step_device_dt(dt_dev)
        ev[k][2].record(b.stream)
        b.fill_guards()
        ev[k][3].record(b.stream)
        b.cfl_dt_device(dt_dev)
        ev[k][4].record(b.stream)
    b.stream.synchronize()
    mean = lambda i, j: float(np.mean([ev[k][i].elapsed_time(ev[k][j]) for k in range(args.steps)]))
    t_fc, t_step, t_fill, t_cfl = mean(0, 1), mean(1, 2), mean(2, 3), mean(3, 4)
    # the step with the HLL face flux instead of HLLD (same kernel, runtime switch)
    b.set_riemann(capi.MHD_RIEMANN_HLL)
    nh = max(2, min(args.steps, 5))
    evh = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nh + 1)]
    for k in range(nh + 1):            # the first is a warm-up
        b.fill_cfl_device(dt_dev)
        evh[k][0].record(b.stream)
        b.step_device_dt(dt_dev)
        evh[k][1].record(b.stream)
    b.stream.synchronize()
    t_step_hll = float(np.mean([evh[k][0].elapsed_time(evh[k][1]) for k in range(1, nh + 1)]))
    b.set_riemann(capi.MHD_RIEMANN_HLLD)
    code, msg = b.error()
    if code != 0:
        raise RuntimeError(f"device error during the benchmark: {msg}")

    # ---- the plain path: one launch per patch (same kernel), eager
    kp = 0 if args.no_plain else max(2, min(args.steps, 4))
    plain = None
    if kp:
        b.set_mode(capi.MHD_MODE_PER_PATCH, cfg)
        b.fill_guards()
        b.cfl_dt_device(dt_dev)
        b.step_device_dt(dt_dev)
        b.stream.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(b.stream)
        for _ in range(kp):
            b.fill_guards()
            b.cfl_dt_device(dt_dev)
            b.step_device_dt(dt_dev)
        p1.record(b.stream)
        b.stream.synchronize()
        plain = cells * kp / (p0.elapsed_time(p1) * 1e-3)
        b.set_mode(capi.MHD_MODE_PERSISTENT, cfg)

    # ---- asynchronous stepping from the starting state (before the end-to-end legs, which
    # advance the host copy in place)
    async_rec = async_leg(b, host, geom) if rank == 0 and not args.no_extra else None

    # ---- end to end through the C ABI on host buffers (H2D + fill + dt + step + D2H per step)
    e2e = None if args.no_e2e else e2e_leg(b, host, host_int, cells, ws, max(2, min(args.steps, 20)))
    del host, host_int          # the pinned host copies (11.5 GB FP32) are not used past here

    # ---- roofline of the dominant kernel (the fused step): SIMT-arithmetic bound; the
    # peak is the FMA rate the library's probe kernel measures on this GPU
    step_s = t_step * 1e-3
    alu_peak = fma_rate(dtype, str(dev)) / 1e12
    derived = SMS * FP32_LANES * 2 * sm_max_mhz * 1e6 / 1e12 if rb == 4 else None
    flops = FLOPS_PER_CELL * cells / step_s / 1e12
    hbm = BYTES_PER_CELL[rb] * cells / step_s / 1e9
    tpc = STEP_DRAM_BYTES_PER_CELL.get((rb, args.patch, tuple(tile)))
    roof = {"bound": "alu", "achieved": flops, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": flops / alu_peak, "traffic": tpc * cells if tpc else None,
            "kernel": "step_kernel",
            "peak_source": f"measured: FMA-chain probe (mhd_probe_fma_rate), {args.dtype}",
            "derived_peak": derived,
            "derived_peak_source": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz",
            "flops_per_cell": FLOPS_PER_CELL,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per cell of a 192^3 "
                              "capture, times the cells of one launch" if tpc else None}
    hbm_roof = {"bound": "hbm", "achieved": hbm, "peak": hbm_gbs, "unit": "GB/s", "frac": hbm / hbm_gbs,
                "bytes_per_cell": BYTES_PER_CELL[rb], "peak_source": peak_src,
                "frac_of_whole_step": (BYTES_PER_CELL[rb] * value / ws / 1e9) / hbm_gbs}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": workload_name(args, geom.npatch) if ws == 1 else
                      f"the {workload_name(args, geom.npatch)} repeated {ws} times along z, split into one slab of "
                      f"{int(geom.domain[2] // geom.patch_n[0][2])} patch layers per GPU",
                      "cells": cells, "patches": geom.npatch, "patch": args.patch,
                      "tile": {"x": tile[0], "y": tile[1], "threads": tile[2]},
                      "l2": f"inputs larger than L2 (state {b.nbytes / 1e9:.2f} GB per buffer)",
                      "parallelism": "single GPU" if ws == 1 else
                      f"z-slab split over {ws} GPUs: per step one patch layer sent each way per rank (NCCL "
                      "send/recv) and an allreduce-min of dt; value counts the cells of all slabs"},
           "roofline": roof, "hbm_roofline": hbm_roof,
           "kernels_ms": {"fill_cfl": t_fc, "step": t_step, "fill_guards_alone": t_fill, "cfl_dt_alone": t_cfl,
                          "step_hll_flux": t_step_hll},
           "plain_per_patch": {"value": plain, "unit": UNIT, "launches_per_step": geom.npatch + 2,
                               "path": "guard fill + CFL dt + one step launch per patch, eager"},
           "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
           "setup_s": {"generate": t_gen}}
    if rank == 0 and not args.no_extra:
        out["async"] = async_rec
        out["ragged"] = ragged_leg(dev, max(3, min(args.steps, 10)))
        out["adjoint_forward_ratio"] = {"workload": "64^3 periodic box, 8 patches of 32^3, fixed dt",
                                        "f64": adjoint_leg(dev, torch.float64),
                                        "f32": adjoint_leg(dev, torch.float32)}
    if rank == 0 and not args.no_cpu:
        box = workload(args.ncell, args.patch)
        out["cpu_baseline"] = cpu_baseline(CPU_SAMPLE_PATCHES, box=box)
        # one host core: ns per cell-update, the per-core kind of figure the paper quotes
        nt = torch.get_num_threads()
        torch.set_num_threads(1)
        try:
            one = cpu_baseline(CPU_CHUNK, box=box)
        finally:
            torch.set_num_threads(nt)
        del box
        out["cpu_baseline"]["single_core"] = {"ns_per_cell_update": 1e9 / one["value"], "cores": 1,
                                              "sample": one["sample"]}
        out["cpu_baseline"]["other_configs"] = cpu_baseline_configs()
    b.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--ncell", type=int, default=512)
    ap.add_argument("--patch", type=int, default=32)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-launch-per-patch comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--config", type=int, default=-1, help="tile configuration (default: autotune)")
    ap.add_argument("--no-extra", action="store_true", help="skip the ragged-box and adjoint legs")
    ap.add_argument("--leg", default=None, choices=["async", "ragged", "adjoint", "e2e"],
                    help="run only this secondary leg and print its record (for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
