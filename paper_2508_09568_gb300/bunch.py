"""Python handle of a device-resident MHD bunch (thin wrapper over the C ABI).

PyTorch provides the device memory (two state buffers) and the CUDA stream; every
operation is one or more calls into libmhdbunch.so.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np
import torch

from . import capi
from .workloads import Geometry


def _check_dt_dev(dt_dev: torch.Tensor, count: int = 1):
    """dt on the device: `count` float64 elements of a contiguous CUDA tensor."""
    if not (isinstance(dt_dev, torch.Tensor) and dt_dev.is_cuda and dt_dev.dtype == torch.float64
            and dt_dev.is_contiguous() and dt_dev.numel() >= count):
        raise ValueError(f"dt_dev must be a contiguous CUDA float64 tensor of at least {count} element(s)")


def _check_buffer(t: torch.Tensor, dtype, nbytes: int, cuda: bool, what: str):
    """A contiguous tensor of the bunch's dtype holding exactly nbytes, on the device
    (cuda) or in host memory."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{what} must be a torch tensor")
    if t.is_cuda != cuda:
        raise ValueError(f"{what} must be in {'device' if cuda else 'host'} memory")
    if t.dtype != dtype:
        raise ValueError(f"{what} has dtype {t.dtype}, the bunch computes in {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() * t.element_size() != nbytes:
        raise ValueError(f"{what} holds {t.numel() * t.element_size()} bytes, the layout needs {nbytes}")


class MHDBunch:
    """A bunch of patches on one GPU.

    geom     workloads.Geometry (patch sizes, origins, box, dx, boundary kinds, guard)
    dtype    torch.float32 or torch.float64 (arithmetic precision of the kernels)
    riemann  face-flux solver: capi.MHD_RIEMANN_HLLD (default) or capi.MHD_RIEMANN_HLL
    bind     allocate and bind the two device state buffers (False: the handle holds no
             state on the device; only advance_out_of_core, which streams host state, runs)
    slab     (z0, z1): own only the patch layers z0 <= layer < z1 of the box plus two halo
             layers (mhd_bunch_set_slab; domain.SlabDomain drives it)
    """

    def __init__(self, geom: Geometry, dtype=torch.float32, gamma=5.0 / 3.0, courant=0.8, limiter=0,
                 device="cuda:0", stream: torch.cuda.Stream | None = None, riemann: int = 0, bind: bool = True,
                 slab: tuple | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("MHDBunch needs a CUDA device (no CPU fallback)")
        self.lib = capi.load()
        self.geom = geom
        self._params = dict(gamma=gamma, courant=courant, limiter=limiter, riemann=riemann)
        self._twin = None
        self.dtype = dtype
        self.device = torch.device(device)
        self.rb = 4 if dtype == torch.float32 else 8
        torch.cuda.set_device(self.device)
        # a dedicated stream by default: the legacy default stream cannot be captured in a graph
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = ct.c_void_p()
        pn = np.ascontiguousarray(geom.patch_n.astype(np.int32))
        capi.check(self.lib.mhd_bunch_create_ragged(pn.ctypes.data_as(capi.I32P), geom.npatch, int(geom.guard), 8,
                                                    self.rb, ct.byref(h)))
        self.h = h
        try:
            dx = np.ascontiguousarray(geom.dx, dtype=np.float64)
            org = np.ascontiguousarray(geom.origin, dtype=np.int64)
            dom = np.ascontiguousarray(geom.domain, dtype=np.int64)
            bc = np.ascontiguousarray(geom.bc.reshape(-1), dtype=np.int32)
            capi.check(self.lib.mhd_bunch_set_geometry(h, dx.ctypes.data_as(capi.DP), org.ctypes.data_as(capi.I64P),
                                                       dom.ctypes.data_as(capi.I64P), bc.ctypes.data_as(capi.I32P)))
            capi.check(self.lib.mhd_bunch_set_params(h, float(gamma), float(courant), int(limiter)))
            capi.check(self.lib.mhd_bunch_set_riemann(h, int(riemann)))
            self.slab = None if slab is None else (int(slab[0]), int(slab[1]))
            if self.slab is not None:
                capi.check(self.lib.mhd_bunch_set_slab(h, self.slab[0], self.slab[1]))
            nbytes = ct.c_size_t()
            offs = np.zeros(geom.npatch, dtype=np.int64)
            capi.check(self.lib.mhd_bunch_state_size(h, ct.byref(nbytes), offs.ctypes.data_as(capi.I64P)))
            if self.slab is None and not np.array_equal(offs, geom.offsets()):
                raise RuntimeError("library state layout differs from the workload layout")
            self.nbytes = nbytes.value
            n = self.nbytes // self.rb
            self.buf = None
            if not bind:
                return
            with torch.cuda.stream(self.stream):
                self.buf = [torch.full((n,), float("nan"), dtype=dtype, device=self.device) for _ in range(2)]
            capi.check(self.lib.mhd_bunch_bind(h, ct.c_void_p(self.buf[0].data_ptr()),
                                               ct.c_void_p(self.buf[1].data_ptr()),
                                               ct.c_void_p(self.stream.cuda_stream)))
        except Exception:
            self.lib.mhd_bunch_destroy(h)
            self.h = None
            raise

    # -- state ------------------------------------------------------------------------
    def current(self) -> torch.Tensor:
        p = ct.c_void_p()
        capi.check(self.lib.mhd_bunch_current(self.h, ct.byref(p)))
        for t in self.buf:
            if t.data_ptr() == p.value:
                return t
        raise RuntimeError("current buffer not found")

    def upload(self, flat: np.ndarray):
        cur = self.current()
        src = torch.from_numpy(np.ascontiguousarray(flat).astype(np.float64 if self.rb == 8 else np.float32))
        with torch.cuda.stream(self.stream):
            cur.copy_(src.to(self.device, non_blocking=False))

    def download(self) -> np.ndarray:
        self.stream.synchronize()
        return self.current().cpu().numpy()

    # -- the path -------------------------------------------------------------------------
    def fill_guards(self):
        capi.check(self.lib.mhd_bunch_fill_guards(self.h))

    def cfl_dt(self) -> float:
        dt = ct.c_double()
        capi.check(self.lib.mhd_bunch_cfl_dt(self.h, ct.byref(dt)))
        return dt.value

    def cfl_dt_device(self, dt_dev: torch.Tensor):
        _check_dt_dev(dt_dev)
        capi.check(self.lib.mhd_bunch_cfl_dt_device(self.h, ct.c_void_p(dt_dev.data_ptr())))

    def fill_cfl_device(self, dt_dev: torch.Tensor):
        """Guard fill then CFL dt into dt_dev (one pass on regular grids)."""
        _check_dt_dev(dt_dev)
        capi.check(self.lib.mhd_bunch_fill_cfl_device(self.h, ct.c_void_p(dt_dev.data_ptr())))

    def step(self, dt: float):
        capi.check(self.lib.mhd_bunch_step(self.h, float(dt)))

    def step_device_dt(self, dt_dev: torch.Tensor):
        _check_dt_dev(dt_dev)
        capi.check(self.lib.mhd_bunch_step_device_dt(self.h, ct.c_void_p(dt_dev.data_ptr())))

    def set_riemann(self, riemann: int):
        """Face-flux solver of later steps: capi.MHD_RIEMANN_HLLD or capi.MHD_RIEMANN_HLL."""
        capi.check(self.lib.mhd_bunch_set_riemann(self.h, int(riemann)))
        self._params["riemann"] = int(riemann)

    def set_bunches(self, bunches):
        """Bunches (lists of patch indices covering every patch once) for MHD_MODE_BUNCH_LISTS."""
        lists = [np.asarray(q, dtype=np.int32) for q in bunches]
        patches = np.ascontiguousarray(np.concatenate(lists), dtype=np.int32)
        starts = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(q) for q in lists])]), dtype=np.int32)
        capi.check(self.lib.mhd_bunch_set_bunches(self.h, patches.ctypes.data_as(capi.I32P),
                                                  starts.ctypes.data_as(capi.I32P), len(lists)))

    def set_mode(self, mode: int, config: int = -1):
        capi.check(self.lib.mhd_bunch_set_mode(self.h, int(mode), int(config)))

    def num_configs(self) -> int:
        n = ct.c_int()
        capi.check(self.lib.mhd_bunch_num_configs(self.h, ct.byref(n)))
        return n.value

    def config_info(self, k: int):
        tx, ty, nt = ct.c_int(), ct.c_int(), ct.c_int()
        capi.check(self.lib.mhd_bunch_config_info(self.h, k, ct.byref(tx), ct.byref(ty), ct.byref(nt)))
        return tx.value, ty.value, nt.value

    def autotune(self, cache_path: str | None = None) -> int:
        c = ct.c_int()
        capi.check(self.lib.mhd_bunch_autotune(self.h, cache_path.encode() if cache_path else None, ct.byref(c)))
        return c.value

    def graph_capture(self, nsteps: int, dt_dev: torch.Tensor | None = None):
        if dt_dev is not None:
            _check_dt_dev(dt_dev, max(int(nsteps), 1))
        ptr = ct.c_void_p(dt_dev.data_ptr()) if dt_dev is not None else None
        capi.check(self.lib.mhd_bunch_graph_capture(self.h, int(nsteps), ptr))

    def graph_launch(self):
        capi.check(self.lib.mhd_bunch_graph_launch(self.h))

    def advance_host(self, host_state: torch.Tensor, nsteps: int) -> float:
        """End to end on host memory (pinned torch tensor in the state layout), in place."""
        _check_buffer(host_state, self.dtype, self.nbytes, False, "host_state")
        t = ct.c_double()
        capi.check(self.lib.mhd_bunch_advance_host(self.h, ct.c_void_p(host_state.data_ptr()), int(nsteps),
                                                   ct.byref(t)))
        return t.value

    def advance_streamed(self, host_state: torch.Tensor, nsteps: int, nchunks: int = 8) -> float:
        """nsteps steps of a host-resident state (a contiguous CPU tensor of the state layout,
        pinned for overlap) streamed through the GPU every step in nchunks chunks; returns the
        simulated time."""
        _check_buffer(host_state, self.dtype, self.nbytes, False, "host_state")
        t = ct.c_double()
        capi.check(self.lib.mhd_bunch_advance_streamed(self.h, ct.c_void_p(host_state.data_ptr()), nsteps, nchunks,
                                                       ct.byref(t)))
        return t.value

    def interior_size(self):
        """(bytes, per-patch element offsets) of the interior layout (mhd_bunch_interior_size)."""
        nbytes = ct.c_size_t()
        offs = np.zeros(self.geom.npatch, dtype=np.int64)
        capi.check(self.lib.mhd_bunch_interior_size(self.h, ct.byref(nbytes), offs.ctypes.data_as(capi.I64P)))
        return nbytes.value, offs

    def advance_streamed_interior(self, host_interior: torch.Tensor, nsteps: int, nchunks: int = 8) -> float:
        """As advance_streamed with the host state in the interior layout (owned cells only,
        per patch [8][nz][ny][nx]; workloads.to_interior builds one); returns the simulated
        time."""
        _check_buffer(host_interior, self.dtype, self.interior_size()[0], False, "host_interior")
        t = ct.c_double()
        capi.check(self.lib.mhd_bunch_advance_streamed_interior(self.h, ct.c_void_p(host_interior.data_ptr()), nsteps,
                                                                nchunks, ct.byref(t)))
        return t.value

    def advance_out_of_core(self, host_state: torch.Tensor, host_scratch: torch.Tensor, nsteps: int,
                            device_budget: int) -> float:
        """nsteps steps of a host-resident state in the interior layout (pinned CPU tensors;
        host_scratch of the same size is overwritten) using at most device_budget bytes of
        device memory for the working set (mhd_bunch_advance_out_of_core); the new state is
        in host_state; returns the simulated time.  self.io_bytes: (host -> device,
        device -> host) bytes of the call."""
        nb = self.interior_size()[0]
        _check_buffer(host_state, self.dtype, nb, False, "host_state")
        _check_buffer(host_scratch, self.dtype, nb, False, "host_scratch")
        t = ct.c_double()
        io = (ct.c_size_t * 2)()
        capi.check(self.lib.mhd_bunch_advance_out_of_core(self.h, ct.c_void_p(host_state.data_ptr()),
                                                          ct.c_void_p(host_scratch.data_ptr()), int(nsteps),
                                                          ct.c_size_t(int(device_budget)),
                                                          ct.c_void_p(self.stream.cuda_stream), ct.byref(t), io))
        self.io_bytes = (io[0], io[1])
        return t.value

    def advance_async(self, t_span: float, max_rounds: int = 100000):
        """Asynchronous per-patch stepping by t_span (mhd_bunch_advance_async); returns
        (rounds, patch_updates)."""
        r = ct.c_int()
        u = ct.c_int64()
        capi.check(self.lib.mhd_bunch_advance_async(self.h, float(t_span), int(max_rounds), ct.byref(r), ct.byref(u)))
        return r.value, u.value

    def async_rounds(self, nrounds: int):
        """[(patches int32, dts float64)] of the last advance_async, one entry per round."""
        out = []
        for k in range(nrounds):
            n = ct.c_int()
            capi.check(self.lib.mhd_bunch_async_round(self.h, k, None, None, 0, ct.byref(n)))
            pp = np.zeros(n.value, dtype=np.int32)
            dd = np.zeros(n.value, dtype=np.float64)
            capi.check(self.lib.mhd_bunch_async_round(self.h, k, pp.ctypes.data_as(capi.I32P),
                                                      dd.ctypes.data_as(capi.DP), n.value, ct.byref(n)))
            out.append((pp, dd))
        return out

    def step_adjoint(self, dt: float, U_n: torch.Tensor, lam_next: torch.Tensor, lam: torch.Tensor):
        for t, what in ((U_n, "U_n"), (lam_next, "lam_next"), (lam, "lam")):
            _check_buffer(t, self.dtype, self.nbytes, True, what)
        capi.check(self.lib.mhd_bunch_step_adjoint(self.h, float(dt), ct.c_void_p(U_n.data_ptr()),
                                                   ct.c_void_p(lam_next.data_ptr()), ct.c_void_p(lam.data_ptr())))

    def error(self):
        code = ct.c_int()
        msg = ct.create_string_buffer(256)
        capi.check(self.lib.mhd_bunch_get_error(self.h, ct.byref(code), msg, 256))
        return code.value, msg.value.decode()

    def launch_count(self) -> int:
        n = ct.c_int64()
        capi.check(self.lib.mhd_bunch_launch_count(self.h, ct.byref(n)))
        return n.value

    def slab_info(self):
        """(owned layers, patches per layer, bytes of one layer in the interior layout)."""
        nl, ppl, lb = ct.c_int(), ct.c_int64(), ct.c_size_t()
        capi.check(self.lib.mhd_bunch_slab_info(self.h, ct.byref(nl), ct.byref(ppl), ct.byref(lb)))
        return nl.value, ppl.value, lb.value

    def slab_pack(self, bottom: torch.Tensor | None, top: torch.Tensor | None):
        """Interiors of the bottom / top owned layers into device tensors (on the bunch stream)."""
        capi.check(self.lib.mhd_bunch_slab_pack(self.h, None if bottom is None else ct.c_void_p(bottom.data_ptr()),
                                                None if top is None else ct.c_void_p(top.data_ptr())))

    def slab_unpack(self, below: torch.Tensor | None, above: torch.Tensor | None):
        """The neighbours' layers into the halo slots (on the bunch stream)."""
        capi.check(self.lib.mhd_bunch_slab_unpack(self.h, None if below is None else ct.c_void_p(below.data_ptr()),
                                                  None if above is None else ct.c_void_p(above.data_ptr())))

    def twin(self) -> "MHDBunch":
        """A second handle on the same geometry and parameters with its own stream, state
        buffers and work arrays (created on first use, closed with this one), so that two
        step sequences can run concurrently; every mode and tile configuration computes the
        same state, so the twin's steps equal this handle's."""
        if self._twin is None:
            self._twin = MHDBunch(self.geom, self.dtype, device=str(self.device), **self._params)
        return self._twin

    def close(self):
        if getattr(self, "_twin", None) is not None:
            self._twin.close()
            self._twin = None
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.mhd_bunch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fma_rate(dtype=torch.float32, device="cuda") -> float:
    """Attainable SIMT FMA rate (flop/s, 2 per FMA) of the device, measured by the
    library's probe kernel on a fresh stream (mhd_probe_fma_rate)."""
    lib = capi.load()
    rb = 4 if dtype == torch.float32 else 8
    with torch.cuda.device(torch.device(device)):
        st = torch.cuda.Stream()
        r = ct.c_double()
        capi.check(lib.mhd_probe_fma_rate(rb, ct.c_void_p(st.cuda_stream), ct.byref(r)))
    return r.value
