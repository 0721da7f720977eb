"""ctypes binding of libmhdbunch.so: the C ABI of include/mhd_bunch.h, same names.

Argument marshalling only; every step of the update runs in the library's CUDA kernels.
Loading fails loudly (OSError / RuntimeError) when the library is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

from . import build as _build

MHD_OK, MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_EPHYS, MHD_EBOUNDS, MHD_ETIMEOUT, MHD_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
MHD_BC_PERIODIC, MHD_BC_OUTFLOW = 0, 1
MHD_LIMITER_MINMOD, MHD_LIMITER_MC = 0, 1
MHD_RIEMANN_HLLD, MHD_RIEMANN_HLL = 0, 1
MHD_MODE_PER_PATCH, MHD_MODE_BUNCHED, MHD_MODE_PERSISTENT, MHD_MODE_MIXED, MHD_MODE_BUNCH_LISTS = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "MHD_OK", -1: "MHD_EINVAL", -2: "MHD_ENOMEM", -3: "MHD_ECUDA", -4: "MHD_EPHYS",
                -5: "MHD_EBOUNDS", -6: "MHD_ETIMEOUT", -7: "MHD_ESTATE"}

P = ct.c_void_p
I = ct.c_int
D = ct.c_double
I64P = ct.POINTER(ct.c_int64)
I32P = ct.POINTER(ct.c_int32)
DP = ct.POINTER(ct.c_double)
HP = ct.POINTER(ct.c_void_p)

# name -> (restype, argtypes); the exported symbols of the C ABI
SIGNATURES = {
    "mhd_bunch_create": (I, [I, I, I, I, I, I, I, HP]),
    "mhd_bunch_create_ragged": (I, [I32P, I, I, I, I, HP]),
    "mhd_bunch_set_geometry": (I, [P, DP, I64P, I64P, I32P]),
    "mhd_bunch_set_params": (I, [P, D, D, I]),
    "mhd_bunch_set_riemann": (I, [P, I]),
    "mhd_bunch_set_bunches": (I, [P, I32P, I32P, I]),
    "mhd_bunch_state_size": (I, [P, ct.POINTER(ct.c_size_t), I64P]),
    "mhd_bunch_bind": (I, [P, P, P, P]),
    "mhd_bunch_current": (I, [P, HP]),
    "mhd_bunch_fill_guards": (I, [P]),
    "mhd_bunch_cfl_dt": (I, [P, DP]),
    "mhd_bunch_cfl_dt_device": (I, [P, P]),
    "mhd_bunch_fill_cfl_device": (I, [P, P]),
    "mhd_bunch_step": (I, [P, D]),
    "mhd_bunch_step_device_dt": (I, [P, P]),
    "mhd_bunch_set_mode": (I, [P, I, I]),
    "mhd_bunch_num_configs": (I, [P, ct.POINTER(I)]),
    "mhd_bunch_config_info": (I, [P, I, ct.POINTER(I), ct.POINTER(I), ct.POINTER(I)]),
    "mhd_bunch_autotune": (I, [P, ct.c_char_p, ct.POINTER(I)]),
    "mhd_bunch_graph_capture": (I, [P, I, P]),
    "mhd_bunch_graph_launch": (I, [P]),
    "mhd_bunch_advance_host": (I, [P, P, I, DP]),
    "mhd_bunch_advance_streamed": (I, [P, P, I, I, DP]),
    "mhd_bunch_interior_size": (I, [P, ct.POINTER(ct.c_size_t), I64P]),
    "mhd_bunch_advance_streamed_interior": (I, [P, P, I, I, DP]),
    "mhd_bunch_set_slab": (I, [P, I, I]),
    "mhd_bunch_slab_info": (I, [P, ct.POINTER(I), I64P, ct.POINTER(ct.c_size_t)]),
    "mhd_bunch_slab_pack": (I, [P, P, P]),
    "mhd_bunch_slab_unpack": (I, [P, P, P]),
    "mhd_bunch_advance_out_of_core": (I, [P, P, P, I, ct.c_size_t, P, DP, ct.POINTER(ct.c_size_t)]),
    "mhd_bunch_advance_async": (I, [P, D, I, ct.POINTER(I), I64P]),
    "mhd_bunch_async_round": (I, [P, I, I32P, DP, I, ct.POINTER(I)]),
    "mhd_bunch_step_adjoint": (I, [P, D, P, P, P]),
    "mhd_bunch_get_error": (I, [P, ct.POINTER(I), ct.c_char_p, ct.c_size_t]),
    "mhd_bunch_launch_count": (I, [P, I64P]),
    "mhd_bunch_destroy": (None, [P]),
    "mhd_last_error": (ct.c_char_p, []),
    "mhd_cfl_dt_uniform_noalloc": (I, [P, I, I, I, I, I, I, DP, D, D, P, P]),
    "mhd_probe_fma_rate": (I, [I, P, DP]),
}
MHD_NOALLOC_MAX_PATCHES = 16384

_LIB = None


class MHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmhdbunch.so (building it in-tree first if asked).  Raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise OSError(f"libmhdbunch.so not built ({path}); run paper_2508_09568_gb300.build.build()")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(code: int):
    if code != MHD_OK:
        msg = load().mhd_last_error()
        raise MHDError(code, msg.decode() if msg else "")
    return code
