"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares.

No kernel runs here (no GPU needed); argument validation that happens before any CUDA call
is checked too.
"""
import ctypes as ct
import os
import re

import pytest

from paper_2508_09568_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mhd_bunch.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def test_header_declares_the_boundary():
    names = declared()
    for required in ("mhd_bunch_create", "mhd_bunch_fill_guards", "mhd_bunch_cfl_dt", "mhd_bunch_step",
                     "mhd_bunch_step_adjoint", "mhd_bunch_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    lib2 = ct.CDLL(capi.lib_path())
    for n in names:
        assert hasattr(lib2, n), n
    # and the binding covers exactly the declared API
    assert sorted(capi.SIGNATURES) == names


def test_library_is_built_for_sm103a(lib):
    # the link step embeds the sm_103a image; cuobjdump is not needed: the build command is fixed
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.getsize(capi.lib_path()) > 100_000


def test_argument_validation_before_any_device_call(lib):
    h = ct.c_void_p()
    assert lib.mhd_bunch_create(8, 8, 8, 3, 7, 4, 4, ct.byref(h)) == capi.MHD_EINVAL   # nvar
    assert b"nvar" in lib.mhd_last_error()
    assert lib.mhd_bunch_create(8, 8, 8, 2, 8, 4, 4, ct.byref(h)) == capi.MHD_EINVAL   # guard < 3
    assert lib.mhd_bunch_create(8, 8, 8, 3, 8, 4, 2, ct.byref(h)) == capi.MHD_EINVAL   # real_bytes
    assert lib.mhd_bunch_create(8, 8, 8, 3, 8, 0, 4, ct.byref(h)) == capi.MHD_EINVAL   # npatch
    assert lib.mhd_bunch_create(8, 1, 8, 3, 8, 4, 4, ct.byref(h)) == capi.MHD_EINVAL   # x-z only
    assert lib.mhd_bunch_fill_guards(None) == capi.MHD_EINVAL
    assert lib.mhd_bunch_step(None, 0.1) == capi.MHD_EINVAL
    assert lib.mhd_bunch_step_adjoint(None, 0.1, None, None, None) == capi.MHD_EINVAL
    lib.mhd_bunch_destroy(None)   # no-op
    assert lib.mhd_bunch_set_riemann(None, 0) == capi.MHD_EINVAL
    r = ct.c_double()
    assert lib.mhd_probe_fma_rate(2, None, ct.byref(r)) == capi.MHD_EINVAL           # real_bytes
    assert lib.mhd_probe_fma_rate(4, None, None) == capi.MHD_EINVAL                   # no output
    # the largest and smallest patch extents, checked before any allocation
    assert lib.mhd_bunch_create(4097, 8, 8, 3, 8, 4, 4, ct.byref(h)) == capi.MHD_EINVAL
    assert b"too large" in lib.mhd_last_error()
    pn = (ct.c_int32 * 6)(8, 8, 8, 8, 0, 8)
    assert lib.mhd_bunch_create_ragged(pn, 2, 3, 8, 4, ct.byref(h)) == capi.MHD_EINVAL   # extent 0
    pn = (ct.c_int32 * 6)(8, 8, 8, 8, 8, 1)
    assert lib.mhd_bunch_create_ragged(pn, 2, 3, 8, 4, ct.byref(h)) == capi.MHD_EINVAL   # mixed axes
    # every entry point rejects a NULL handle or output without touching the device
    n = ct.c_int()
    i64 = ct.c_int64()
    sz = ct.c_size_t()
    assert lib.mhd_bunch_set_mode(None, capi.MHD_MODE_MIXED, -1) == capi.MHD_EINVAL
    assert lib.mhd_bunch_autotune(None, None, ct.byref(n)) == capi.MHD_EINVAL
    assert lib.mhd_bunch_interior_size(None, ct.byref(sz), None) == capi.MHD_EINVAL
    assert lib.mhd_bunch_advance_streamed(None, None, 1, 1, None) == capi.MHD_EINVAL
    assert lib.mhd_bunch_advance_streamed_interior(None, None, 1, 1, None) == capi.MHD_EINVAL
    assert lib.mhd_bunch_advance_async(None, 1.0, 1, ct.byref(n), ct.byref(i64)) == capi.MHD_EINVAL
    assert lib.mhd_bunch_async_round(None, 0, None, None, 0, ct.byref(n)) == capi.MHD_EINVAL
    assert lib.mhd_bunch_graph_capture(None, 1, None) == capi.MHD_EINVAL
    assert lib.mhd_bunch_launch_count(None, ct.byref(i64)) == capi.MHD_EINVAL
