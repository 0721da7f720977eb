"""Argument checks of the Python binding (host logic, no GPU): every buffer handed to the
C ABI is checked for memory space, dtype, contiguity and byte count before its pointer
is taken, so that a wrong tensor raises ValueError instead of reaching the library."""
import pytest
import torch

from paper_2508_09568_gb300 import capi
from paper_2508_09568_gb300.autograd import MHDStep, rollout
from paper_2508_09568_gb300.bunch import MHDBunch, _check_buffer, _check_dt_dev


class _StubLib:
    """Records the calls a handle makes; every call succeeds."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return capi.MHD_OK
        return call


def _handle(dtype=torch.float32, nelem=64):
    b = object.__new__(MHDBunch)     # no device: only the host-side checks run
    b.lib = _StubLib()
    b.h = None
    b._twin = None
    b.dtype = dtype
    b.rb = 4 if dtype == torch.float32 else 8
    b.nbytes = nelem * b.rb
    return b


def test_check_buffer_accepts_the_layout_and_rejects_the_rest():
    _check_buffer(torch.zeros(64), torch.float32, 256, False, "x")
    with pytest.raises(ValueError, match="dtype"):
        _check_buffer(torch.zeros(32, dtype=torch.float64), torch.float32, 256, False, "x")   # same bytes
    with pytest.raises(ValueError, match="bytes"):
        _check_buffer(torch.zeros(63), torch.float32, 256, False, "x")
    with pytest.raises(ValueError, match="contiguous"):
        _check_buffer(torch.zeros(128)[::2], torch.float32, 256, False, "x")
    with pytest.raises(ValueError, match="contiguous"):
        _check_buffer(torch.zeros(()).expand(64), torch.float32, 256, False, "x")
    with pytest.raises(ValueError, match="device memory"):
        _check_buffer(torch.zeros(64), torch.float32, 256, True, "x")
    with pytest.raises(ValueError, match="torch tensor"):
        _check_buffer(None, torch.float32, 256, False, "x")


def test_host_paths_check_before_calling_the_library():
    b = _handle()
    b.advance_host(torch.zeros(64), 1)
    b.advance_streamed(torch.zeros(64), 1, 2)
    assert b.lib.calls == ["mhd_bunch_advance_host", "mhd_bunch_advance_streamed"]
    for bad in (torch.zeros(32, dtype=torch.float64), torch.zeros(65), torch.zeros(128)[::2]):
        with pytest.raises(ValueError):
            b.advance_host(bad, 1)
        with pytest.raises(ValueError):
            b.advance_streamed(bad, 1, 2)
    assert len(b.lib.calls) == 2


def test_device_paths_reject_host_tensors():
    b = _handle(torch.float64)
    x = torch.zeros(64, dtype=torch.float64)
    with pytest.raises(ValueError, match="device memory"):
        b.step_adjoint(0.1, x, x, x)
    for f in (b.cfl_dt_device, b.fill_cfl_device, b.step_device_dt, lambda t: b.graph_capture(1, t)):
        with pytest.raises(ValueError, match="dt_dev"):
            f(torch.zeros(1, dtype=torch.float64))
    with pytest.raises(ValueError, match="dt_dev"):
        _check_dt_dev(torch.zeros(0, dtype=torch.float64))
    assert b.lib.calls == []


def test_autograd_entry_points_check_the_state():
    b = _handle(torch.float64)
    with pytest.raises(ValueError, match="device memory"):
        MHDStep.apply(torch.zeros(64, dtype=torch.float64, requires_grad=True), b, 0.1)
    with pytest.raises(ValueError, match="device memory"):
        rollout(torch.zeros(64, dtype=torch.float64, requires_grad=True), b, 0.1, 4, 2)
    assert b.lib.calls == []
