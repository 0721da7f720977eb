"""torch.autograd integration of the MHD bunch step and its hand-written adjoint.

MHDStep.apply(U, bunch, dt) advances a state tensor (the flat state layout of the bunch, on
its GPU) by one step at fixed dt; its backward calls mhd_bunch_step_adjoint.  rollout()
runs many steps keeping only every ckpt-th state; its backward recomputes each segment
forward from its checkpoint and sweeps the adjoint back through it, so the memory held is
about nsteps/ckpt + 2 ckpt states.  The recompute of segment k-1 runs on a twin handle
(bunch.twin(): its own stream and work arrays) while the adjoint sweeps segment k on the
bunch's stream; an event per segment orders the sweep after its recompute.  Both the forward and the backward run in the library's
CUDA kernels; torch only holds the buffers.
"""
from __future__ import annotations

import ctypes as ct

import torch

from . import capi
from .bunch import _check_buffer


def _step_into(bunch, U_in: torch.Tensor, U_out: torch.Tensor, dt: float):
    """U_out <- step(fill(U_in)) on the bunch's stream (U_in's ghosts are rewritten)."""
    lib = bunch.lib
    capi.check(lib.mhd_bunch_bind(bunch.h, ct.c_void_p(U_in.data_ptr()), ct.c_void_p(U_out.data_ptr()),
                                  ct.c_void_p(bunch.stream.cuda_stream)))
    capi.check(lib.mhd_bunch_fill_guards(bunch.h))
    capi.check(lib.mhd_bunch_step(bunch.h, float(dt)))


def _restore(bunch):
    capi.check(bunch.lib.mhd_bunch_bind(bunch.h, ct.c_void_p(bunch.buf[0].data_ptr()),
                                        ct.c_void_p(bunch.buf[1].data_ptr()),
                                        ct.c_void_p(bunch.stream.cuda_stream)))


def _adjoint(bunch, U: torch.Tensor, lam_next: torch.Tensor, dt: float) -> torch.Tensor:
    lam = torch.empty_like(U)
    bunch.step_adjoint(dt, U, lam_next.contiguous(), lam)
    return lam


class MHDStep(torch.autograd.Function):
    """One fixed-dt step: U^{n+1} = step(fill(U^n)); backward = the discrete adjoint."""

    @staticmethod
    def forward(ctx, U, bunch, dt):
        _check_buffer(U, bunch.dtype, bunch.nbytes, True, "U")
        cur = torch.cuda.current_stream(U.device)
        bunch.stream.wait_stream(cur)
        with torch.cuda.stream(bunch.stream):
            # the copy and the output live on the bunch stream, ordered before its kernels
            U_in = U.detach().clone()
            out = torch.empty_like(U_in)
            _step_into(bunch, U_in, out, dt)
            _restore(bunch)
        cur.wait_stream(bunch.stream)
        out.record_stream(cur)
        ctx.bunch, ctx.dt = bunch, float(dt)
        ctx.save_for_backward(U.detach())
        return out

    @staticmethod
    def backward(ctx, g):
        (U,) = ctx.saved_tensors
        cur = torch.cuda.current_stream(U.device)
        ctx.bunch.stream.wait_stream(cur)
        with torch.cuda.stream(ctx.bunch.stream):
            lam = _adjoint(ctx.bunch, U, g, ctx.dt)
        cur.wait_stream(ctx.bunch.stream)
        lam.record_stream(cur)
        return lam, None, None


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, bunch, dt, nsteps, ckpt):
        _check_buffer(U0, bunch.dtype, bunch.nbytes, True, "U0")
        if int(nsteps) < 1 or int(ckpt) < 1:
            raise ValueError("nsteps and ckpt must be at least 1")
        cur_stream = torch.cuda.current_stream(U0.device)
        bunch.stream.wait_stream(cur_stream)
        ckpts = []
        with torch.cuda.stream(bunch.stream):
            cur = U0.detach().clone()
            for s in range(nsteps):
                if s % ckpt == 0:
                    ckpts.append(cur.clone())
                nxt = torch.empty_like(cur)
                _step_into(bunch, cur, nxt, dt)
                cur = nxt
            _restore(bunch)
        cur_stream.wait_stream(bunch.stream)
        cur.record_stream(cur_stream)
        ctx.bunch, ctx.dt, ctx.nsteps, ctx.ckpt = bunch, float(dt), int(nsteps), int(ckpt)
        ctx.ckpts = ckpts
        return cur

    @staticmethod
    def backward(ctx, g):
        bunch, dt, n, k = ctx.bunch, ctx.dt, ctx.nsteps, ctx.ckpt
        cur_stream = torch.cuda.current_stream(g.device)
        bunch.stream.wait_stream(cur_stream)
        twin = bunch.twin()
        # the checkpoints were written on the bunch's stream
        twin.stream.wait_stream(bunch.stream)

        def recompute(seg):
            # the segment's inputs from its checkpoint, on the twin's stream (each step's
            # guard fill rewrites the ghosts of its input, which the adjoint fills anew)
            s0 = seg * k
            s1 = min(n, s0 + k)
            with torch.cuda.stream(twin.stream):
                states = [ctx.ckpts[seg]]
                for _ in range(s0, s1 - 1):
                    nxt = torch.empty_like(states[-1])
                    _step_into(twin, states[-1], nxt, dt)
                    states.append(nxt)
                done = torch.cuda.Event()
                done.record(twin.stream)
            for t in states:
                t.record_stream(bunch.stream)
            return states, done

        with torch.cuda.stream(bunch.stream):
            lam = g.contiguous().clone()
        nseg = len(ctx.ckpts)
        pending = recompute(nseg - 1)
        for seg in reversed(range(nseg)):
            states, done = pending
            if seg > 0:
                pending = recompute(seg - 1)
            bunch.stream.wait_event(done)
            with torch.cuda.stream(bunch.stream):
                for U in reversed(states):
                    lam = _adjoint(bunch, U, lam, dt)
        with torch.cuda.stream(bunch.stream):
            _restore(bunch)
        cur_stream.wait_stream(bunch.stream)
        lam.record_stream(cur_stream)
        ctx.ckpts = None
        return lam, None, None, None, None


def rollout(U0: torch.Tensor, bunch, dt: float, nsteps: int, ckpt: int = 10) -> torch.Tensor:
    """nsteps fixed-dt steps from U0 with checkpoint-every-ckpt-steps recomputation in backward."""
    return _Rollout.apply(U0, bunch, dt, nsteps, ckpt)
