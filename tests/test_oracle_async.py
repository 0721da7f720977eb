"""Pins of the oracle's asynchronous stepping (patches at their own times; the DISPATCH
mode of Sec. 2.2 read as R20): the neighbour lists, the time-interpolated guard fill, the
readiness rule and the replay of a schedule, each checked against something other than
itself — brute force over the box's cells, the synchronous guard fill (pinned against
numpy.pad) and the synchronous step of the oracle, and linearity in time.
"""
import numpy as np
import torch

from oracle import mhd as O
from paper_2508_09568_gb300 import workloads as W


def _owner_brute(geom, c):
    """The patch containing box cell c = (x, y, z), by scanning every patch's box."""
    for q in range(geom.npatch):
        o, n = geom.origin[q], geom.patch_n[q]
        if all(o[d] <= c[d] < o[d] + n[d] for d in range(3)):
            return q
    raise AssertionError(c)


def _wrap(i, N, lo, hi):
    if i < 0:
        return i % N if lo == W.BC_PERIODIC else 0
    if i >= N:
        return i % N if hi == W.BC_PERIODIC else N - 1
    return i


def test_neighbours_by_brute_force():
    for geom, U, meta in (W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=1), W.ragged_small()):
        nb = O.neighbours(geom)
        g = geom.gvec
        for p in range(geom.npatch):
            o, n = geom.origin[p], geom.patch_n[p]
            want = set()
            for z in range(o[2] - g[2], o[2] + n[2] + g[2]):
                for y in range(o[1] - g[1], o[1] + n[1] + g[1]):
                    for x in range(o[0] - g[0], o[0] + n[0] + g[0]):
                        c = [_wrap(v, int(geom.domain[d]), *geom.bc[d]) for d, v in enumerate((x, y, z))]
                        want.add(_owner_brute(geom, c))
            assert nb[p] == want - {p}, p


def test_fill_at_equal_times_is_the_synchronous_fill():
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=2)
    ob = O.Bunch(geom, meta["gamma"])
    P = ob.split(W.to_patches(U, geom))
    sync = ob.fill_guards(P)
    other = [u * 1.5 for u in P]        # a different previous slice: unused at w = 1
    t = [0.3] * geom.npatch
    for p in range(geom.npatch):
        assert torch.equal(O.fill_guards_at(P, other, t, [0.1] * geom.npatch, geom, p), sync[p])
        assert torch.equal(O.fill_guards_at(P, other, t, t, geom, p), sync[p])   # equal slice times


def test_fill_interpolates_linearly_in_time():
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=3)
    ob = O.Bunch(geom, meta["gamma"])
    A = ob.split(W.to_patches(U, geom))
    geom2, U2, _ = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=4)
    B = ob.split(W.to_patches(U2, geom2))
    fa, fb = ob.fill_guards(A), ob.fill_guards(B)
    g = geom.gvec
    for p in range(geom.npatch):
        t_old = [0.0] * geom.npatch
        t_cur = [1.0] * geom.npatch
        t_cur[p] = 0.25                  # patch p at a quarter of its neighbours' step
        got = O.fill_guards_at(B, A, t_cur, t_old, geom, p)
        want = 0.75 * fa[p] + 0.25 * fb[p]
        n = geom.patch_n[p]
        want[:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]] = \
            B[p][:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]    # its own cells: its current slice
        assert torch.allclose(got, want, rtol=1e-14, atol=1e-14), p


def test_fill_is_exact_for_fields_linear_in_time():
    """Every patch holds two slices of one field linear in time, f(t) = A + t B, at slice
    times of its own (all different); a patch's guard fill at its own time t_p, inside every
    neighbour's slice interval, is the window of f(t_p): linear interpolation between a
    neighbour's two slices reproduces a linear function of time at any t_p."""
    geom, A, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=7)
    _, Bf, _ = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=8)
    ob = O.Bunch(geom, meta["gamma"])
    PA, PB = ob.split(W.to_patches(A, geom)), ob.split(W.to_patches(Bf, geom))
    rng = np.random.default_rng(21)
    P = geom.npatch
    t_old = list(rng.uniform(0.0, 0.3, P))
    t_cur = list(rng.uniform(0.7, 1.0, P))
    old = [PA[q] + t_old[q] * PB[q] for q in range(P)]
    cur = [PA[q] + t_cur[q] * PB[q] for q in range(P)]
    GA = torch.tensor(A)
    GB = torch.tensor(Bf)
    for p in range(P):
        t_p = float(rng.uniform(0.35, 0.65))      # inside every neighbour's interval
        t = list(t_cur)
        t[p] = t_p
        cur_p = list(cur)
        cur_p[p] = PA[p] + t_p * PB[p]
        got = O.fill_guards_at(cur_p, old, t, t_old, geom, p)
        want = O.window(GA + t_p * GB, geom.origin[p], geom.patch_n[p], geom.gvec, geom.domain, geom.bc)
        assert torch.allclose(got, want, rtol=0, atol=1e-13), p


def test_readiness_rule_closed_forms():
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=5)
    ab = O.AsyncBunch(geom, meta["gamma"])
    P = geom.npatch
    assert ab.ready([0.0] * P, 1.0) == list(range(P))          # all at one time: all ready
    t = [0.0] * P
    t[0] = 0.5                                                  # one patch ahead of its neighbours
    assert ab.ready(t, 1.0) == list(range(1, P))
    t = [0.5] * P
    t[0] = 0.0                                                  # one patch behind: only it
    assert ab.ready(t, 1.0) == [0]
    assert ab.ready([1.0] * P, 1.0) == []                       # everyone arrived


def test_replay_of_a_synchronous_schedule_is_the_synchronous_run():
    geom, U, meta = W.small_box(ncell=(24, 16, 16), patch=(8, 8, 8), seed=6, amp=0.6)
    ob = O.Bunch(geom, meta["gamma"])
    P0 = ob.split(W.to_patches(U, geom))
    P, dts = P0, []
    for _ in range(3):
        dt = float(ob.cfl_dt(ob.fill_guards(P)))
        dts.append(dt)
        P = ob.step(P, dt)
    t_span = dts[0] + dts[1] + dts[2]
    ab = O.AsyncBunch(geom, meta["gamma"])
    rounds = [(list(range(geom.npatch)), [dt] * geom.npatch) for dt in dts]
    final, ready_sets, local_dts, t_cur = ab.replay(P0, rounds, t_span)
    assert all(rs == list(range(geom.npatch)) for rs in ready_sets)
    for r, dt in enumerate(dts):                    # the global dt is the minimum of the local ones
        assert min(local_dts[r]) <= dt * (1 + 1e-14) or r == len(dts) - 1
    for a, b in zip(final, P):
        assert torch.allclose(a, b, rtol=1e-14, atol=1e-14)
    assert all(abs(t - t_span) <= 1e-15 for t in t_cur)
