"""Pins of the oracle's HLL face flux (Harten, Lax & van Leer 1983; the paper's mockup solver,
Sec. 2.4) and of the whole step run with it.

Expected values come from outside the HLL code: the physical flux of Eq. 6 retyped from
the equation, the HLLD solver (whose own consistency and exactness are pinned separately),
the two Rankine-Hugoniot relations that define the single HLL state, a closed form of the
numerical diffusion HLL puts on an isolated contact, and the exact Sod solution.
"""
import numpy as np
import pytest
import torch

from oracle import exact_riemann as ER
from oracle import mhd
from paper_2508_09568_gb300 import workloads as W

G = 5.0 / 3.0


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64))


def rand_state(rng, n, bscale=1.0):
    rho = rng.uniform(0.3, 2.0, n)
    un, ut1, ut2 = rng.normal(0, 1, (3, n))
    P = rng.uniform(0.2, 2.0, n)
    bt1, bt2 = rng.normal(0, bscale, (2, n))
    return [rho, un, ut1, ut2, P, bt1, bt2]


def conserved(S, bn, g):
    rho, un, ut1, ut2, pg, bt1, bt2 = [np.asarray(a) for a in S]
    E = pg / (g - 1) + 0.5 * rho * (un ** 2 + ut1 ** 2 + ut2 ** 2) + 0.5 * (bn ** 2 + bt1 ** 2 + bt2 ** 2)
    return [rho, rho * un, rho * ut1, rho * ut2, E]


def physical_flux(S, bn, g):
    """Eq. 6 in the face frame, retyped."""
    rho, un, ut1, ut2, pg, bt1, bt2 = [np.asarray(a) for a in S]
    b2 = bn ** 2 + bt1 ** 2 + bt2 ** 2
    Ptot = pg + 0.5 * b2
    E = pg / (g - 1) + 0.5 * rho * (un ** 2 + ut1 ** 2 + ut2 ** 2) + 0.5 * b2
    udb = un * bn + ut1 * bt1 + ut2 * bt2
    return [rho * un, rho * un ** 2 + Ptot - bn ** 2, rho * ut1 * un - bt1 * bn,
            rho * ut2 * un - bt2 * bn, un * (E + Ptot) - bn * udb]


def fast(S, bn, g):
    """Fast magnetosonic speed along the normal, textbook form."""
    rho, un, ut1, ut2, pg, bt1, bt2 = [np.asarray(a) for a in S]
    a2 = g * pg / rho
    b2 = (bn ** 2 + bt1 ** 2 + bt2 ** 2) / rho
    return np.sqrt(0.5 * (a2 + b2 + np.sqrt((a2 + b2) ** 2 - 4 * a2 * bn ** 2 / rho)))


def call(fn, L, R, bn):
    if fn is mhd.hll:
        out = fn([T(a) for a in L], [T(a) for a in R], T(bn), G)
    else:
        out = fn([T(a) for a in L], [T(a) for a in R], T(bn), G, 1e-12)
    return [f.numpy() for f in out]


def test_consistency_equal_states_against_hlld_and_eq6():
    rng = np.random.default_rng(11)
    S = rand_state(rng, 400)
    bn = rng.normal(0, 1, 400)
    F = call(mhd.hll, S, S, bn)
    Fd = call(mhd.hlld, S, S, bn)
    Fp = physical_flux(S, bn, G)
    for a, b, c in zip(F, Fd, Fp):
        assert np.allclose(a, c, rtol=1e-12, atol=1e-12)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_supersonic_states_take_the_upwind_flux():
    """All signals to the right (left): the flux is F(L) (F(R)), as HLLD's is."""
    rng = np.random.default_rng(12)
    L, R = rand_state(rng, 300), rand_state(rng, 300)
    bn = rng.normal(0, 0.5, 300)
    for sgn in (+1, -1):
        L2, R2 = list(L), list(R)
        L2[1] = sgn * (np.abs(L[1]) + 8.0)
        R2[1] = sgn * (np.abs(R[1]) + 8.0)
        F = call(mhd.hll, L2, R2, bn)
        Fd = call(mhd.hlld, L2, R2, bn)
        up = physical_flux(L2 if sgn > 0 else R2, bn, G)
        for a, b, c in zip(F, Fd, up):
            assert np.allclose(a, c, rtol=1e-12, atol=1e-12)
            assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_subsonic_flux_satisfies_both_jump_relations():
    """With S_L < 0 < S_R the HLL flux is F_L + S_L (U* - U_L) = F_R + S_R (U* - U_R) for the
    single state U* = (S_R U_R - S_L U_L - (F_R - F_L)) / (S_R - S_L); speeds from the
    textbook fast speed."""
    rng = np.random.default_rng(13)
    L, R = rand_state(rng, 500, 0.7), rand_state(rng, 500, 0.7)
    L[1] *= 0.2
    R[1] *= 0.2
    bn = rng.normal(0, 0.7, 500)
    cmax = np.maximum(fast(L, bn, G), fast(R, bn, G))
    SL = np.minimum(L[1], R[1]) - cmax
    SR = np.maximum(L[1], R[1]) + cmax
    assert np.all(SL < 0) and np.all(SR > 0)
    UL, UR = conserved(L, bn, G), conserved(R, bn, G)
    FL, FR = physical_flux(L, bn, G), physical_flux(R, bn, G)
    F = call(mhd.hll, L, R, bn)
    for c in range(5):
        Us = (SR * UR[c] - SL * UL[c] - (FR[c] - FL[c])) / (SR - SL)
        scale = np.abs(FL[c]) + np.abs(FR[c]) + np.abs(SL * UL[c]) + np.abs(SR * UR[c]) + 1.0
        assert np.all(np.abs(F[c] - (FL[c] + SL * (Us - UL[c]))) <= 1e-12 * scale)
        assert np.all(np.abs(F[c] - (FR[c] + SR * (Us - UR[c]))) <= 1e-12 * scale)


def test_isolated_contact_is_smeared_by_the_closed_form_diffusion():
    """A stationary contact (u = 0, equal pressure, B = 0, density jump): HLLD resolves it
    exactly (zero mass flux), HLL carries the mass flux -c (rho_R - rho_L) / 2 with
    c = max of the two sound speeds."""
    rng = np.random.default_rng(14)
    n = 200
    rl, rr = rng.uniform(0.2, 2, n), rng.uniform(0.2, 2, n)
    P = rng.uniform(0.3, 2, n)
    z = np.zeros(n)
    L = [rl, z, z, z, P, z, z]
    R = [rr, z, z, z, P, z, z]
    F = call(mhd.hll, L, R, z)
    Fd = call(mhd.hlld, L, R, z)
    c = np.maximum(np.sqrt(G * P / rl), np.sqrt(G * P / rr))
    assert np.allclose(Fd[0], 0.0, atol=1e-14)
    assert np.allclose(F[0], -0.5 * c * (rr - rl), rtol=1e-12, atol=1e-14)
    assert np.allclose(F[1], P, rtol=1e-12)          # momentum flux: the pressure, unchanged


def _sod_errors(N, riemann):
    geom, U, meta = W.sod(ncell=N, npatch=16)
    B = mhd.Bunch(geom, meta["gamma"], courant=0.8, riemann=riemann)
    P = B.split(W.to_patches(U, geom))
    P, t, k = B.run(P, t_end=0.2)
    G_ = W.from_patches(B.join(P), geom)
    rho = G_[0, 0, 0]
    xl = np.arange(N) / N
    r, ue, pe = ER.cell_average(xl, xl + 1.0 / N, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1), 1.4)
    return np.abs(rho - r).mean()


def test_sod_with_hll_converges_and_is_more_diffusive_than_hlld():
    e = [_sod_errors(N, mhd.RIEMANN_HLL) for N in (64, 128, 256)]
    assert e[0] > e[1] > e[2]
    assert e[2] < 6e-3
    assert e[2] > _sod_errors(256, mhd.RIEMANN_HLLD)


def test_hll_step_conserves_and_keeps_divb_3d():
    geom, U, meta = W.small_box(ncell=(16, 16, 16), patch=(8, 8, 8), seed=15)
    B = mhd.Bunch(geom, meta["gamma"], riemann=mhd.RIEMANN_HLL)
    P = B.split(W.to_patches(U, geom))
    P, t, k = B.run(P, nsteps=4)
    G0 = U
    G1 = W.from_patches(B.join(P), geom)
    for v in (0, 1, 2, 3, 4):
        assert abs(G1[v].sum() - G0[v].sum()) <= 1e-12 * np.abs(G0[v]).sum()
    dx = geom.dx

    def divb(G_):
        return (np.roll(G_[5], -1, 2) - G_[5]) / dx[0] + (np.roll(G_[6], -1, 1) - G_[6]) / dx[1] + \
            (np.roll(G_[7], -1, 0) - G_[7]) / dx[2]
    assert np.max(np.abs(divb(G1) - divb(G0))) * dx[0] < 1e-12
