"""Pins of the oracle's HLLD face flux (Sec. 2.1.2, flux of Eq. 6) and 2D HLL edge EMF (Sec. 2.1.3).

Every reference value here is written independently of the oracle: the physical flux of
Eq. 6 is retyped from the equation, HLLC (the B = 0 limit) from its textbook definition,
the exactness of HLLD on isolated contacts and rotational discontinuities follows from
its construction (Miyoshi & Kusano 2005), the invariance of a face Riemann problem under
rotation of the transverse plane is a symmetry of the equations, and the 1D HLL induction
flux from the HLL formula applied to the induction equation.
"""
import math

import numpy as np
import pytest
import torch

from oracle import mhd

G = 5.0 / 3.0


def T(x):
    return torch.tensor(np.asarray(x, dtype=np.float64))


def rand_state(rng, n, bscale=1.0):
    rho = rng.uniform(0.3, 2.0, n)
    un, ut1, ut2 = rng.normal(0, 1, (3, n))
    P = rng.uniform(0.2, 2.0, n)
    bt1, bt2 = rng.normal(0, bscale, (2, n))
    return [rho, un, ut1, ut2, P, bt1, bt2]


def physical_flux(S, bn, g):
    """Eq. 6 in the face frame, retyped: (rho un, rho un^2 + P - Bn^2, rho ut un - Bt Bn, u(E+P) - Bn u.B)."""
    rho, un, ut1, ut2, pg, bt1, bt2 = [np.asarray(a) for a in S]
    b2 = bn ** 2 + bt1 ** 2 + bt2 ** 2
    Ptot = pg + 0.5 * b2
    E = pg / (g - 1) + 0.5 * rho * (un ** 2 + ut1 ** 2 + ut2 ** 2) + 0.5 * b2
    udb = un * bn + ut1 * bt1 + ut2 * bt2
    return [rho * un, rho * un ** 2 + Ptot - bn ** 2, rho * ut1 * un - bt1 * bn,
            rho * ut2 * un - bt2 * bn, un * (E + Ptot) - bn * udb]


def call_hlld(L, R, bn, eps=1e-12):
    return [f.numpy() for f in mhd.hlld([T(a) for a in L], [T(a) for a in R], T(bn), G, eps)]


def test_consistency_equal_states():
    rng = np.random.default_rng(1)
    S = rand_state(rng, 500)
    bn = rng.normal(0, 1, 500)
    F = call_hlld(S, S, bn)
    Fp = physical_flux(S, bn, G)
    for a, b in zip(F, Fp):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_mirror_symmetry():
    """x -> -x with (un, Bn) -> (-un, -Bn): F(mir R, mir L) = (-F_rho, F_mn, -F_mt, -F_mt, -F_E)."""
    rng = np.random.default_rng(2)
    L, R = rand_state(rng, 400), rand_state(rng, 400)
    bn = rng.normal(0, 1, 400)

    def mir(S):
        return [S[0], -S[1], S[2], S[3], S[4], S[5], S[6]]

    F = call_hlld(L, R, bn)
    Fm = call_hlld(mir(R), mir(L), -bn)
    sign = [-1, 1, -1, -1, -1]
    for a, b, s in zip(F, Fm, sign):
        assert np.allclose(s * a, b, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("solver", ["hlld", "hll"])
def test_rotation_about_the_face_normal(solver):
    """Turning the transverse plane by an angle (velocity and field together) is a symmetry
    of the face Riemann problem: the mass, normal-momentum and energy fluxes are unchanged
    and the transverse momentum flux turns with the plane."""
    rng = np.random.default_rng(14)
    n = 600
    L, R = rand_state(rng, n), rand_state(rng, n)
    bn = rng.normal(0, 1, n)
    th = rng.uniform(0, 2 * np.pi, n)
    c, s_ = np.cos(th), np.sin(th)

    def turn(S):
        rho, un, ut1, ut2, P, bt1, bt2 = S
        return [rho, un, c * ut1 - s_ * ut2, s_ * ut1 + c * ut2, P, c * bt1 - s_ * bt2, s_ * bt1 + c * bt2]

    def flux(A, B):
        if solver == "hlld":
            return call_hlld(A, B, bn)
        return [f.numpy() for f in mhd.hll([T(a) for a in A], [T(a) for a in B], T(bn), G)]

    F, Fr = flux(L, R), flux(turn(L), turn(R))
    scale = max(np.abs(f).max() for f in F)
    for k in (0, 1, 4):
        assert np.max(np.abs(Fr[k] - F[k])) <= 1e-12 * scale, k
    assert np.max(np.abs(Fr[2] - (c * F[2] - s_ * F[3]))) <= 1e-12 * scale
    assert np.max(np.abs(Fr[3] - (s_ * F[2] + c * F[3]))) <= 1e-12 * scale


@pytest.mark.parametrize("alpha", [1e-14, 1e12])
def test_scaling_of_density_pressure_and_field(alpha):
    """Ideal MHD is invariant under rho -> a rho, P -> a P, B -> sqrt(a) B with the
    velocities unchanged (all signal speeds stay the same); every face flux then scales by
    a.  This includes the solver's degenerate-state test, which compares D with Bn^2."""
    rng = np.random.default_rng(15)
    n = 800
    L, R = rand_state(rng, n), rand_state(rng, n)
    bn = rng.normal(0, 1, n)
    bn[:100] = 1e-9 * bn[:100]                # nearly degenerate (Bn -> 0) faces too
    def scale(S):
        rho, un, ut1, ut2, P, bt1, bt2 = S
        r = math.sqrt(alpha)
        return [alpha * rho, un, ut1, ut2, alpha * P, r * bt1, r * bt2]
    F = call_hlld(L, R, bn)
    Fs = call_hlld(scale(L), scale(R), math.sqrt(alpha) * bn)
    for k in range(5):
        assert np.allclose(Fs[k], alpha * F[k], rtol=1e-9, atol=1e-12 * alpha * np.abs(F[k]).max()), k


def test_flux_is_continuous_in_states():
    rng = np.random.default_rng(3)
    L, R = rand_state(rng, 200), rand_state(rng, 200)
    bn = rng.normal(0, 1, 200)
    F0 = call_hlld(L, R, bn)
    h = 1e-7
    L2 = [a + h * rng.normal(0, 1, 200) for a in L]
    F1 = call_hlld(L2, R, bn)
    for a, b in zip(F0, F1):
        assert np.max(np.abs(a - b)) < 1e-4


def test_isolated_contact_is_exact():
    """Density jump only (u, P, B continuous, Bn != 0): HLLD returns the exact flux, no diffusion."""
    rng = np.random.default_rng(4)
    n = 100
    rhoL, rhoR = rng.uniform(0.2, 3, n), rng.uniform(0.2, 3, n)
    un = np.zeros(n)
    ut1, ut2 = rng.normal(0, 1, (2, n))
    P = rng.uniform(0.5, 2, n)
    bt1, bt2 = rng.normal(0, 1, (2, n))
    bn = rng.uniform(0.3, 1.5, n) * rng.choice([-1, 1], n)
    L = [rhoL, un, ut1, ut2, P, bt1, bt2]
    R = [rhoR, un, ut1, ut2, P, bt1, bt2]
    F = call_hlld(L, R, bn)
    Fex = physical_flux(L, bn, G)   # un = 0: mass and energy fluxes vanish on both sides
    for a, b in zip(F, Fex):
        assert np.allclose(a, b, rtol=1e-11, atol=1e-12)
    assert np.max(np.abs(F[0])) < 1e-12


def test_isolated_rotational_discontinuity_is_exact():
    """A stationary Alfven (rotational) discontinuity: un = |Bn|/sqrt(rho) (wave at rest),
    transverse B rotates at constant |Bt|, ut jumps by -sgn(Bn) dBt/sqrt(rho).  HLLD resolves
    it exactly, so its flux equals the physical flux of either side."""
    rng = np.random.default_rng(5)
    n = 50
    rho = rng.uniform(0.5, 2, n)
    bn = rng.uniform(0.5, 1.5, n)
    P = rng.uniform(0.5, 2, n)
    bt = rng.uniform(0.3, 1.0, n)
    thL, thR = rng.uniform(0, 2 * np.pi, (2, n))
    un = -bn / np.sqrt(rho)  # left-moving Alfven wave in the fluid frame, at rest in the lab
    ut1L = rng.normal(0, 0.3, n)
    ut2L = rng.normal(0, 0.3, n)
    b1L, b2L = bt * np.cos(thL), bt * np.sin(thL)
    b1R, b2R = bt * np.cos(thR), bt * np.sin(thR)
    # across the wave: rho [ut] (un - S) = ... -> [ut] = [Bt] * Bn / (rho (un - S)) with S = 0
    ut1R = ut1L + (b1R - b1L) * bn / (rho * un)
    ut2R = ut2L + (b2R - b2L) * bn / (rho * un)
    L = [rho, un, ut1L, ut2L, P, b1L, b2L]
    R = [rho, un, ut1R, ut2R, P, b1R, b2R]
    FL, FR = physical_flux(L, bn, G), physical_flux(R, bn, G)
    for a, b in zip(FL, FR):   # the set-up is a true discontinuity: both sides share the flux
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
    F = call_hlld(L, R, bn)
    for a, b in zip(F, FL):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-10)


def hllc_textbook(L, R, g):
    """HLLC flux for the Euler equations (Toro ch. 10) with the same wave-speed estimates."""
    rL, uL, vL, wL, pL = [np.asarray(a) for a in L[:5]]
    rR, uR, vR, wR, pR = [np.asarray(a) for a in R[:5]]
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    SL = np.minimum(uL, uR) - np.maximum(aL, aR)
    SR = np.maximum(uL, uR) + np.maximum(aL, aR)
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def cons(r, u, v, w, p):
        E = p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)
        return np.stack([r, r * u, r * v, r * w, E])

    def flux(r, u, v, w, p):
        E = p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)
        return np.stack([r * u, r * u * u + p, r * u * v, r * u * w, u * (E + p)])

    def ustar(r, u, v, w, p, S):
        E = p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)
        c = r * (S - u) / (S - Ss)
        return np.stack([c, c * Ss, c * v, c * w, c * (E / r + (Ss - u) * (Ss + p / (r * (S - u))))])

    UL, UR = cons(rL, uL, vL, wL, pL), cons(rR, uR, vR, wR, pR)
    FL, FR = flux(rL, uL, vL, wL, pL), flux(rR, uR, vR, wR, pR)
    FsL = FL + SL * (ustar(rL, uL, vL, wL, pL, SL) - UL)
    FsR = FR + SR * (ustar(rR, uR, vR, wR, pR, SR) - UR)
    return np.where(SL >= 0, FL, np.where(Ss >= 0, FsL, np.where(SR >= 0, FsR, FR)))


def test_zero_field_reduces_to_hllc():
    rng = np.random.default_rng(6)
    n = 400
    L, R = rand_state(rng, n, 0.0), rand_state(rng, n, 0.0)
    L[1] *= 3
    R[1] *= 3   # include supersonic faces so every region is visited
    F = call_hlld(L, R, np.zeros(n))
    Fc = hllc_textbook(L, R, G)
    for k in range(5):
        assert np.allclose(F[k], Fc[k], rtol=1e-11, atol=1e-12)


def test_fast_speed_equals_textbook_form():
    """The expanded discriminant equals a^2 - 4 gamma P bn^2 / rho^2 away from degeneracy."""
    rng = np.random.default_rng(10)
    n = 1000
    rho, P = rng.uniform(0.2, 3, n), rng.uniform(0.1, 3, n)
    bn, b1, b2 = rng.normal(0, 1, (3, n))
    a = (G * P + bn ** 2 + b1 ** 2 + b2 ** 2) / rho
    ref = np.sqrt(0.5 * (a + np.sqrt(a * a - 4 * G * P * bn ** 2 / rho ** 2)))
    got = mhd.fast_speed(T(rho), T(P), T(bn), T(b1), T(b2), G).numpy()
    assert np.allclose(got, ref, rtol=1e-13)


def test_fast_speed_closed_forms():
    rho, P = T([1.3]), T([0.7])
    cs2 = G * 0.7 / 1.3
    # no field: sound speed
    assert math.isclose(float(mhd.fast_speed(rho, P, T([0.0]), T([0.0]), T([0.0]), G)), math.sqrt(cs2), rel_tol=1e-14)
    # field along the normal: max(cs, ca)
    b = 2.0
    ca2 = b * b / 1.3
    assert math.isclose(float(mhd.fast_speed(rho, P, T([b]), T([0.0]), T([0.0]), G)), math.sqrt(max(cs2, ca2)), rel_tol=1e-14)
    # field across the normal: sqrt(cs^2 + ca^2)
    assert math.isclose(float(mhd.fast_speed(rho, P, T([0.0]), T([b]), T([0.0]), G)), math.sqrt(cs2 + ca2), rel_tol=1e-14)


# ---------------------------------------------------------------------------------------
# 2D HLL upwind EMF
# ---------------------------------------------------------------------------------------

def _corner(rng, n):
    return dict(rho=T(rng.uniform(0.5, 2, n)), P=T(rng.uniform(0.5, 2, n)), ua=T(rng.normal(0, 1, n)),
                ub=T(rng.normal(0, 1, n)), ue=T(rng.normal(0, 1, n)), Ba=T(rng.normal(0, 1, n)),
                Bb=T(rng.normal(0, 1, n)), Be=T(rng.normal(0, 1, n)))


def _cf(s, along_a):
    rho, P = s["rho"].numpy(), s["P"].numpy()
    bn = (s["Ba"] if along_a else s["Bb"]).numpy()
    b2 = s["Ba"].numpy() ** 2 + s["Bb"].numpy() ** 2 + s["Be"].numpy() ** 2
    a2, ca2 = G * P / rho, b2 / rho
    return np.sqrt(0.5 * (a2 + ca2 + np.sqrt((a2 + ca2) ** 2 - 4 * a2 * bn ** 2 / rho)))


def hll_1d(F_l, F_r, U_l, U_r, s_l, s_r):
    """1D HLL flux of a single conserved quantity, textbook form with speeds clipped at 0."""
    sl, sr = np.minimum(s_l, 0.0), np.maximum(s_r, 0.0)
    return (sr * F_l - sl * F_r + sl * sr * (U_r - U_l)) / (sr - sl)


def test_emf_reduces_to_1d_hll_along_a():
    """States uniform along b (S = N): E_e equals the 1D HLL flux of B_b along a.

    Induction along a: d B_b/dt + d_a (ua Bb - ub Ba) = 0, so F_a(B_b) = E_e.
    """
    rng = np.random.default_rng(7)
    n = 300
    W, E = _corner(rng, n), _corner(rng, n)
    E["Ba"] = W["Ba"].clone()   # the a-normal field is single valued across the face
    emf = mhd.emf_2d(W, E, W, E, G).numpy()
    e = lambda s: (s["ua"] * s["Bb"] - s["ub"] * s["Ba"]).numpy()
    s_l = np.minimum(W["ua"].numpy() - _cf(W, True), E["ua"].numpy() - _cf(E, True))
    s_r = np.maximum(W["ua"].numpy() + _cf(W, True), E["ua"].numpy() + _cf(E, True))
    ref = hll_1d(e(W), e(E), W["Bb"].numpy(), E["Bb"].numpy(), s_l, s_r)
    assert np.allclose(emf, ref, rtol=1e-11, atol=1e-12)


def test_emf_reduces_to_1d_hll_along_b():
    """States uniform along a (W = E): flux of B_a along b is -E_e, so E_e = -HLL(-E)."""
    rng = np.random.default_rng(8)
    n = 300
    S, N = _corner(rng, n), _corner(rng, n)
    N["Bb"] = S["Bb"].clone()
    emf = mhd.emf_2d(S, S, N, N, G).numpy()
    f = lambda s: -(s["ua"] * s["Bb"] - s["ub"] * s["Ba"]).numpy()
    s_l = np.minimum(S["ub"].numpy() - _cf(S, False), N["ub"].numpy() - _cf(N, False))
    s_r = np.maximum(S["ub"].numpy() + _cf(S, False), N["ub"].numpy() + _cf(N, False))
    ref = -hll_1d(f(S), f(N), S["Ba"].numpy(), N["Ba"].numpy(), s_l, s_r)
    assert np.allclose(emf, ref, rtol=1e-11, atol=1e-12)


def test_emf_uniform_state_is_u_cross_b():
    rng = np.random.default_rng(9)
    s = _corner(rng, 100)
    emf = mhd.emf_2d(s, s, s, s, G).numpy()
    ref = (s["ua"] * s["Bb"] - s["ub"] * s["Ba"]).numpy()
    assert np.allclose(emf, ref, rtol=1e-12, atol=1e-13)
