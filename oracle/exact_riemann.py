"""Exact solution of the Riemann problem of the 1D Euler equations.  TEST INFRASTRUCTURE ONLY.

With B = 0 the MHD system of Sec. 2.1 reduces to the Euler equations, and the Sod shock
tube of Sec. 3.1 is a Riemann problem; its exact self-similar solution (the reference the
paper's Sod comparison appeals to) is computed here with the textbook construction:
the star pressure is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock
(Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction branch otherwise,
solved by Newton iteration; the solution is then sampled at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:   # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:        # rarefaction
        f = 2.0 * a / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
        df = 1.0 / (rho * a) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma, tol=1e-15, maxit=200):
    """(p*, u*, rho*_L, rho*_R) of the Riemann problem."""
    aL, aR = math.sqrt(gamma * pL / rhoL), math.sqrt(gamma * pR / rhoR)
    # two-rarefaction initial guess
    z = (gamma - 1.0) / (2.0 * gamma)
    p = ((aL + aR - 0.5 * (gamma - 1.0) * (uR - uL)) / (aL / pL ** z + aR / pR ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(maxit):
        fL, dL = _fk(p, rhoL, pL, gamma)
        fR, dR = _fk(p, rhoR, pR, gamma)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fk(p, rhoL, pL, gamma)
    fR, _ = _fk(p, rhoR, pR, gamma)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if p > pL:
        rsL = rhoL * (p / pL + g1) / (g1 * p / pL + 1.0)
    else:
        rsL = rhoL * (p / pL) ** (1.0 / gamma)
    if p > pR:
        rsR = rhoR * (p / pR + g1) / (g1 * p / pR + 1.0)
    else:
        rsR = rhoR * (p / pR) ** (1.0 / gamma)
    return p, u, rsL, rsR


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t (array)."""
    ps, us, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    aL, aR = math.sqrt(gamma * pL / rhoL), math.sqrt(gamma * pR / rhoR)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    g = gamma
    for n, s in enumerate(xi.ravel()):
        if s <= us:  # left of contact
            if ps > pL:  # left shock
                SL = uL - aL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                st = (rhoL, uL, pL) if s <= SL else (rsL, us, ps)
            else:        # left rarefaction
                SHL = uL - aL
                asL = aL * (ps / pL) ** ((g - 1) / (2 * g))
                STL = us - asL
                if s <= SHL:
                    st = (rhoL, uL, pL)
                elif s >= STL:
                    st = (rsL, us, ps)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * aL) * (uL - s)
                    st = (rhoL * c ** (2 / (g - 1)),
                          2 / (g + 1) * (aL + (g - 1) / 2 * uL + s),
                          pL * c ** (2 * g / (g - 1)))
        else:        # right of contact
            if ps > pR:  # right shock
                SR = uR + aR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                st = (rsR, us, ps) if s <= SR else (rhoR, uR, pR)
            else:        # right rarefaction
                SHR = uR + aR
                asR = aR * (ps / pR) ** ((g - 1) / (2 * g))
                STR = us + asR
                if s >= SHR:
                    st = (rhoR, uR, pR)
                elif s <= STR:
                    st = (rsR, us, ps)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * aR) * (uR - s)
                    st = (rhoR * c ** (2 / (g - 1)),
                          2 / (g + 1) * (-aR + (g - 1) / 2 * uR + s),
                          pR * c ** (2 * g / (g - 1)))
        rho.flat[n], u.flat[n], p.flat[n] = st
    return rho, u, p


def cell_average(x_lo, x_hi, t, x0, left, right, gamma, sub=64):
    """Cell averages of (rho, u, p) of the exact solution over [x_lo, x_hi] cells (midpoint rule)."""
    x_lo = np.asarray(x_lo)
    h = (x_hi - x_lo) / sub
    acc = [np.zeros_like(x_lo, dtype=np.float64) for _ in range(3)]
    for k in range(sub):
        xs = x_lo + (k + 0.5) * h
        r, u, p = sample((xs - x0) / t, *left, *right, gamma)
        for a, v in zip(acc, (r, u, p)):
            a += v / sub
    return acc
