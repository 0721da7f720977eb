"""FP64 CPU oracle of the MHD bunch update.  TEST INFRASTRUCTURE ONLY.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It shares no code with the CUDA path; it is written from the paper's
method description (Haahr et al., "GPU accelerated MHD in the DISPATCH framework using
directive-based programming"), stage by stage, in plain PyTorch CPU tensor operations
in float64 on whole arrays, with no fusion, blocking or reordering.

One step advances every patch of a bunch by the same dt (synchronous time):

  a1  guard fill          ghost cells copy the cells of the box they stand for
  a2  CFL time step       dt = C / max_cells sum_d (|u_d| + c_f,d) / dx_d
  a3  primitives          Sec. 2.1 (state vector Eq. 6, adiabatic EOS)
  a4  limited slopes      Sec. 2.1.4
  a5  Hancock predictor   Sec. 2.1.4 (primitive Euler half step; face B from the
                          arithmetic edge EMF of Eqs. 7-11, Sec. 2.1.3)
  a6  face states         Sec. 2.1.4
  a7  HLLD face flux      Sec. 2.1.2 (Miyoshi & Kusano 2005), flux of Eq. 6; or the HLL
                          flux of the paper's mockup solver (Sec. 2.4)
  a8  edge EMF            Sec. 2.1.3, Fig. 3 (corner states LB/RB/LT/RT -> SW/SE/NW/NE,
                          two-dimensional HLL upwind EMF)
  a9  update              finite-volume update of rho, rho*u, E; constrained transport
                          for B, Eq. 12 and its cyclic permutations

Readings where the paper is silent (each also listed in the design notes):
  * units with mu_0 = 1 (the flux of Eq. 6 has -B_x^2 and the energy 1/2 B^2);
  * EMF = u x B with dB/dt = +curl(EMF): Eq. 7 computes (u x B)_z and Eq. 12 adds
    +d_y E_z - d_z E_y, so the "-" of the Ohm's law sentence is the physical E;
  * slope limiter: minmod (option: monotonised central) on primitive variables;
  * the time-n edge EMF of Eqs. 7-11 predicts the face field to t+dt/2 by Eq. 12 with
    dt/2; the cell-centred predicted field is the mean of the two predicted faces;
  * HLLD wave speeds S_L = min(u_L,u_R) - max(cf_L,cf_R), S_R = max(u_L,u_R) +
    max(cf_L,cf_R); degenerate star state when |D| <= eps * Bn^2; ties at x/t = 0 take
    the left state;
  * the 2D Riemann solver of Sec. 2.1.3 ("HLLD 2D") is not written out in the paper;
    this oracle uses the two-dimensional HLL upwind EMF with the B-jump terms signed so
    that it reduces to the 1D HLL induction flux when the states do not vary across one
    direction;
  * collapsed axes (extent 1) carry no ghosts, no slopes and no flux differences.

Array convention: a batch of padded patches is a tensor (P, 8, Z, Y, X); x is the last
axis.  Face fields: Bx[..., i] is the low x-face of cell i.  Edge EMFs: Ez[k, j, i] is at
(x_{i-1/2}, y_{j-1/2}, z_k), Ex[k, j, i] at (x_i, y_{j-1/2}, z_{k-1/2}), Ey[k, j, i] at
(x_{i-1/2}, y_j, z_{k-1/2}).  Stencil neighbours are taken with torch.roll over the whole
padded patch; the outermost layers are then garbage and only the interior is kept (its
dependency radius, two cells plus the far face, fits inside a guard of 3).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64
RHO, MX, MY, MZ, EN, BX, BY, BZ = range(8)
BC_PERIODIC, BC_OUTFLOW = 0, 1
LIMITER_MINMOD, LIMITER_MC = 0, 1
RIEMANN_HLLD, RIEMANN_HLL = 0, 1      # face-flux solver of a7
AXIS = {0: -1, 1: -2, 2: -3}     # direction (x, y, z) -> tensor axis

# degenerate-star threshold of the HLLD solver, relative to Bn^2, per arithmetic precision
HLLD_EPS = {8: 1e-12, 4: 1e-6}


# ----------------------------------------------------------------------------------------
# small helpers
# ----------------------------------------------------------------------------------------

def m(a, d):
    """a at index i-1 along direction d."""
    return torch.roll(a, shifts=1, dims=AXIS[d])


def p(a, d):
    """a at index i+1 along direction d."""
    return torch.roll(a, shifts=-1, dims=AXIS[d])


def minmod(a, b):
    """minmod(a, b) = 0 if a*b <= 0 else the argument of smaller magnitude (ties: a)."""
    pick = torch.where(a.abs() <= b.abs(), a, b)
    return torch.where(a * b > 0, pick, torch.zeros_like(a))


def mc(a, b):
    """Monotonised central limiter: 0 if a*b <= 0, else sign * min(2|a|, 2|b|, |a+b|/2)."""
    c = 0.5 * (a + b)
    m2 = torch.where((2 * a).abs() <= (2 * b).abs(), 2 * a, 2 * b)
    pick = torch.where(c.abs() <= m2.abs(), c, m2)
    return torch.where(a * b > 0, pick, torch.zeros_like(a))


def limited(q, d, limiter):
    """Limited undivided slope of q along d (Sec. 2.1.4: slopes from neighbour differences)."""
    lim = minmod if limiter == LIMITER_MINMOD else mc
    return lim(q - m(q, d), p(q, d) - q)


def safe_sqrt(x):
    """sqrt(max(x, 0)) with derivative 0 at 0 (subgradient reading for the adjoint)."""
    pos = x > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))), torch.zeros_like(x))


def fmax(a, b):
    """max(a, b), ties -> a (first argument)."""
    return torch.where(a >= b, a, b)


def fmin(a, b):
    """min(a, b), ties -> a (first argument)."""
    return torch.where(a <= b, a, b)


def fast_speed(rho, P, bn, bt1, bt2, gamma):
    """Fast magnetosonic speed along the normal whose field component is bn.

    c_f^2 = 1/2 [ (cs^2 + ca^2) + sqrt( (cs^2 + ca^2)^2 - 4 cs^2 can^2 ) ]
    with cs^2 = gamma P / rho, ca^2 = B^2 / rho, can^2 = bn^2 / rho.  The discriminant is
    evaluated in the algebraically identical expanded form
    (cs^2 - can^2)^2 + cat^2 (2 (cs^2 + can^2) + cat^2), cat^2 = (bt1^2 + bt2^2) / rho,
    whose terms are all non-negative (no cancellation when cs ~ can and B is along n).
    """
    cs2 = gamma * P / rho
    can2 = bn * bn / rho
    cat2 = (bt1 * bt1 + bt2 * bt2) / rho
    d = cs2 - can2
    disc = d * d + cat2 * (2.0 * (cs2 + can2) + cat2)
    return torch.sqrt(0.5 * (cs2 + can2 + cat2 + safe_sqrt(disc)))


# ----------------------------------------------------------------------------------------
# a1: guard fill
# ----------------------------------------------------------------------------------------

def _wrap(idx, n, lo, hi):
    out = idx.clone()
    below, above = idx < 0, idx >= n
    out[below] = torch.remainder(idx[below], n) if lo == BC_PERIODIC else 0
    out[above] = torch.remainder(idx[above], n) if hi == BC_PERIODIC else n - 1
    return out


def window(global_U, origin, n, gvec, domain, bc):
    """Padded patch (8, Z, Y, X) whose every cell (ghosts included) holds the box cell it covers.

    Ghost positions beyond the box are mapped by the boundary kind: periodic wrap or
    zero-gradient (copy of the edge cell; for a normal face field the copy of the last
    owned face, which keeps the discrete divergence of the ghost cell at zero).
    """
    idx = []
    for d in range(3):
        r = torch.arange(int(n[d]) + 2 * int(gvec[d])) + int(origin[d]) - int(gvec[d])
        idx.append(_wrap(r, int(domain[d]), int(bc[d][0]), int(bc[d][1])))
    ix, iy, iz = idx
    return global_U[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def assemble(patches, geom_n, geom_origin, gvec, domain):
    """Global interior field (8, Nz, Ny, Nx) from a list of padded patches."""
    G = torch.full((8, int(domain[2]), int(domain[1]), int(domain[0])), float("nan"), dtype=F64)
    for Up, n, o in zip(patches, geom_n, geom_origin):
        g = gvec
        G[:, o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = \
            Up[:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
    return G


def fill_guards(patches, geom):
    """a1 for a whole bunch: every ghost cell gets the value of the box cell it stands for.

    patches: list of padded patches (8, Z, Y, X) (interiors valid).  Returns a new list.
    """
    G = assemble(patches, geom.patch_n, geom.origin, geom.gvec, geom.domain)
    return [window(G, geom.origin[i], geom.patch_n[i], geom.gvec, geom.domain, geom.bc)
            for i in range(len(patches))]


# ----------------------------------------------------------------------------------------
# a3: primitive variables
# ----------------------------------------------------------------------------------------

def primitives(U, gamma):
    """(rho, u, v, w, P_gas, Bxc, Byc, Bzc) from the conserved state (Eq. 6, EOS of Sec. 2.1).

    The cell-centred field is the mean of the two faces of the cell.
    """
    rho = U[:, RHO]
    u, v, w = U[:, MX] / rho, U[:, MY] / rho, U[:, MZ] / rho
    bxc = 0.5 * (U[:, BX] + p(U[:, BX], 0))
    byc = 0.5 * (U[:, BY] + p(U[:, BY], 1))
    bzc = 0.5 * (U[:, BZ] + p(U[:, BZ], 2))
    P = (gamma - 1.0) * (U[:, EN] - 0.5 * rho * (u * u + v * v + w * w)
                         - 0.5 * (bxc * bxc + byc * byc + bzc * bzc))
    return [rho, u, v, w, P, bxc, byc, bzc]


# ----------------------------------------------------------------------------------------
# a2: CFL time step
# ----------------------------------------------------------------------------------------

def cfl_rate(U, active, dx, gamma):
    """Per cell sum over active axes of (|u_d| + c_f,d) / dx_d."""
    rho, u, v, w, P, bxc, byc, bzc = primitives(U, gamma)
    vel = [u, v, w]
    bc = [bxc, byc, bzc]
    rate = torch.zeros_like(rho)
    for d in range(3):
        if not active[d]:
            continue
        cf = fast_speed(rho, P, bc[d], bc[(d + 1) % 3], bc[(d + 2) % 3], gamma)
        rate = rate + (vel[d].abs() + cf) / dx[d]
    return rate


def cfl_dt(patches, geom, gamma, courant):
    """a2: dt = C / max over all interior cells of the bunch of cfl_rate."""
    g = geom.gvec
    rmax = torch.zeros((), dtype=F64)
    for Up, n in zip(patches, geom.patch_n):
        r = cfl_rate(Up[None], geom.active, geom.dx, gamma)[0]
        r = r[g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
        rmax = torch.maximum(rmax, r.max())
    return courant / rmax


# ----------------------------------------------------------------------------------------
# a7: HLLD Riemann solver (Miyoshi & Kusano 2005), Sec. 2.1.2
# ----------------------------------------------------------------------------------------

def hlld(L, R, bn, gamma, eps):
    """HLLD flux through a face with normal field bn.

    L, R: lists (rho, un, ut1, ut2, P, bt1, bt2) of the left and right states.
    Returns the fluxes of (rho, rho*un, rho*ut1, rho*ut2, E) (the flux of Eq. 6 in the
    frame of the face) of the region that covers x/t = 0 among the six of the solver.
    """
    def side(S):
        rho, un, ut1, ut2, P, bt1, bt2 = S
        b2 = bn * bn + bt1 * bt1 + bt2 * bt2
        pT = P + 0.5 * b2
        E = P / (gamma - 1.0) + 0.5 * rho * (un * un + ut1 * ut1 + ut2 * ut2) + 0.5 * b2
        cf = fast_speed(rho, P, bn, bt1, bt2, gamma)
        vb = un * bn + ut1 * bt1 + ut2 * bt2
        U = [rho, rho * un, rho * ut1, rho * ut2, E]
        F = [rho * un,
             rho * un * un + pT - bn * bn,
             rho * ut1 * un - bt1 * bn,
             rho * ut2 * un - bt2 * bn,
             (E + pT) * un - bn * vb]
        return dict(rho=rho, un=un, ut1=ut1, ut2=ut2, bt1=bt1, bt2=bt2, pT=pT, E=E, cf=cf,
                    vb=vb, U=U, F=F)

    l, r = side(L), side(R)
    cmax = fmax(l["cf"], r["cf"])
    SL = fmin(l["un"], r["un"]) - cmax
    SR = fmax(l["un"], r["un"]) + cmax
    dl = (SL - l["un"]) * l["rho"]
    dr = (SR - r["un"]) * r["rho"]
    den = dr - dl
    SM = (dr * r["un"] - dl * l["un"] - r["pT"] + l["pT"]) / den
    pTs = (dr * l["pT"] - dl * r["pT"] + dl * dr * (r["un"] - l["un"])) / den

    def star(s, S):
        rhos = s["rho"] * (S - s["un"]) / (S - SM)
        D = s["rho"] * (S - s["un"]) * (S - SM) - bn * bn
        degen = D.abs() <= eps * bn * bn
        Dsafe = torch.where(degen, torch.ones_like(D), D)
        num_u = bn * (SM - s["un"]) / Dsafe
        num_b = (s["rho"] * (S - s["un"]) ** 2 - bn * bn) / Dsafe
        ut1 = torch.where(degen, s["ut1"], s["ut1"] - s["bt1"] * num_u)
        ut2 = torch.where(degen, s["ut2"], s["ut2"] - s["bt2"] * num_u)
        bt1 = torch.where(degen, s["bt1"], s["bt1"] * num_b)
        bt2 = torch.where(degen, s["bt2"], s["bt2"] * num_b)
        vbs = SM * bn + ut1 * bt1 + ut2 * bt2
        Es = ((S - s["un"]) * s["E"] - s["pT"] * s["un"] + pTs * SM + bn * (s["vb"] - vbs)) / (S - SM)
        U = [rhos, rhos * SM, rhos * ut1, rhos * ut2, Es]
        return dict(rho=rhos, ut1=ut1, ut2=ut2, bt1=bt1, bt2=bt2, vb=vbs, E=Es, U=U)

    ls, rs = star(l, SL), star(r, SR)
    sl, sr = torch.sqrt(ls["rho"]), torch.sqrt(rs["rho"])
    SsL = SM - bn.abs() / sl
    SsR = SM + bn.abs() / sr
    sgn = torch.sign(bn)
    ssum = sl + sr
    ut1d = (sl * ls["ut1"] + sr * rs["ut1"] + (rs["bt1"] - ls["bt1"]) * sgn) / ssum
    ut2d = (sl * ls["ut2"] + sr * rs["ut2"] + (rs["bt2"] - ls["bt2"]) * sgn) / ssum
    bt1d = (sl * rs["bt1"] + sr * ls["bt1"] + sl * sr * (rs["ut1"] - ls["ut1"]) * sgn) / ssum
    bt2d = (sl * rs["bt2"] + sr * ls["bt2"] + sl * sr * (rs["ut2"] - ls["ut2"]) * sgn) / ssum
    vbd = SM * bn + ut1d * bt1d + ut2d * bt2d
    EdL = ls["E"] - sl * (ls["vb"] - vbd) * sgn
    EdR = rs["E"] + sr * (rs["vb"] - vbd) * sgn
    UdL = [ls["rho"], ls["rho"] * SM, ls["rho"] * ut1d, ls["rho"] * ut2d, EdL]
    UdR = [rs["rho"], rs["rho"] * SM, rs["rho"] * ut1d, rs["rho"] * ut2d, EdR]

    out = []
    for c in range(5):
        FL, FR = l["F"][c], r["F"][c]
        FsL = FL + SL * (ls["U"][c] - l["U"][c])
        FsR = FR + SR * (rs["U"][c] - r["U"][c])
        FdL = FsL + SsL * (UdL[c] - ls["U"][c])
        FdR = FsR + SsR * (UdR[c] - rs["U"][c])
        f = torch.where(SR >= 0, FsR, FR)
        f = torch.where(SsR >= 0, FdR, f)
        f = torch.where(SM >= 0, FdL, f)
        f = torch.where(SsL >= 0, FsL, f)
        f = torch.where(SL >= 0, FL, f)
        out.append(f)
    return out


# ----------------------------------------------------------------------------------------
# a7 variant: HLL face flux (Harten, Lax & van Leer 1983), the simple solver the paper's
# mockup used before the HLLD solver (Sec. 2.4)
# ----------------------------------------------------------------------------------------

def hll(L, R, bn, gamma):
    """HLL flux through a face with normal field bn.

    One intermediate state between the fastest left- and right-going signals, with the
    same estimates as hlld: S_L = min(u_L, u_R) - max(cf_L, cf_R), S_R = max(u_L, u_R) +
    max(cf_L, cf_R).  The flux at x/t = 0 is F_L when S_L >= 0, otherwise the HLL flux
    (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) when S_R >= 0, otherwise F_R.
    L, R and the result as in hlld.
    """
    def conserved_and_flux(S):
        rho, un, ut1, ut2, P, bt1, bt2 = S
        b2 = bn * bn + bt1 * bt1 + bt2 * bt2
        pT = P + 0.5 * b2
        E = P / (gamma - 1.0) + 0.5 * rho * (un * un + ut1 * ut1 + ut2 * ut2) + 0.5 * b2
        U = [rho, rho * un, rho * ut1, rho * ut2, E]
        F = [rho * un,
             rho * un * un + pT - bn * bn,
             rho * ut1 * un - bt1 * bn,
             rho * ut2 * un - bt2 * bn,
             (E + pT) * un - bn * (un * bn + ut1 * bt1 + ut2 * bt2)]
        return U, F, fast_speed(rho, P, bn, bt1, bt2, gamma)

    UL, FL, cfl = conserved_and_flux(L)
    UR, FR, cfr = conserved_and_flux(R)
    cmax = fmax(cfl, cfr)
    SL = fmin(L[1], R[1]) - cmax
    SR = fmax(L[1], R[1]) + cmax
    out = []
    for c in range(5):
        fh = (SR * FL[c] - SL * FR[c] + SL * SR * (UR[c] - UL[c])) / (SR - SL)
        out.append(torch.where(SL >= 0, FL[c], torch.where(SR >= 0, fh, FR[c])))
    return out


# ----------------------------------------------------------------------------------------
# a8: two-dimensional HLL upwind EMF at an edge, Sec. 2.1.3 / Fig. 3
# ----------------------------------------------------------------------------------------

def emf_2d(SW, SE, NW, NE, gamma):
    """EMF along an edge from the four corner states around it.

    Each state is a dict with rho, P, ua, ub, ue (velocity along the two transverse
    directions a, b and the edge direction e) and Ba, Bb, Be.  E/W are the sides along a,
    N/S along b.  E_e = ua*Bb - ub*Ba for each state.
    """
    def e(s):
        return s["ua"] * s["Bb"] - s["ub"] * s["Ba"]

    def cf(s, along_a):
        bn = s["Ba"] if along_a else s["Bb"]
        bt = s["Bb"] if along_a else s["Ba"]
        return fast_speed(s["rho"], s["P"], bn, bt, s["Be"], gamma)

    states = [SW, SE, NW, NE]
    up_a = [s["ua"] + cf(s, True) for s in states]
    dn_a = [s["ua"] - cf(s, True) for s in states]
    up_b = [s["ub"] + cf(s, False) for s in states]
    dn_b = [s["ub"] - cf(s, False) for s in states]
    zero = torch.zeros_like(SW["rho"])
    SE_ = fmax(fmax(fmax(fmax(up_a[0], up_a[1]), up_a[2]), up_a[3]), zero)
    SWs = fmin(fmin(fmin(fmin(dn_a[0], dn_a[1]), dn_a[2]), dn_a[3]), zero)
    SN = fmax(fmax(fmax(fmax(up_b[0], up_b[1]), up_b[2]), up_b[3]), zero)
    SS = fmin(fmin(fmin(fmin(dn_b[0], dn_b[1]), dn_b[2]), dn_b[3]), zero)
    da = SE_ - SWs
    db = SN - SS
    num = SE_ * SN * e(SW) - SE_ * SS * e(NW) - SWs * SN * e(SE) + SWs * SS * e(NE)
    bb_e, bb_w = SE["Bb"], SW["Bb"]      # B_b on the east / west side (single valued)
    ba_n, ba_s = NW["Ba"], SW["Ba"]      # B_a on the north / south side
    return num / (da * db) + SE_ * SWs / da * (bb_e - bb_w) - SN * SS / db * (ba_n - ba_s)


# ----------------------------------------------------------------------------------------
# one step (a3 - a9) for a batch of padded patches
# ----------------------------------------------------------------------------------------

def step(Up, dt, active, dx, gamma, limiter=LIMITER_MINMOD, eps=HLLD_EPS[8], gvec=None, n=None,
         riemann=RIEMANN_HLLD):
    """Advance padded patches (P, 8, Z, Y, X) by dt; returns the new padded tensor.

    riemann selects the face-flux solver of a7: RIEMANN_HLLD (Sec. 2.1.2) or RIEMANN_HLL.

    Only interior cells (and their owned low faces) of the result are meaningful; the
    ghost layers of the result are copies of the input ghosts.
    """
    Up = Up.to(F64)
    dx = [float(a) for a in dx]
    act = [bool(a) for a in active]
    hdt = 0.5 * dt
    zero = torch.zeros_like(Up[:, 0])

    # a3 primitives at time n
    W = primitives(Up, gamma)
    rho, u, v, w, P = W[:5]
    vel = [u, v, w]
    bf = [Up[:, BX], Up[:, BY], Up[:, BZ]]   # face fields at time n

    # a4 limited slopes of the 8 primitives and the transverse slopes of the face fields
    dW = [[limited(q, d, limiter) if act[d] else zero for q in W] for d in range(3)]
    dbf = [[limited(bf[c], d, limiter) if (act[d] and d != c) else zero for d in range(3)]
           for c in range(3)]   # dbf[c][d]: slope of face field c along d

    # Eqs. 7-11: time-n edge EMF from 4-cell velocity averages and 2-face field averages.
    # E_e at the edge low in (a, b) with (e, a, b) cyclic: E_e = va*Bb - vb*Ba.
    def avg4(q, a, b):
        return 0.25 * (q + m(q, a) + m(q, b) + m(m(q, a), b))

    def emf_n(e):
        a, b = (e + 1) % 3, (e + 2) % 3
        va, vb_ = avg4(vel[a], a, b), avg4(vel[b], a, b)
        Ba = 0.5 * (bf[a] + m(bf[a], b))
        Bb = 0.5 * (bf[b] + m(bf[b], a))
        return va * Bb - vb_ * Ba

    En = [emf_n(e) for e in range(3)]

    # Eq. 12 over dt/2: predicted face fields; dB_c/dt = d_a E_b... in cyclic form
    # dBx/dt = d_y Ez - d_z Ey ; dBy/dt = d_z Ex - d_x Ez ; dBz/dt = d_x Ey - d_y Ex
    def curl_term(E, c, k):
        a, b = (c + 1) % 3, (c + 2) % 3
        t = torch.zeros_like(E[0])
        if act[a]:
            t = t + k * (p(E[b], a) - E[b]) / dx[a]
        if act[b]:
            t = t - k * (p(E[a], b) - E[a]) / dx[b]
        return t

    bh = [bf[c] + curl_term(En, c, hdt) for c in range(3)]
    bch = [0.5 * (bh[c] + p(bh[c], c)) for c in range(3)]

    # a5 Hancock predictor in primitive form (Euler half step with the slopes)
    D = [[dW[d][q] / dx[d] if act[d] else zero for q in range(8)] for d in range(3)]
    divu = D[0][1] + D[1][2] + D[2][3]
    bcn = W[5:8]

    def adv(q):
        return u * D[0][q] + v * D[1][q] + w * D[2][q]

    rho_h = rho - hdt * (adv(0) + rho * divu)
    P_h = P - hdt * (adv(4) + gamma * P * divu)
    vel_h = []
    for c in range(3):
        a, b = (c + 1) % 3, (c + 2) % 3
        # (1/rho)[ d_c P + B_a d_c B_a + B_b d_c B_b - B_a d_a B_c - B_b d_b B_c ]
        lor = (D[c][4] + bcn[a] * D[c][5 + a] + bcn[b] * D[c][5 + b]
               - bcn[a] * D[a][5 + c] - bcn[b] * D[b][5 + c])
        vel_h.append(vel[c] - hdt * (adv(1 + c) + lor / rho))
    Wh = [rho_h, vel_h[0], vel_h[1], vel_h[2], P_h, bch[0], bch[1], bch[2]]

    # a6 + a7: face states and HLLD fluxes of (rho, m_x, m_y, m_z, E) on low faces
    flux = []
    for d in range(3):
        if not act[d]:
            flux.append(None)
            continue
        t1, t2 = (d + 1) % 3, (d + 2) % 3
        plus = [Wh[q] + 0.5 * dW[d][q] for q in range(8)]     # state at the high face
        minus = [Wh[q] - 0.5 * dW[d][q] for q in range(8)]    # state at the low face
        Lq = [m(q, d) for q in plus]    # left state of the low face of cell i (cell i-1)
        Rq = minus
        L = [Lq[0], Lq[1 + d], Lq[1 + t1], Lq[1 + t2], Lq[4], Lq[5 + t1], Lq[5 + t2]]
        R = [Rq[0], Rq[1 + d], Rq[1 + t1], Rq[1 + t2], Rq[4], Rq[5 + t1], Rq[5 + t2]]
        f = hlld(L, R, bh[d], gamma, eps) if riemann == RIEMANN_HLLD else hll(L, R, bh[d], gamma)
        F = [None] * 5
        F[0], F[4] = f[0], f[4]
        F[1 + d], F[1 + t1], F[1 + t2] = f[1], f[2], f[3]
        flux.append(F)

    # a8: corner states and edge EMF at t+dt/2 for each edge direction e, (a, b) cyclic.
    def corner(c_a, c_b, e):
        """Predicted state of each cell at its corner (sa, sb) in the (a, b) plane."""
        a, b = (e + 1) % 3, (e + 2) % 3
        q = [Wh[k] + 0.5 * (c_a * dW[a][k] + c_b * dW[b][k]) for k in range(8)]
        ba_face = bh[a] if c_a < 0 else p(bh[a], a)
        bb_face = bh[b] if c_b < 0 else p(bh[b], b)
        dba = dbf[a][b] if c_a < 0 else p(dbf[a][b], a)
        dbb = dbf[b][a] if c_b < 0 else p(dbf[b][a], b)
        return dict(rho=q[0], P=q[4], ua=q[1 + a], ub=q[1 + b], ue=q[1 + e],
                    Ba=ba_face + 0.5 * c_b * dba, Bb=bb_face + 0.5 * c_a * dbb, Be=q[5 + e])

    def shift(s, fn):
        return {k: fn(t) for k, t in s.items()}

    Eh = [None, None, None]
    for e in range(3):
        a, b = (e + 1) % 3, (e + 2) % 3
        if not (act[a] or act[b]):
            Eh[e] = None
            continue
        RT, LT, RB, LB = corner(+1, +1, e), corner(-1, +1, e), corner(+1, -1, e), corner(-1, -1, e)
        SW = shift(RT, lambda t: m(m(t, a), b))
        SE = shift(LT, lambda t: m(t, b))
        NW = shift(RB, lambda t: m(t, a))
        NE = LB
        Eh[e] = emf_2d(SW, SE, NW, NE, gamma)

    # a9: conservative update and constrained transport (Eq. 12)
    out = Up.clone()
    for k, var in enumerate([RHO, MX, MY, MZ, EN]):
        du = torch.zeros_like(rho)
        for d in range(3):
            if act[d]:
                du = du - dt * (p(flux[d][k], d) - flux[d][k]) / dx[d]
        out[:, var] = Up[:, var] + du
    for c in range(3):
        a, b = (c + 1) % 3, (c + 2) % 3
        t = torch.zeros_like(rho)
        if act[a] and Eh[b] is not None:
            t = t + dt * (p(Eh[b], a) - Eh[b]) / dx[a]
        if act[b] and Eh[a] is not None:
            t = t - dt * (p(Eh[a], b) - Eh[a]) / dx[b]
        out[:, BX + c] = Up[:, BX + c] + t
    if gvec is not None and n is not None:
        # keep the input ghosts: only interior cells are part of the update
        res = Up.clone()
        g = gvec
        sl = (slice(None), slice(None), slice(g[2], g[2] + n[2]), slice(g[1], g[1] + n[1]),
              slice(g[0], g[0] + n[0]))
        res[sl] = out[sl]
        return res
    return out


# ----------------------------------------------------------------------------------------
# bunch driver: a flat buffer in the shared layout
# ----------------------------------------------------------------------------------------

class Bunch:
    """Oracle view of a flat bunch buffer (float64), following the shared layout."""

    def __init__(self, geom, gamma, courant=0.8, limiter=LIMITER_MINMOD, eps=HLLD_EPS[8], riemann=RIEMANN_HLLD):
        self.geom = geom
        self.gamma = float(gamma)
        self.courant = float(courant)
        self.limiter = int(limiter)
        self.eps = float(eps)
        self.riemann = int(riemann)

    def split(self, flat):
        g = self.geom
        offs = g.offsets()
        out = []
        for i in range(g.npatch):
            Z, Y, X = g.padded(i)
            out.append(torch.as_tensor(np.asarray(flat[offs[i]:offs[i] + 8 * X * Y * Z]),
                                       dtype=F64).reshape(8, Z, Y, X))
        return out

    def join(self, patches):
        return torch.cat([q.reshape(-1) for q in patches]).numpy()

    def fill_guards(self, patches):
        return fill_guards(patches, self.geom)

    def cfl_dt(self, patches):
        return float(cfl_dt(patches, self.geom, self.gamma, self.courant))

    def step(self, patches, dt):
        """Guard fill then one update of every patch; returns the new list of patches."""
        geom = self.geom
        filled = self.fill_guards(patches)
        out = []
        # equal-size patches are advanced together
        sizes = {}
        for i in range(geom.npatch):
            sizes.setdefault(tuple(geom.patch_n[i]), []).append(i)
        res = [None] * geom.npatch
        for n, idx in sizes.items():
            batch = torch.stack([filled[i] for i in idx])
            new = step(batch, dt, geom.active, geom.dx, self.gamma, self.limiter, self.eps,
                       gvec=geom.gvec, n=n, riemann=self.riemann)
            for j, i in enumerate(idx):
                res[i] = new[j]
        return res

    def run(self, patches, t_end=None, nsteps=None, dt_fixed=None):
        """Advance to t_end (last step clipped) or for nsteps; returns (patches, t, steps)."""
        t, k = 0.0, 0
        while True:
            if nsteps is not None and k >= nsteps:
                break
            if t_end is not None and t >= t_end * (1 - 1e-14):
                break
            if dt_fixed is not None:
                dt = dt_fixed
            else:
                dt = self.cfl_dt(self.fill_guards(patches))
            if t_end is not None and t + dt > t_end:
                dt = t_end - t
            patches = self.step(patches, dt)
            t += dt
            k += 1
        return patches, t, k


# ----------------------------------------------------------------------------------------
# Asynchronous per-patch stepping (DISPATCH's patches at their own times, Sec. 2.2, updated
# in bunches of the ready ones, Sec. 2.4).  Readings: each patch keeps two time slices; a
# patch is ready when it is short of the target time and no neighbour (a patch owning a cell
# of its guard zone) is at an earlier time; its guard values are the neighbours' two slices
# interpolated linearly in time to its own time; it steps by its own CFL dt clipped to the
# target time.
# ----------------------------------------------------------------------------------------

def owner_map(geom):
    """Patch index of every box cell (Nz, Ny, Nx)."""
    own = np.full((int(geom.domain[2]), int(geom.domain[1]), int(geom.domain[0])), -1, dtype=np.int64)
    for p in range(geom.npatch):
        o, n = geom.origin[p], geom.patch_n[p]
        own[o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = p
    return own


def _window_index(geom, p):
    """Box indices (iz, iy, ix) covered by padded patch p (wrap / clamp by the boundary kinds)."""
    idx = []
    for d in range(3):
        r = torch.arange(int(geom.patch_n[p][d]) + 2 * int(geom.gvec[d])) + int(geom.origin[p][d]) - int(geom.gvec[d])
        idx.append(_wrap(r, int(geom.domain[d]), int(geom.bc[d][0]), int(geom.bc[d][1])).numpy())
    return idx[2], idx[1], idx[0]


def neighbours(geom):
    """For each patch the set of other patches that own a cell of its guard zone."""
    own = owner_map(geom)
    out = []
    for p in range(geom.npatch):
        iz, iy, ix = _window_index(geom, p)
        covered = own[np.ix_(iz, iy, ix)]
        out.append(set(int(q) for q in np.unique(covered)) - {p})
    return out


def fill_guards_at(cur, old, t_cur, t_old, geom, p):
    """Padded patch p with every guard cell at time t_cur[p]: the box cell's patch q gives
    old_q + w (cur_q - old_q), w = (t_cur[p] - t_old[q]) / (t_cur[q] - t_old[q]) (the current
    slice when w >= 1 or the two slice times are equal, the previous one when w <= 0)."""
    blended = []
    for q in range(geom.npatch):
        den = t_cur[q] - t_old[q]
        w = (t_cur[p] - t_old[q]) / den if den > 0 else 1.0
        if w >= 1.0:
            blended.append(cur[q])
        elif w <= 0.0:
            blended.append(old[q])
        else:
            blended.append(old[q] + w * (cur[q] - old[q]))
    G = assemble(blended, geom.patch_n, geom.origin, geom.gvec, geom.domain)
    return window(G, geom.origin[p], geom.patch_n[p], geom.gvec, geom.domain, geom.bc)


class AsyncBunch:
    """Asynchronous stepping of a bunch (FP64), for checking a recorded schedule."""

    def __init__(self, geom, gamma, courant=0.8, limiter=LIMITER_MINMOD, eps=HLLD_EPS[8], riemann=RIEMANN_HLLD):
        self.geom = geom
        self.gamma, self.courant = float(gamma), float(courant)
        self.limiter, self.eps, self.riemann = int(limiter), float(eps), int(riemann)
        self.nbrs = neighbours(geom)

    def ready(self, t_cur, t_span):
        return [p for p in range(self.geom.npatch)
                if t_cur[p] < t_span and all(t_cur[q] >= t_cur[p] for q in self.nbrs[p])]

    def local_dt(self, filled, p):
        g, n = self.geom.gvec, self.geom.patch_n[p]
        r = cfl_rate(filled[None], self.geom.active, self.geom.dx, self.gamma)[0]
        r = r[g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
        return float(self.courant / r.max())

    def replay(self, patches, rounds, t_span):
        """Apply a recorded schedule [(patches, dts), ...] to the list of padded patches.

        Returns (final patches, the ready set the rule gives before each round, the local
        CFL dt of each listed patch clipped to t_span, final times)."""
        geom = self.geom
        P = geom.npatch
        cur = [u.clone() for u in patches]
        old = [u.clone() for u in patches]
        t_cur, t_old = [0.0] * P, [0.0] * P
        ready_sets, local_dts = [], []
        for plist, dts in rounds:
            ready_sets.append(self.ready(t_cur, t_span))
            filled = {int(p): fill_guards_at(cur, old, t_cur, t_old, geom, int(p)) for p in plist}
            ldt = []
            for p in plist:
                p = int(p)
                ldt.append(min(self.local_dt(filled[p], p), t_span - t_cur[p]))
            local_dts.append(ldt)
            new = {}
            for p, dt in zip(plist, dts):
                p = int(p)
                n = geom.patch_n[p]
                new[p] = step(filled[p][None], float(dt), geom.active, geom.dx, self.gamma, self.limiter, self.eps,
                              gvec=geom.gvec, n=n, riemann=self.riemann)[0]
            for p, dt in zip(plist, dts):
                p = int(p)
                old[p] = cur[p]
                cur[p] = new[p]
                t_old[p] = t_cur[p]
                t_cur[p] = t_cur[p] + float(dt) if float(dt) < t_span - t_cur[p] else t_span
            # (a clipped last step lands exactly on t_span)
        return cur, ready_sets, local_dts, t_cur
