// Per-cell / per-face / per-edge arithmetic of the MHD bunch update (device code).
//
// Method: Haahr et al., Sec. 2.1 (ideal MHD, state vector and x-flux of Eq. 6, adiabatic
// EOS), Sec. 2.1.2 (HLLD solver, after Miyoshi & Kusano 2005), Sec. 2.1.3 (staggered
// field, arithmetic edge EMF of Eqs. 7-11, constrained transport Eq. 12, 2D Riemann
// problem at cell edges from the LB/RB/LT/RT corner states of Fig. 3), Sec. 2.1.4 (MUSCL
// slopes and Hancock half-step predictor).  Readings for what the paper leaves open are
// stated where they are used (EMF = u x B with dB/dt = +curl EMF; minmod/MC limiter;
// two-dimensional HLL edge EMF; HLLD degenerate threshold eps * Bn^2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mhd_ops.cuh"

namespace mhd {

// Variable order of the state and of the primitive vector.
enum { V_RHO = 0, V_MX = 1, V_MY = 2, V_MZ = 3, V_EN = 4, V_BX = 5, V_BY = 6, V_BZ = 7 };
// Primitive order: rho, u, v, w, P_gas, Bx_c, By_c, Bz_c.
enum { Q_RHO = 0, Q_U = 1, Q_V = 2, Q_W = 3, Q_P = 4, Q_BX = 5, Q_BY = 6, Q_BZ = 7 };

// max/min with ties going to the first argument (the subgradient choice of the adjoint)
template <typename R>
MHD_HD R fmax1(R a, R b) { return a >= b ? a : b; }
template <typename R>
MHD_HD R fmin1(R a, R b) { return a <= b ? a : b; }

// Limited undivided slope from the two one-sided differences a = q_i - q_{i-1},
// b = q_{i+1} - q_i (Sec. 2.1.4).  limiter 0: minmod, 1: monotonised central.
// Zero when a*b <= 0; otherwise the selected candidate (ties: the first).
template <typename R>
MHD_HD R limited(R a, R b, int limiter) {
    R pick;
    if (limiter == 0) {
        pick = sel(le(rabs(a), rabs(b)), a, b);
    } else {
        const R c = R(0.5) * (a + b);
        const R a2 = a + a, b2 = b + b;
        const R m2v = sel(le(rabs(a2), rabs(b2)), a2, b2);
        pick = sel(le(rabs(c), rabs(m2v)), c, m2v);
    }
    return sel(gt(a * b, R(0)), pick, R(0));
}

// Fast magnetosonic speed along a normal with field component bn (transverse bt1, bt2).
// cf^2 = 1/2 (cs^2 + ca^2 + sqrt(disc)), disc = (cs^2 + ca^2)^2 - 4 cs^2 can^2 evaluated
// as (cs^2 - can^2)^2 + cat^2 (2 (cs^2 + can^2) + cat^2) (identical, no cancellation).
template <typename R>
MHD_HD R fast_speed(R rho_inv, R gP, R bn, R bt1, R bt2) {
    // (products that feed sums are unfusable: every kernel rounds the speed the same way)
    const R cs2 = mul_(gP, rho_inv);
    const R can2 = mul_(mul_(bn, bn), rho_inv);
    const R cat2 = mul_(fma_(bt1, bt1, bt2 * bt2), rho_inv);
    const R d = cs2 - can2;
    const R disc = fma_(d, d, cat2 * fma_(R(2), cs2 + can2, cat2));
    // 1/2 (s + sqrt(disc)) as one fused step after the square root (halving is exact, so
    // this rounds as 1/2 * (s + sqrt(disc)) does)
    return rsqrt_(fma_(R(0.5), rsqrt_(disc), R(0.5) * (cs2 + can2 + cat2)));
}

// Primitive state from the conserved one; the cell-centred field is the mean of the two
// faces of the cell (Sec. 2.1 EOS: P = (gamma-1)(E - rho u^2/2 - B^2/2)).
template <typename R>
MHD_HD void cons_to_prim(R rho, R mx, R my, R mz, R E, R bxc, R byc, R bzc, R gm1, R q[8]) {
    const R ri = rdiv(R(1), rho);
    const R u = mx * ri, v = my * ri, w = mz * ri;
    q[Q_RHO] = rho;
    q[Q_U] = u;
    q[Q_V] = v;
    q[Q_W] = w;
    // P = (gamma-1) (E - rho |u|^2 / 2 - |B|^2 / 2), both subtractions fused
    const R kin = fma_(u, u, fma_(v, v, w * w));
    const R mag = fma_(bxc, bxc, fma_(byc, byc, bzc * bzc));
    q[Q_P] = gm1 * fma_(R(-0.5), mag, fma_(R(-0.5) * rho, kin, E));
    q[Q_BX] = bxc;
    q[Q_BY] = byc;
    q[Q_BZ] = bzc;
}

// Hancock half step in primitive form (Sec. 2.1.4): W^{n+1/2} = W - dt/2 * (A_x W_x +
// A_y W_y + A_z W_z) for (rho, u, v, w, P) with the ideal-MHD primitive Jacobians; the
// field components of the result are set by the caller from the predicted faces.
// D[d][k]: slope of primitive k along d divided by dx_d (zero on collapsed axes).
template <typename R>
MHD_HD void hancock(const R q[8], const R D[3][8], R hdt, R gamma, R out[5]) {
    const R u = q[Q_U], v = q[Q_V], w = q[Q_W], rho = q[Q_RHO], P = q[Q_P];
    const R divu = D[0][Q_U] + D[1][Q_V] + D[2][Q_W];
    const R ri = rdiv(R(1), rho);
    // advective derivative u . grad of primitive k
    auto adv = [&](int k) { return fma_(u, D[0][k], fma_(v, D[1][k], w * D[2][k])); };
    out[0] = rho - hdt * fma_(rho, divu, adv(Q_RHO));
    out[4] = P - hdt * fma_(gamma * P, divu, adv(Q_P));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        // (1/rho)[d_c P + B_a d_c B_a + B_b d_c B_b - B_a d_a B_c - B_b d_b B_c]
        const R lor = fma_(q[Q_BX + a], D[c][Q_BX + a] - D[a][Q_BX + c],
                           fma_(q[Q_BX + b], D[c][Q_BX + b] - D[b][Q_BX + c], D[c][Q_P]));
        out[1 + c] = q[Q_U + c] - hdt * fma_(lor, ri, adv(Q_U + c));
    }
}

// The same half step from the undivided slopes dW[d][k] and the inverse cell sizes dxi[d]
// (D = dW * dxi folded into the products that use it; equal to hancock up to rounding).
// The step kernel's prep uses this form: one multiply less on each slope's path.
template <typename R>
MHD_HD void hancock_dw(const R q[8], const R dW[3][8], const R dxi[3], R hdt, R gamma, R out[5]) {
    const R u = q[Q_U], v = q[Q_V], w = q[Q_W], rho = q[Q_RHO], P = q[Q_P];
    const R us = u * dxi[0], vs = v * dxi[1], ws = w * dxi[2];
    const R divu = fma_(dxi[0], dW[0][Q_U], fma_(dxi[1], dW[1][Q_V], dxi[2] * dW[2][Q_W]));
    const R ri = rdiv(R(1), rho);
    auto adv = [&](int k) { return fma_(us, dW[0][k], fma_(vs, dW[1][k], ws * dW[2][k])); };
    out[0] = rho - hdt * fma_(rho, divu, adv(Q_RHO));
    out[4] = P - hdt * fma_(gamma * P, divu, adv(Q_P));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        const R ja = fma_(dxi[c], dW[c][Q_BX + a], -(dxi[a] * dW[a][Q_BX + c]));
        const R jb = fma_(dxi[c], dW[c][Q_BX + b], -(dxi[b] * dW[b][Q_BX + c]));
        const R lor = fma_(q[Q_BX + a], ja, fma_(q[Q_BX + b], jb, dxi[c] * dW[c][Q_P]));
        out[1 + c] = q[Q_U + c] - hdt * fma_(lor, ri, adv(Q_U + c));
    }
}

// HLLD flux (Sec. 2.1.2; Miyoshi & Kusano 2005) through a face with normal field bn.
// Left/right states: rho, un, ut1, ut2, P, bt1, bt2.  F receives the fluxes of
// (rho, rho*un, rho*ut1, rho*ut2, E) of the region covering x/t = 0.
// Wave speeds S_L = min(un_L, un_R) - max(cf_L, cf_R), S_R = max(..) + max(..);
// the star state is degenerate when |D| <= eps*bn^2 (then transverse v, B keep their
// outer values); ties at x/t = 0 take the left state.  Every lane takes the same path:
// the states of all regions are formed and the one at x/t = 0 is selected.
template <typename R>
MHD_HD void hlld(const R L[7], const R Rt[7], R bn, R gamma, R gm1i, R eps, R F[5]) {
    const R zero = R(0), half = R(0.5);
    const R bn2 = bn * bn;
    // outer states
    const R rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4], byl = L[5], bzl = L[6];
    const R rr = Rt[0], ur = Rt[1], vr = Rt[2], wr = Rt[3], pr = Rt[4], byr = Rt[5], bzr = Rt[6];
    const R b2l = fma_(byl, byl, fma_(bzl, bzl, bn2)), b2r = fma_(byr, byr, fma_(bzr, bzr, bn2));
    const R ptl = fma_(half, b2l, pl), ptr = fma_(half, b2r, pr);
    const R el = fma_(pl, gm1i, half * fma_(rl, fma_(ul, ul, fma_(vl, vl, wl * wl)), b2l));
    const R er = fma_(pr, gm1i, half * fma_(rr, fma_(ur, ur, fma_(vr, vr, wr * wr)), b2r));
    const R cfl = fast_speed(rdiv(R(1), rl), gamma * pl, bn, byl, bzl);
    const R cfr = fast_speed(rdiv(R(1), rr), gamma * pr, bn, byr, bzr);
    const R vbl = fma_(ul, bn, fma_(vl, byl, wl * bzl)), vbr = fma_(ur, bn, fma_(vr, byr, wr * bzr));
    const R cmax = fmax_(cfl, cfr);
    const R sl = fmin_(ul, ur) - cmax;
    const R sr = fmax_(ul, ur) + cmax;
    const R sul = sl - ul, sur = sr - ur;
    const R dl = sul * rl, dr = sur * rr;
    const R deni = rdiv(R(1), dr - dl);
    const R sm = (fma_(dr, ur, -dl * ul) - ptr + ptl) * deni;
    const R pts = fma_(dl * dr, ur - ul, fma_(dr, ptl, -dl * ptr)) * deni;

    // star states
    const R sml = sl - sm, smr = sr - sm;
    const R sli = rdiv(R(1), sml), sri = rdiv(R(1), smr);
    const R rsl = dl * sli, rsr = dr * sri;
    const R Dl = fma_(dl, sml, -bn2), Dr = fma_(dr, smr, -bn2);
    const auto degl = le(rabs(Dl), eps * bn2), degr = le(rabs(Dr), eps * bn2);
    const R Dli = sel(degl, zero, rdiv(R(1), Dl)), Dri = sel(degr, zero, rdiv(R(1), Dr));
    const R nul = bn * (sm - ul) * Dli, nur = bn * (sm - ur) * Dri;
    const R nbl = fma_(dl, sul, -bn2) * Dli, nbr = fma_(dr, sur, -bn2) * Dri;
    const R vsl = sel(degl, vl, fma_(-byl, nul, vl)), wsl = sel(degl, wl, fma_(-bzl, nul, wl));
    const R vsr = sel(degr, vr, fma_(-byr, nur, vr)), wsr = sel(degr, wr, fma_(-bzr, nur, wr));
    const R bysl = sel(degl, byl, byl * nbl), bzsl = sel(degl, bzl, bzl * nbl);
    const R bysr = sel(degr, byr, byr * nbr), bzsr = sel(degr, bzr, bzr * nbr);
    const R vbsl = fma_(sm, bn, fma_(vsl, bysl, wsl * bzsl)), vbsr = fma_(sm, bn, fma_(vsr, bysr, wsr * bzsr));
    const R esl = fma_(sul, el, fma_(-ptl, ul, fma_(pts, sm, bn * (vbl - vbsl)))) * sli;
    const R esr = fma_(sur, er, fma_(-ptr, ur, fma_(pts, sm, bn * (vbr - vbsr)))) * sri;

    // double-star states
    const R sql = rsqrt_(rsl), sqr = rsqrt_(rsr);
    const R abn = rabs(bn);
    const R ssl = sm - rdiv(abn, sql), ssr = sm + rdiv(abn, sqr);
    // sign of bn (+-1; at bn = 0 the double-star region has zero width, ssl = sm = ssr, and
    // is never the one selected, so its value there does not matter)
    const R sgn = copysign(R(1), bn);
    const R isum = rdiv(R(1), sql + sqr);
    const R vss = fma_(sql, vsl, fma_(sqr, vsr, (bysr - bysl) * sgn)) * isum;
    const R wss = fma_(sql, wsl, fma_(sqr, wsr, (bzsr - bzsl) * sgn)) * isum;
    const R sq2 = sql * sqr * sgn;
    const R byss = fma_(sql, bysr, fma_(sqr, bysl, sq2 * (vsr - vsl))) * isum;
    const R bzss = fma_(sql, bzsr, fma_(sqr, bzsl, sq2 * (wsr - wsl))) * isum;
    const R vbss = fma_(sm, bn, fma_(vss, byss, wss * bzss));
    const R essl = fma_(-sql * sgn, vbsl - vbss, esl);
    const R essr = fma_(sqr * sgn, vbsr - vbss, esr);

    // region at x/t = 0 (priority: the leftmost wave with speed >= 0):
    // L (sl >= 0), *L, **L, **R, *R, R
    const auto gl = ge(sl, zero), gsl = ge(ssl, zero), gm = ge(sm, zero), gsr = ge(ssr, zero), gr = ge(sr, zero);
    const auto left = mor(gl, mor(gsl, gm));                       // L, *L or **L
    const auto outer = mor(gl, mnot(mor(gsl, mor(gm, mor(gsr, gr)))));   // L or R
    const auto dstar = mand(mnot(mor(gl, gsl)), mor(gm, gsr));    // **L or **R
    // flux of the outer state on the chosen side
    const R r0 = sel(left, rl, rr), u0 = sel(left, ul, ur), v0 = sel(left, vl, vr), w0 = sel(left, wl, wr);
    const R by0 = sel(left, byl, byr), bz0 = sel(left, bzl, bzr), pt0 = sel(left, ptl, ptr);
    const R e0 = sel(left, el, er), vb0 = sel(left, vbl, vbr);
    const R m0 = r0 * u0;
    R f0 = m0;
    R f1 = fma_(m0, u0, pt0 - bn2);
    R f2v = fma_(m0, v0, -by0 * bn);
    R f3 = fma_(m0, w0, -bz0 * bn);
    R f4 = fma_(e0 + pt0, u0, -bn * vb0);
    // F* = F + S (U* - U)
    const R S = sel(left, sl, sr);
    const R rs = sel(left, rsl, rsr);
    const R vs = sel(left, vsl, vsr), ws = sel(left, wsl, wsr), es = sel(left, esl, esr);
    const R us1 = rs * sm, us2 = rs * vs, us3 = rs * ws;
    const R g0 = fma_(S, rs - r0, f0);
    const R g1 = fma_(S, us1 - m0, f1);
    const R g2 = fma_(S, fma_(-r0, v0, us2), f2v);
    const R g3 = fma_(S, fma_(-r0, w0, us3), f3);
    const R g4 = fma_(S, es - e0, f4);
    // F** = F* + S* (U** - U*); the density and normal momentum are unchanged
    const R Ss = sel(left, ssl, ssr);
    const R ess = sel(left, essl, essr);
    const R h2 = fma_(Ss, fma_(rs, vss, -us2), g2);
    const R h3 = fma_(Ss, fma_(rs, wss, -us3), g3);
    const R h4 = fma_(Ss, ess - es, g4);
    F[0] = sel(outer, f0, g0);
    F[1] = sel(outer, f1, g1);
    F[2] = sel(outer, f2v, sel(dstar, h2, g2));
    F[3] = sel(outer, f3, sel(dstar, h3, g3));
    F[4] = sel(outer, f4, sel(dstar, h4, g4));
}

// HLL flux (Harten, Lax & van Leer 1983; the simple solver of the paper's mockup, Sec. 2.4)
// through a face with normal field bn: one intermediate state between the fastest signals
// S_L, S_R (the same estimates as hlld).  States and result as in hlld; the flux at x/t = 0
// is F_L when S_L >= 0, the HLL flux when S_R >= 0 > S_L, otherwise F_R.
template <typename R>
MHD_HD void hll(const R L[7], const R Rt[7], R bn, R gamma, R gm1i, R F[5]) {
    const R zero = R(0), half = R(0.5);
    const R bn2 = bn * bn;
    const R rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4], byl = L[5], bzl = L[6];
    const R rr = Rt[0], ur = Rt[1], vr = Rt[2], wr = Rt[3], pr = Rt[4], byr = Rt[5], bzr = Rt[6];
    const R b2l = fma_(byl, byl, fma_(bzl, bzl, bn2)), b2r = fma_(byr, byr, fma_(bzr, bzr, bn2));
    const R ptl = fma_(half, b2l, pl), ptr = fma_(half, b2r, pr);
    const R el = fma_(pl, gm1i, half * fma_(rl, fma_(ul, ul, fma_(vl, vl, wl * wl)), b2l));
    const R er = fma_(pr, gm1i, half * fma_(rr, fma_(ur, ur, fma_(vr, vr, wr * wr)), b2r));
    const R cfl = fast_speed(rdiv(R(1), rl), gamma * pl, bn, byl, bzl);
    const R cfr = fast_speed(rdiv(R(1), rr), gamma * pr, bn, byr, bzr);
    const R vbl = fma_(ul, bn, fma_(vl, byl, wl * bzl)), vbr = fma_(ur, bn, fma_(vr, byr, wr * bzr));
    const R cmax = fmax_(cfl, cfr);
    const R sl = fmin_(ul, ur) - cmax;
    const R sr = fmax_(ul, ur) + cmax;
    const R ml = rl * ul, mr = rr * ur;
    const R UL[5] = {rl, ml, rl * vl, rl * wl, el};
    const R UR[5] = {rr, mr, rr * vr, rr * wr, er};
    const R FL[5] = {ml, fma_(ml, ul, ptl - bn2), fma_(ml, vl, -byl * bn), fma_(ml, wl, -bzl * bn),
                     fma_(el + ptl, ul, -bn * vbl)};
    const R FR[5] = {mr, fma_(mr, ur, ptr - bn2), fma_(mr, vr, -byr * bn), fma_(mr, wr, -bzr * bn),
                     fma_(er + ptr, ur, -bn * vbr)};
    const R di = rdiv(R(1), sr - sl);
    const R slr = sl * sr;
    const auto gl = ge(sl, zero), gr = ge(sr, zero);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const R fh = fma_(sr, FL[c], fma_(-sl, FR[c], slr * (UR[c] - UL[c]))) * di;
        F[c] = sel(gl, FL[c], sel(gr, fh, FR[c]));
    }
}

// A predicted state at a cell corner around an edge (Fig. 3): density, gas pressure,
// the velocity components along the edge's two transverse axes a, b, and the field
// components along a, b and the edge direction e.
template <typename R>
struct Corner {
    R rho, p, ua, ub, Ba, Bb, Be;
};

// Two-dimensional HLL upwind EMF at an edge from the four corner states SW, SE, NW, NE
// (E/W along a, N/S along b), with E_e = ua*Bb - ub*Ba per state:
// E = [S_E S_N E_SW - S_E S_S E_NW - S_W S_N E_SE + S_W S_S E_NE] / ((S_E-S_W)(S_N-S_S))
//     + S_E S_W/(S_E-S_W) (Bb_E - Bb_W) - S_N S_S/(S_N-S_S) (Ba_N - Ba_S),
// S_E = max(0, max ua+cf_a), S_W = min(0, min ua-cf_a), S_N, S_S likewise along b.
// It reduces to the 1D HLL induction flux when the states do not vary along a or b.
template <typename R>
MHD_HD R emf2d(const Corner<R>& SW, const Corner<R>& SE, const Corner<R>& NW, const Corner<R>& NE, R gamma) {
    R ap[4], am[4], bp[4], bm[4];
    const Corner<R>* st[4] = {&SW, &SE, &NW, &NE};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const Corner<R>& s = *st[k];
        const R ri = rdiv(R(1), s.rho), gP = gamma * s.p;
        const R cfa = fast_speed(ri, gP, s.Ba, s.Bb, s.Be);
        const R cfb = fast_speed(ri, gP, s.Bb, s.Ba, s.Be);
        ap[k] = s.ua + cfa;
        am[k] = s.ua - cfa;
        bp[k] = s.ub + cfb;
        bm[k] = s.ub - cfb;
    }
    const R zero = R(0);
    const R sE = fmax_(fmax_(fmax_(ap[0], ap[1]), fmax_(ap[2], ap[3])), zero);
    const R sW = fmin_(fmin_(fmin_(am[0], am[1]), fmin_(am[2], am[3])), zero);
    const R sN = fmax_(fmax_(fmax_(bp[0], bp[1]), fmax_(bp[2], bp[3])), zero);
    const R sS = fmin_(fmin_(fmin_(bm[0], bm[1]), fmin_(bm[2], bm[3])), zero);
    const R da = sE - sW, db = sN - sS;
    const R eSW = fma_(SW.ua, SW.Bb, -SW.ub * SW.Ba);
    const R eSE = fma_(SE.ua, SE.Bb, -SE.ub * SE.Ba);
    const R eNW = fma_(NW.ua, NW.Bb, -NW.ub * NW.Ba);
    const R eNE = fma_(NE.ua, NE.Bb, -NE.ub * NE.Ba);
    // [S_E (S_N E_SW - S_S E_NW) - S_W (S_N E_SE - S_S E_NE)] / (da db)
    const R num = fma_(sE, fma_(sN, eSW, -sS * eNW), -sW * fma_(sN, eSE, -sS * eNE));
    const R ida = rdiv(R(1), da), idb = rdiv(R(1), db);
    return fma_(sE * sW * ida, SE.Bb - SW.Bb, fma_(num * ida, idb, -(sN * sS * idb) * (NW.Ba - SW.Ba)));
}

}  // namespace mhd
