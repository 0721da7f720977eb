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

#ifndef MHD_HD
#define MHD_HD __host__ __device__ __forceinline__
#endif

namespace mhd {

// Variable order of the state and of the primitive vector.
enum { V_RHO = 0, V_MX = 1, V_MY = 2, V_MZ = 3, V_EN = 4, V_BX = 5, V_BY = 6, V_BZ = 7 };
// Primitive order: rho, u, v, w, P_gas, Bx_c, By_c, Bz_c.
enum { Q_RHO = 0, Q_U = 1, Q_V = 2, Q_W = 3, Q_P = 4, Q_BX = 5, Q_BY = 6, Q_BZ = 7 };

template <typename R>
MHD_HD R rabs(R x) { return x < R(0) ? -x : x; }

MHD_HD float rsqrt_(float x) { return sqrtf(x); }
MHD_HD double rsqrt_(double x) { return sqrt(x); }

// Quotient.  Single precision on the device: the hardware approximate division
// (__fdividef, a reciprocal and a multiply, within 2 ulp for divisors below 2^126 in
// magnitude, which every divisor of the scheme is); double precision and host code: the
// IEEE operation.
MHD_HD float rdiv(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
MHD_HD double rdiv(double a, double b) { return a / b; }

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
        pick = rabs(a) <= rabs(b) ? a : b;
    } else {
        R c = R(0.5) * (a + b);
        R m2 = rabs(R(2) * a) <= rabs(R(2) * b) ? R(2) * a : R(2) * b;
        pick = rabs(c) <= rabs(m2) ? c : m2;
    }
    return (a * b > R(0)) ? pick : R(0);
}

// Fast magnetosonic speed along a normal with field component bn (transverse bt1, bt2).
// cf^2 = 1/2 (cs^2 + ca^2 + sqrt(disc)), disc = (cs^2 + ca^2)^2 - 4 cs^2 can^2 evaluated
// as (cs^2 - can^2)^2 + cat^2 (2 (cs^2 + can^2) + cat^2) (identical, no cancellation).
template <typename R>
MHD_HD R fast_speed(R rho_inv, R gP, R bn, R bt1, R bt2) {
    R cs2 = gP * rho_inv;
    R can2 = bn * bn * rho_inv;
    R cat2 = (bt1 * bt1 + bt2 * bt2) * rho_inv;
    R d = cs2 - can2;
    R disc = d * d + cat2 * (R(2) * (cs2 + can2) + cat2);
    return rsqrt_(R(0.5) * (cs2 + can2 + cat2 + rsqrt_(disc)));
}

// Primitive state from the conserved one; the cell-centred field is the mean of the two
// faces of the cell (Sec. 2.1 EOS: P = (gamma-1)(E - rho u^2/2 - B^2/2)).
template <typename R>
MHD_HD void cons_to_prim(R rho, R mx, R my, R mz, R E, R bxc, R byc, R bzc,
                                             R gm1, R q[8]) {
    R ri = rdiv(R(1), rho);
    R u = mx * ri, v = my * ri, w = mz * ri;
    q[Q_RHO] = rho;
    q[Q_U] = u;
    q[Q_V] = v;
    q[Q_W] = w;
    q[Q_P] = gm1 * (E - R(0.5) * rho * (u * u + v * v + w * w)
                    - R(0.5) * (bxc * bxc + byc * byc + bzc * bzc));
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
#define ADV(k) (u * D[0][k] + v * D[1][k] + w * D[2][k])
    out[0] = rho - hdt * (ADV(Q_RHO) + rho * divu);
    out[4] = P - hdt * (ADV(Q_P) + gamma * P * divu);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        // (1/rho)[d_c P + B_a d_c B_a + B_b d_c B_b - B_a d_a B_c - B_b d_b B_c]
        R lor = D[c][Q_P] + q[Q_BX + a] * D[c][Q_BX + a] + q[Q_BX + b] * D[c][Q_BX + b]
                - q[Q_BX + a] * D[a][Q_BX + c] - q[Q_BX + b] * D[b][Q_BX + c];
        out[1 + c] = q[Q_U + c] - hdt * (ADV(Q_U + c) + lor * ri);
    }
#undef ADV
}

// HLLD flux (Sec. 2.1.2; Miyoshi & Kusano 2005) through a face with normal field bn.
// Left/right states: rho, un, ut1, ut2, P, bt1, bt2.  F receives the fluxes of
// (rho, rho*un, rho*ut1, rho*ut2, E) of the region covering x/t = 0.
// Wave speeds S_L = min(un_L, un_R) - max(cf_L, cf_R), S_R = max(..) + max(..);
// the star state is degenerate when |D| <= eps*bn^2 (then transverse v, B keep their
// outer values); ties at x/t = 0 take the left state.
template <typename R>
MHD_HD void hlld(const R L[7], const R Rt[7], R bn, R gamma, R gm1i, R eps,
                                     R F[5]) {
    const R bn2 = bn * bn;
    // outer states
    const R rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4], byl = L[5], bzl = L[6];
    const R rr = Rt[0], ur = Rt[1], vr = Rt[2], wr = Rt[3], pr = Rt[4], byr = Rt[5], bzr = Rt[6];
    const R b2l = bn2 + byl * byl + bzl * bzl, b2r = bn2 + byr * byr + bzr * bzr;
    const R ptl = pl + R(0.5) * b2l, ptr = pr + R(0.5) * b2r;
    const R el = pl * gm1i + R(0.5) * rl * (ul * ul + vl * vl + wl * wl) + R(0.5) * b2l;
    const R er = pr * gm1i + R(0.5) * rr * (ur * ur + vr * vr + wr * wr) + R(0.5) * b2r;
    const R cfl = fast_speed(rdiv(R(1), rl), gamma * pl, bn, byl, bzl);
    const R cfr = fast_speed(rdiv(R(1), rr), gamma * pr, bn, byr, bzr);
    const R vbl = ul * bn + vl * byl + wl * bzl, vbr = ur * bn + vr * byr + wr * bzr;
    const R cmax = fmax1(cfl, cfr);
    const R sl = fmin1(ul, ur) - cmax;
    const R sr = fmax1(ul, ur) + cmax;
    const R dl = (sl - ul) * rl, dr = (sr - ur) * rr;
    const R deni = rdiv(R(1), dr - dl);
    const R sm = (dr * ur - dl * ul - ptr + ptl) * deni;
    const R pts = (dr * ptl - dl * ptr + dl * dr * (ur - ul)) * deni;

    // star states
    const R sli = rdiv(R(1), sl - sm), sri = rdiv(R(1), sr - sm);
    const R rsl = rl * (sl - ul) * sli, rsr = rr * (sr - ur) * sri;
    const R Dl = rl * (sl - ul) * (sl - sm) - bn2, Dr = rr * (sr - ur) * (sr - sm) - bn2;
    const bool degl = rabs(Dl) <= eps * bn2, degr = rabs(Dr) <= eps * bn2;
    const R Dli = degl ? R(0) : rdiv(R(1), Dl), Dri = degr ? R(0) : rdiv(R(1), Dr);
    const R nul = bn * (sm - ul) * Dli, nur = bn * (sm - ur) * Dri;
    const R nbl = (rl * (sl - ul) * (sl - ul) - bn2) * Dli, nbr = (rr * (sr - ur) * (sr - ur) - bn2) * Dri;
    const R vsl = degl ? vl : vl - byl * nul, wsl = degl ? wl : wl - bzl * nul;
    const R vsr = degr ? vr : vr - byr * nur, wsr = degr ? wr : wr - bzr * nur;
    const R bysl = degl ? byl : byl * nbl, bzsl = degl ? bzl : bzl * nbl;
    const R bysr = degr ? byr : byr * nbr, bzsr = degr ? bzr : bzr * nbr;
    const R vbsl = sm * bn + vsl * bysl + wsl * bzsl, vbsr = sm * bn + vsr * bysr + wsr * bzsr;
    const R esl = ((sl - ul) * el - ptl * ul + pts * sm + bn * (vbl - vbsl)) * sli;
    const R esr = ((sr - ur) * er - ptr * ur + pts * sm + bn * (vbr - vbsr)) * sri;

    // double-star states
    const R sql = rsqrt_(rsl), sqr = rsqrt_(rsr);
    const R abn = rabs(bn);
    const R ssl = sm - rdiv(abn, sql), ssr = sm + rdiv(abn, sqr);
    const R sgn = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0));
    const R isum = rdiv(R(1), sql + sqr);
    const R vss = (sql * vsl + sqr * vsr + (bysr - bysl) * sgn) * isum;
    const R wss = (sql * wsl + sqr * wsr + (bzsr - bzsl) * sgn) * isum;
    const R byss = (sql * bysr + sqr * bysl + sql * sqr * (vsr - vsl) * sgn) * isum;
    const R bzss = (sql * bzsr + sqr * bzsl + sql * sqr * (wsr - wsl) * sgn) * isum;
    const R vbss = sm * bn + vss * byss + wss * bzss;
    const R essl = esl - sql * (vbsl - vbss) * sgn;
    const R essr = esr + sqr * (vbsr - vbss) * sgn;

    // region at x/t = 0 (priority: the leftmost wave with speed >= 0)
    int reg = 5;                  // 0 L, 1 *L, 2 **L, 3 **R, 4 *R, 5 R
    if (sr >= R(0)) reg = 4;
    if (ssr >= R(0)) reg = 3;
    if (sm >= R(0)) reg = 2;
    if (ssl >= R(0)) reg = 1;
    if (sl >= R(0)) reg = 0;
    const bool left = reg <= 2;
    // flux of the outer state on the chosen side
    const R r0 = left ? rl : rr, u0 = left ? ul : ur, v0 = left ? vl : vr, w0 = left ? wl : wr;
    const R by0 = left ? byl : byr, bz0 = left ? bzl : bzr, pt0 = left ? ptl : ptr;
    const R e0 = left ? el : er, vb0 = left ? vbl : vbr;
    R f0 = r0 * u0;
    R f1 = r0 * u0 * u0 + pt0 - bn2;
    R f2 = r0 * v0 * u0 - by0 * bn;
    R f3 = r0 * w0 * u0 - bz0 * bn;
    R f4 = (e0 + pt0) * u0 - bn * vb0;
    if (reg != 0 && reg != 5) {
        const R S = left ? sl : sr;
        const R rs = left ? rsl : rsr;
        const R vs = left ? vsl : vsr, ws = left ? wsl : wsr, es = left ? esl : esr;
        // F* = F + S (U* - U)
        const R us0 = rs, us1 = rs * sm, us2 = rs * vs, us3 = rs * ws, us4 = es;
        f0 = f0 + S * (us0 - r0);
        f1 = f1 + S * (us1 - r0 * u0);
        f2 = f2 + S * (us2 - r0 * v0);
        f3 = f3 + S * (us3 - r0 * w0);
        f4 = f4 + S * (us4 - e0);
        if (reg == 2 || reg == 3) {
            // F** = F* + S* (U** - U*)
            const R Ss = left ? ssl : ssr;
            const R ess = left ? essl : essr;
            f0 = f0 + Ss * (rs - us0);
            f1 = f1 + Ss * (rs * sm - us1);
            f2 = f2 + Ss * (rs * vss - us2);
            f3 = f3 + Ss * (rs * wss - us3);
            f4 = f4 + Ss * (ess - us4);
        }
    }
    F[0] = f0;
    F[1] = f1;
    F[2] = f2;
    F[3] = f3;
    F[4] = f4;
}

// HLL flux (Harten, Lax & van Leer 1983; the simple solver of the paper's mockup, Sec. 2.4)
// through a face with normal field bn: one intermediate state between the fastest signals
// S_L, S_R (the same estimates as hlld).  States and result as in hlld; the flux at x/t = 0
// is F_L when S_L >= 0, the HLL flux when S_R >= 0 > S_L, otherwise F_R.
template <typename R>
MHD_HD void hll(const R L[7], const R Rt[7], R bn, R gamma, R gm1i, R F[5]) {
    const R bn2 = bn * bn;
    const R rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4], byl = L[5], bzl = L[6];
    const R rr = Rt[0], ur = Rt[1], vr = Rt[2], wr = Rt[3], pr = Rt[4], byr = Rt[5], bzr = Rt[6];
    const R b2l = bn2 + byl * byl + bzl * bzl, b2r = bn2 + byr * byr + bzr * bzr;
    const R ptl = pl + R(0.5) * b2l, ptr = pr + R(0.5) * b2r;
    const R el = pl * gm1i + R(0.5) * rl * (ul * ul + vl * vl + wl * wl) + R(0.5) * b2l;
    const R er = pr * gm1i + R(0.5) * rr * (ur * ur + vr * vr + wr * wr) + R(0.5) * b2r;
    const R cfl = fast_speed(rdiv(R(1), rl), gamma * pl, bn, byl, bzl);
    const R cfr = fast_speed(rdiv(R(1), rr), gamma * pr, bn, byr, bzr);
    const R vbl = ul * bn + vl * byl + wl * bzl, vbr = ur * bn + vr * byr + wr * bzr;
    const R cmax = fmax1(cfl, cfr);
    const R sl = fmin1(ul, ur) - cmax;
    const R sr = fmax1(ul, ur) + cmax;
    const R UL[5] = {rl, rl * ul, rl * vl, rl * wl, el};
    const R UR[5] = {rr, rr * ur, rr * vr, rr * wr, er};
    const R FL[5] = {rl * ul, rl * ul * ul + ptl - bn2, rl * vl * ul - byl * bn, rl * wl * ul - bzl * bn,
                     (el + ptl) * ul - bn * vbl};
    const R FR[5] = {rr * ur, rr * ur * ur + ptr - bn2, rr * vr * ur - byr * bn, rr * wr * ur - bzr * bn,
                     (er + ptr) * ur - bn * vbr};
    const R di = rdiv(R(1), sr - sl);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const R fh = (sr * FL[c] - sl * FR[c] + sl * sr * (UR[c] - UL[c])) * di;
        F[c] = sl >= R(0) ? FL[c] : (sr >= R(0) ? fh : FR[c]);
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
MHD_HD R emf2d(const Corner<R>& SW, const Corner<R>& SE, const Corner<R>& NW,
                                   const Corner<R>& NE, R gamma) {
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
    const R sE = fmax1(fmax1(fmax1(fmax1(ap[0], ap[1]), ap[2]), ap[3]), R(0));
    const R sW = fmin1(fmin1(fmin1(fmin1(am[0], am[1]), am[2]), am[3]), R(0));
    const R sN = fmax1(fmax1(fmax1(fmax1(bp[0], bp[1]), bp[2]), bp[3]), R(0));
    const R sS = fmin1(fmin1(fmin1(fmin1(bm[0], bm[1]), bm[2]), bm[3]), R(0));
    const R da = sE - sW, db = sN - sS;
    const R eSW = SW.ua * SW.Bb - SW.ub * SW.Ba;
    const R eSE = SE.ua * SE.Bb - SE.ub * SE.Ba;
    const R eNW = NW.ua * NW.Bb - NW.ub * NW.Ba;
    const R eNE = NE.ua * NE.Bb - NE.ub * NE.Ba;
    const R num = sE * sN * eSW - sE * sS * eNW - sW * sN * eSE + sW * sS * eNE;
    return rdiv(num, da * db) + rdiv(sE * sW, da) * (SE.Bb - SW.Bb) - rdiv(sN * sS, db) * (NW.Ba - SW.Ba);
}

}  // namespace mhd
