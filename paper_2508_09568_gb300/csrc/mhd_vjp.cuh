// Hand-written reverse-mode derivatives (vector-Jacobian products) of the per-element
// arithmetic in mhd_math.cuh, for the discrete adjoint of one bunch step at fixed dt.
//
// Each *_vjp function re-evaluates the forward expression it differentiates (the same
// sequence as the forward code) and then accumulates (+=) the cotangents of its inputs
// from the cotangent of its output, sweeping the forward assignments in reverse order.
// Non-differentiable points take the branch the forward took: the limiter passes the
// cotangent to the argument it selected (ties: the first; none when the arguments differ
// in sign or one is zero), max/min pass it to the selected argument (ties: the first),
// sqrt has derivative 0 at 0, and the HLLD region / degenerate-star choices are constant.
#pragma once

#include "mhd_math.cuh"

namespace mhd {

// d limited(a, b): lo -> la, lb
template <typename R>
MHD_HD void limited_vjp(R a, R b, int limiter, R lo, R& la, R& lb) {
    if (!(a * b > R(0))) return;
    if (limiter == 0) {
        if (rabs(a) <= rabs(b)) la += lo;
        else lb += lo;
    } else {
        const R c = R(0.5) * (a + b);
        const bool pa = rabs(R(2) * a) <= rabs(R(2) * b);
        const R m2 = pa ? R(2) * a : R(2) * b;
        if (rabs(c) <= rabs(m2)) {
            la += R(0.5) * lo;
            lb += R(0.5) * lo;
        } else if (pa) {
            la += R(2) * lo;
        } else {
            lb += R(2) * lo;
        }
    }
}

// slope of q from (qm, q0, qp): lo -> lqm, lq0, lqp
template <typename R>
MHD_HD void slope_vjp(R qm, R q0, R qp, int limiter, R lo, R& lqm, R& lq0, R& lqp) {
    R la = R(0), lb = R(0);
    limited_vjp(q0 - qm, qp - q0, limiter, lo, la, lb);
    lqm -= la;
    lq0 += la - lb;
    lqp += lb;
}

// d fast_speed (in terms of rho and P): lcf -> lrho, lP, lbn, lbt1, lbt2
template <typename R>
MHD_HD void fast_speed_vjp(R rho, R P, R bn, R bt1, R bt2, R gamma, R lcf, R& lrho, R& lP, R& lbn, R& lbt1,
                           R& lbt2) {
    const R ri = R(1) / rho;
    const R cs2 = gamma * P * ri;
    const R can2 = bn * bn * ri;
    const R cat2 = (bt1 * bt1 + bt2 * bt2) * ri;
    const R d = cs2 - can2;
    const R disc = d * d + cat2 * (R(2) * (cs2 + can2) + cat2);
    const R s = rsqrt_(disc);
    const R h = R(0.5) * (cs2 + can2 + cat2 + s);
    const R cf = rsqrt_(h);
    const R lh = cf > R(0) ? lcf / (R(2) * cf) : R(0);
    const R ls = R(0.5) * lh;
    const R ldisc = disc > R(0) ? ls / (R(2) * s) : R(0);
    const R lcs2 = R(0.5) * lh + ldisc * (R(2) * d + R(2) * cat2);
    const R lcan2 = R(0.5) * lh + ldisc * (R(-2) * d + R(2) * cat2);
    const R lcat2 = R(0.5) * lh + ldisc * (R(2) * (cs2 + can2) + R(2) * cat2);
    lP += lcs2 * gamma * ri;
    lbn += lcan2 * R(2) * bn * ri;
    lbt1 += lcat2 * R(2) * bt1 * ri;
    lbt2 += lcat2 * R(2) * bt2 * ri;
    lrho -= (lcs2 * cs2 + lcan2 * can2 + lcat2 * cat2) * ri;
}

// d cons_to_prim: lq[8] -> lU (rho, mx, my, mz, E) and lbc[3] (cell-centred field)
template <typename R>
MHD_HD void cons_to_prim_vjp(R rho, R mx, R my, R mz, R E, R bxc, R byc, R bzc, R gm1, const R lq[8], R lU[5],
                             R lbc[3]) {
    (void)E;
    const R ri = R(1) / rho;
    const R u = mx * ri, v = my * ri, w = mz * ri;
    const R lP = lq[Q_P];
    // P = gm1 (E - rho |u|^2 / 2 - |bc|^2 / 2), u = m / rho
    R lu = lq[Q_U] - lP * gm1 * rho * u;
    R lv = lq[Q_V] - lP * gm1 * rho * v;
    R lw = lq[Q_W] - lP * gm1 * rho * w;
    R lrho = lq[Q_RHO] - lP * gm1 * R(0.5) * (u * u + v * v + w * w);
    lU[4] += lP * gm1;
    lbc[0] += lq[Q_BX] - lP * gm1 * bxc;
    lbc[1] += lq[Q_BY] - lP * gm1 * byc;
    lbc[2] += lq[Q_BZ] - lP * gm1 * bzc;
    lU[1] += lu * ri;
    lU[2] += lv * ri;
    lU[3] += lw * ri;
    lrho -= (lu * u + lv * v + lw * w) * ri;
    lU[0] += lrho;
}

// d hancock: lout[5] -> lq[8] (primitives at time n) and lD[3][8] (slopes / dx)
template <typename R>
MHD_HD void hancock_vjp(const R q[8], const R D[3][8], R hdt, R gamma, const R lout[5], R lq[8], R lD[3][8]) {
    const R u = q[Q_U], v = q[Q_V], w = q[Q_W], rho = q[Q_RHO], P = q[Q_P];
    const R vel[3] = {u, v, w};
    const R divu = D[0][Q_U] + D[1][Q_V] + D[2][Q_W];
    const R ri = R(1) / rho;
    R ladv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ladv[k] = R(0);
    R ldivu = R(0), lri = R(0);
    // out0 = rho - hdt (adv0 + rho divu)
    lq[Q_RHO] += lout[0] * (R(1) - hdt * divu);
    ldivu -= hdt * lout[0] * rho;
    ladv[Q_RHO] -= hdt * lout[0];
    // out4 = P - hdt (adv4 + gamma P divu)
    lq[Q_P] += lout[4] * (R(1) - hdt * gamma * divu);
    ldivu -= hdt * lout[4] * gamma * P;
    ladv[Q_P] -= hdt * lout[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        const R lor = D[c][Q_P] + q[Q_BX + a] * D[c][Q_BX + a] + q[Q_BX + b] * D[c][Q_BX + b]
                      - q[Q_BX + a] * D[a][Q_BX + c] - q[Q_BX + b] * D[b][Q_BX + c];
        const R lo = lout[1 + c];
        lq[Q_U + c] += lo;
        ladv[Q_U + c] -= hdt * lo;
        const R llor = -hdt * lo * ri;
        lri -= hdt * lo * lor;
        lD[c][Q_P] += llor;
        lq[Q_BX + a] += llor * (D[c][Q_BX + a] - D[a][Q_BX + c]);
        lq[Q_BX + b] += llor * (D[c][Q_BX + b] - D[b][Q_BX + c]);
        lD[c][Q_BX + a] += llor * q[Q_BX + a];
        lD[c][Q_BX + b] += llor * q[Q_BX + b];
        lD[a][Q_BX + c] -= llor * q[Q_BX + a];
        lD[b][Q_BX + c] -= llor * q[Q_BX + b];
    }
    // adv(k) = u D0k + v D1k + w D2k
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k == Q_BX || k == Q_BY || k == Q_BZ) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lq[Q_U + d] += ladv[k] * D[d][k];
            lD[d][k] += ladv[k] * vel[d];
        }
    }
    lD[0][Q_U] += ldivu;
    lD[1][Q_V] += ldivu;
    lD[2][Q_W] += ldivu;
    lq[Q_RHO] -= lri * ri * ri;
}

// d hlld: lF[5] -> lL[7], lR[7], lbn.  Same forward sequence as hlld().
template <typename R>
MHD_HD void hlld_vjp(const R L[7], const R Rt[7], R bn, R gamma, R gm1i, R eps, const R lF[5], R lL[7], R lR[7],
                     R& lbn) {
    // ----- forward (as hlld)
    const R bn2 = bn * bn;
    const R rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4], byl = L[5], bzl = L[6];
    const R rr = Rt[0], ur = Rt[1], vr = Rt[2], wr = Rt[3], pr = Rt[4], byr = Rt[5], bzr = Rt[6];
    const R b2l = bn2 + byl * byl + bzl * bzl, b2r = bn2 + byr * byr + bzr * bzr;
    const R ptl = pl + R(0.5) * b2l, ptr = pr + R(0.5) * b2r;
    const R el = pl * gm1i + R(0.5) * rl * (ul * ul + vl * vl + wl * wl) + R(0.5) * b2l;
    const R er = pr * gm1i + R(0.5) * rr * (ur * ur + vr * vr + wr * wr) + R(0.5) * b2r;
    const R cfl = fast_speed(R(1) / rl, gamma * pl, bn, byl, bzl);
    const R cfr = fast_speed(R(1) / rr, gamma * pr, bn, byr, bzr);
    const R vbl = ul * bn + vl * byl + wl * bzl, vbr = ur * bn + vr * byr + wr * bzr;
    const bool cl = cfl >= cfr;            // max picks cf_L
    const R cmax = cl ? cfl : cfr;
    const bool ml = ul <= ur;              // min picks u_L
    const bool Ml = ul >= ur;              // max picks u_L
    const R sl = (ml ? ul : ur) - cmax;
    const R sr = (Ml ? ul : ur) + cmax;
    const R dl = (sl - ul) * rl, dr = (sr - ur) * rr;
    const R den = dr - dl;
    const R deni = R(1) / den;
    const R smn = dr * ur - dl * ul - ptr + ptl;
    const R ptn = dr * ptl - dl * ptr + dl * dr * (ur - ul);
    const R sm = smn * deni;
    const R pts = ptn * deni;
    // star states, per side
    struct Star {
        R S, sa, ssm, ssmi, rs, D, nu, nb, vs, ws, bys, bzs, vbs, nes, es;
        bool deg;
    };
    auto star = [&](R S, R r, R u, R v, R w, R by, R bz, R pt, R e, R vb) {
        Star t;
        t.S = S;
        t.sa = S - u;
        t.ssm = S - sm;
        t.ssmi = R(1) / t.ssm;
        t.rs = r * t.sa * t.ssmi;
        t.D = r * t.sa * t.ssm - bn2;
        t.deg = rabs(t.D) <= eps * bn2;
        const R Di = t.deg ? R(0) : R(1) / t.D;
        t.nu = bn * (sm - u) * Di;
        t.nb = (r * t.sa * t.sa - bn2) * Di;
        t.vs = t.deg ? v : v - by * t.nu;
        t.ws = t.deg ? w : w - bz * t.nu;
        t.bys = t.deg ? by : by * t.nb;
        t.bzs = t.deg ? bz : bz * t.nb;
        t.vbs = sm * bn + t.vs * t.bys + t.ws * t.bzs;
        t.nes = t.sa * e - pt * u + pts * sm + bn * (vb - t.vbs);
        t.es = t.nes * t.ssmi;
        return t;
    };
    const Star A = star(sl, rl, ul, vl, wl, byl, bzl, ptl, el, vbl);
    const Star B = star(sr, rr, ur, vr, wr, byr, bzr, ptr, er, vbr);
    const R sql = rsqrt_(A.rs), sqr = rsqrt_(B.rs);
    const R abn = rabs(bn);
    const R ssl = sm - abn / sql, ssr = sm + abn / sqr;
    const R sgn = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0));
    const R isum = R(1) / (sql + sqr);
    const R nv = sql * A.vs + sqr * B.vs + (B.bys - A.bys) * sgn;
    const R nw = sql * A.ws + sqr * B.ws + (B.bzs - A.bzs) * sgn;
    const R nby = sql * B.bys + sqr * A.bys + sql * sqr * (B.vs - A.vs) * sgn;
    const R nbz = sql * B.bzs + sqr * A.bzs + sql * sqr * (B.ws - A.ws) * sgn;
    const R vss = nv * isum, wss = nw * isum, byss = nby * isum, bzss = nbz * isum;
    const R vbss = sm * bn + vss * byss + wss * bzss;
    const R essl = A.es - sql * (A.vbs - vbss) * sgn;
    const R essr = B.es + sqr * (B.vbs - vbss) * sgn;
    int reg = 5;
    if (sr >= R(0)) reg = 4;
    if (ssr >= R(0)) reg = 3;
    if (sm >= R(0)) reg = 2;
    if (ssl >= R(0)) reg = 1;
    if (sl >= R(0)) reg = 0;
    const bool left = reg <= 2;

    // ----- reverse
    R g_rl = 0, g_ul = 0, g_vl = 0, g_wl = 0, g_pl = 0, g_byl = 0, g_bzl = 0;
    R g_rr = 0, g_ur = 0, g_vr = 0, g_wr = 0, g_pr = 0, g_byr = 0, g_bzr = 0;
    R g_bn = 0, g_bn2 = 0, g_ptl = 0, g_ptr = 0, g_el = 0, g_er = 0, g_vbl = 0, g_vbr = 0;
    R g_sl = 0, g_sr = 0, g_sm = 0, g_pts = 0;
    // per-side star adjoints
    R gA_rs = 0, gA_vs = 0, gA_ws = 0, gA_bys = 0, gA_bzs = 0, gA_vbs = 0, gA_es = 0;
    R gB_rs = 0, gB_vs = 0, gB_ws = 0, gB_bys = 0, gB_bzs = 0, gB_vbs = 0, gB_es = 0;
    R g_sql = 0, g_sqr = 0, g_abn = 0;

    // outer flux of the chosen side
    {
        const R r0 = left ? rl : rr, u0 = left ? ul : ur, v0 = left ? vl : vr, w0 = left ? wl : wr;
        const R by0 = left ? byl : byr, bz0 = left ? bzl : bzr, pt0 = left ? ptl : ptr;
        const R e0 = left ? el : er, vb0 = left ? vbl : vbr;
        R g_r0 = lF[0] * u0 + lF[1] * u0 * u0 + lF[2] * v0 * u0 + lF[3] * w0 * u0;
        R g_u0 = lF[0] * r0 + lF[1] * R(2) * r0 * u0 + lF[2] * r0 * v0 + lF[3] * r0 * w0 + lF[4] * (e0 + pt0);
        R g_v0 = lF[2] * r0 * u0, g_w0 = lF[3] * r0 * u0;
        R g_pt0 = lF[1] + lF[4] * u0;
        g_bn2 -= lF[1];
        R g_by0 = -lF[2] * bn, g_bz0 = -lF[3] * bn;
        g_bn -= lF[2] * by0 + lF[3] * bz0 + lF[4] * vb0;
        R g_e0 = lF[4] * u0;
        R g_vb0 = -lF[4] * bn;
        if (reg != 0 && reg != 5) {
            const Star& T = left ? A : B;
            const R S = T.S;
            const R us0 = T.rs, us1 = T.rs * sm, us2 = T.rs * T.vs, us3 = T.rs * T.ws, us4 = T.es;
            // f += S (U* - U)
            R gS = lF[0] * (us0 - r0) + lF[1] * (us1 - r0 * u0) + lF[2] * (us2 - r0 * v0) +
                   lF[3] * (us3 - r0 * w0) + lF[4] * (us4 - e0);
            g_r0 -= S * (lF[0] + lF[1] * u0 + lF[2] * v0 + lF[3] * w0);
            g_u0 -= S * lF[1] * r0;
            g_v0 -= S * lF[2] * r0;
            g_w0 -= S * lF[3] * r0;
            g_e0 -= S * lF[4];
            R gUs0 = S * lF[0], gUs1 = S * lF[1], gUs2 = S * lF[2], gUs3 = S * lF[3], gUs4 = S * lF[4];
            R g_rs = 0, g_vs = 0, g_ws = 0, g_es = 0;
            if (reg == 2 || reg == 3) {
                // f += S* (U** - U*), U** - U* = (0, 0, rs (vss - vs), rs (wss - ws), ess - es)
                const R Ss = left ? ssl : ssr;
                const R ess = left ? essl : essr;
                const R gSs = lF[2] * T.rs * (vss - T.vs) + lF[3] * T.rs * (wss - T.ws) + lF[4] * (ess - T.es);
                g_rs += Ss * (lF[2] * (vss - T.vs) + lF[3] * (wss - T.ws));
                const R g_vss = Ss * lF[2] * T.rs, g_wss = Ss * lF[3] * T.rs;
                g_vs -= Ss * lF[2] * T.rs;
                g_ws -= Ss * lF[3] * T.rs;
                const R g_ess = Ss * lF[4];
                g_es -= Ss * lF[4];
                R g_vbss = 0;
                if (left) {   // essl = esl - sql (vbsl - vbss) sgn ; ssl = sm - abn / sql
                    gA_es += g_ess;
                    g_sql -= g_ess * (A.vbs - vbss) * sgn;
                    gA_vbs -= g_ess * sql * sgn;
                    g_vbss += g_ess * sql * sgn;
                    g_sm += gSs;
                    g_abn -= gSs / sql;
                    g_sql += gSs * abn / (sql * sql);
                } else {      // essr = esr + sqr (vbsr - vbss) sgn ; ssr = sm + abn / sqr
                    gB_es += g_ess;
                    g_sqr += g_ess * (B.vbs - vbss) * sgn;
                    gB_vbs += g_ess * sqr * sgn;
                    g_vbss -= g_ess * sqr * sgn;
                    g_sm += gSs;
                    g_abn += gSs / sqr;
                    g_sqr -= gSs * abn / (sqr * sqr);
                }
                // vbss = sm bn + vss byss + wss bzss
                g_sm += g_vbss * bn;
                g_bn += g_vbss * sm;
                const R g_vss2 = g_vss + g_vbss * byss, g_wss2 = g_wss + g_vbss * bzss;
                const R g_byss = g_vbss * vss, g_bzss = g_vbss * wss;
                // x = n * isum
                const R g_nv = g_vss2 * isum, g_nw = g_wss2 * isum, g_nby = g_byss * isum, g_nbz = g_bzss * isum;
                const R g_isum = g_vss2 * nv + g_wss2 * nw + g_byss * nby + g_bzss * nbz;
                // nv = sql vsl + sqr vsr + (bysr - bysl) sgn
                g_sql += g_nv * A.vs;
                gA_vs += g_nv * sql;
                g_sqr += g_nv * B.vs;
                gB_vs += g_nv * sqr;
                gB_bys += g_nv * sgn;
                gA_bys -= g_nv * sgn;
                // nw
                g_sql += g_nw * A.ws;
                gA_ws += g_nw * sql;
                g_sqr += g_nw * B.ws;
                gB_ws += g_nw * sqr;
                gB_bzs += g_nw * sgn;
                gA_bzs -= g_nw * sgn;
                // nby = sql bysr + sqr bysl + sql sqr (vsr - vsl) sgn
                g_sql += g_nby * (B.bys + sqr * (B.vs - A.vs) * sgn);
                g_sqr += g_nby * (A.bys + sql * (B.vs - A.vs) * sgn);
                gB_bys += g_nby * sql;
                gA_bys += g_nby * sqr;
                gB_vs += g_nby * sql * sqr * sgn;
                gA_vs -= g_nby * sql * sqr * sgn;
                // nbz
                g_sql += g_nbz * (B.bzs + sqr * (B.ws - A.ws) * sgn);
                g_sqr += g_nbz * (A.bzs + sql * (B.ws - A.ws) * sgn);
                gB_bzs += g_nbz * sql;
                gA_bzs += g_nbz * sqr;
                gB_ws += g_nbz * sql * sqr * sgn;
                gA_ws -= g_nbz * sql * sqr * sgn;
                // isum = 1 / (sql + sqr)
                g_sql -= g_isum * isum * isum;
                g_sqr -= g_isum * isum * isum;
            }
            // U* = (rs, rs sm, rs vs, rs ws, es)
            g_rs += gUs0 + gUs1 * sm + gUs2 * T.vs + gUs3 * T.ws;
            g_sm += gUs1 * T.rs;
            g_vs += gUs2 * T.rs;
            g_ws += gUs3 * T.rs;
            g_es += gUs4;
            if (left) {
                gA_rs += g_rs;
                gA_vs += g_vs;
                gA_ws += g_ws;
                gA_es += g_es;
                g_sl += gS;
            } else {
                gB_rs += g_rs;
                gB_vs += g_vs;
                gB_ws += g_ws;
                gB_es += g_es;
                g_sr += gS;
            }
        }
        if (left) {
            g_rl += g_r0; g_ul += g_u0; g_vl += g_v0; g_wl += g_w0; g_ptl += g_pt0;
            g_byl += g_by0; g_bzl += g_bz0; g_el += g_e0; g_vbl += g_vb0;
        } else {
            g_rr += g_r0; g_ur += g_u0; g_vr += g_v0; g_wr += g_w0; g_ptr += g_pt0;
            g_byr += g_by0; g_bzr += g_bz0; g_er += g_e0; g_vbr += g_vb0;
        }
    }
    // sql = sqrt(rsl), sqr = sqrt(rsr)
    gA_rs += g_sql / (R(2) * sql);
    gB_rs += g_sqr / (R(2) * sqr);
    // star states (reverse), side by side
    auto star_rev = [&](const Star& T, R r, R u, R v, R w, R by, R bz, R pt, R e, R vb, R g_rs, R g_vs, R g_ws,
                        R g_bys, R g_bzs, R g_vbs, R g_es, R& g_r, R& g_u, R& g_v, R& g_w, R& g_by, R& g_bz,
                        R& g_pt, R& g_e, R& g_vb, R& g_S) {
        (void)v;
        (void)w;
        // es = nes * ssmi
        const R g_nes = g_es * T.ssmi;
        R g_ssm = -g_es * T.es * T.ssmi;
        // nes = sa e - pt u + pts sm + bn (vb - vbs)
        R g_sa = g_nes * e;
        g_e += g_nes * T.sa;
        g_pt -= g_nes * u;
        g_u -= g_nes * pt;
        g_pts += g_nes * sm;
        g_sm += g_nes * pts;
        g_bn += g_nes * (vb - T.vbs);
        g_vb += g_nes * bn;
        g_vbs -= g_nes * bn;
        // vbs = sm bn + vs bys + ws bzs
        g_sm += g_vbs * bn;
        g_bn += g_vbs * sm;
        g_vs += g_vbs * T.bys;
        g_bys += g_vbs * T.vs;
        g_ws += g_vbs * T.bzs;
        g_bzs += g_vbs * T.ws;
        if (!T.deg) {
            R g_nu = 0, g_nb = 0;
            g_v += g_vs;
            g_by -= g_vs * T.nu;
            g_nu -= g_vs * by;
            g_w += g_ws;
            g_bz -= g_ws * T.nu;
            g_nu -= g_ws * bz;
            g_by += g_bys * T.nb;
            g_nb += g_bys * by;
            g_bz += g_bzs * T.nb;
            g_nb += g_bzs * bz;
            const R Di = R(1) / T.D;
            // nu = bn (sm - u) / D
            g_bn += g_nu * (sm - u) * Di;
            g_sm += g_nu * bn * Di;
            g_u -= g_nu * bn * Di;
            R g_D = -g_nu * T.nu * Di;
            // nb = (r sa^2 - bn2) / D
            g_r += g_nb * T.sa * T.sa * Di;
            g_sa += g_nb * R(2) * r * T.sa * Di;
            g_bn2 -= g_nb * Di;
            g_D -= g_nb * T.nb * Di;
            // D = r sa ssm - bn2
            g_r += g_D * T.sa * T.ssm;
            g_sa += g_D * r * T.ssm;
            g_ssm += g_D * r * T.sa;
            g_bn2 -= g_D;
        } else {
            g_v += g_vs;
            g_w += g_ws;
            g_by += g_bys;
            g_bz += g_bzs;
        }
        // rs = r sa ssmi
        g_r += g_rs * T.sa * T.ssmi;
        g_sa += g_rs * r * T.ssmi;
        g_ssm -= g_rs * T.rs * T.ssmi;
        // ssm = S - sm ; sa = S - u
        g_S += g_ssm + g_sa;
        g_sm -= g_ssm;
        g_u -= g_sa;
    };
    star_rev(B, rr, ur, vr, wr, byr, bzr, ptr, er, vbr, gB_rs, gB_vs, gB_ws, gB_bys, gB_bzs, gB_vbs, gB_es, g_rr, g_ur,
             g_vr, g_wr, g_byr, g_bzr, g_ptr, g_er, g_vbr, g_sr);
    star_rev(A, rl, ul, vl, wl, byl, bzl, ptl, el, vbl, gA_rs, gA_vs, gA_ws, gA_bys, gA_bzs, gA_vbs, gA_es, g_rl, g_ul,
             g_vl, g_wl, g_byl, g_bzl, g_ptl, g_el, g_vbl, g_sl);
    // sm = smn / den ; pts = ptn / den
    const R g_smn = g_sm * deni, g_ptn = g_pts * deni;
    R g_den = -(g_sm * sm + g_pts * pts) * deni;
    // ptn = dr ptl - dl ptr + dl dr (ur - ul)
    R g_dr = g_ptn * (ptl + dl * (ur - ul));
    R g_dl = g_ptn * (-ptr + dr * (ur - ul));
    g_ptl += g_ptn * dr;
    g_ptr -= g_ptn * dl;
    g_ur += g_ptn * dl * dr;
    g_ul -= g_ptn * dl * dr;
    // smn = dr ur - dl ul - ptr + ptl
    g_dr += g_smn * ur;
    g_ur += g_smn * dr;
    g_dl -= g_smn * ul;
    g_ul -= g_smn * dl;
    g_ptr -= g_smn;
    g_ptl += g_smn;
    // den = dr - dl
    g_dr += g_den;
    g_dl -= g_den;
    // dl = (sl - ul) rl ; dr = (sr - ur) rr
    g_sl += g_dl * rl;
    g_ul -= g_dl * rl;
    g_rl += g_dl * (sl - ul);
    g_sr += g_dr * rr;
    g_ur -= g_dr * rr;
    g_rr += g_dr * (sr - ur);
    // sl = min(ul, ur) - cmax ; sr = max(ul, ur) + cmax
    const R g_cmax = g_sr - g_sl;
    if (ml) g_ul += g_sl;
    else g_ur += g_sl;
    if (Ml) g_ul += g_sr;
    else g_ur += g_sr;
    R g_cfl = cl ? g_cmax : R(0), g_cfr = cl ? R(0) : g_cmax;
    // vb = u bn + v by + w bz
    g_ul += g_vbl * bn; g_bn += g_vbl * ul; g_vl += g_vbl * byl; g_byl += g_vbl * vl; g_wl += g_vbl * bzl;
    g_bzl += g_vbl * wl;
    g_ur += g_vbr * bn; g_bn += g_vbr * ur; g_vr += g_vbr * byr; g_byr += g_vbr * vr; g_wr += g_vbr * bzr;
    g_bzr += g_vbr * wr;
    // fast speeds
    fast_speed_vjp(rl, pl, bn, byl, bzl, gamma, g_cfl, g_rl, g_pl, g_bn, g_byl, g_bzl);
    fast_speed_vjp(rr, pr, bn, byr, bzr, gamma, g_cfr, g_rr, g_pr, g_bn, g_byr, g_bzr);
    // e = p gm1i + rho |u|^2 / 2 + b2 / 2 ; pt = p + b2 / 2
    R g_b2l = R(0.5) * g_el + R(0.5) * g_ptl, g_b2r = R(0.5) * g_er + R(0.5) * g_ptr;
    g_pl += g_el * gm1i + g_ptl;
    g_pr += g_er * gm1i + g_ptr;
    g_rl += g_el * R(0.5) * (ul * ul + vl * vl + wl * wl);
    g_rr += g_er * R(0.5) * (ur * ur + vr * vr + wr * wr);
    g_ul += g_el * rl * ul; g_vl += g_el * rl * vl; g_wl += g_el * rl * wl;
    g_ur += g_er * rr * ur; g_vr += g_er * rr * vr; g_wr += g_er * rr * wr;
    // b2 = bn2 + by^2 + bz^2
    g_bn2 += g_b2l + g_b2r;
    g_byl += R(2) * byl * g_b2l; g_bzl += R(2) * bzl * g_b2l;
    g_byr += R(2) * byr * g_b2r; g_bzr += R(2) * bzr * g_b2r;
    // bn2 = bn^2 ; abn = |bn|
    g_bn += R(2) * bn * g_bn2 + g_abn * sgn;
    lL[0] += g_rl; lL[1] += g_ul; lL[2] += g_vl; lL[3] += g_wl; lL[4] += g_pl; lL[5] += g_byl; lL[6] += g_bzl;
    lR[0] += g_rr; lR[1] += g_ur; lR[2] += g_vr; lR[3] += g_wr; lR[4] += g_pr; lR[5] += g_byr; lR[6] += g_bzr;
    lbn += g_bn;
}

// d hll: lF[5] -> lL[7], lR[7], lbn.  Same forward sequence as hll(); the region (L, HLL
// state, R) and the max / min selections of the wave speeds are constant.
template <typename R>
MHD_HD void hll_vjp(const R L[7], const R Rt[7], R bn, R gamma, R gm1i, const R lF[5], R lL[7], R lR[7], R& lbn) {
    // ----- forward (as hll)
    const R bn2 = bn * bn;
    const R* st[2] = {L, Rt};
    R U[2][5], F[2][5], cf[2], e[2], pt[2], vb[2];
    for (int k = 0; k < 2; ++k) {
        const R r = st[k][0], u = st[k][1], v = st[k][2], w = st[k][3], p = st[k][4], by = st[k][5], bz = st[k][6];
        const R b2 = bn2 + by * by + bz * bz;
        pt[k] = p + R(0.5) * b2;
        e[k] = p * gm1i + R(0.5) * r * (u * u + v * v + w * w) + R(0.5) * b2;
        cf[k] = fast_speed(rdiv(R(1), r), gamma * p, bn, by, bz);
        vb[k] = u * bn + v * by + w * bz;
        U[k][0] = r;
        U[k][1] = r * u;
        U[k][2] = r * v;
        U[k][3] = r * w;
        U[k][4] = e[k];
        F[k][0] = r * u;
        F[k][1] = r * u * u + pt[k] - bn2;
        F[k][2] = r * v * u - by * bn;
        F[k][3] = r * w * u - bz * bn;
        F[k][4] = (e[k] + pt[k]) * u - bn * vb[k];
    }
    const R ul = L[1], ur = Rt[1];
    const bool cl = cf[0] >= cf[1];
    const R cmax = cl ? cf[0] : cf[1];
    const bool ml = ul <= ur, Ml = ul >= ur;
    const R sl = (ml ? ul : ur) - cmax;
    const R sr = (Ml ? ul : ur) + cmax;
    // ----- reverse
    R lU[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}}, lFs[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
    R lsl = R(0), lsr = R(0);
    if (sl >= R(0)) {
        for (int c = 0; c < 5; ++c) lFs[0][c] = lF[c];
    } else if (sr >= R(0)) {
        const R di = R(1) / (sr - sl);
        for (int c = 0; c < 5; ++c) {
            const R dU = U[1][c] - U[0][c];
            const R fh = (sr * F[0][c] - sl * F[1][c] + sl * sr * dU) * di;
            lFs[0][c] = lF[c] * sr * di;
            lFs[1][c] = -lF[c] * sl * di;
            lU[1][c] = lF[c] * sl * sr * di;
            lU[0][c] = -lF[c] * sl * sr * di;
            lsr += lF[c] * (F[0][c] + sl * dU - fh) * di;
            lsl += lF[c] * (-F[1][c] + sr * dU + fh) * di;
        }
    } else {
        for (int c = 0; c < 5; ++c) lFs[1][c] = lF[c];
    }
    // wave speeds: sl = min(ul, ur) - cmax, sr = max(ul, ur) + cmax
    R* lst[2] = {lL, lR};
    lst[ml ? 0 : 1][1] += lsl;
    lst[Ml ? 0 : 1][1] += lsr;
    const R lcmax = lsr - lsl;
    R lcf[2] = {cl ? lcmax : R(0), cl ? R(0) : lcmax};
    for (int k = 0; k < 2; ++k) {
        const R r = st[k][0], u = st[k][1], v = st[k][2], w = st[k][3], p = st[k][4], by = st[k][5], bz = st[k][6];
        R lr = R(0), lu = R(0), lv = R(0), lw = R(0), lp = R(0), lby = R(0), lbz = R(0);
        fast_speed_vjp(r, p, bn, by, bz, gamma, lcf[k], lr, lp, lbn, lby, lbz);
        const R* g = lFs[k];
        const R* h = lU[k];
        // U = (r, r u, r v, r w, e)
        lr += h[0] + h[1] * u + h[2] * v + h[3] * w;
        lu += h[1] * r;
        lv += h[2] * r;
        lw += h[3] * r;
        R le = h[4];
        // F0 = r u
        lr += g[0] * u;
        lu += g[0] * r;
        // F1 = r u^2 + pt - bn^2
        lr += g[1] * u * u;
        lu += g[1] * R(2) * r * u;
        R lpt = g[1];
        lbn -= g[1] * R(2) * bn;
        // F2 = r v u - by bn, F3 = r w u - bz bn
        lr += g[2] * v * u + g[3] * w * u;
        lv += g[2] * r * u;
        lw += g[3] * r * u;
        lu += g[2] * r * v + g[3] * r * w;
        lby -= g[2] * bn;
        lbz -= g[3] * bn;
        lbn -= g[2] * by + g[3] * bz;
        // F4 = (e + pt) u - bn vb, vb = u bn + v by + w bz
        le += g[4] * u;
        lpt += g[4] * u;
        lu += g[4] * (e[k] + pt[k]);
        lbn -= g[4] * vb[k];
        const R lvb = -g[4] * bn;
        lu += lvb * bn;
        lbn += lvb * u;
        lv += lvb * by;
        lby += lvb * v;
        lw += lvb * bz;
        lbz += lvb * w;
        // e = p/(gamma-1) + r (u^2 + v^2 + w^2)/2 + b2/2, pt = p + b2/2, b2 = bn^2 + by^2 + bz^2
        lp += le * gm1i + lpt;
        lr += le * R(0.5) * (u * u + v * v + w * w);
        lu += le * r * u;
        lv += le * r * v;
        lw += le * r * w;
        const R lb2 = R(0.5) * (le + lpt);
        lbn += lb2 * R(2) * bn;
        lby += lb2 * R(2) * by;
        lbz += lb2 * R(2) * bz;
        R* o = lst[k];
        o[0] += lr;
        o[1] += lu;
        o[2] += lv;
        o[3] += lw;
        o[4] += lp;
        o[5] += lby;
        o[6] += lbz;
    }
}

// d emf2d: lE -> cotangents of the four corner states (rho, p, ua, ub, Ba, Bb, Be each)
template <typename R>
MHD_HD void emf2d_vjp(const Corner<R>& SW, const Corner<R>& SE, const Corner<R>& NW, const Corner<R>& NE, R gamma,
                      R lE, Corner<R>& gSW, Corner<R>& gSE, Corner<R>& gNW, Corner<R>& gNE) {
    const Corner<R>* st[4] = {&SW, &SE, &NW, &NE};
    Corner<R>* gs[4] = {&gSW, &gSE, &gNW, &gNE};
    R ap[4], am[4], bp[4], bm[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const Corner<R>& s = *st[k];
        const R ri = R(1) / s.rho, gP = gamma * s.p;
        const R cfa = fast_speed(ri, gP, s.Ba, s.Bb, s.Be);
        const R cfb = fast_speed(ri, gP, s.Bb, s.Ba, s.Be);
        ap[k] = s.ua + cfa;
        am[k] = s.ua - cfa;
        bp[k] = s.ub + cfb;
        bm[k] = s.ub - cfb;
    }
    // folds with the selected index (-1: the clip at zero won)
    auto fold_max = [](const R* x, int& k) {
        R m = x[0];
        k = 0;
        for (int j = 1; j < 4; ++j)
            if (!(m >= x[j])) {
                m = x[j];
                k = j;
            }
        if (!(m >= R(0))) {
            m = R(0);
            k = -1;
        }
        return m;
    };
    auto fold_min = [](const R* x, int& k) {
        R m = x[0];
        k = 0;
        for (int j = 1; j < 4; ++j)
            if (!(m <= x[j])) {
                m = x[j];
                k = j;
            }
        if (!(m <= R(0))) {
            m = R(0);
            k = -1;
        }
        return m;
    };
    int kE, kW, kN, kS;
    const R sE = fold_max(ap, kE), sW = fold_min(am, kW), sN = fold_max(bp, kN), sS = fold_min(bm, kS);
    const R da = sE - sW, db = sN - sS;
    R e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = st[k]->ua * st[k]->Bb - st[k]->ub * st[k]->Ba;
    const R num = sE * sN * e[0] - sE * sS * e[2] - sW * sN * e[1] + sW * sS * e[3];
    const R q = da * db;
    const R t2 = sE * sW / da, t3 = sN * sS / db;
    const R jb = SE.Bb - SW.Bb, ja = NW.Ba - SW.Ba;
    // E = num / q + t2 jb - t3 ja
    const R g_num = lE / q;
    const R g_q = -lE * num / (q * q);
    R g_da = g_q * db, g_db = g_q * da;
    const R g_t2 = lE * jb, g_t3 = -lE * ja;
    const R g_jb = lE * t2, g_ja = -lE * t3;
    R g_sE = g_t2 * sW / da, g_sW = g_t2 * sE / da;
    g_da -= g_t2 * t2 / da;
    R g_sN = g_t3 * sS / db, g_sS = g_t3 * sN / db;
    g_db -= g_t3 * t3 / db;
    gSE.Bb += g_jb;
    gSW.Bb -= g_jb;
    gNW.Ba += g_ja;
    gSW.Ba -= g_ja;
    g_sE += g_num * (sN * e[0] - sS * e[2]);
    g_sN += g_num * (sE * e[0] - sW * e[1]);
    g_sS += g_num * (-sE * e[2] + sW * e[3]);
    g_sW += g_num * (-sN * e[1] + sS * e[3]);
    R g_e[4] = {g_num * sE * sN, -g_num * sW * sN, -g_num * sE * sS, g_num * sW * sS};
    g_sE += g_da;
    g_sW -= g_da;
    g_sN += g_db;
    g_sS -= g_db;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        gs[k]->ua += g_e[k] * st[k]->Bb;
        gs[k]->Bb += g_e[k] * st[k]->ua;
        gs[k]->ub -= g_e[k] * st[k]->Ba;
        gs[k]->Ba -= g_e[k] * st[k]->ub;
    }
    // speeds -> corner velocities and fast speeds
    // (each corner tests whether it was selected, so that every index is a compile-time
    // constant and the corner cotangents stay in registers)
    R g_cfa[4] = {0, 0, 0, 0}, g_cfb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k == kE) {
            gs[k]->ua += g_sE;
            g_cfa[k] += g_sE;
        }
        if (k == kW) {
            gs[k]->ua += g_sW;
            g_cfa[k] -= g_sW;
        }
        if (k == kN) {
            gs[k]->ub += g_sN;
            g_cfb[k] += g_sN;
        }
        if (k == kS) {
            gs[k]->ub += g_sS;
            g_cfb[k] -= g_sS;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const Corner<R>& s = *st[k];
        fast_speed_vjp(s.rho, s.p, s.Ba, s.Bb, s.Be, gamma, g_cfa[k], gs[k]->rho, gs[k]->p, gs[k]->Ba, gs[k]->Bb,
                       gs[k]->Be);
        fast_speed_vjp(s.rho, s.p, s.Bb, s.Ba, s.Be, gamma, g_cfb[k], gs[k]->rho, gs[k]->p, gs[k]->Bb, gs[k]->Ba,
                       gs[k]->Be);
    }
}

}  // namespace mhd
