// Fused bunch-update kernel: steps a3-a9 of one time step for tiles of patches.
//
// One CTA owns a tile of TX x TY columns of one patch and marches through its z-planes.
// Per plane it stages, in shared memory:
//   W ring   : primitive variables + face fields of the three planes c-1, c, c+1
//              over the tile plus a halo of 2 cells (+1 face on the high side);
//   prep     : predicted state W^{n+1/2}, limited slopes, predicted low-face fields and
//              their transverse slopes of planes c-1 and c, over the tile plus 1 halo;
//   fluxes   : HLLD fluxes of the x-, y-faces and the z-edge EMF of the plane, and the
//              z-faces / x-, y-edge EMFs between planes c-1 and c (double buffered);
// and writes the interior cells and owned faces of plane c-1 of U^{n+1}.  Every face
// flux and edge EMF of the tile is computed once; faces and edges on tile borders are
// recomputed by the neighbouring tile with the same code and inputs, so shared values
// agree bit for bit (exact conservation and div B across tiles and patches).
//
// Scheme: Sec. 2.1 (Eq. 6 flux, EOS), Sec. 2.1.2 (HLLD), Sec. 2.1.3 (Eqs. 7-12, Fig. 3),
// Sec. 2.1.4 (MUSCL-Hancock).  See mhd_math.cuh for the per-element arithmetic.
#pragma once

#include "mhd_common.cuh"
#include "mhd_math.cuh"

namespace mhd {

template <typename R, int NDIM_, int TX_, int TY_, int NT_>
struct StepCfg {
    static constexpr int NDIM = NDIM_, TX = TX_, TY = (NDIM_ >= 2 ? TY_ : 1), NT = NT_;
    static constexpr bool AY = NDIM >= 2, AZ = NDIM >= 3;
    // W ring: tile-local i in [-2, TX+2], j in [-2, TY+2] (y collapsed: j = 0)
    static constexpr int LOX = 2, LOY = AY ? 2 : 0;
    static constexpr int LX = TX + 5, LY = AY ? TY + 5 : 1;
    static constexpr int LSZ = LX * LY;
    static constexpr int NWV = 11;          // 8 primitives + 3 face fields
    static constexpr int NWSLOT = AZ ? 3 : 1;
    // prep: i in [-1, TX], j in [-1, TY]
    static constexpr int POX = 1, POY = AY ? 1 : 0;
    static constexpr int PX = TX + 2, PY = AY ? TY + 2 : 1;
    static constexpr int PSZ = PX * PY;
    static constexpr int NPV = 38;          // Wh(8) + dW(21) + bh(3) + face slopes(6)
    static constexpr int NPSLOT = AZ ? 2 : 1;
    // flux buffers
    static constexpr int FXN = (TX + 1) * TY;
    static constexpr int FYN = AY ? TX * (TY + 1) : 0;
    static constexpr int EZN = (TX + 1) * (AY ? TY + 1 : 1);
    static constexpr int FZN = AZ ? TX * TY : 0;
    static constexpr int EXN = AY ? TX * (TY + 1) : 0;
    static constexpr int EYN = (TX + 1) * TY;
    static constexpr int INB = 5 * FXN + 5 * FYN + EZN;     // in-plane buffer
    static constexpr int ZB = 5 * FZN + EXN + EYN;          // inter-plane buffer
    static constexpr int NINB = AZ ? 2 : 1, NZB = AZ ? 2 : 1;
    static constexpr size_t SMEM_REALS = (size_t)NWSLOT * NWV * LSZ + (size_t)NPSLOT * NPV * PSZ +
                                         (size_t)NINB * INB + (size_t)NZB * ZB;
    static constexpr size_t SMEM_BYTES = SMEM_REALS * sizeof(R) + 16;
    // Work segments of the flux stage.  Each walks rows of the prep pitch PX (idle lanes
    // at the row ends) so that a warp's shared-memory reads of the prep arrays are
    // contiguous (no bank conflicts); each is padded to a warp multiple.
    static constexpr int pad32(int n) { return (n + 31) / 32 * 32; }
    static constexpr int RFX = TY, RFY = AY ? TY + 1 : 0, REZ = AY ? TY + 1 : 1;
    static constexpr int RFZ = AZ ? TY : 0, REX = AY ? TY + 1 : 0, REY = TY;
    static constexpr int S_FX = pad32(RFX * PX), S_FY = pad32(RFY * PX), S_EZ = pad32(REZ * PX);
    static constexpr int S_FZ = pad32(RFZ * PX), S_EX = pad32(REX * PX), S_EY = pad32(REY * PX);
    // update stage rows of pitch TX+1
    static constexpr int S_UP = TY * (TX + 1);
};

// prep slot variable indices
#define PV_WH(k) (k)
// slope of primitive k along d (the slope of the normal field component along its own
// axis is never used and not stored)
#define PV_DW(d, k) (8 + 7 * (d) + ((k) < 5 + (d) ? (k) : (k) - 1))
#define PV_BH(c) (29 + (c))
#define PV_FS(c, k) (32 + 2 * (c) + (k))   // slope of face field c along (c+k+1)%3

template <typename R, typename C>
struct StepSmem {
    R* w;     // [NWSLOT][NWV][LSZ]
    R* prep;  // [NPSLOT][NPV][PSZ]
    R* inb;   // [NINB][INB]
    R* zb;    // [NZB][ZB]
    __device__ __forceinline__ R* W(int slot) const { return w + (size_t)slot * C::NWV * C::LSZ; }
    __device__ __forceinline__ R* P(int slot) const { return prep + (size_t)slot * C::NPV * C::PSZ; }
    __device__ __forceinline__ R* I(int slot) const { return inb + (size_t)slot * C::INB; }
    __device__ __forceinline__ R* Z(int slot) const { return zb + (size_t)slot * C::ZB; }
};

template <typename C>
__device__ __forceinline__ int lidx(int i, int j) {   // W ring cell index
    return (j + C::LOY) * C::LX + (i + C::LOX);
}
template <typename C>
__device__ __forceinline__ int pidx(int i, int j) {   // prep cell index
    return (j + C::POY) * C::PX + (i + C::POX);
}

// ---------------------------------------------------------------------------------------
// stage 1: load one plane of U^n into the W ring (raw), and the next plane's Bz.
// ASYNC: element copies global -> shared with cp.async (the issuing threads do not wait;
// cp_async_wait_all before the barrier that publishes the plane), so that the copies of
// plane m+1 can be issued before the flux stage of plane m-1 and complete under it.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* smem_dst, const R* gsrc) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename R, typename C, bool ASYNC = false>
__device__ __forceinline__ void stage_load(const R* __restrict__ U, const PatchDev& pt, int x0, int y0,
                                           int m, R* Wslot, R* bznext) {
    const int gx = pt.gx, gy = pt.gy, gz = pt.gz;
    const int X = pt.X, Y = pt.Y, Z = pt.Z;
    const int64_t vol = (int64_t)X * Y * Z;
    const R* base = U + pt.off;
    for (int w = threadIdx.x; w < C::LSZ; w += C::NT) {
        const int li = w % C::LX, lj = w / C::LX;
        const int i = li - C::LOX, j = lj - C::LOY;
        const int x = x0 + i + gx, y = (C::AY ? y0 + j + gy : 0), z = m + gz;
        const bool in = x >= 0 && x < X && y >= 0 && y < Y && z >= 0 && z < Z;
        if (in) {
            const int64_t o = ((int64_t)z * Y + y) * X + x;
            const bool hasnext = C::AZ ? (z + 1 < Z) : true;
            const R* nxt = base + 7 * vol + o + (C::AZ ? (int64_t)X * Y : 0);
            if constexpr (ASYNC) {
                constexpr int dst[8] = {0, 1, 2, 3, 4, 8, 9, 10};
#pragma unroll
                for (int v = 0; v < 8; ++v) cp_async_elem(&Wslot[dst[v] * C::LSZ + w], base + v * vol + o);
                if (hasnext) cp_async_elem(&bznext[w], nxt);
                else bznext[w] = R(0);
            } else {
                Wslot[0 * C::LSZ + w] = base[0 * vol + o];
                Wslot[1 * C::LSZ + w] = base[1 * vol + o];
                Wslot[2 * C::LSZ + w] = base[2 * vol + o];
                Wslot[3 * C::LSZ + w] = base[3 * vol + o];
                Wslot[4 * C::LSZ + w] = base[4 * vol + o];
                Wslot[8 * C::LSZ + w] = base[5 * vol + o];
                Wslot[9 * C::LSZ + w] = base[6 * vol + o];
                Wslot[10 * C::LSZ + w] = base[7 * vol + o];
                bznext[w] = hasnext ? *nxt : R(0);
            }
        } else {
            // outside the padded patch: a benign state, never used by owned outputs
            Wslot[0 * C::LSZ + w] = R(1);
            Wslot[1 * C::LSZ + w] = R(0);
            Wslot[2 * C::LSZ + w] = R(0);
            Wslot[3 * C::LSZ + w] = R(0);
            Wslot[4 * C::LSZ + w] = R(1);
            Wslot[8 * C::LSZ + w] = R(0);
            Wslot[9 * C::LSZ + w] = R(0);
            Wslot[10 * C::LSZ + w] = R(0);
            bznext[w] = R(0);
        }
    }
}

// stage 2: conserved -> primitive in place (a3)
template <typename R, typename C>
__device__ __forceinline__ void stage_convert(R* Wslot, const R* bznext, R gm1) {
    for (int w = threadIdx.x; w < C::LSZ; w += C::NT) {
        const int li = w % C::LX, lj = w / C::LX;
        const R bx0 = Wslot[8 * C::LSZ + w];
        const R bx1 = (li + 1 < C::LX) ? Wslot[8 * C::LSZ + w + 1] : R(0);
        const R by0 = Wslot[9 * C::LSZ + w];
        R by1;
        if (C::AY) by1 = (lj + 1 < C::LY) ? Wslot[9 * C::LSZ + w + C::LX] : R(0);
        else by1 = by0;
        const R bz0 = Wslot[10 * C::LSZ + w];
        const R bz1 = bznext[w];
        R q[8];
        cons_to_prim(Wslot[0 * C::LSZ + w], Wslot[1 * C::LSZ + w], Wslot[2 * C::LSZ + w],
                     Wslot[3 * C::LSZ + w], Wslot[4 * C::LSZ + w], R(0.5) * (bx0 + bx1),
                     R(0.5) * (by0 + by1), R(0.5) * (bz0 + bz1), gm1, q);
#pragma unroll
        for (int k = 1; k < 8; ++k) Wslot[k * C::LSZ + w] = q[k];
    }
}

// ---------------------------------------------------------------------------------------
// stage 3: prep (a4 slopes, time-n edge EMF, predicted faces, a5 Hancock predictor)
// ---------------------------------------------------------------------------------------
template <typename R, typename C>
struct PrepCtx {
    const R* Wm;   // plane c-1
    const R* W0;   // plane c
    const R* Wp;   // plane c+1
    R hdt, gamma, dxi[3];
    int limiter;
};

// value of W-ring variable k at (i+di, j+dj) on plane c+dk (dk in -1..1)
template <typename R, typename C>
__device__ __forceinline__ R wv(const PrepCtx<R, C>& X, int k, int i, int j, int dk) {
    const R* s = (!C::AZ || dk == 0) ? X.W0 : (dk < 0 ? X.Wm : X.Wp);
    return s[k * C::LSZ + lidx<C>(i, C::AY ? j : 0)];
}

// time-n edge EMF (Eqs. 7-11): E_e = <v_a><B_b> - <v_b><B_a> on the edge low in (a, b) of
// cell (i, j, dk).  <v> averages the four cells around the edge, <B_a> the two a-faces,
// <B_b> the two b-faces.  Collapsed axes map the -1 neighbour onto the cell itself.
template <typename R, typename C>
__device__ __forceinline__ R emf_n(const PrepCtx<R, C>& X, int e, int i, int j, int dk) {
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    // offsets of the "-1" neighbour along a and b in (i, j, k)
    auto off = [&](int d, int& oi, int& oj, int& ok) {
        oi = (d == 0) ? -1 : 0;
        oj = (d == 1 && C::AY) ? -1 : 0;
        ok = (d == 2 && C::AZ) ? -1 : 0;
    };
    int ai, aj, ak, bi, bj, bk;
    off(a, ai, aj, ak);
    off(b, bi, bj, bk);
    const int qa = Q_U + a, qb = Q_U + b;
    // (pairwise sums: two dependent additions instead of three)
    const R va = R(0.25) * ((wv(X, qa, i, j, dk) + wv(X, qa, i + ai, j + aj, dk + ak)) +
                            (wv(X, qa, i + bi, j + bj, dk + bk) +
                             wv(X, qa, i + ai + bi, j + aj + bj, dk + ak + bk)));
    const R vb = R(0.25) * ((wv(X, qb, i, j, dk) + wv(X, qb, i + ai, j + aj, dk + ak)) +
                            (wv(X, qb, i + bi, j + bj, dk + bk) +
                             wv(X, qb, i + ai + bi, j + aj + bj, dk + ak + bk)));
    const R Ba = R(0.5) * (wv(X, 8 + a, i, j, dk) + wv(X, 8 + a, i + bi, j + bj, dk + bk));
    const R Bb = R(0.5) * (wv(X, 8 + b, i, j, dk) + wv(X, 8 + b, i + ai, j + aj, dk + ak));
    return va * Bb - vb * Ba;
}

template <typename R, typename C>
__device__ __forceinline__ void prep_cell(const PrepCtx<R, C>& X, int i, int j, R* Pslot, int pid) {
    const int li = lidx<C>(i, C::AY ? j : 0);
    R q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = X.W0[k * C::LSZ + li];
    // a4: limited slopes of the primitives along each active axis
    R dW[3][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        dW[0][k] = limited(q[k] - wv(X, k, i - 1, j, 0), wv(X, k, i + 1, j, 0) - q[k], X.limiter);
        dW[1][k] = C::AY ? limited(q[k] - wv(X, k, i, j - 1, 0), wv(X, k, i, j + 1, 0) - q[k], X.limiter) : R(0);
        dW[2][k] = C::AZ ? limited(q[k] - wv(X, k, i, j, -1), wv(X, k, i, j, 1) - q[k], X.limiter) : R(0);
    }
    // transverse slopes of the low face fields of this cell
    const R bx = wv(X, 8, i, j, 0), by = wv(X, 9, i, j, 0), bz = wv(X, 10, i, j, 0);
    const R fs_bx_y = C::AY ? limited(bx - wv(X, 8, i, j - 1, 0), wv(X, 8, i, j + 1, 0) - bx, X.limiter) : R(0);
    const R fs_bx_z = C::AZ ? limited(bx - wv(X, 8, i, j, -1), wv(X, 8, i, j, 1) - bx, X.limiter) : R(0);
    const R fs_by_z = C::AZ ? limited(by - wv(X, 9, i, j, -1), wv(X, 9, i, j, 1) - by, X.limiter) : R(0);
    const R fs_by_x = limited(by - wv(X, 9, i - 1, j, 0), wv(X, 9, i + 1, j, 0) - by, X.limiter);
    const R fs_bz_x = limited(bz - wv(X, 10, i - 1, j, 0), wv(X, 10, i + 1, j, 0) - bz, X.limiter);
    const R fs_bz_y = C::AY ? limited(bz - wv(X, 10, i, j - 1, 0), wv(X, 10, i, j + 1, 0) - bz, X.limiter) : R(0);

    // time-n edge EMFs around the cell (Eqs. 7-11); edge index = low corner cell
    const int jy = C::AY ? 1 : 0;
    const int kz = C::AZ ? 1 : 0;
    // Ez at (i-1/2 + di, j-1/2 + dj) for di, dj in {0, 1}
    const R ez00 = emf_n(X, 2, i, j, 0), ez10 = emf_n(X, 2, i + 1, j, 0);
    const R ez01 = emf_n(X, 2, i, j + jy, 0), ez11 = emf_n(X, 2, i + 1, j + jy, 0);
    // Ex at (i, j-1/2 + dj, k-1/2 + dk)
    const R ex00 = emf_n(X, 0, i, j, 0), ex10 = emf_n(X, 0, i, j + jy, 0);
    const R ex01 = emf_n(X, 0, i, j, kz), ex11 = emf_n(X, 0, i, j + jy, kz);
    // Ey at (i-1/2 + di, j, k-1/2 + dk)
    const R ey00 = emf_n(X, 1, i, j, 0), ey10 = emf_n(X, 1, i + 1, j, 0);
    const R ey01 = emf_n(X, 1, i, j, kz), ey11 = emf_n(X, 1, i + 1, j, kz);

    // face fields predicted to t + dt/2 by Eq. 12 over dt/2 (with EMF = u x B):
    // dBx/dt = d_y Ez - d_z Ey, dBy/dt = d_z Ex - d_x Ez, dBz/dt = d_x Ey - d_y Ex
    const R h = X.hdt;
    R tx0 = R(0), tx1 = R(0), ty0 = R(0), ty1 = R(0), tz0 = R(0), tz1 = R(0);
    if (C::AY) {
        tx0 += h * X.dxi[1] * (ez01 - ez00);
        tx1 += h * X.dxi[1] * (ez11 - ez10);
        tz0 -= h * X.dxi[1] * (ex10 - ex00);
        tz1 -= h * X.dxi[1] * (ex11 - ex01);
    }
    if (C::AZ) {
        tx0 -= h * X.dxi[2] * (ey01 - ey00);
        tx1 -= h * X.dxi[2] * (ey11 - ey10);
        ty0 += h * X.dxi[2] * (ex01 - ex00);
        ty1 += h * X.dxi[2] * (ex11 - ex10);
    }
    ty0 -= h * X.dxi[0] * (ez10 - ez00);
    ty1 -= h * X.dxi[0] * (ez11 - ez01);
    tz0 += h * X.dxi[0] * (ey10 - ey00);
    tz1 += h * X.dxi[0] * (ey11 - ey01);
    const R bxh0 = bx + tx0, bxh1 = wv(X, 8, i + 1, j, 0) + tx1;
    const R byh0 = by + ty0, byh1 = (C::AY ? wv(X, 9, i, j + 1, 0) : by) + ty1;
    const R bzh0 = bz + tz0, bzh1 = (C::AZ ? wv(X, 10, i, j, 1) : bz) + tz1;

    // a5: Hancock predictor
    R hq[5];
    hancock_dw(q, dW, X.dxi, X.hdt, X.gamma, hq);

#pragma unroll
    for (int k = 0; k < 5; ++k) Pslot[PV_WH(k) * C::PSZ + pid] = hq[k];
    Pslot[PV_WH(5) * C::PSZ + pid] = R(0.5) * (bxh0 + bxh1);
    Pslot[PV_WH(6) * C::PSZ + pid] = R(0.5) * (byh0 + byh1);
    Pslot[PV_WH(7) * C::PSZ + pid] = R(0.5) * (bzh0 + bzh1);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k != 5 + d) Pslot[PV_DW(d, k) * C::PSZ + pid] = dW[d][k];
    Pslot[PV_BH(0) * C::PSZ + pid] = bxh0;
    Pslot[PV_BH(1) * C::PSZ + pid] = byh0;
    Pslot[PV_BH(2) * C::PSZ + pid] = bzh0;
    Pslot[PV_FS(0, 0) * C::PSZ + pid] = fs_bx_y;
    Pslot[PV_FS(0, 1) * C::PSZ + pid] = fs_bx_z;
    Pslot[PV_FS(1, 0) * C::PSZ + pid] = fs_by_z;
    Pslot[PV_FS(1, 1) * C::PSZ + pid] = fs_by_x;
    Pslot[PV_FS(2, 0) * C::PSZ + pid] = fs_bz_x;
    Pslot[PV_FS(2, 1) * C::PSZ + pid] = fs_bz_y;
}

// ---------------------------------------------------------------------------------------
// stage 4: fluxes (a6 face states + a7 HLLD) and edge EMFs (a8)
// ---------------------------------------------------------------------------------------
template <typename R, typename C>
__device__ __forceinline__ R pv(const R* P, int v, int pid) { return P[v * C::PSZ + pid]; }

// flux through the low d-face of cell (pidR) with left cell (pidL) (possibly in another
// slot for d = z).  F receives (rho, mx, my, mz, E) fluxes.
template <typename R, typename C>
__device__ __forceinline__ void face_flux(const R* PL, int pidL, const R* PR, int pidR, int d, R gamma,
                                          R gm1i, R eps, int riemann, R F[5]) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    R L[7], Rr[7];
    const int ks[7] = {Q_RHO, Q_U + d, Q_U + t1, Q_U + t2, Q_P, Q_BX + t1, Q_BX + t2};
#pragma unroll
    for (int n = 0; n < 7; ++n) {
        const int k = ks[n];
        L[n] = pv<R, C>(PL, PV_WH(k), pidL) + R(0.5) * pv<R, C>(PL, PV_DW(d, k), pidL);
        Rr[n] = pv<R, C>(PR, PV_WH(k), pidR) - R(0.5) * pv<R, C>(PR, PV_DW(d, k), pidR);
    }
    const R bn = pv<R, C>(PR, PV_BH(d), pidR);
    R f[5];
    if (riemann == 1) hll(L, Rr, bn, gamma, gm1i, f);
    else hlld(L, Rr, bn, gamma, gm1i, eps, f);
    F[0] = f[0];
    F[4] = f[4];
    F[1 + d] = f[1];
    F[1 + t1] = f[2];
    F[1 + t2] = f[3];
}

// corner state (sa, sb) of a cell for edge direction e with (a, b) = ((e+1)%3, (e+2)%3).
// Ba: the a-face on side sa (value and its slope along b), Bb: the b-face on side sb.
template <typename R, typename C>
__device__ __forceinline__ Corner<R> corner(const R* P, int pid, int e, R sa, R sb, R ba_face,
                                            R ba_slope, R bb_face, R bb_slope) {
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    auto ext = [&](int k) {
        return pv<R, C>(P, PV_WH(k), pid) +
               R(0.5) * (sa * pv<R, C>(P, PV_DW(a, k), pid) + sb * pv<R, C>(P, PV_DW(b, k), pid));
    };
    Corner<R> s;
    s.rho = ext(Q_RHO);
    s.p = ext(Q_P);
    s.ua = ext(Q_U + a);
    s.ub = ext(Q_U + b);
    s.Be = ext(Q_BX + e);
    s.Ba = ba_face + R(0.5) * sb * ba_slope;
    s.Bb = bb_face + R(0.5) * sa * bb_slope;
    return s;
}

// ---------------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------------
template <typename R>
struct StepArgs {
    const R* __restrict__ U;
    R* __restrict__ Unew;
    // asynchronous stepping (both null otherwise): patch p reads its current time slice
    // from buffer slice[p] (U when 0, Unew when 1) and writes the new one into the other
    // buffer, advancing by its own dt_patch[p]
    const int* __restrict__ slice;
    const double* __restrict__ dt_patch;
    const PatchDev* __restrict__ patches;
    const int4* __restrict__ tiles;
    int ntiles;
    const int* ntiles_dev;  // ASYNC: tile count written by the device scheduler (null: ntiles)
    int dynamic;          // 1: pull tiles from *work (persistent), 0: one tile per CTA
    int* work;            // [0] next tile, [1] finished CTAs
    const double* dt_ptr; // device dt (if not null)
    double dt_val;
    double gamma, eps;
    double dxi[3];
    int limiter;
    int riemann;          // face flux: 0 HLLD, 1 HLL
    unsigned* err;
};

// a9 for one plane u of the tile: conservative update and constrained transport (Eq. 12)
// from the in-plane buffer of plane u and the inter-plane buffers of levels u-1/2, u+1/2.
// Threads walk rows of pitch TX+1 (one idle lane per row) so flux reads are contiguous.
template <typename R, typename C>
__device__ __forceinline__ void stage_update(const StepSmem<R, C>& S, const R* __restrict__ U, R* __restrict__ Unew,
                                             const PatchDev& pt, int x0, int y0, int u, int wx, int wy, R dtdx0,
                                             R dtdx1, R dtdx2, unsigned* err) {
    const R* IB = S.I(C::AZ ? (u & 1) : 0);
    const R* Fx = IB;
    const R* Fy = IB + 5 * C::FXN;
    const R* Ez = Fy + 5 * C::FYN;
    const R* ZL = S.Z(C::AZ ? (u & 1) : 0);        // level u-1/2
    const R* ZH = S.Z(C::AZ ? ((u + 1) & 1) : 0);  // level u+1/2
    const R* FzL = ZL;
    const R* FzH = ZH;
    const R* ExL = ZL + 5 * C::FZN;
    const R* ExH = ZH + 5 * C::FZN;
    const R* EyL = ExL + C::EXN;
    const R* EyH = ExH + C::EXN;
    const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
    for (int w = threadIdx.x; w < C::S_UP; w += C::NT) {
        const int i = w % (C::TX + 1), j = w / (C::TX + 1);
        if (i >= wx || j >= wy) continue;
        const int x = x0 + i + pt.gx, y = C::AY ? y0 + j + pt.gy : 0, z = u + pt.gz;
        const int64_t o = pt.off + ((int64_t)z * pt.Y + y) * pt.X + x;
        const int fx = j * (C::TX + 1) + i;   // x-faces, Ez, Ey: pitch TX+1
        const int fy = j * C::TX + i;         // y-faces, z-faces, Ex: pitch TX
        R du[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            R d = dtdx0 * (Fx[v * C::FXN + fx + 1] - Fx[v * C::FXN + fx]);
            if (C::AY) d += dtdx1 * (Fy[v * C::FYN + fy + C::TX] - Fy[v * C::FYN + fy]);
            if (C::AZ) d += dtdx2 * (FzH[v * C::FZN + fy] - FzL[v * C::FZN + fy]);
            du[v] = -d;
        }
        R dbx = R(0), dby, dbz;
        if (C::AY) dbx += dtdx1 * (Ez[fx + (C::TX + 1)] - Ez[fx]);
        if (C::AZ) dbx -= dtdx2 * (EyH[fx] - EyL[fx]);
        dby = -dtdx0 * (Ez[fx + 1] - Ez[fx]);
        if (C::AZ) dby += dtdx2 * (ExH[fy] - ExL[fy]);
        dbz = dtdx0 * (EyL[fx + 1] - EyL[fx]);
        if (C::AY) dbz -= dtdx1 * (ExL[fy + C::TX] - ExL[fy]);
        const R* Ub = U + o;
        R* Un = Unew + o;
        R nv[8];
#pragma unroll
        for (int v = 0; v < 5; ++v) nv[v] = Ub[v * vol] + du[v];
        nv[5] = Ub[5 * vol] + dbx;
        nv[6] = Ub[6 * vol] + dby;
        nv[7] = Ub[7 * vol] + dbz;
#pragma unroll
        for (int v = 0; v < 8; ++v) Un[v * vol] = nv[v];
        if (!(nv[0] > R(0)) || !finite_(nv[4])) atomicOr(err, ERR_PHYS);
    }
}

// PREFETCH (3D): the raw plane m+1 is copied with cp.async into the W-ring slot of plane
// c-1 (free once plane c is prepared) while the flux stage of plane c runs, instead of
// being loaded at the start of the next iteration; its conversion then shares the phase of
// the update, so a plane takes three barriers (update + convert / prep / flux).
// ASYNC: asynchronous stepping (a.slice, a.dt_patch): per-tile slice choice and dt; a
// separate instantiation so that the synchronous step keeps its kernel-wide constants.
template <typename R, int NDIM, int TX, int TY, int NT, int MINB, bool PREFETCH, bool ASYNC>
__global__ void __launch_bounds__(NT, MINB) step_kernel(StepArgs<R> a) {
    using C = StepCfg<R, NDIM, TX, TY, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    StepSmem<R, C> S;
    S.w = sm;
    S.prep = S.w + (size_t)C::NWSLOT * C::NWV * C::LSZ;
    S.inb = S.prep + (size_t)C::NPSLOT * C::NPV * C::PSZ;
    S.zb = S.inb + (size_t)C::NINB * C::INB;
    __shared__ R bznext[C::LSZ];
    __shared__ int s_tile;

    const double dt0 = a.dt_ptr ? *a.dt_ptr : a.dt_val;
    const R gamma = R(a.gamma), gm1 = R(a.gamma - 1.0), gm1i = R(1.0 / (a.gamma - 1.0));
    const R eps = R(a.eps);
    R hdt = R(0.5 * dt0);
    R dtdx0 = R(dt0 * a.dxi[0]), dtdx1 = R(dt0 * a.dxi[1]), dtdx2 = R(dt0 * a.dxi[2]);

    int t;
    if (a.dynamic) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&a.work[0], 1);
        __syncthreads();
        t = s_tile;
    } else {
        t = blockIdx.x;
    }
    int ntiles = a.ntiles;
    if constexpr (ASYNC) {
        if (a.ntiles_dev) ntiles = min(*a.ntiles_dev, a.ntiles);
    }
    while (t < ntiles) {
        const int4 tl = a.tiles[t];
        const PatchDev pt = a.patches[tl.x];
        const R* __restrict__ Uc = a.U;
        R* __restrict__ Un = a.Unew;
        if constexpr (ASYNC) {
            const double dtd = a.dt_patch[tl.x];
            hdt = R(0.5 * dtd);
            dtdx0 = R(dtd * a.dxi[0]);
            dtdx1 = R(dtd * a.dxi[1]);
            dtdx2 = R(dtd * a.dxi[2]);
            if (a.slice[tl.x]) {
                Uc = a.Unew;
                Un = const_cast<R*>(a.U);
            }
        }
        const int x0 = tl.y, y0 = tl.z;
        const int wx = min(C::TX, pt.nx - x0), wy = C::AY ? min(C::TY, pt.ny - y0) : 1;
        const int nz = C::AZ ? pt.nz : 1;
        // 3D: iteration s loads plane s-2, prepares plane s-3 (fluxes of that plane and
        // of the level below it) and updates plane s-5 (whose last inter-plane level was
        // computed in iteration s-1); one extra iteration finishes the last update.
        const int niter = C::AZ ? nz + 5 : 1;

        PrepCtx<R, C> X;
        X.hdt = hdt;
        X.gamma = gamma;
        X.dxi[0] = R(a.dxi[0]);
        X.dxi[1] = R(a.dxi[1]);
        X.dxi[2] = R(a.dxi[2]);
        X.limiter = a.limiter;

        constexpr bool PF = PREFETCH && C::AZ;
        for (int s = 0; s < niter; ++s) {
            const int m = C::AZ ? s - 2 : 0;     // plane loaded
            const int c = C::AZ ? s - 3 : 0;     // plane prepared
            // ---- load plane m (+ the update of plane s-5, which reads only flux buffers);
            // with the prefetch, plane m was issued in the previous iteration's flux stage
            R* Wm_slot = S.W(C::AZ ? (m + 3) % 3 : 0);
            if constexpr (PF) {
                // plane m arrived under the previous iteration's flux stage (waited for and
                // published by its closing barrier); only the first plane is loaded here
                if (s == 0) {
                    stage_load<R, C, true>(Uc, pt, x0, y0, m, Wm_slot, bznext);
                    cp_async_wait_all();
                    __syncthreads();
                }
            } else if (!C::AZ || m <= nz + 1) {
                stage_load<R, C, false>(Uc, pt, x0, y0, m, Wm_slot, bznext);
            }
            if (C::AZ && s >= 5)
                stage_update<R, C>(S, Uc, Un, pt, x0, y0, s - 5, wx, wy, dtdx0, dtdx1, dtdx2, a.err);
            if constexpr (!PF) __syncthreads();
            if (C::AZ && m > nz + 1) break;      // the last update is done
            // PREFETCH: the conversion shares the update's phase (the update reads only the
            // flux buffers and U^n, the conversion only its ring slot and bznext)
            stage_convert<R, C>(Wm_slot, bznext, gm1);
            __syncthreads();
            // ---- prep plane c: threads walk rows of the W-ring pitch LX so that the
            // stencil reads of the W ring are contiguous; active lanes cover i in [-1, TX]
            if (c >= -1) {
                X.W0 = S.W(C::AZ ? (c + 3) % 3 : 0);
                X.Wm = S.W(C::AZ ? (c + 2) % 3 : 0);
                X.Wp = S.W(C::AZ ? (c + 4) % 3 : 0);
                R* Ps = S.P(C::AZ ? (c + 2) & 1 : 0);
                for (int w = threadIdx.x; w < C::PY * C::LX; w += C::NT) {
                    const int i = w % C::LX - C::LOX, j = w / C::LX - C::POY;
                    if (i < -1 || i > C::TX) continue;
                    prep_cell<R, C>(X, i, j, Ps, pidx<C>(i, j));
                }
            }
            __syncthreads();
            // ---- prefetch plane m+1 into the slot of plane c-1 (read by nobody from here on)
            if (PF && m + 1 <= nz + 1) stage_load<R, C, true>(Uc, pt, x0, y0, m + 1, S.W((m + 4) % 3), bznext);
            // ---- fluxes of plane c and between planes c-1 and c
            if (c >= 0) {
                const R* P0 = S.P(C::AZ ? (c + 2) & 1 : 0);
                const R* Pm = S.P(C::AZ ? (c + 1) & 1 : 0);
                R* IB = S.I(C::AZ ? (c & 1) : 0);
                R* ZB = S.Z(C::AZ ? (c & 1) : 0);
                R* Fx = IB;
                R* Fy = IB + 5 * C::FXN;
                R* Ez = Fy + 5 * C::FYN;
                R* Fz = ZB;
                R* Ex = ZB + 5 * C::FZN;
                R* Ey = Ex + C::EXN;
                const bool inplane = c < nz;
                constexpr int TOT = C::S_FX + C::S_FY + C::S_EZ + C::S_FZ + C::S_EX + C::S_EY;
                for (int w = threadIdx.x; w < TOT; w += C::NT) {
                    int r = w;
                    if (r < C::S_FX) {   // x-face i-1/2 of cell (i, j): i in [0, TX], j in [0, TY)
                        const int i = r % C::PX, j = r / C::PX;
                        if (inplane && i <= C::TX && j < C::RFX) {
                            R F[5];
                            face_flux<R, C>(P0, pidx<C>(i - 1, j), P0, pidx<C>(i, j), 0, gamma, gm1i, eps, a.riemann, F);
                            const int o = j * (C::TX + 1) + i;
#pragma unroll
                            for (int v = 0; v < 5; ++v) Fx[v * C::FXN + o] = F[v];
                        }
                        continue;
                    }
                    r -= C::S_FX;
                    if (r < C::S_FY) {   // y-face j-1/2 of cell (i, j): i in [0, TX), j in [0, TY]
                        const int i = r % C::PX - 1, j = r / C::PX;
                        if (C::AY && inplane && i >= 0 && i < C::TX && j < C::RFY) {
                            R F[5];
                            face_flux<R, C>(P0, pidx<C>(i, j - 1), P0, pidx<C>(i, j), 1, gamma, gm1i, eps, a.riemann, F);
                            const int o = j * C::TX + i;
#pragma unroll
                            for (int v = 0; v < 5; ++v) Fy[v * C::FYN + o] = F[v];
                        }
                        continue;
                    }
                    r -= C::S_FY;
                    if (r < C::S_EZ) {   // Ez at (i-1/2, j-1/2): i in [0, TX], j in [0, TY]
                        const int i = r % C::PX, j = r / C::PX;
                        if (inplane && i <= C::TX && j < C::REZ) {
                            const int jm = C::AY ? j - 1 : j;
                            // cells: SW=(i-1,j-1) RT, SE=(i,j-1) LT, NW=(i-1,j) RB, NE=(i,j) LB
                            const int pSW = pidx<C>(i - 1, jm), pSE = pidx<C>(i, jm);
                            const int pNW = pidx<C>(i - 1, j), pNE = pidx<C>(i, j);
                            // Ba = Bx face on side sa (+ slope along y): the x-face between
                            // cells i-1 and i is the low face of cell i; Bb = By face on side
                            // sb (+ slope along x): the low y-face of row j
                            const R bxS = pv<R, C>(P0, PV_BH(0), pSE), bxN = pv<R, C>(P0, PV_BH(0), pNE);
                            const R sxS = pv<R, C>(P0, PV_FS(0, 0), pSE), sxN = pv<R, C>(P0, PV_FS(0, 0), pNE);
                            const R byW = pv<R, C>(P0, PV_BH(1), pNW), byE = pv<R, C>(P0, PV_BH(1), pNE);
                            const R syW = pv<R, C>(P0, PV_FS(1, 1), pNW), syE = pv<R, C>(P0, PV_FS(1, 1), pNE);
                            const Corner<R> SW = corner<R, C>(P0, pSW, 2, R(1), R(1), bxS, sxS, byW, syW);
                            const Corner<R> SE = corner<R, C>(P0, pSE, 2, R(-1), R(1), bxS, sxS, byE, syE);
                            const Corner<R> NW = corner<R, C>(P0, pNW, 2, R(1), R(-1), bxN, sxN, byW, syW);
                            const Corner<R> NE = corner<R, C>(P0, pNE, 2, R(-1), R(-1), bxN, sxN, byE, syE);
                            Ez[j * (C::TX + 1) + i] = emf2d(SW, SE, NW, NE, gamma);
                        }
                        continue;
                    }
                    r -= C::S_EZ;
                    if (r < C::S_FZ) {   // z-face c-1/2 of cell (i, j): i in [0, TX), j in [0, TY)
                        const int i = r % C::PX - 1, j = r / C::PX;
                        if (C::AZ && i >= 0 && i < C::TX && j < C::RFZ) {
                            const int p = pidx<C>(i, j);
                            R F[5];
                            face_flux<R, C>(Pm, p, P0, p, 2, gamma, gm1i, eps, a.riemann, F);
                            const int o = j * C::TX + i;
#pragma unroll
                            for (int v = 0; v < 5; ++v) Fz[v * C::FZN + o] = F[v];
                        }
                        continue;
                    }
                    r -= C::S_FZ;
                    if (r < C::S_EX) {   // Ex at (i, j-1/2, c-1/2): a = y, b = z; i in [0, TX), j in [0, TY]
                        const int i = r % C::PX - 1, j = r / C::PX;
                        if (C::AY && i >= 0 && i < C::TX && j < C::REX) {
                            const int pS = pidx<C>(i, j - 1), pN = pidx<C>(i, j);
                            // SW = (j-1, c-1) corner (+y,+z); SE = (j, c-1) (-y,+z);
                            // NW = (j-1, c) (+y,-z); NE = (j, c) (-y,-z)
                            // Ba = By face at side sy: the low y-face of row j (both planes)
                            const R byB = pv<R, C>(Pm, PV_BH(1), pN), byT = pv<R, C>(P0, PV_BH(1), pN);
                            const R syB = pv<R, C>(Pm, PV_FS(1, 0), pN), syT = pv<R, C>(P0, PV_FS(1, 0), pN);
                            // Bb = Bz face at side sz: the face between c-1 and c = low face of plane c
                            const R bzW = pv<R, C>(P0, PV_BH(2), pS), bzE = pv<R, C>(P0, PV_BH(2), pN);
                            const R szW = pv<R, C>(P0, PV_FS(2, 1), pS), szE = pv<R, C>(P0, PV_FS(2, 1), pN);
                            const Corner<R> SW = corner<R, C>(Pm, pS, 0, R(1), R(1), byB, syB, bzW, szW);
                            const Corner<R> SE = corner<R, C>(Pm, pN, 0, R(-1), R(1), byB, syB, bzE, szE);
                            const Corner<R> NW = corner<R, C>(P0, pS, 0, R(1), R(-1), byT, syT, bzW, szW);
                            const Corner<R> NE = corner<R, C>(P0, pN, 0, R(-1), R(-1), byT, syT, bzE, szE);
                            Ex[j * C::TX + i] = emf2d(SW, SE, NW, NE, gamma);
                        }
                        continue;
                    }
                    r -= C::S_EX;
                    {   // Ey at (i-1/2, j, c-1/2): a = z, b = x; i in [0, TX], j in [0, TY)
                        const int i = r % C::PX, j = r / C::PX;
                        if (i <= C::TX && j < C::REY) {
                            const int pW = pidx<C>(i - 1, j), pE = pidx<C>(i, j);
                            // SW = (x=i-1, c-1) corner (+z,+x); SE = (i-1, c) (-z,+x);
                            // NW = (i, c-1) (+z,-x); NE = (i, c) (-z,-x)
                            // Ba = Bz face at side sz: low face of plane c (shared); slope along x
                            const R bzS = pv<R, C>(P0, PV_BH(2), pW), bzN = pv<R, C>(P0, PV_BH(2), pE);
                            const R szS = pv<R, C>(P0, PV_FS(2, 0), pW), szN = pv<R, C>(P0, PV_FS(2, 0), pE);
                            // Bb = Bx face at side sx: low face of cell i (shared); slope along z
                            const R bxW = pv<R, C>(Pm, PV_BH(0), pE), bxE = pv<R, C>(P0, PV_BH(0), pE);
                            const R sxW = pv<R, C>(Pm, PV_FS(0, 1), pE), sxE = pv<R, C>(P0, PV_FS(0, 1), pE);
                            const Corner<R> SW = corner<R, C>(Pm, pW, 1, R(1), R(1), bzS, szS, bxW, sxW);
                            const Corner<R> SE = corner<R, C>(P0, pW, 1, R(-1), R(1), bzS, szS, bxE, sxE);
                            const Corner<R> NW = corner<R, C>(Pm, pE, 1, R(1), R(-1), bzN, szN, bxW, sxW);
                            const Corner<R> NE = corner<R, C>(P0, pE, 1, R(-1), R(-1), bzN, szN, bxE, sxE);
                            Ey[j * (C::TX + 1) + i] = emf2d(SW, SE, NW, NE, gamma);
                        }
                    }
                }
            }
            if (PF) cp_async_wait_all();   // plane m+1, published by the barrier below
            __syncthreads();
            if (!C::AZ) {
                stage_update<R, C>(S, Uc, Un, pt, x0, y0, 0, wx, wy, dtdx0, dtdx1, dtdx2, a.err);
            }
        }
        // next tile
        if (a.dynamic) {
            __syncthreads();
            if (threadIdx.x == 0) s_tile = atomicAdd(&a.work[0], 1);
            __syncthreads();
            t = s_tile;
        } else {
            t = ntiles;
        }
    }
    if (a.dynamic && threadIdx.x == 0) {
        // the last CTA to finish resets the work counters for the next launch
        __threadfence();
        if (atomicAdd(&a.work[1], 1) == (int)gridDim.x - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace mhd
