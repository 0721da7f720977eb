// Discrete adjoint of one bunch step at fixed dt (3D bunches).
//
// lam = (dU^{n+1}/dU^n)^T lam_next, where U^{n+1} = step(fill(U^n)) is the forward
// update of mhd_step.cuh (a3-a9) applied after the guard fill (a1).  The forward
// intermediates are recomputed into global work arrays (one value per padded cell and
// field), then every stage is reversed in turn.  Each reverse kernel handles one item
// (cell, face or edge), calls the hand-written VJP of its arithmetic (mhd_vjp.cuh) and
// adds the resulting cotangents to the cells / faces / edges it read, with atomic adds.
// The last kernel is the transpose of the guard fill: the cotangent that reached a ghost
// copy is added to the interior cell it copies.
//
// Occupancy: the face and edge kernels (the HLLD / 2D-HLL VJPs) are capped at 128
// registers (two 256-thread blocks per SM) and take their direction from the grid's z
// index, so each thread handles one face or edge; the slope kernel is capped at 128
// registers and the other cell kernels at 85.
//
// Work arrays (fields of one value per padded cell; index coff[p] + (z*Y + y)*X + x):
//   W(8) primitives, DW(24) slopes [d][k], FS(6) face-field slopes, EN(3) time-n edge
//   EMFs, BH(3) predicted low-face fields, WH(8) predicted cell state; and the same 52
//   fields again for their cotangents.  The state cotangent lives in the output buffer.
#pragma once

#include "mhd_aux.cuh"
#include "mhd_common.cuh"
#include "mhd_math.cuh"
#include "mhd_vjp.cuh"

namespace mhd {

enum { AF_W = 0, AF_DW = 8, AF_FS = 32, AF_EN = 38, AF_BH = 41, AF_WH = 44, AF_N = 52 };

template <typename R>
struct AdjArgs {
    const R* U;          // padded U^n with filled ghosts (state layout)
    const R* lam_next;   // cotangent of U^{n+1} (state layout; interior entries used)
    R* lam;              // cotangent of U^n (state layout), accumulated
    R* F;                // forward work fields [AF_N][ncell]
    R* G;                // cotangent work fields [AF_N][ncell]
    int64_t ncell;       // cells of all padded patches
    const PatchDev* patches;
    int npatch;
    double gamma, eps, dt;
    double dxi[3];
    int limiter;
    int riemann;         // face flux: 0 HLLD, 1 HLL
};

// cell-field index helper for one patch
struct Cell {
    int64_t base;   // coff of the patch
    int X, Y, Z;
    __device__ __forceinline__ int64_t at(int x, int y, int z) const { return base + ((int64_t)z * Y + y) * X + x; }
};

__device__ __forceinline__ void unit(int d, int& ox, int& oy, int& oz) {
    ox = d == 0;
    oy = d == 1;
    oz = d == 2;
}

// Iterate the cells of the box [lo, hi] (inclusive, padded indices) of every patch.
// lo/hi are offsets from (g, g + n) per axis: lo = g + lo_off, hi = g + n - 1 + hi_off.
#define ADJ_FOR_REGION(a, LO, HI, ...)                                                        \
    for (int p = blockIdx.y; p < (a).npatch; p += gridDim.y) {                                 \
        const PatchDev pt = (a).patches[p];                                                    \
        const Cell C{pt.off / 8, pt.X, pt.Y, pt.Z};                                            \
        const int x0 = pt.gx + (LO), y0 = pt.gy + (LO), z0 = pt.gz + (LO);                     \
        const int x1 = pt.gx + pt.nx - 1 + (HI), y1 = pt.gy + pt.ny - 1 + (HI),                \
                  z1 = pt.gz + pt.nz - 1 + (HI);                                               \
        const int ex = x1 - x0 + 1, ey = y1 - y0 + 1, ez = z1 - z0 + 1;                        \
        const int64_t cnt = (int64_t)ex * ey * ez;                                             \
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < cnt;              \
             k += (int64_t)gridDim.x * blockDim.x) {                                           \
            const int x = x0 + (int)(k % ex), y = y0 + (int)((k / ex) % ey),                   \
                      z = z0 + (int)(k / ((int64_t)ex * ey));                                  \
            __VA_ARGS__                                                                        \
        }                                                                                      \
    }

template <typename R>
__device__ __forceinline__ R* fld(R* base, int f, int64_t ncell) { return base + (int64_t)f * ncell; }

// the state variable v of the cell with field index i (state layout: 8 vars per patch)
template <typename R>
__device__ __forceinline__ int64_t sidx(const PatchDev& pt, const Cell& C, int v, int64_t i) {
    const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
    return pt.off + v * vol + (i - C.base);
}

// ---------------------------------------------------------------------------------------
// forward recompute
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void adj_fwd_prim(AdjArgs<R> a) {
    const R gm1 = R(a.gamma - 1.0);
    ADJ_FOR_REGION(a, -2, 2, {
        const int64_t i = C.at(x, y, z);
        const R* u = a.U;
        R q[8];
        const R bxc = R(0.5) * (u[sidx<R>(pt, C, 5, i)] + u[sidx<R>(pt, C, 5, C.at(x + 1, y, z))]);
        const R byc = R(0.5) * (u[sidx<R>(pt, C, 6, i)] + u[sidx<R>(pt, C, 6, C.at(x, y + 1, z))]);
        const R bzc = R(0.5) * (u[sidx<R>(pt, C, 7, i)] + u[sidx<R>(pt, C, 7, C.at(x, y, z + 1))]);
        cons_to_prim(u[sidx<R>(pt, C, 0, i)], u[sidx<R>(pt, C, 1, i)], u[sidx<R>(pt, C, 2, i)],
                     u[sidx<R>(pt, C, 3, i)], u[sidx<R>(pt, C, 4, i)], bxc, byc, bzc, gm1, q);
        for (int v = 0; v < 8; ++v) fld(a.F, AF_W + v, a.ncell)[i] = q[v];
    })
}

template <typename R>
__global__ void adj_fwd_slopes(AdjArgs<R> a) {
    ADJ_FOR_REGION(a, -1, 2, {
        const int64_t i = C.at(x, y, z);
        const bool inner = x <= pt.gx + pt.nx && y <= pt.gy + pt.ny && z <= pt.gz + pt.nz;
        for (int d = 0; d < 3; ++d) {
            int ox, oy, oz;
            unit(d, ox, oy, oz);
            const int64_t im = C.at(x - ox, y - oy, z - oz), ip = C.at(x + ox, y + oy, z + oz);
            if (inner)
                for (int k = 0; k < 8; ++k) {
                    const R* w = fld(a.F, AF_W + k, a.ncell);
                    fld(a.F, AF_DW + 8 * d + k, a.ncell)[i] = limited(w[i] - w[im], w[ip] - w[i], a.limiter);
                }
        }
        // transverse slopes of the three low face fields
        for (int c = 0; c < 3; ++c)
            for (int kk = 0; kk < 2; ++kk) {
                const int t = (c + kk + 1) % 3;
                int ox, oy, oz;
                unit(t, ox, oy, oz);
                const R bm = a.U[sidx<R>(pt, C, 5 + c, C.at(x - ox, y - oy, z - oz))];
                const R b0 = a.U[sidx<R>(pt, C, 5 + c, i)];
                const R bp = a.U[sidx<R>(pt, C, 5 + c, C.at(x + ox, y + oy, z + oz))];
                fld(a.F, AF_FS + 2 * c + kk, a.ncell)[i] = limited(b0 - bm, bp - b0, a.limiter);
            }
    })
}

// time-n edge EMF of Eqs. 7-11 on the edge low in (a, b) of the cell
template <typename R>
__device__ __forceinline__ R en_value(const AdjArgs<R>& a, const PatchDev& pt, const Cell& C, int e, int x, int y,
                                      int z, R* va_out = nullptr, R* vb_out = nullptr, R* Ba_out = nullptr,
                                      R* Bb_out = nullptr) {
    const int A = (e + 1) % 3, B = (e + 2) % 3;
    int ax, ay, az, bx, by, bz;
    unit(A, ax, ay, az);
    unit(B, bx, by, bz);
    const int64_t c0 = C.at(x, y, z), cA = C.at(x - ax, y - ay, z - az), cB = C.at(x - bx, y - by, z - bz),
                  cAB = C.at(x - ax - bx, y - ay - by, z - az - bz);
    const R* ua = fld(a.F, AF_W + 1 + A, a.ncell);
    const R* ub = fld(a.F, AF_W + 1 + B, a.ncell);
    const R va = R(0.25) * (ua[c0] + ua[cA] + ua[cB] + ua[cAB]);
    const R vb = R(0.25) * (ub[c0] + ub[cA] + ub[cB] + ub[cAB]);
    const R Ba = R(0.5) * (a.U[sidx<R>(pt, C, 5 + A, c0)] + a.U[sidx<R>(pt, C, 5 + A, cB)]);
    const R Bb = R(0.5) * (a.U[sidx<R>(pt, C, 5 + B, c0)] + a.U[sidx<R>(pt, C, 5 + B, cA)]);
    if (va_out) {
        *va_out = va;
        *vb_out = vb;
        *Ba_out = Ba;
        *Bb_out = Bb;
    }
    return va * Bb - vb * Ba;
}

template <typename R>
__global__ void adj_fwd_en(AdjArgs<R> a) {
    ADJ_FOR_REGION(a, -1, 2, {
        const int64_t i = C.at(x, y, z);
        for (int e = 0; e < 3; ++e) fld(a.F, AF_EN + e, a.ncell)[i] = en_value(a, pt, C, e, x, y, z);
    })
}

// is the low c-face of cell (x,y,z) inside the predicted-face region (normal axis
// [g-1, g+n+1], transverse axes [g-1, g+n])?
__device__ __forceinline__ bool bh_region(const PatchDev& pt, int c, int x, int y, int z) {
    const int lim[3] = {pt.gx + pt.nx, pt.gy + pt.ny, pt.gz + pt.nz};
    const int v[3] = {x, y, z};
    for (int d = 0; d < 3; ++d)
        if (d != c && v[d] > lim[d]) return false;
    return true;
}

template <typename R>
__global__ void adj_fwd_bh(AdjArgs<R> a) {
    const R hdt = R(0.5 * a.dt);
    ADJ_FOR_REGION(a, -1, 2, {
        const int64_t i = C.at(x, y, z);
        for (int c = 0; c < 3; ++c) {
            if (!bh_region(pt, c, x, y, z)) continue;
            const int A = (c + 1) % 3, B = (c + 2) % 3;
            int ax, ay, az, bx, by, bz;
            unit(A, ax, ay, az);
            unit(B, bx, by, bz);
            const R* EA = fld(a.F, AF_EN + A, a.ncell);
            const R* EB = fld(a.F, AF_EN + B, a.ncell);
            // dB_c/dt = d_A E_B - d_B E_A
            const R t = hdt * R(a.dxi[A]) * (EB[C.at(x + ax, y + ay, z + az)] - EB[i]) -
                        hdt * R(a.dxi[B]) * (EA[C.at(x + bx, y + by, z + bz)] - EA[i]);
            fld(a.F, AF_BH + c, a.ncell)[i] = a.U[sidx<R>(pt, C, 5 + c, i)] + t;
        }
    })
}

template <typename R>
__device__ __forceinline__ void load_q_D(const AdjArgs<R>& a, int64_t i, R q[8], R D[3][8]) {
    for (int k = 0; k < 8; ++k) q[k] = fld(a.F, AF_W + k, a.ncell)[i];
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < 8; ++k) D[d][k] = fld(a.F, AF_DW + 8 * d + k, a.ncell)[i] * R(a.dxi[d]);
}

template <typename R>
__global__ void adj_fwd_wh(AdjArgs<R> a) {
    const R hdt = R(0.5 * a.dt), gamma = R(a.gamma);
    ADJ_FOR_REGION(a, -1, 1, {
        const int64_t i = C.at(x, y, z);
        R q[8], D[3][8], out[5];
        load_q_D(a, i, q, D);
        hancock(q, D, hdt, gamma, out);
        for (int k = 0; k < 5; ++k) fld(a.F, AF_WH + k, a.ncell)[i] = out[k];
        for (int c = 0; c < 3; ++c) {
            int ox, oy, oz;
            unit(c, ox, oy, oz);
            const R* bh = fld(a.F, AF_BH + c, a.ncell);
            fld(a.F, AF_WH + 5 + c, a.ncell)[i] = R(0.5) * (bh[i] + bh[C.at(x + ox, y + oy, z + oz)]);
        }
    })
}

// ---------------------------------------------------------------------------------------
// reverse
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void aadd(R* p, R v) {
    if (v != R(0)) atomicAdd(p, v);
}

// cotangent of U^{n+1} at a state entry if it is an interior cell / owned face, else 0
template <typename R>
__device__ __forceinline__ R lnext(const AdjArgs<R>& a, const PatchDev& pt, const Cell& C, int v, int x, int y,
                                   int z) {
    if (x < pt.gx || x >= pt.gx + pt.nx || y < pt.gy || y >= pt.gy + pt.ny || z < pt.gz || z >= pt.gz + pt.nz)
        return R(0);
    return a.lam_next[sidx<R>(pt, C, v, C.at(x, y, z))];
}

// lam = lam_next on interior entries (the identity part of U^{n+1} = U^n + ...), 0 elsewhere
template <typename R>
__global__ void adj_init(AdjArgs<R> a) {
    ADJ_FOR_REGION(a, -pt.gx, pt.gx, {
        for (int v = 0; v < 8; ++v) a.lam[sidx<R>(pt, C, v, C.at(x, y, z))] = lnext(a, pt, C, v, x, y, z);
    })
}

// faces: the HLLD flux through the low c-face of cells with normal index in [g, g+n] and
// transverse indices in the interior
template <typename R>
__global__ void __launch_bounds__(256, 2) adj_faces(AdjArgs<R> a) {
    const R gamma = R(a.gamma), gm1i = R(1.0 / (a.gamma - 1.0)), eps = R(a.eps);
    ADJ_FOR_REGION(a, 0, 1, {
        const int64_t i = C.at(x, y, z);
        for (int c = blockIdx.z; c < 3; c += gridDim.z) {   // face direction: one per grid z-slice
            const int t1 = (c + 1) % 3, t2 = (c + 2) % 3;
            const int v3[3] = {x, y, z};
            const int lim[3] = {pt.gx + pt.nx, pt.gy + pt.ny, pt.gz + pt.nz};
            if (v3[t1] >= lim[t1] || v3[t2] >= lim[t2]) continue;
            int ox, oy, oz;
            unit(c, ox, oy, oz);
            const int64_t im = C.at(x - ox, y - oy, z - oz);
            const R dtdx = R(a.dt * a.dxi[c]);
            // lF = dt/dx (lam'(cell) - lam'(cell - e_c)) for rho, m_c, m_t1, m_t2, E
            const int vs[5] = {0, 1 + c, 1 + t1, 1 + t2, 4};
            R lF[5];
            bool any = false;
            for (int n = 0; n < 5; ++n) {
                lF[n] = dtdx * (lnext(a, pt, C, vs[n], x, y, z) - lnext(a, pt, C, vs[n], x - ox, y - oy, z - oz));
                any |= lF[n] != R(0);
            }
            if (!any) continue;
            const int ks[7] = {Q_RHO, Q_U + c, Q_U + t1, Q_U + t2, Q_P, Q_BX + t1, Q_BX + t2};
            R L[7], Rr[7];
            for (int n = 0; n < 7; ++n) {
                const int k = ks[n];
                L[n] = fld(a.F, AF_WH + k, a.ncell)[im] + R(0.5) * fld(a.F, AF_DW + 8 * c + k, a.ncell)[im];
                Rr[n] = fld(a.F, AF_WH + k, a.ncell)[i] - R(0.5) * fld(a.F, AF_DW + 8 * c + k, a.ncell)[i];
            }
            const R bn = fld(a.F, AF_BH + c, a.ncell)[i];
            R lL[7] = {0, 0, 0, 0, 0, 0, 0}, lR[7] = {0, 0, 0, 0, 0, 0, 0}, lbn = R(0);
            if (a.riemann == 1) hll_vjp(L, Rr, bn, gamma, gm1i, lF, lL, lR, lbn);
            else hlld_vjp(L, Rr, bn, gamma, gm1i, eps, lF, lL, lR, lbn);
            for (int n = 0; n < 7; ++n) {
                const int k = ks[n];
                aadd(&fld(a.G, AF_WH + k, a.ncell)[im], lL[n]);
                aadd(&fld(a.G, AF_DW + 8 * c + k, a.ncell)[im], R(0.5) * lL[n]);
                aadd(&fld(a.G, AF_WH + k, a.ncell)[i], lR[n]);
                aadd(&fld(a.G, AF_DW + 8 * c + k, a.ncell)[i], R(-0.5) * lR[n]);
            }
            aadd(&fld(a.G, AF_BH + c, a.ncell)[i], lbn);
        }
    })
}

// corner state (sa, sb) of cell X for edge e, with the a-face / b-face fields it uses
template <typename R>
__device__ __forceinline__ Corner<R> adj_corner(const AdjArgs<R>& a, const Cell& C, int e, int X0, int Y0, int Z0,
                                                int sa, int sb, int64_t& fa, int64_t& fb) {
    const int A = (e + 1) % 3, B = (e + 2) % 3;
    int ax, ay, az, bx, by, bz;
    unit(A, ax, ay, az);
    unit(B, bx, by, bz);
    const int64_t i = C.at(X0, Y0, Z0);
    fa = sa > 0 ? C.at(X0 + ax, Y0 + ay, Z0 + az) : i;   // cell whose low a-face it is
    fb = sb > 0 ? C.at(X0 + bx, Y0 + by, Z0 + bz) : i;
    auto ext = [&](int k) {
        return fld(a.F, AF_WH + k, a.ncell)[i] +
               R(0.5) * (R(sa) * fld(a.F, AF_DW + 8 * A + k, a.ncell)[i] + R(sb) * fld(a.F, AF_DW + 8 * B + k, a.ncell)[i]);
    };
    Corner<R> s;
    s.rho = ext(Q_RHO);
    s.p = ext(Q_P);
    s.ua = ext(Q_U + A);
    s.ub = ext(Q_U + B);
    s.Be = ext(Q_BX + e);
    s.Ba = fld(a.F, AF_BH + A, a.ncell)[fa] + R(0.5) * R(sb) * fld(a.F, AF_FS + 2 * A + 0, a.ncell)[fa];
    s.Bb = fld(a.F, AF_BH + B, a.ncell)[fb] + R(0.5) * R(sa) * fld(a.F, AF_FS + 2 * B + 1, a.ncell)[fb];
    return s;
}

template <typename R>
__device__ __forceinline__ void adj_corner_scatter(const AdjArgs<R>& a, const Cell& C, int e, int X0, int Y0, int Z0,
                                                   int sa, int sb, int64_t fa, int64_t fb, const Corner<R>& g) {
    const int A = (e + 1) % 3, B = (e + 2) % 3;
    const int64_t i = C.at(X0, Y0, Z0);
    const int ks[5] = {Q_RHO, Q_P, Q_U + A, Q_U + B, Q_BX + e};
    const R gv[5] = {g.rho, g.p, g.ua, g.ub, g.Be};
    for (int n = 0; n < 5; ++n) {
        aadd(&fld(a.G, AF_WH + ks[n], a.ncell)[i], gv[n]);
        aadd(&fld(a.G, AF_DW + 8 * A + ks[n], a.ncell)[i], R(0.5) * R(sa) * gv[n]);
        aadd(&fld(a.G, AF_DW + 8 * B + ks[n], a.ncell)[i], R(0.5) * R(sb) * gv[n]);
    }
    aadd(&fld(a.G, AF_BH + A, a.ncell)[fa], g.Ba);
    aadd(&fld(a.G, AF_FS + 2 * A + 0, a.ncell)[fa], R(0.5) * R(sb) * g.Ba);
    aadd(&fld(a.G, AF_BH + B, a.ncell)[fb], g.Bb);
    aadd(&fld(a.G, AF_FS + 2 * B + 1, a.ncell)[fb], R(0.5) * R(sa) * g.Bb);
}

// edges: the 2D HLL EMF on the edge low in (a, b) of cells with a, b indices in [g, g+n]
// and the e index in the interior
template <typename R>
__global__ void __launch_bounds__(256, 2) adj_edges(AdjArgs<R> a) {
    const R gamma = R(a.gamma);
    ADJ_FOR_REGION(a, 0, 1, {
        for (int e = blockIdx.z; e < 3; e += gridDim.z) {   // edge direction: one per grid z-slice
            const int A = (e + 1) % 3, B = (e + 2) % 3;
            const int v3[3] = {x, y, z};
            const int lim[3] = {pt.gx + pt.nx, pt.gy + pt.ny, pt.gz + pt.nz};
            if (v3[e] >= lim[e]) continue;
            int ax, ay, az, bx, by, bz;
            unit(A, ax, ay, az);
            unit(B, bx, by, bz);
            // lE = dt/dx_B (lam_A(cell - e_B) - lam_A(cell)) + dt/dx_A (lam_B(cell) - lam_B(cell - e_A))
            const R lE = R(a.dt * a.dxi[B]) * (lnext(a, pt, C, 5 + A, x - bx, y - by, z - bz) -
                                               lnext(a, pt, C, 5 + A, x, y, z)) +
                         R(a.dt * a.dxi[A]) * (lnext(a, pt, C, 5 + B, x, y, z) -
                                               lnext(a, pt, C, 5 + B, x - ax, y - ay, z - az));
            if (lE == R(0)) continue;
            // SW = (-a,-b) corner (+,+); SE = (-b) corner (-,+); NW = (-a) corner (+,-); NE = cell (-,-)
            int64_t fa[4], fb[4];
            const int cx[4] = {x - ax - bx, x - bx, x - ax, x};
            const int cy[4] = {y - ay - by, y - by, y - ay, y};
            const int cz[4] = {z - az - bz, z - bz, z - az, z};
            const int sa[4] = {1, -1, 1, -1}, sb[4] = {1, 1, -1, -1};
            Corner<R> s[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] = adj_corner(a, C, e, cx[k], cy[k], cz[k], sa[k], sb[k], fa[k], fb[k]);
            Corner<R> g[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) g[k] = Corner<R>{0, 0, 0, 0, 0, 0, 0};
            emf2d_vjp(s[0], s[1], s[2], s[3], gamma, lE, g[0], g[1], g[2], g[3]);
#pragma unroll
            for (int k = 0; k < 4; ++k) adj_corner_scatter(a, C, e, cx[k], cy[k], cz[k], sa[k], sb[k], fa[k], fb[k], g[k]);
        }
    })
}

// predictor: lWH -> lW, lDW (Hancock) and lBH (cell-centred predicted field = face mean)
template <typename R>
__global__ void __launch_bounds__(256, 3) adj_pred(AdjArgs<R> a) {
    const R hdt = R(0.5 * a.dt), gamma = R(a.gamma);
    ADJ_FOR_REGION(a, -1, 1, {
        const int64_t i = C.at(x, y, z);
        R lo[5], lb[3];
        bool any = false;
        for (int k = 0; k < 5; ++k) {
            lo[k] = fld(a.G, AF_WH + k, a.ncell)[i];
            any |= lo[k] != R(0);
        }
        for (int c = 0; c < 3; ++c) lb[c] = fld(a.G, AF_WH + 5 + c, a.ncell)[i];   // before any atomic add
        if (any) {
            R q[8], D[3][8], lq[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lD[3][8];
            for (int d = 0; d < 3; ++d)
                for (int k = 0; k < 8; ++k) lD[d][k] = R(0);
            load_q_D(a, i, q, D);
            hancock_vjp(q, D, hdt, gamma, lo, lq, lD);
            for (int k = 0; k < 8; ++k) aadd(&fld(a.G, AF_W + k, a.ncell)[i], lq[k]);
            for (int d = 0; d < 3; ++d)
                for (int k = 0; k < 8; ++k) aadd(&fld(a.G, AF_DW + 8 * d + k, a.ncell)[i], lD[d][k] * R(a.dxi[d]));
        }
        for (int c = 0; c < 3; ++c) {
            const R l = lb[c];
            if (l == R(0)) continue;
            int ox, oy, oz;
            unit(c, ox, oy, oz);
            aadd(&fld(a.G, AF_BH + c, a.ncell)[i], R(0.5) * l);
            aadd(&fld(a.G, AF_BH + c, a.ncell)[C.at(x + ox, y + oy, z + oz)], R(0.5) * l);
        }
    })
}

// predicted faces: bh_c = B_c + dt/2 (dx_A^-1 (EN_B(+A) - EN_B) - dx_B^-1 (EN_A(+B) - EN_A))
template <typename R>
__global__ void __launch_bounds__(256, 3) adj_bh(AdjArgs<R> a) {
    const R hdt = R(0.5 * a.dt);
    ADJ_FOR_REGION(a, -1, 2, {
        const int64_t i = C.at(x, y, z);
        for (int c = 0; c < 3; ++c) {
            if (!bh_region(pt, c, x, y, z)) continue;
            const R l = fld(a.G, AF_BH + c, a.ncell)[i];
            if (l == R(0)) continue;
            const int A = (c + 1) % 3, B = (c + 2) % 3;
            int ax, ay, az, bx, by, bz;
            unit(A, ax, ay, az);
            unit(B, bx, by, bz);
            aadd(&a.lam[sidx<R>(pt, C, 5 + c, i)], l);
            const R kA = hdt * R(a.dxi[A]) * l, kB = hdt * R(a.dxi[B]) * l;
            aadd(&fld(a.G, AF_EN + B, a.ncell)[C.at(x + ax, y + ay, z + az)], kA);
            aadd(&fld(a.G, AF_EN + B, a.ncell)[i], -kA);
            aadd(&fld(a.G, AF_EN + A, a.ncell)[C.at(x + bx, y + by, z + bz)], -kB);
            aadd(&fld(a.G, AF_EN + A, a.ncell)[i], kB);
        }
    })
}

// time-n edge EMF: E = <v_a><B_b> - <v_b><B_a>
template <typename R>
__global__ void __launch_bounds__(256, 3) adj_en(AdjArgs<R> a) {
    ADJ_FOR_REGION(a, -1, 2, {
        const int64_t i = C.at(x, y, z);
        for (int e = 0; e < 3; ++e) {
            const R l = fld(a.G, AF_EN + e, a.ncell)[i];
            if (l == R(0)) continue;
            const int A = (e + 1) % 3, B = (e + 2) % 3;
            int ax, ay, az, bx, by, bz;
            unit(A, ax, ay, az);
            unit(B, bx, by, bz);
            R va, vb, Ba, Bb;
            en_value(a, pt, C, e, x, y, z, &va, &vb, &Ba, &Bb);
            const int64_t cs[4] = {i, C.at(x - ax, y - ay, z - az), C.at(x - bx, y - by, z - bz),
                                   C.at(x - ax - bx, y - ay - by, z - az - bz)};
            for (int k = 0; k < 4; ++k) {
                aadd(&fld(a.G, AF_W + 1 + A, a.ncell)[cs[k]], R(0.25) * l * Bb);
                aadd(&fld(a.G, AF_W + 1 + B, a.ncell)[cs[k]], R(-0.25) * l * Ba);
            }
            aadd(&a.lam[sidx<R>(pt, C, 5 + B, i)], R(0.5) * l * va);
            aadd(&a.lam[sidx<R>(pt, C, 5 + B, cs[1])], R(0.5) * l * va);
            aadd(&a.lam[sidx<R>(pt, C, 5 + A, i)], R(-0.5) * l * vb);
            aadd(&a.lam[sidx<R>(pt, C, 5 + A, cs[2])], R(-0.5) * l * vb);
        }
    })
}

// limited slopes of the primitives and of the face fields
template <typename R>
__global__ void __launch_bounds__(256, 2) adj_slopes(AdjArgs<R> a) {
    ADJ_FOR_REGION(a, -1, 2, {
        const int64_t i = C.at(x, y, z);
        const bool inner = x <= pt.gx + pt.nx && y <= pt.gy + pt.ny && z <= pt.gz + pt.nz;
        // Every load of a group is issued before its atomic adds: the fields read here (slope
        // cotangents, primitives, U) are never written by this kernel, but the compiler
        // cannot tell them from the accumulated ones and would otherwise wait for each load.
        if (inner)
            for (int d = 0; d < 3; ++d) {
                int ox, oy, oz;
                unit(d, ox, oy, oz);
                const int64_t im = C.at(x - ox, y - oy, z - oz), ip = C.at(x + ox, y + oy, z + oz);
                R l[8], wm[8], w0[8], wp[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const R* w = fld(a.F, AF_W + k, a.ncell);
                    l[k] = fld(a.G, AF_DW + 8 * d + k, a.ncell)[i];
                    wm[k] = w[im];
                    w0[k] = w[i];
                    wp[k] = w[ip];
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (l[k] == R(0)) continue;
                    R lm = 0, l0 = 0, lp = 0;
                    slope_vjp(wm[k], w0[k], wp[k], a.limiter, l[k], lm, l0, lp);
                    R* gw = fld(a.G, AF_W + k, a.ncell);
                    aadd(&gw[im], lm);
                    aadd(&gw[i], l0);
                    aadd(&gw[ip], lp);
                }
            }
        R lf[6], um[6], u0[6], up[6];
        int64_t fim[6], fip[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int c = f >> 1, kk = f & 1;
            const int t = (c + kk + 1) % 3;
            int ox, oy, oz;
            unit(t, ox, oy, oz);
            fim[f] = C.at(x - ox, y - oy, z - oz);
            fip[f] = C.at(x + ox, y + oy, z + oz);
            lf[f] = fld(a.G, AF_FS + f, a.ncell)[i];
            um[f] = a.U[sidx<R>(pt, C, 5 + c, fim[f])];
            u0[f] = a.U[sidx<R>(pt, C, 5 + c, i)];
            up[f] = a.U[sidx<R>(pt, C, 5 + c, fip[f])];
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (lf[f] == R(0)) continue;
            const int c = f >> 1;
            R lm = 0, l0 = 0, lp = 0;
            slope_vjp(um[f], u0[f], up[f], a.limiter, lf[f], lm, l0, lp);
            aadd(&a.lam[sidx<R>(pt, C, 5 + c, fim[f])], lm);
            aadd(&a.lam[sidx<R>(pt, C, 5 + c, i)], l0);
            aadd(&a.lam[sidx<R>(pt, C, 5 + c, fip[f])], lp);
        }
    })
}

// primitives: lW -> lU (rho, momenta, E) and the two faces of each field component
template <typename R>
__global__ void __launch_bounds__(256, 3) adj_prim(AdjArgs<R> a) {
    const R gm1 = R(a.gamma - 1.0);
    ADJ_FOR_REGION(a, -2, 2, {
        const int64_t i = C.at(x, y, z);
        R lq[8];
        bool any = false;
        for (int k = 0; k < 8; ++k) {
            lq[k] = fld(a.G, AF_W + k, a.ncell)[i];
            any |= lq[k] != R(0);
        }
        if (!any) continue;
        const R* u = a.U;
        const int64_t ix = C.at(x + 1, y, z), iy = C.at(x, y + 1, z), iz = C.at(x, y, z + 1);
        const R bxc = R(0.5) * (u[sidx<R>(pt, C, 5, i)] + u[sidx<R>(pt, C, 5, ix)]);
        const R byc = R(0.5) * (u[sidx<R>(pt, C, 6, i)] + u[sidx<R>(pt, C, 6, iy)]);
        const R bzc = R(0.5) * (u[sidx<R>(pt, C, 7, i)] + u[sidx<R>(pt, C, 7, iz)]);
        R lU[5] = {0, 0, 0, 0, 0}, lbc[3] = {0, 0, 0};
        cons_to_prim_vjp(u[sidx<R>(pt, C, 0, i)], u[sidx<R>(pt, C, 1, i)], u[sidx<R>(pt, C, 2, i)],
                         u[sidx<R>(pt, C, 3, i)], u[sidx<R>(pt, C, 4, i)], bxc, byc, bzc, gm1, lq, lU, lbc);
        for (int v = 0; v < 5; ++v) aadd(&a.lam[sidx<R>(pt, C, v, i)], lU[v]);
        const int64_t hi[3] = {ix, iy, iz};
        for (int c = 0; c < 3; ++c) {
            aadd(&a.lam[sidx<R>(pt, C, 5 + c, i)], R(0.5) * lbc[c]);
            aadd(&a.lam[sidx<R>(pt, C, 5 + c, hi[c])], R(0.5) * lbc[c]);
        }
    })
}

// transpose of the guard fill: every ghost adds its cotangent to the interior cell it
// copies (same owner lookup as fill_kernel) and is then cleared
template <typename R>
__global__ void adj_fill_transpose(R* lam, const PatchDev* __restrict__ patches, int npatch, FillGeom fg,
                                   unsigned* err) {
    for (int p = blockIdx.y; p < npatch; p += gridDim.y) {
        const PatchDev pt = patches[p];
        const int ng = ghost_count(pt);
        const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += gridDim.x * blockDim.x) {
            int x, y, z;
            ghost_coord(pt, k, x, y, z);
            const int gxg = wrap_axis(pt.ox + x - pt.gx, fg.N[0], fg.bc[0][0], fg.bc[0][1]);
            const int gyg = wrap_axis(pt.oy + y - pt.gy, fg.N[1], fg.bc[1][0], fg.bc[1][1]);
            const int gzg = wrap_axis(pt.oz + z - pt.gz, fg.N[2], fg.bc[2][0], fg.bc[2][1]);
            const int ow = fg.owner[((gzg / fg.bs[2]) * fg.M[1] + gyg / fg.bs[1]) * fg.M[0] + gxg / fg.bs[0]];
            if (ow < 0 || ow >= npatch) {
                atomicOr(err, ERR_BOUNDS);
                continue;
            }
            const PatchDev src = patches[ow];
            const int sx = gxg - src.ox + src.gx, sy = gyg - src.oy + src.gy, sz = gzg - src.oz + src.gz;
            const int64_t svol = (int64_t)src.X * src.Y * src.Z;
            R* s = lam + src.off + ((int64_t)sz * src.Y + sy) * src.X + sx;
            R* d = lam + pt.off + ((int64_t)z * pt.Y + y) * pt.X + x;
            // the ghost's 8 cotangents are loaded before the atomic adds into its source (an
            // interior cell, never a ghost, so the two never alias)
            R g[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) g[v] = d[v * vol];
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                d[v * vol] = R(0);
                if (g[v] != R(0)) atomicAdd(&s[v * svol], g[v]);
            }
        }
    }
}

// the same for equal patches on a regular grid: sources from the neighbour table (as
// fill_grid_kernel), one CTA per padded z-plane of a patch walking the plane's ghost cells
template <typename R>
__global__ void adj_fill_transpose_grid(R* lam, const PatchDev* __restrict__ patches,
                                        const int64_t* __restrict__ nboff, int Zp) {
    const int p = blockIdx.x / Zp, z = blockIdx.x - p * Zp;
    const PatchDev pt = patches[p];
    const int64_t* nb = nboff + (int64_t)p * 27;
    const int X = pt.X, Y = pt.Y, gx = pt.gx, gy = pt.gy;
    const int64_t vol = (int64_t)X * Y * pt.Z;
    const int iz = z - pt.gz;
    const bool zghost = iz < 0 || iz >= pt.nz;
    const int nfull = zghost ? X * Y : 2 * gy * X;
    const int ncnt = zghost ? X * Y : nfull + pt.ny * 2 * gx;
    R* plane = lam + pt.off + (int64_t)z * X * Y;
    for (int k = threadIdx.x; k < ncnt; k += blockDim.x) {
        int x, y;
        if (k < nfull) {
            const int r = k / X;
            x = k - r * X;
            y = zghost ? r : (r < gy ? r : pt.ny + r);
        } else {
            const int k2 = k - nfull;
            const int r = k2 / (2 * gx), c = k2 - r * (2 * gx);
            y = gy + r;
            x = c < gx ? c : pt.nx + c;
        }
        R* s = lam + neighbour_source(pt, nb, x - gx, y - gy, iz);
        R* d = plane + (int64_t)y * X + x;
        R g[8];   // loaded before the atomic adds (source interior, destination ghost)
#pragma unroll
        for (int v = 0; v < 8; ++v) g[v] = d[v * vol];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            d[v * vol] = R(0);
            if (g[v] != R(0)) atomicAdd(&s[v * vol], g[v]);
        }
    }
}

}  // namespace mhd
