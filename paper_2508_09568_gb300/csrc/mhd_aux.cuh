// Guard fill (a1) and CFL time step (a2) kernels.
#pragma once

#include "mhd_common.cuh"
#include "mhd_math.cuh"

namespace mhd {

// ---------------------------------------------------------------------------------------
// a1: guard fill.  Every ghost cell of every patch receives the value (all 8 variables)
// of the box cell it stands for: its global index is wrapped (periodic) or clamped
// (zero-gradient outflow) into the box, the owning patch is read from the owner map and
// the value is copied from that patch's interior.  Sources are always interior cells and
// destinations always ghost cells, so the kernel is race free.  DISPATCH fills ghost
// zones from neighbouring patches (Sec. 2.2, Sec. 3.1); here all patches share one time.
// ---------------------------------------------------------------------------------------

// number of ghost cells of a padded patch
__device__ __forceinline__ int ghost_count(const PatchDev& p) {
    return p.X * p.Y * p.Z - p.nx * p.ny * p.nz;
}

// k-th ghost cell of a patch -> local padded coordinates (slabs: z, then y, then x)
__device__ __forceinline__ void ghost_coord(const PatchDev& p, int k, int& x, int& y, int& z) {
    const int cz = 2 * p.gz * p.X * p.Y;
    const int cy = 2 * p.gy * p.X * p.nz;
    if (k < cz) {
        const int per = p.gz * p.X * p.Y;
        const int side = k / per, r = k - side * per;
        z = (side ? p.gz + p.nz : 0) + r / (p.X * p.Y);
        const int r2 = r % (p.X * p.Y);
        y = r2 / p.X;
        x = r2 % p.X;
        return;
    }
    k -= cz;
    if (k < cy) {
        const int per = p.gy * p.X * p.nz;
        const int side = k / per, r = k - side * per;
        z = p.gz + r / (p.gy * p.X);
        const int r2 = r % (p.gy * p.X);
        y = (side ? p.gy + p.ny : 0) + r2 / p.X;
        x = r2 % p.X;
        return;
    }
    k -= cy;
    const int per = p.gx * p.ny * p.nz;
    const int side = k / per, r = k - side * per;
    z = p.gz + r / (p.gx * p.ny);
    const int r2 = r % (p.gx * p.ny);
    y = p.gy + r2 / p.gx;
    x = (side ? p.gx + p.nx : 0) + r2 % p.gx;
}

__device__ __forceinline__ int wrap_axis(int g, int N, int lo, int hi) {
    if (g < 0) return lo == 0 ? ((g % N) + N) % N : 0;
    if (g >= N) return hi == 0 ? g % N : N - 1;
    return g;
}

template <typename R>
__global__ void fill_kernel(R* __restrict__ U, const PatchDev* __restrict__ patches, int npatch,
                            FillGeom fg, unsigned* err) {
    // four ghost cells per thread and pass: their owner lookups and loads all in flight
    // before the stores
    constexpr int NC = 4;
    for (int p = blockIdx.y; p < npatch; p += gridDim.y) {
        const PatchDev pt = patches[p];
        const int ng = ghost_count(pt);
        const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
        const int stride = gridDim.x * blockDim.x;
        for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < ng; k0 += NC * stride) {
            const R* s[NC];
            R* d[NC];
            int64_t svol[NC];
            bool on[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = k0 + c * stride;
                on[c] = k < ng;
                s[c] = U;
                d[c] = U;
                svol[c] = 0;
                if (!on[c]) continue;
                int x, y, z;
                ghost_coord(pt, k, x, y, z);
                const int gxg = wrap_axis(pt.ox + x - pt.gx, fg.N[0], fg.bc[0][0], fg.bc[0][1]);
                const int gyg = wrap_axis(pt.oy + y - pt.gy, fg.N[1], fg.bc[1][0], fg.bc[1][1]);
                const int gzg = wrap_axis(pt.oz + z - pt.gz, fg.N[2], fg.bc[2][0], fg.bc[2][1]);
                const int ow = fg.owner[((gzg / fg.bs[2]) * fg.M[1] + gyg / fg.bs[1]) * fg.M[0] + gxg / fg.bs[0]];
                if (ow < 0 || ow >= npatch) {
                    atomicOr(err, ERR_BOUNDS);
                    on[c] = false;
                    continue;
                }
                const PatchDev src = patches[ow];
                const int sx = gxg - src.ox + src.gx, sy = gyg - src.oy + src.gy, sz = gzg - src.oz + src.gz;
                svol[c] = (int64_t)src.X * src.Y * src.Z;
                s[c] = U + src.off + ((int64_t)sz * src.Y + sy) * src.X + sx;
                d[c] = U + pt.off + ((int64_t)z * pt.Y + y) * pt.X + x;
            }
            R v[NC][8];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int q = 0; q < 8; ++q) v[c][q] = on[c] ? s[c][q * svol[c]] : R(0);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (on[c]) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) d[c][q * vol] = v[c][q];
                }
        }
    }
}

// a1 for bunches of equal patches on a regular grid (the same values as fill_kernel): the
// source of every ghost cell comes from the patch's neighbour table instead of the owner
// map.  One CTA per padded z-plane of a patch (blockIdx.x = patch * Z + plane) walks only
// the plane's ghost cells: the whole plane outside the interior z range, else the ghost
// rows (taken whole) and the ghost columns of the interior rows.
template <typename R>
__global__ void __launch_bounds__(128) fill_grid_kernel(R* __restrict__ U, const PatchDev* __restrict__ patches,
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
    R* plane = U + pt.off + (int64_t)z * X * Y;
    // plane coordinates of the k-th ghost cell of the plane
    auto coord = [&](int k, int& x, int& y) {
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
    };
    // four cells per thread and pass: all their loads in flight before the stores
    constexpr int NC = 4;
    for (int k0 = threadIdx.x; k0 < ncnt; k0 += NC * blockDim.x) {
        const R* src[NC];
        R* dst[NC];
        bool on[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int k = k0 + c * blockDim.x;
            on[c] = k < ncnt;
            int x = 0, y = 0;
            if (on[c]) coord(k, x, y);
            src[c] = U + neighbour_source(pt, nb, on[c] ? x - gx : 0, on[c] ? y - gy : 0, iz);
            dst[c] = plane + (int64_t)y * X + x;
        }
        R v[NC][8];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int q = 0; q < 8; ++q) v[c][q] = on[c] ? src[c][q * vol] : R(0);
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (on[c]) {
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[c][q * vol] = v[c][q];
            }
    }
}

// ---------------------------------------------------------------------------------------
// a2: CFL time step.  rate = sum over active axes of (|u_d| + c_f,d) / dx_d per interior
// cell; each block reduces its patches' maximum (warp shuffles, then shared memory) into
// partial[block]; the last block to finish reduces the partials and writes
// dt = courant / max_rate into *dt_out (double).  Non-finite rates set ERR_PHYS.
// ---------------------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ R block_max(R v, R* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : R(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            R w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
    }
    return v;   // valid in thread 0
}

template <typename R>
struct CflArgs {
    const R* __restrict__ U;
    const PatchDev* __restrict__ patches;
    int npatch;
    double gamma, courant;
    double dxi[3];
    int act[3];
    R* partial;            // [gridDim.x] scratch
    unsigned* counter;     // scratch, zero before the launch, left at zero after
    double* dt_out;
    unsigned* err;
};

// CFL rate of the interior cell c (pointer to its rho) of a patch: sum over active axes of
// (|u_d| + c_f,d) / dx_d, with the cell-centred field the mean of the cell's two faces
// (the same with the cell's three high faces given)
// (from the cell's 8 values u)
template <typename R>
__device__ __forceinline__ R cell_rate_vals(const R u[8], R bxh, R byh, R bzh, bool act1, bool act2, R gamma,
                                            R gm1, R dxi0, R dxi1, R dxi2) {
    const R bxc = R(0.5) * (u[5] + bxh);
    const R byc = act1 ? R(0.5) * (u[6] + byh) : u[6];
    const R bzc = act2 ? R(0.5) * (u[7] + bzh) : u[7];
    R q[8];
    cons_to_prim(u[0], u[1], u[2], u[3], u[4], bxc, byc, bzc, gm1, q);
    const R ri = rdiv(R(1), q[Q_RHO]), gP = gamma * q[Q_P];
    R rate = mul_(rabs(q[Q_U]) + fast_speed(ri, gP, bxc, byc, bzc), dxi0);
    if (act1) rate = fma_(rabs(q[Q_V]) + fast_speed(ri, gP, byc, bzc, bxc), dxi1, rate);
    if (act2) rate = fma_(rabs(q[Q_W]) + fast_speed(ri, gP, bzc, bxc, byc), dxi2, rate);
    return rate;
}

template <typename R>
__device__ __forceinline__ R cell_rate_faces(const R* c, int64_t vol, R bxh, R byh, R bzh, bool act1, bool act2,
                                             R gamma, R gm1, R dxi0, R dxi1, R dxi2) {
    R u[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) u[v] = c[v * vol];
    return cell_rate_vals(u, bxh, byh, bzh, act1, act2, gamma, gm1, dxi0, dxi1, dxi2);
}

template <typename R>
__device__ __forceinline__ R cell_rate(const R* c, int64_t vol, int sy, int sz, bool act1, bool act2, R gamma,
                                       R gm1, R dxi0, R dxi1, R dxi2) {
    return cell_rate_faces(c, vol, c[5 * vol + 1], act1 ? c[6 * vol + sy] : R(0), act2 ? c[7 * vol + sz] : R(0),
                           act1, act2, gamma, gm1, dxi0, dxi1, dxi2);
}

template <typename R>
__global__ void cfl_kernel(CflArgs<R> a) {
    __shared__ R red[32];
    __shared__ bool last;
    const R gamma = R(a.gamma), gm1 = R(a.gamma - 1.0);
    const R dxi0 = R(a.dxi[0]), dxi1 = R(a.dxi[1]), dxi2 = R(a.dxi[2]);
    R vmax = R(0);
    bool bad = false;
    // one warp per row of a patch (x along the lanes): the (z, y) of a row is computed once
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = blockIdx.x; p < a.npatch; p += gridDim.x) {
        const PatchDev pt = a.patches[p];
        const int rows = pt.ny * pt.nz;
        const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
        const int sy = pt.X, sz = pt.X * pt.Y;
        for (int r = wid; r < rows; r += nw) {
            const int z = r / pt.ny + pt.gz, y = r - (r / pt.ny) * pt.ny + pt.gy;
            const R* row = a.U + pt.off + ((int64_t)z * pt.Y + y) * pt.X + pt.gx;
            for (int x = lane; x < pt.nx; x += 32) {
                const R rate = cell_rate(row + x, vol, sy, sz, a.act[1] != 0, a.act[2] != 0, gamma, gm1, dxi0,
                                         dxi1, dxi2);
                if (!finite_(rate)) bad = true;
                else vmax = rate > vmax ? rate : vmax;
            }
        }
    }
    if (bad) atomicOr(a.err, ERR_PHYS);
    R bm = block_max(vmax, red);
    if (threadIdx.x == 0) {
        a.partial[blockIdx.x] = bm;
        __threadfence();
        last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        R v = R(0);
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
            R w = ((volatile R*)a.partial)[k];
            v = w > v ? w : v;
        }
        __syncthreads();
        v = block_max(v, red);
        if (threadIdx.x == 0) {
            *a.dt_out = a.courant / (double)v;
            *a.counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// a1 + a2 fused for bunches of equal patches on a regular grid (the values of
// fill_grid_kernel and the dt of cfl_kernel, bitwise): one CTA per padded z-plane of a
// patch fills the plane's ghost cells, then (interior planes) takes the CFL rates of the
// plane's cells.  Their high x- and y-faces are ghost cells the CTA has just written; the
// high z-face of the top interior plane is read where the fill takes it from.  Each CTA
// writes its maximum to partial[blockIdx.x]; the last CTA writes dt = courant / max.
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) fill_cfl_grid_kernel(R* __restrict__ U, const PatchDev* __restrict__ patches,
                                                           const int64_t* __restrict__ nboff, int Zp, R gamma, R gm1,
                                                           double courant, R dxi0, R dxi1, R dxi2, int act1,
                                                           int act2, R* partial,
                                                           unsigned* counter, double* dt_out, unsigned* err) {
    __shared__ R red[32];
    __shared__ bool last;
    const int p = blockIdx.x / Zp, z = blockIdx.x - p * Zp;
    const PatchDev pt = patches[p];
    const int64_t* nb = nboff + (int64_t)p * 27;
    const int X = pt.X, Y = pt.Y, gx = pt.gx, gy = pt.gy;
    const int64_t vol = (int64_t)X * Y * pt.Z;
    const int iz = z - pt.gz;
    const bool zghost = iz < 0 || iz >= pt.nz;
    R* plane = U + pt.off + (int64_t)z * X * Y;
    {   // ghost cells of the plane, as fill_grid_kernel
        const int nfull = zghost ? X * Y : 2 * gy * X;
        const int ncnt = zghost ? X * Y : nfull + pt.ny * 2 * gx;
        auto coord = [&](int k, int& x, int& y) {
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
        };
        constexpr int NC = 4;
        for (int k0 = threadIdx.x; k0 < ncnt; k0 += NC * blockDim.x) {
            const R* src[NC];
            R* dst[NC];
            bool on[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = k0 + c * blockDim.x;
                on[c] = k < ncnt;
                int x = 0, y = 0;
                if (on[c]) coord(k, x, y);
                src[c] = U + neighbour_source(pt, nb, on[c] ? x - gx : 0, on[c] ? y - gy : 0, iz);
                dst[c] = plane + (int64_t)y * X + x;
            }
            R v[NC][8];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int q = 0; q < 8; ++q) v[c][q] = on[c] ? src[c][q * vol] : R(0);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (on[c]) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[c][q * vol] = v[c][q];
                }
        }
    }
    __syncthreads();   // the plane's ghost faces are in place
    R vmax = R(0);
    bool bad = false;
    if (!zghost) {
        const bool top = iz + 1 == pt.nz;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        // each warp takes RR rows at a time, every load of the RR cells before the rates
        constexpr int RR = 4;
        for (int y0 = wid * RR; y0 < pt.ny; y0 += nw * RR) {
            for (int x = lane; x < pt.nx; x += 32) {
                R u[RR][8], bxh[RR], byh[RR], bzh[RR];
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int yy = min(y0 + r, pt.ny - 1);
                    const R* c = plane + (int64_t)(yy + gy) * X + gx + x;
#pragma unroll
                    for (int v = 0; v < 8; ++v) u[r][v] = c[v * vol];
                    bxh[r] = c[5 * vol + 1];
                    byh[r] = act1 ? c[6 * vol + X] : R(0);
                    bzh[r] = R(0);
                    if (act2)
                        bzh[r] = top ? U[7 * vol + neighbour_source(pt, nb, x, yy, pt.nz)] : c[7 * vol + (int64_t)X * Y];
                }
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    if (y0 + r >= pt.ny) continue;
                    const R rate = cell_rate_vals(u[r], bxh[r], byh[r], bzh[r], act1 != 0, act2 != 0, gamma, gm1, dxi0,
                                                  dxi1, dxi2);
                    if (!finite_(rate)) bad = true;
                    else vmax = rate > vmax ? rate : vmax;
                }
            }
        }
    }
    if (bad) atomicOr(err, ERR_PHYS);
    const R bm = block_max(vmax, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = bm;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        R v = R(0);
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
            const R w = ((volatile R*)partial)[k];
            v = w > v ? w : v;
        }
        __syncthreads();
        v = block_max(v, red);
        if (threadIdx.x == 0) {
            *dt_out = courant / (double)v;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// a1 + a2 fused, with the interior staged through shared memory, for regular grids whose
// plane fits (the ghost values and the dt of fill_cfl_grid_kernel, bitwise).  One CTA per
// padded z-plane of a patch.  An interior plane brings the rows of its own plane that hold
// interior cells (rows gy .. gy+ny-1 of each variable, rounded out to 16-byte bounds: one
// contiguous block per variable) and the same rows of B_z in the plane above (the cells'
// high z-faces) into shared memory with bulk copies (TMA) on an mbarrier, and the high x-
// and y-faces of its last column and row, and for the top interior plane the high z-faces
// from the neighbour above, with element copies (cp.async).  While those are in
// flight, every thread copies its ghost cells of the plane through registers, three cells
// (FP64: one) at a time with all their loads before their stores, the sources found from
// the patch's 27 neighbour offsets held in shared memory; a z-ghost plane only copies
// ghost cells.
// Then the CTA waits once (each thread for its element copies, one thread on the mbarrier,
// then a barrier) and takes the rates of its interior cells from shared memory.  Ghost
// sources are interior cells and destinations ghost cells, and the staged rows are
// interior cells and the high faces, which no CTA writes, so nothing read here is written
// by the launch.
// The wait on the bulk copies is bounded (one second of %globaltimer; the waiting thread
// is suspended between polls): past it the CTA sets ERR_TIMEOUT, waits once more
// (bounded) for its copies, skips the rates and reports an infinite rate, so the launch
// still completes and the dt is not a valid one.
// Dynamic shared memory, in elements: PL[8][r1 - r0] PZ[r1 - r0] FX[ny] FY[nx]
// (fill_cfl_staged_smem).  Rows whose address or byte size, or a plane whose X*Y reals,
// are not a multiple of 16 bytes (no bulk copy) are brought in with element copies of the
// interior cells instead.
// ---------------------------------------------------------------------------------------

// elements [r0, r1) of a padded plane staged for the rates: rows gy .. gy+ny-1 rounded out
// to 16-byte bounds (within the plane)
template <typename R>
__host__ __device__ inline void fill_cfl_staged_rows(int X, int Y, int ny, int gy, int& r0, int& r1) {
    constexpr int EQ = 16 / (int)sizeof(R);
    r0 = (gy * X) / EQ * EQ;
    r1 = ((gy + ny) * X + EQ - 1) / EQ * EQ;
    if (r1 > X * Y) r1 = X * Y;
}

template <typename R>
__host__ __device__ inline size_t fill_cfl_staged_smem(int X, int Y, int nx, int ny, int gx, int gy) {
    (void)gx;
    int r0, r1;
    fill_cfl_staged_rows<R>(X, Y, ny, gy, r0, r1);
    return ((size_t)9 * (r1 - r0) + ny + nx) * sizeof(R);
}
// planes whose staging needs more than this take fill_cfl_grid_kernel (two CTAs per SM fit)
constexpr size_t FILL_CFL_STAGED_MAX_SMEM = 113 * 1024;

template <typename R>
inline bool fill_cfl_staged_fits(const PatchDev& h0) {
    return fill_cfl_staged_smem<R>(h0.X, h0.Y, h0.nx, h0.ny, h0.gx, h0.gy) <= FILL_CFL_STAGED_MAX_SMEM;
}

template <typename R>
__device__ __forceinline__ void cp_async_elem_aux(R* smem_dst, const R* gsrc) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// phase 0 of the mbarrier at bar completed within limit_ns (false: gave up); between polls
// the thread is suspended (up to 20 us, or until the phase completes)
__device__ __forceinline__ bool mbar_wait0(unsigned bar, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(20000u)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// (x, y) of the items k = k0, k0 + S, k0 + 2S, ... of a row-major index space of rows w
// wide, stepped without a division per item (one division per thread at the start)
struct Walk2 {
    int x, y, sx, sy, w;
    __device__ __forceinline__ Walk2(int k0, int w_, int S) : w(w_) {
        y = k0 / w;
        x = k0 - y * w;
        sy = S / w;
        sx = S - sy * w;
    }
    __device__ __forceinline__ void next() {
        x += sx;
        y += sy;
        if (x >= w) {
            x -= w;
            ++y;
        }
    }
};

template <typename R>
__global__ void __launch_bounds__(256, 4) fill_cfl_staged_kernel(R* __restrict__ U, const PatchDev* __restrict__ patches,
                                                             const int64_t* __restrict__ nboff, int Zp, R gamma, R gm1,
                                                             double courant, R dxi0, R dxi1, R dxi2, int act1,
                                                             int act2, R* partial, unsigned* counter, double* dt_out,
                                                             unsigned* err) {
    extern __shared__ __align__(128) unsigned char fc_smem[];
    __shared__ R red[32];
    __shared__ bool last;
    __shared__ int s_ok;
    __shared__ int64_t s_nb[27];
    __shared__ __align__(8) uint64_t bar_mem;
    const int p = blockIdx.x / Zp, z = blockIdx.x - p * Zp;
    const PatchDev pt = patches[p];
    const int X = pt.X, Y = pt.Y, gx = pt.gx, gy = pt.gy, nx = pt.nx, ny = pt.ny;
    const int XY = X * Y;
    const int64_t vol = (int64_t)XY * pt.Z;
    const int iz = z - pt.gz;
    const bool zghost = iz < 0 || iz >= pt.nz;
    const int nfull = zghost ? XY : 2 * gy * X;
    const int nin = nx * ny;
    R* plane = U + pt.off + (int64_t)z * XY;
    int r0, r1;
    fill_cfl_staged_rows<R>(X, Y, ny, gy, r0, r1);
    const int NR = r1 - r0;
    R* PL = reinterpret_cast<R*>(fc_smem);   // PL[q * NR + c - r0]: element c of variable q's plane
    R* PZ = PL + 8 * NR;   // PZ[c - r0]: the high z-face of the cell at c (B_z of the plane above)
    R* FX = PZ + NR;
    R* FY = FX + ny;
    const unsigned bar = static_cast<unsigned>(__cvta_generic_to_shared(&bar_mem));
    // the patch's neighbour offsets, read once per CTA
    if (threadIdx.x < 27) s_nb[threadIdx.x] = nboff[(int64_t)p * 27 + threadIdx.x];
    const bool bulk = !zghost && ((reinterpret_cast<uintptr_t>(plane + r0) | ((size_t)NR * sizeof(R)) |
                                   ((size_t)XY * sizeof(R))) & 15) == 0;
    if (bulk && threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    // 1. the staged rows and high faces in flight (below the top interior plane the high
    // z-faces are variable 7 of the next plane's staged rows: a ninth bulk copy)
    const bool top = iz + 1 == pt.nz;
    const int nbulk = (act2 && !top) ? 9 : 8;
    if (bulk) {
        if (threadIdx.x == 0) {
            const unsigned bytes = (unsigned)(NR * sizeof(R));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(nbulk * bytes)
                         : "memory");
#pragma unroll 1
            for (int q = 0; q < nbulk; ++q) {
                const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(PL + q * NR));
                const R* src = q < 8 ? plane + q * vol + r0 : plane + 7 * vol + XY + r0;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
                    "l"(src), "r"(bytes), "r"(bar)
                    : "memory");
            }
        }
    } else if (!zghost) {
        Walk2 w(threadIdx.x, nx, blockDim.x);
        for (int k = threadIdx.x; k < nin; k += blockDim.x, w.next()) {
            const int c = (w.y + gy) * X + w.x + gx;
#pragma unroll
            for (int q = 0; q < 8; ++q) cp_async_elem_aux(PL + q * NR + c - r0, plane + q * vol + c);
            if (act2 && !top) cp_async_elem_aux(PZ + c - r0, plane + 7 * vol + XY + c);
        }
    }
    if (!zghost) {
        if (act2 && top) {
            Walk2 w(threadIdx.x, nx, blockDim.x);
            for (int k = threadIdx.x; k < nin; k += blockDim.x, w.next())
                cp_async_elem_aux(PZ + (w.y + gy) * X + w.x + gx - r0,
                                  U + 7 * vol + neighbour_source(pt, s_nb, w.x, w.y, pt.nz));
        }
        for (int k = threadIdx.x; k < ny + nx; k += blockDim.x) {
            if (k < ny) cp_async_elem_aux(FX + k, U + 5 * vol + neighbour_source(pt, s_nb, nx, k, iz));
            else if (act1) cp_async_elem_aux(FY + (k - ny), U + 6 * vol + neighbour_source(pt, s_nb, k - ny, ny, iz));
        }
    }
    // 2. the ghost cells of the plane through registers, NC per thread at a time (index k
    // over the full rows, then the x-ghost runs of the interior rows), all loads of a group
    // before its stores
    {
        constexpr int NC = sizeof(R) == 4 ? 3 : 1;
        const int ncnt = zghost ? XY : nfull + ny * 2 * gx;
        for (int k0 = threadIdx.x; k0 < ncnt; k0 += NC * blockDim.x) {
            R v[NC][8];
            R* dst[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = k0 + c * (int)blockDim.x;
                dst[c] = nullptr;
                if (k < ncnt) {
                    int x, y;
                    if (k < nfull) {
                        const int r = k / X;
                        x = k - r * X;
                        y = zghost ? r : (r < gy ? r : ny + r);
                    } else {
                        const int k2 = k - nfull;
                        const int r = k2 / (2 * gx), cc = k2 - r * (2 * gx);
                        y = gy + r;
                        x = cc < gx ? cc : nx + cc;
                    }
                    const R* src = U + neighbour_source(pt, s_nb, x - gx, y - gy, iz);
                    dst[c] = plane + y * X + x;
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[c][q] = src[q * vol];
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (dst[c]) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[c][q * vol] = v[c][q];
                }
        }
    }
    // 3. one wait: each thread for its element copies, thread 0 for the bulk copies (the
    // barrier then publishes both)
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (threadIdx.x == 0) s_ok = bulk ? (int)mbar_wait0(bar, 1000000000ull) : 1;
    __syncthreads();
    R vmax = R(0);
    bool bad = false;
    if (!s_ok) {
        // copies that did not land in time: wait once more (bounded) so that none is still
        // writing this CTA's shared memory when it exits, and report
        if (threadIdx.x == 0) {
            mbar_wait0(bar, 1000000000ull);
            atomicOr(err, ERR_TIMEOUT);
        }
        vmax = R(INFINITY);
    } else if (!zghost) {
        // 4. the rates of the interior cells
        Walk2 w(threadIdx.x, nx, blockDim.x);
        for (int k = threadIdx.x; k < nin; k += blockDim.x, w.next()) {
            const int y = w.y, x = w.x;
            const int c = (y + gy) * X + x + gx - r0;
            R u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) u[q] = PL[q * NR + c];
            const R bxh = x + 1 < nx ? PL[5 * NR + c + 1] : FX[y];
            const R byh = act1 ? (y + 1 < ny ? PL[6 * NR + c + X] : FY[x]) : R(0);
            const R bzh = act2 ? PZ[c] : R(0);
            const R rate = cell_rate_vals(u, bxh, byh, bzh, act1 != 0, act2 != 0, gamma, gm1, dxi0, dxi1, dxi2);
            if (!finite_(rate)) bad = true;
            else vmax = rate > vmax ? rate : vmax;
        }
    }
    if (bad) atomicOr(err, ERR_PHYS);
    const R bm = block_max(vmax, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = bm;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        R v = R(0);
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
            const R w = ((volatile R*)partial)[k];
            v = w > v ? w : v;
        }
        __syncthreads();
        v = block_max(v, red);
        if (threadIdx.x == 0) {
            *dt_out = courant / (double)v;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Asynchronous stepping (patches at their own times, two time slices each: the current one
// in buffer slice[p] of (U0, U1), the previous one in the other).
// ---------------------------------------------------------------------------------------

// a1 at each listed patch's own time t_cur[p]: a ghost cell takes the value of the box cell
// it stands for (owner map, wrap / clamp as fill_kernel) interpolated linearly in time
// between the owner's two slices, w = (t_cur[p] - t_old[q]) / (t_cur[q] - t_old[q]); w >= 1
// (or equal slice times) takes the current slice exactly, w <= 0 the previous one.
template <typename R>
__global__ void fill_interp_kernel(R* __restrict__ U0, R* __restrict__ U1, const PatchDev* __restrict__ patches,
                                   int npatch, const int* __restrict__ list, int nlist, const int* nlist_dev,
                                   const int* __restrict__ slice, const double* __restrict__ t_old,
                                   const double* __restrict__ t_cur, FillGeom fg, unsigned* err) {
    const int nl = nlist_dev ? min(*nlist_dev, nlist) : nlist;
    for (int L = blockIdx.y; L < nl; L += gridDim.y) {
        const int p = list[L];
        const PatchDev pt = patches[p];
        const int ng = ghost_count(pt);
        const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
        R* Up = (slice[p] ? U1 : U0) + pt.off;
        const double tp = t_cur[p];
        // two ghost cells per thread and pass, both slices of both sources loaded before
        // the stores
        constexpr int NC = 2;
        const int stride = gridDim.x * blockDim.x;
        for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < ng; k0 += NC * stride) {
            const R* cur[NC];
            const R* old[NC];
            R* d[NC];
            int64_t svol[NC];
            double w[NC];
            bool on[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = k0 + c * stride;
                on[c] = k < ng;
                cur[c] = old[c] = U0;
                d[c] = Up;
                svol[c] = 0;
                w[c] = 1.0;
                if (!on[c]) continue;
                int x, y, z;
                ghost_coord(pt, k, x, y, z);
                const int gxg = wrap_axis(pt.ox + x - pt.gx, fg.N[0], fg.bc[0][0], fg.bc[0][1]);
                const int gyg = wrap_axis(pt.oy + y - pt.gy, fg.N[1], fg.bc[1][0], fg.bc[1][1]);
                const int gzg = wrap_axis(pt.oz + z - pt.gz, fg.N[2], fg.bc[2][0], fg.bc[2][1]);
                const int ow = fg.owner[((gzg / fg.bs[2]) * fg.M[1] + gyg / fg.bs[1]) * fg.M[0] + gxg / fg.bs[0]];
                if (ow < 0 || ow >= npatch) {
                    atomicOr(err, ERR_BOUNDS);
                    on[c] = false;
                    continue;
                }
                const PatchDev src = patches[ow];
                const int64_t so = src.off +
                                   ((int64_t)(gzg - src.oz + src.gz) * src.Y + (gyg - src.oy + src.gy)) * src.X +
                                   (gxg - src.ox + src.gx);
                svol[c] = (int64_t)src.X * src.Y * src.Z;
                cur[c] = (slice[ow] ? U1 : U0) + so;
                old[c] = (slice[ow] ? U0 : U1) + so;
                const double den = t_cur[ow] - t_old[ow];
                w[c] = den > 0.0 ? (tp - t_old[ow]) / den : 1.0;
                d[c] = Up + ((int64_t)z * pt.Y + y) * pt.X + x;
            }
            R vc[NC][8], vo[NC][8];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    vc[c][q] = on[c] ? cur[c][q * svol[c]] : R(0);
                    vo[c][q] = on[c] ? old[c][q * svol[c]] : R(0);
                }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (!on[c]) continue;
                const R wr = R(w[c]);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const R o = vo[c][q];
                    d[c][q * vol] = w[c] >= 1.0 ? vc[c][q] : (w[c] <= 0.0 ? o : o + wr * (vc[c][q] - o));
                }
            }
        }
    }
}

// The same for equal patches on a regular grid: sources from the neighbour table (as
// fill_grid_kernel; the patch owning a source is its state offset over pstride, the state
// stride of one patch, the patches being stored back to back), one CTA per padded z-plane of
// a listed patch (blockIdx.x = plane), four ghost cells per thread and pass with both slices
// of their sources loaded before the stores; the same values as fill_interp_kernel.
template <typename R>
__global__ void __launch_bounds__(128) fill_interp_grid_kernel(R* __restrict__ U0, R* __restrict__ U1,
                                                              const PatchDev* __restrict__ patches,
                                                              const int64_t* __restrict__ nboff,
                                                              const int* __restrict__ list, int nlist,
                                                              const int* nlist_dev, int64_t pstride,
                                                              const int* __restrict__ slice,
                                                              const double* __restrict__ t_old,
                                                              const double* __restrict__ t_cur) {
    __shared__ double s_w[27];   // time weight of the slices of the patch in each direction
    __shared__ int s_sq[27];     // its current slice
    const int nl = nlist_dev ? min(*nlist_dev, nlist) : nlist;
    const int z = blockIdx.x;
    for (int L = blockIdx.y; L < nl; L += gridDim.y) {
        const int p = list[L];
        const PatchDev pt = patches[p];
        if (z >= pt.Z) continue;
        const int64_t* nb = nboff + (int64_t)p * 27;
        // the weight depends on the source patch only: once per direction, not per ghost cell
        // (an FP64 division per cell kept the small FP64 pipe busy)
        __syncthreads();
        if (threadIdx.x < 27) {
            const int q = (int)(nb[threadIdx.x] / pstride);
            const double den = t_cur[q] - t_old[q];
            s_w[threadIdx.x] = den > 0.0 ? (t_cur[p] - t_old[q]) / den : 1.0;
            s_sq[threadIdx.x] = slice[q];
        }
        __syncthreads();
        const int X = pt.X, Y = pt.Y, gx = pt.gx, gy = pt.gy;
        const int64_t vol = (int64_t)X * Y * pt.Z;
        const int iz = z - pt.gz;
        const bool zghost = iz < 0 || iz >= pt.nz;
        const int nfull = zghost ? X * Y : 2 * gy * X;
        const int ncnt = zghost ? X * Y : nfull + pt.ny * 2 * gx;
        R* plane = (slice[p] ? U1 : U0) + pt.off + (int64_t)z * X * Y;
        constexpr int NC = 4;
        for (int k0 = threadIdx.x; k0 < ncnt; k0 += NC * blockDim.x) {
            int64_t so[NC];
            int64_t dof[NC];
            double w[NC];
            int sq[NC];
            bool on[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = k0 + c * blockDim.x;
                on[c] = k < ncnt;
                int x = 0, y = 0;
                if (on[c]) {
                    if (k < nfull) {
                        const int r = k / X;
                        x = k - r * X;
                        y = zghost ? r : (r < gy ? r : pt.ny + r);
                    } else {
                        const int k2 = k - nfull;
                        const int r = k2 / (2 * gx), cc = k2 - r * (2 * gx);
                        y = gy + r;
                        x = cc < gx ? cc : pt.nx + cc;
                    }
                }
                int dir;
                so[c] = neighbour_source_dir(pt, nb, on[c] ? x - gx : 0, on[c] ? y - gy : 0, on[c] ? iz : 0, dir);
                sq[c] = s_sq[dir];
                w[c] = s_w[dir];
                dof[c] = (int64_t)y * X + x;
            }
            R vc[NC][8], vo[NC][8];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const R* cur = (sq[c] ? U1 : U0) + so[c];
                const R* old = (sq[c] ? U0 : U1) + so[c];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    vc[c][v] = on[c] ? cur[v * vol] : R(0);
                    vo[c][v] = on[c] ? old[v * vol] : R(0);
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (!on[c]) continue;
                const R wr = R(w[c]);
                R* d = plane + dof[c];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const R o = vo[c][v];
                    d[v * vol] = w[c] >= 1.0 ? vc[c][v] : (w[c] <= 0.0 ? o : o + wr * (vc[c][v] - o));
                }
            }
        }
    }
}

// a2 per listed patch: the maximum CFL rate over the patch's interior cells of its current
// slice, as the bit pattern of a non-negative double in rate_max[p] (zeroed beforehand;
// blocks along x share a patch and combine with an integer atomic max, which orders
// non-negative doubles as their values, so the result is exact and order independent).
// The dt, courant / max rate, is taken by the asynchronous scheduler.  Non-finite rates
// set ERR_PHYS and are left out of the maximum.
template <typename R>
__global__ void cfl_patch_kernel(const R* __restrict__ U0, const R* __restrict__ U1,
                                 const PatchDev* __restrict__ patches, const int* __restrict__ list, int nlist,
                                 const int* nlist_dev, const int* __restrict__ slice, double gamma_d, double dxi0_d,
                                 double dxi1_d, double dxi2_d, int act1, int act2, unsigned long long* rate_max,
                                 unsigned* err) {
    __shared__ R red[32];
    const int nl = nlist_dev ? min(*nlist_dev, nlist) : nlist;
    const R gamma = R(gamma_d), gm1 = R(gamma_d - 1.0);
    const R dxi0 = R(dxi0_d), dxi1 = R(dxi1_d), dxi2 = R(dxi2_d);
    for (int L = blockIdx.y; L < nl; L += gridDim.y) {
        const int p = list[L];
        const PatchDev pt = patches[p];
        const int n = pt.nx * pt.ny * pt.nz;
        const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
        const R* base = (slice[p] ? U1 : U0) + pt.off;
        R vmax = R(0);
        bool bad = false;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const int x = k % pt.nx + pt.gx, y = (k / pt.nx) % pt.ny + pt.gy, z = k / (pt.nx * pt.ny) + pt.gz;
            const R* c = base + ((int64_t)z * pt.Y + y) * pt.X + x;
            const R rate = cell_rate(c, vol, pt.X, pt.X * pt.Y, act1 != 0, act2 != 0, gamma, gm1, dxi0, dxi1, dxi2);
            if (!finite_(rate)) bad = true;
            else vmax = rate > vmax ? rate : vmax;
        }
        if (bad) atomicOr(err, ERR_PHYS);
        const R bm = block_max(vmax, red);
        if (threadIdx.x == 0 && bm > R(0))
            atomicMax(&rate_max[p], (unsigned long long)__double_as_longlong((double)bm));
        __syncthreads();
    }
}

}  // namespace mhd
