// Instantiation helpers shared by the per-precision translation units.
#pragma once

#include <algorithm>

#include "mhd_adjoint.cuh"
#include "mhd_aux.cuh"
#include "mhd_launch.h"
#include "mhd_step.cuh"

namespace mhd {

template <typename R>
static StepArgs<R> to_args(const StepHostArgs& h) {
    StepArgs<R> a;
    a.U = static_cast<const R*>(h.U);
    a.Unew = static_cast<R*>(h.Unew);
    a.slice = h.slice;
    a.dt_patch = h.dt_patch;
    a.patches = h.patches;
    a.tiles = h.tiles;
    a.ntiles = h.ntiles;
    a.ntiles_dev = h.ntiles_dev;
    a.dynamic = h.dynamic;
    a.work = h.work;
    a.dt_ptr = h.dt_ptr;
    a.dt_val = h.dt_val;
    a.gamma = h.gamma;
    a.eps = h.eps;
    for (int d = 0; d < 3; ++d) a.dxi[d] = h.dxi[d];
    a.limiter = h.limiter;
    a.riemann = h.riemann;
    a.err = h.err;
    return a;
}

template <typename R, int NDIM, int TX, int TY, int NT, int MINB = 1, bool PREFETCH = false>
struct StepInst {
    using C = StepCfg<R, NDIM, TX, TY, NT>;
    static_assert(C::SMEM_BYTES * MINB <= 227 * 1024, "tile too large for shared memory");
    static cudaError_t prepare() {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<R, NDIM, TX, TY, NT, MINB, PREFETCH, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(step_kernel<R, NDIM, TX, TY, NT, MINB, PREFETCH, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
    }
    static cudaError_t occupancy(int* blocks) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, step_kernel<R, NDIM, TX, TY, NT, MINB, PREFETCH, false>,
                                                             NT, C::SMEM_BYTES);
    }
    // asynchronous stepping (a.slice set) runs its own instantiation
    static cudaError_t launch(const void* args, int grid, cudaStream_t s) {
        const StepArgs<R> a = to_args<R>(*static_cast<const StepHostArgs*>(args));
        if (a.slice)
            step_kernel<R, NDIM, TX, TY, NT, MINB, PREFETCH, true><<<grid, NT, C::SMEM_BYTES, s>>>(a);
        else
            step_kernel<R, NDIM, TX, TY, NT, MINB, PREFETCH, false><<<grid, NT, C::SMEM_BYTES, s>>>(a);
        return cudaGetLastError();
    }
    static StepLaunch entry() {
        return StepLaunch{NDIM, C::TX, C::TY, NT, C::SMEM_BYTES, &prepare, &occupancy, &launch};
    }
};

template <typename R>
static cudaError_t launch_fill(void* U, const PatchDev* patches, int npatch, const FillGeom& fg,
                               const int64_t* nboff, int Zp, unsigned* err, cudaStream_t s) {
    if (nboff) {
        fill_grid_kernel<R><<<(unsigned)npatch * (unsigned)Zp, 128, 0, s>>>(static_cast<R*>(U), patches, nboff, Zp);
    } else {
        dim3 grid(8, npatch < 65535 ? npatch : 65535);
        fill_kernel<R><<<grid, 256, 0, s>>>(static_cast<R*>(U), patches, npatch, fg, err);
    }
    return cudaGetLastError();
}

template <typename R>
static cudaError_t prepare_fill_cfl() {
    return cudaFuncSetAttribute(fill_cfl_staged_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FILL_CFL_STAGED_MAX_SMEM);
}

// the staged pass where the plane fits its shared-memory cap, else the register version
template <typename R>
static cudaError_t launch_fill_cfl(void* U, const PatchDev* patches, const PatchDev& h0, int npatch,
                                  const int64_t* nboff, int Zp, double gamma, double courant, const double dxi[3],
                                  const int act[3], void* partial, unsigned* counter, double* dt_out, unsigned* err,
                                  cudaStream_t s) {
    const unsigned grid = (unsigned)npatch * (unsigned)Zp;
    const size_t smem = fill_cfl_staged_smem<R>(h0.X, h0.Y, h0.nx, h0.ny, h0.gx, h0.gy);
    // constants in the kernel's precision, rounded here once (as the kernel would round them)
    const R g = R(gamma), gm1 = R(gamma - 1.0), d0 = R(dxi[0]), d1 = R(dxi[1]), d2 = R(dxi[2]);
    if (fill_cfl_staged_fits<R>(h0))
        fill_cfl_staged_kernel<R><<<grid, 256, smem, s>>>(static_cast<R*>(U), patches, nboff, Zp, g, gm1, courant, d0,
                                                          d1, d2, act[1], act[2], static_cast<R*>(partial), counter,
                                                          dt_out, err);
    else
        fill_cfl_grid_kernel<R><<<grid, 128, 0, s>>>(static_cast<R*>(U), patches, nboff, Zp, g, gm1, courant, d0, d1,
                                                     d2, act[1], act[2], static_cast<R*>(partial), counter, dt_out,
                                                     err);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_fill_interp(void* U0, void* U1, const PatchDev* patches, int npatch, const int* list,
                                     int nlist, const int* nlist_dev, int grid_y, const int* slice,
                                     const double* t_old, const double* t_cur, const FillGeom& fg,
                                     const int64_t* nboff, int Zp, int64_t pstride, unsigned* err, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    const int gy = std::min(std::min(nlist, grid_y > 0 ? grid_y : nlist), 65535);
    if (nboff) {
        fill_interp_grid_kernel<R><<<dim3(Zp, gy), 128, 0, s>>>(static_cast<R*>(U0), static_cast<R*>(U1), patches,
                                                                 nboff, list, nlist, nlist_dev, pstride, slice, t_old,
                                                                 t_cur);
        return cudaGetLastError();
    }
    dim3 grid(32, gy);
    fill_interp_kernel<R><<<grid, 256, 0, s>>>(static_cast<R*>(U0), static_cast<R*>(U1), patches, npatch, list, nlist,
                                               nlist_dev, slice, t_old, t_cur, fg, err);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_cfl_patch(const void* U0, const void* U1, const PatchDev* patches, const int* list,
                                   int nlist, const int* nlist_dev, int grid_y, const int* slice, double gamma,
                                   const double dxi[3], const int act[3], unsigned long long* rate_max,
                                   unsigned* err, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    const int gy = std::min(std::min(nlist, grid_y > 0 ? grid_y : nlist), 65535);
    dim3 grid(16, gy);
    cfl_patch_kernel<R><<<grid, 256, 0, s>>>(static_cast<const R*>(U0), static_cast<const R*>(U1), patches, list,
                                             nlist, nlist_dev, slice, gamma, dxi[0], dxi[1], dxi[2], act[1], act[2],
                                             rate_max, err);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_cfl(const void* U, const PatchDev* patches, int npatch, double gamma, double courant,
                              const double dxi[3], const int act[3], void* partial, int grid, unsigned* counter,
                              double* dt_out, unsigned* err, cudaStream_t s) {
    CflArgs<R> a;
    a.U = static_cast<const R*>(U);
    a.patches = patches;
    a.npatch = npatch;
    a.gamma = gamma;
    a.courant = courant;
    for (int d = 0; d < 3; ++d) {
        a.dxi[d] = dxi[d];
        a.act[d] = act[d];
    }
    a.partial = static_cast<R*>(partial);
    a.counter = counter;
    a.dt_out = dt_out;
    a.err = err;
    cfl_kernel<R><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_adjoint(const AdjHostArgs& h, const FillGeom& fg, unsigned* err, cudaStream_t s,
                                  int* nlaunch) {
    AdjArgs<R> a;
    a.U = static_cast<const R*>(h.U);
    a.lam_next = static_cast<const R*>(h.lam_next);
    a.lam = static_cast<R*>(h.lam);
    a.F = static_cast<R*>(h.F);
    a.G = static_cast<R*>(h.G);
    a.ncell = h.ncell;
    a.patches = h.patches;
    a.npatch = h.npatch;
    a.gamma = h.gamma;
    a.eps = h.eps;
    a.dt = h.dt;
    for (int d = 0; d < 3; ++d) a.dxi[d] = h.dxi[d];
    a.limiter = h.limiter;
    a.riemann = h.riemann;
    // x-blocks per patch: 64, or (FP64, whose kernels are longer) enough for ~8 blocks per
    // SM on small bunches; never more than one thread per padded cell
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    const int bcap = (h.max_cells + 255) / 256;
    const int bwant = sizeof(R) == 8 ? std::max(64, (8 * sms + h.npatch - 1) / h.npatch) : 64;
    const int bx = std::max(1, std::min(bcap, bwant));
    const dim3 grid(bx, h.npatch < 65535 ? h.npatch : 65535), blk(256);
    const dim3 fgrid(bx, h.npatch < 65535 ? h.npatch : 65535);
    const unsigned pgrid = (unsigned)h.npatch * (unsigned)h.Zp;   // planes (regular grids)
    int n = 0;
    if (h.nboff)
        fill_grid_kernel<R><<<pgrid, 128, 0, s>>>(static_cast<R*>(h.U), h.patches, h.nboff, h.Zp);
    else
        fill_kernel<R><<<fgrid, 256, 0, s>>>(static_cast<R*>(h.U), h.patches, h.npatch, fg, err);
    ++n;
    adj_fwd_prim<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_fwd_slopes<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_fwd_en<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_fwd_bh<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_fwd_wh<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_init<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_faces<R><<<dim3(grid.x, grid.y, 3), blk, 0, s>>>(a); ++n;
    adj_edges<R><<<dim3(grid.x, grid.y, 3), blk, 0, s>>>(a); ++n;
    adj_pred<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_bh<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_en<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_slopes<R><<<grid, blk, 0, s>>>(a); ++n;
    adj_prim<R><<<grid, blk, 0, s>>>(a); ++n;
    if (h.nboff)
        adj_fill_transpose_grid<R><<<pgrid, 128, 0, s>>>(static_cast<R*>(h.lam), h.patches, h.nboff, h.Zp);
    else
        adj_fill_transpose<R><<<fgrid, 256, 0, s>>>(static_cast<R*>(h.lam), h.patches, h.npatch, fg, err);
    ++n;
    if (nlaunch) *nlaunch = n;
    return cudaGetLastError();
}

}  // namespace mhd
