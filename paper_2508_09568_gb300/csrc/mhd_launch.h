// Host-side launch table of the per-precision kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <new>
#include <stdexcept>
#include <string>

#include "mhd_common.cuh"

// Catch clauses of every C entry point (a function-try-block; the translation unit defines
// fail(code, message)): no exception crosses the ABI; host allocation failures become
// MHD_ENOMEM, anything else MHD_EINVAL with its text.
#define MHD_CATCH_ALL                                                                         \
    catch (const std::bad_alloc&) {                                                           \
        return fail(MHD_ENOMEM, "host memory allocation failed");                             \
    }                                                                                         \
    catch (const std::length_error&) {                                                        \
        return fail(MHD_ENOMEM, "host allocation too large");                                 \
    }                                                                                         \
    catch (const std::exception& e_) {                                                        \
        return fail(MHD_EINVAL, std::string("internal error: ") + e_.what());                 \
    }                                                                                         \
    catch (...) {                                                                             \
        return fail(MHD_EINVAL, "internal error");                                            \
    }

namespace mhd {

// One compiled configuration of the fused step kernel.
struct StepLaunch {
    int ndim, tx, ty, nt;
    size_t smem;
    cudaError_t (*prepare)();                                   // opt in to large smem
    cudaError_t (*occupancy)(int* blocks_per_sm);
    cudaError_t (*launch)(const void* args, int grid, cudaStream_t s);
};

// arguments of the adjoint step (see mhd_adjoint.cuh), precision independent
struct AdjHostArgs {
    void* U;             // scratch copy of U^n (ghosts filled here)
    const void* lam_next;
    void* lam;
    void* F;             // forward work fields
    void* G;             // cotangent work fields
    int64_t ncell;
    const PatchDev* patches;
    int npatch;
    int max_cells;       // largest padded patch
    double gamma, eps, dt;
    double dxi[3];
    int limiter;
    int riemann;
    const int64_t* nboff;    // regular grids: neighbour table (table-driven fill and transpose), else null
    int Zp;                  // padded z extent (regular grids)
};

// Kernel entry points of one precision (R = float or double).
struct PrecisionKernels {
    const StepLaunch* step;
    int nstep;
    // nboff: neighbour table of a regular grid of equal patches of Zp padded z-planes
    // (table-driven fill), or null (owner-map fill)
    cudaError_t (*fill)(void* U, const PatchDev* patches, int npatch, const FillGeom& fg, const int64_t* nboff,
                        int Zp, unsigned* err, cudaStream_t s);
    // partial: at least cfl_grid reals; counter: one zeroed unsigned
    cudaError_t (*cfl)(const void* U, const PatchDev* patches, int npatch, double gamma, double courant,
                       const double dxi[3], const int act[3], void* partial, int grid, unsigned* counter,
                       double* dt_out, unsigned* err, cudaStream_t s);
    // the whole adjoint kernel sequence (fill of the U copy, forward recompute, reverse);
    // G must be zeroed before the call
    cudaError_t (*adjoint)(const AdjHostArgs& a, const FillGeom& fg, unsigned* err, cudaStream_t s, int* nlaunch);
    int adj_fields;      // work fields per cell in F and in G
    // asynchronous stepping: guard fill of the listed patches at their own times, and
    // their maximum CFL rate (rate_max indexed by patch: the bits of a non-negative double,
    // zeroed beforehand).  The list holds nlist entries, or *nlist_dev (<= nlist) when
    // nlist_dev is not null; grid_y (> 0) caps the blocks along the list.  Regular grids:
    // nboff the neighbour table, Zp the padded z extent and pstride the state stride of one
    // patch (table-driven fill), else nboff null (owner map)
    cudaError_t (*fill_interp)(void* U0, void* U1, const PatchDev* patches, int npatch, const int* list, int nlist,
                               const int* nlist_dev, int grid_y, const int* slice, const double* t_old,
                               const double* t_cur, const FillGeom& fg, const int64_t* nboff, int Zp,
                               int64_t pstride, unsigned* err, cudaStream_t s);
    cudaError_t (*cfl_patch)(const void* U0, const void* U1, const PatchDev* patches, const int* list, int nlist,
                             const int* nlist_dev, int grid_y, const int* slice, double gamma, const double dxi[3],
                             const int act[3], unsigned long long* rate_max, unsigned* err, cudaStream_t s);
    // guard fill + CFL dt in one pass (regular grids: h0 a host copy of the patches' common
    // geometry, nboff the neighbour table, Zp the padded z extent); partial: npatch * Zp
    // reals; counter: one zeroed unsigned
    cudaError_t (*fill_cfl)(void* U, const PatchDev* patches, const PatchDev& h0, int npatch, const int64_t* nboff,
                            int Zp, double gamma, double courant, const double dxi[3], const int act[3], void* partial,
                            unsigned* counter, double* dt_out, unsigned* err, cudaStream_t s);
    cudaError_t (*prepare_fill_cfl)();   // opt the staged fill + CFL pass in to its shared memory
};

const PrecisionKernels& kernels_f32();
const PrecisionKernels& kernels_f64();

// arguments of the step kernel in a precision-independent form (converted per precision)
struct StepHostArgs {
    const void* U;
    void* Unew;
    const int* slice;        // asynchronous stepping (else null): current slice per patch
    const double* dt_patch;  // asynchronous stepping (else null): dt per patch
    const PatchDev* patches;
    const int4* tiles;
    int ntiles;
    const int* ntiles_dev;   // asynchronous stepping: tile count read on the device (<= ntiles), or null
    int dynamic;
    int* work;
    const double* dt_ptr;
    double dt_val;
    double gamma, eps;
    double dxi[3];
    int limiter;
    int riemann;
    unsigned* err;
};

}  // namespace mhd
