// Interior layout for host transfers (mhd_bunch_advance_streamed_interior).
//
// The interior layout holds only the cells a patch owns: patch p starts at element
// ioff[p] and is stored as [8][nz][ny][nx], x fastest (the variables and face-field
// convention of the state layout, ghost cells left out).  It is what a caller keeps on
// the host: ghost cells are derived data, refilled on the device by the guard fill
// before every update, so a step's input and result are the interior alone.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mhd_common.cuh"

namespace mhd {

// Copies the interiors of patches [p0, p1) between the padded state and a buffer in the
// interior layout (to_padded: interior -> state, else state -> interior), as 4-byte words
// (wpr words per real).  Block (z, p - p0): one interior z-plane of one patch; each warp
// copies whole x-rows of nx reals, so both sides are read and written row by row.
__global__ void interior_copy_kernel(unsigned* __restrict__ state, unsigned* __restrict__ interior,
                                     const PatchDev* __restrict__ patches, const int64_t* __restrict__ ioff,
                                     int p0, int p1, int wpr, int to_padded) {
    const int p = p0 + (int)blockIdx.y;
    if (p >= p1) return;
    const PatchDev pt = patches[p];
    const int z = blockIdx.x;
    if (z >= pt.nz) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t vol = (int64_t)pt.X * pt.Y * pt.Z;
    const int rowlen = pt.nx * wpr;
    const int nrow = 8 * pt.ny;
    for (int r = warp; r < nrow; r += nwarp) {
        const int v = r / pt.ny, y = r - v * pt.ny;
        const int64_t s = (pt.off + v * vol + ((int64_t)(z + pt.gz) * pt.Y + (y + pt.gy)) * pt.X + pt.gx) * wpr;
        const int64_t c = (ioff[p] + ((int64_t)v * pt.nz + z) * pt.ny * pt.nx + (int64_t)y * pt.nx) * wpr;
        if (to_padded) {
            for (int k = lane; k < rowlen; k += 32) state[s + k] = interior[c + k];
        } else {
            for (int k = lane; k < rowlen; k += 32) interior[c + k] = state[s + k];
        }
    }
}

}  // namespace mhd
