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
// (wpr words per real).  Block (z, p - p0): one interior z-plane of one patch.  Each warp
// copies kRows x-rows of nx reals at a time, all loads issued before the stores, so that
// enough bytes are in flight for HBM rather than one row's latency per step.
constexpr int kXferRows = 8;

__global__ void __launch_bounds__(256, 4) interior_copy_kernel(unsigned* __restrict__ state,
                                                                unsigned* __restrict__ interior,
                                                                const PatchDev* __restrict__ patches,
                                                                const int64_t* __restrict__ ioff, int p0, int p1,
                                                                int wpr, int to_padded) {
    const int p = p0 + (int)blockIdx.y;
    if (p >= p1) return;
    const PatchDev pt = patches[p];
    const int z = blockIdx.x;
    if (z >= pt.nz) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int vol = pt.X * pt.Y * pt.Z;   // a patch's offsets (words) fit in 32 bits
    const int rowlen = pt.nx * wpr;
    const int nrow = 8 * pt.ny;
    unsigned* sp = state + pt.off * wpr;          // this patch in the state layout
    unsigned* ip = interior + ioff[p] * wpr;      // this patch in the interior layout
    const unsigned* src = to_padded ? ip : sp;
    unsigned* dst = to_padded ? sp : ip;
    for (int r0 = warp * kXferRows; r0 < nrow; r0 += nwarp * kXferRows) {
        int so[kXferRows], io[kXferRows];
#pragma unroll
        for (int u = 0; u < kXferRows; ++u) {
            const int r = min(r0 + u, nrow - 1);
            const int v = r / pt.ny, y = r - v * pt.ny;
            so[u] = (v * vol + ((z + pt.gz) * pt.Y + (y + pt.gy)) * pt.X + pt.gx) * wpr;
            io[u] = ((v * pt.nz + z) * pt.ny + y) * pt.nx * wpr;
        }
        for (int k = lane; k < rowlen; k += 32) {
            unsigned w[kXferRows];
#pragma unroll
            for (int u = 0; u < kXferRows; ++u)
                if (r0 + u < nrow) w[u] = src[(to_padded ? io[u] : so[u]) + k];
#pragma unroll
            for (int u = 0; u < kXferRows; ++u)
                if (r0 + u < nrow) dst[(to_padded ? so[u] : io[u]) + k] = w[u];
        }
    }
}

}  // namespace mhd
