// Shared device-side types of the MHD bunch library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mhd {

// Device patch-table entry (one per patch, about 48 bytes).
struct PatchDev {
    int64_t off;          // element offset of the patch in the state buffer
    int nx, ny, nz;       // active cells
    int X, Y, Z;          // padded extents (active + 2 * ghost on active axes)
    int gx, gy, gz;       // ghost widths
    int ox, oy, oz;       // global index of the first active cell
    int pad;
};

// Geometry needed by the guard fill: box extent, boundary kinds and the owner map
// (a coarse grid of blocks of bs cells, each naming the patch that owns it).
struct FillGeom {
    int N[3];             // box cells
    int bc[3][2];         // boundary kinds
    int bs[3];            // owner-map block size
    int M[3];             // owner-map extent (N / bs)
    const int* owner;     // [M2][M1][M0]
};

// Device error word bits.
enum : unsigned { ERR_PHYS = 1u, ERR_BOUNDS = 2u, ERR_TIMEOUT = 4u };

}  // namespace mhd
