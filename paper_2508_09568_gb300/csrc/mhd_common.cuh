// Shared device-side types of the MHD bunch library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mhd {

// Device patch-table entry (one per patch, 64 bytes).
struct PatchDev {
    int64_t off;          // element offset of the patch in the state buffer
    int nx, ny, nz;       // active cells
    int X, Y, Z;          // padded extents (active + 2 * ghost on active axes)
    int gx, gy, gz;       // ghost widths
    int ox, oy, oz;       // global index of the first active cell
    int clamp;            // bit 2d / 2d+1: the patch's low / high side on axis d is an outflow box face
};

// Source of a ghost cell for bunches of equal patches on a regular grid: element offset in
// the state of the box cell standing at interior-relative coordinates (ix, iy, iz) of patch
// pt (at most one patch extent outside it on each axis), i.e. the cell the guard fill
// copies: in the neighbouring patch (nb[27]: element offsets of the 27 neighbours,
// direction (sx, sy, sz) at (sz+1)*9 + (sy+1)*3 + sx+1, periodic wrap applied), or the
// nearest cell of the patch itself across an outflow box face (zero gradient).
// (dir receives the table index (sz+1)*9 + (sy+1)*3 + sx+1 of the patch holding the source)
__device__ __forceinline__ int64_t neighbour_source_dir(const PatchDev& pt, const int64_t* __restrict__ nb, int ix,
                                                        int iy, int iz, int& dir) {
    int sx = 0, sy = 0, sz = 0;
    if (ix < 0) {
        if (pt.clamp & 1) ix = 0;
        else { sx = -1; ix += pt.nx; }
    } else if (ix >= pt.nx) {
        if (pt.clamp & 2) ix = pt.nx - 1;
        else { sx = 1; ix -= pt.nx; }
    }
    if (iy < 0) {
        if (pt.clamp & 4) iy = 0;
        else { sy = -1; iy += pt.ny; }
    } else if (iy >= pt.ny) {
        if (pt.clamp & 8) iy = pt.ny - 1;
        else { sy = 1; iy -= pt.ny; }
    }
    if (iz < 0) {
        if (pt.clamp & 16) iz = 0;
        else { sz = -1; iz += pt.nz; }
    } else if (iz >= pt.nz) {
        if (pt.clamp & 32) iz = pt.nz - 1;
        else { sz = 1; iz -= pt.nz; }
    }
    dir = (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
    return nb[dir] + ((int64_t)(iz + pt.gz) * pt.Y + (iy + pt.gy)) * pt.X + (ix + pt.gx);
}
__device__ __forceinline__ int64_t neighbour_source(const PatchDev& pt, const int64_t* __restrict__ nb, int ix,
                                                    int iy, int iz) {
    int dir;
    return neighbour_source_dir(pt, nb, ix, iy, iz, dir);
}

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
