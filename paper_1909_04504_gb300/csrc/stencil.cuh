// The cell stencil of the neighbour search (Sec. 2.2 uniform grid): cells no smaller than
// kh / R with R = 1 in 2D (3 x 3 stencil of cells of side >= kh) and R = 2 in 3D
// (5 x 5 x 5 stencil of cells of side >= kh / 2: the stencil volume shrinks from 27 to
// 15.6 (kh)^3, so fewer candidates per neighbour). A row of 2R + 1 cells along x is one
// contiguous run of the cell-sorted arrays.
#pragma once

#include "sph_device.cuh"

namespace sph {

template <int DIM>
struct Stencil {
    static constexpr int R = DIM == 3 ? 2 : 1;   // cells on each side
    static constexpr int RZ = DIM == 3 ? R : 0;
};

__device__ __forceinline__ void cell_of_key(const Grid& G, uint32_t key, int& cx, int& cy, int& cz) {
    cx = (int)(key % (uint32_t)G.nc[0]);
    const uint32_t r = key / (uint32_t)G.nc[0];
    cy = (int)(r % (uint32_t)G.nc[1]);
    cz = (int)(r / (uint32_t)G.nc[1]);
}

// Walks the stencil of cell (cx, cy, cz): rows (dz, dy) in order, and in each row the
// cells [cx - R, cx + R] as contiguous runs: body(jb, je) for each run (a periodic row that
// wraps gives its wrapped cells as separate runs, below-box part first, then above-box,
// then the in-box part).
template <int DIM, class Body>
__device__ __forceinline__ void for_each_run(const Grid& G, const uint32_t* __restrict__ off,
                                             int cx, int cy, int cz, Body body) {
    constexpr int R = Stencil<DIM>::R, RZ = Stencil<DIM>::RZ;
#pragma unroll 1
    for (int dz = -RZ; dz <= RZ; ++dz) {
        int z = cz + dz;
        if (DIM == 3 && (z < 0 || z >= G.nc[2])) {
            if (!G.periodic[2]) continue;
            z = z < 0 ? z + G.nc[2] : z - G.nc[2];
        }
#pragma unroll 1
        for (int dy = -R; dy <= R; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= G.nc[1]) {
                if (!G.periodic[1]) continue;
                y = y < 0 ? y + G.nc[1] : y - G.nc[1];
            }
            const int row = G.nc[0] * (y + G.nc[1] * z);
            int x0 = cx - R, x1 = cx + R;
            if (G.periodic[0]) {
                if (x0 < 0) { body(off[row + G.nc[0] + x0], off[row + G.nc[0]]); x0 = 0; }
                if (x1 >= G.nc[0]) { body(off[row], off[row + x1 - G.nc[0] + 1]); x1 = G.nc[0] - 1; }
            } else {
                if (x0 < 0) x0 = 0;
                if (x1 >= G.nc[0]) x1 = G.nc[0] - 1;
            }
            body(off[row + x0], off[row + x1 + 1]);
        }
    }
}

}  // namespace sph
