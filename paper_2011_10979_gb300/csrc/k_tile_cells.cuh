// k_tile_cells.cuh -- how the several-iterations tile kernels (k_admm_tile.cu, k_cp_tile.cu) deal
// the cells of a phase's square to their threads.
//
// A block owns a TT x TT output tile and stages an FS x FS frame (row pitch FS floats) whose cell
// 0 sits OFF pixels above and left of the tile's corner.  Each phase works on a square of tile
// offsets [LO, HI] (n = HI - LO + 1 >= TT cells a side).  32 consecutive cells of the square would
// straddle two of its rows, FS - n floats apart, and most warps would meet a two-way bank conflict
// on every shared-memory access.  Instead:
//  - 16-pixel tiles: lane t of the run covers frame offset t from the square's first cell, rows
//    counted at the frame pitch, so a warp's addresses are consecutive; the FS - n cells past each
//    row's end idle their lanes (over a 22-cell square with FS = 23, 16 wavefronts per access to a
//    plane against 31);
//  - 32-pixel tiles: a warp task is a whole row of the square's first 32 columns (consecutive
//    addresses) or a run of 32 cells of its remaining n - 32 columns, row by row (at most two-way
//    conflicts there).  Measured per ADMM iteration at 640x480: 6.72 us with consecutive cells of
//    the square, 5.48 pitch-wrapped, 5.41 with row tasks.
// The east, west, north and south neighbours of the cells a warp touches fall in the same number
// of banks as the cells themselves.
#pragma once

namespace tvl1 {

// Calls f(x, i, j) for the in-image cells of the square (x: frame index, (i, j): image pixel);
// (fi, fj) are the image coordinates of frame cell 0.
template <int TT, int FS, int OFF, int NT, int LO, int HI, typename F>
__device__ __forceinline__ void tile_cells(int fi, int fj, int H, int W, F &&f) {
    constexpr int n = HI - LO + 1, x0 = (LO + OFF) * (FS + 1);
    static_assert(n >= TT && LO + OFF >= 0 && HI + OFF < FS, "square inside the frame, no narrower than a tile");
    if constexpr (TT == 16) {
        for (int t = threadIdx.x; t < (n - 1) * FS + n; t += NT) {
            const int r = t / FS, c = t % FS;
            const int i = fi + LO + OFF + r, j = fj + LO + OFF + c;
            if (c < n && i >= 0 && i < H && j >= 0 && j < W) f(x0 + t, i, j);
        }
    } else {
        static_assert(TT == 32, "tile size");
        constexpr int M = n - TT, NTASK = n + (n * M + 31) / 32;
        const int lane = threadIdx.x & 31;
        for (int task = threadIdx.x >> 5; task < NTASK; task += NT / 32) {
            int r = task, c = lane;
            if constexpr (M > 0) {
                if (task >= n) {
                    const int q = (task - n) * 32 + lane;
                    if (q >= n * M) continue;
                    r = q / M;
                    c = TT + q % M;
                }
            }
            const int i = fi + LO + OFF + r, j = fj + LO + OFF + c;
            if (i >= 0 && i < H && j >= 0 && j < W) f(x0 + r * FS + c, i, j);
        }
    }
}

}  // namespace tvl1
