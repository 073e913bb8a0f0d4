// k_admm_roll.cu -- launch policy of the row-streaming ADMM kernel (k_admm_roll.cuh): strip
// height per level and storage-type dispatch.
#include <stdlib.h>

#include "k_admm_roll.cuh"

namespace tvl1 {

int admm_fused_strip_w() { return roll::SW; }
int admm_fused_warps() { return roll::WARPS; }

namespace {
// TVL1_ADMM_ROWS_PER_WARP=1|2|8|32 pins the strip height (read once; for tuning sweeps).
int forced_rows_per_warp() {
    static const int v = [] {
        const char *e = getenv("TVL1_ADMM_ROWS_PER_WARP");
        const int t = e ? atoi(e) : 0;
        return (t == 1 || t == 2 || t == 8 || t == 32) ? t : 0;
    }();
    return v;
}
}  // namespace

int admm_fused_rows_per_warp(long strip_rows) {
    // rows per warp: 32 (halo (32+3)/32) where that still gives about eight warps per SM (large
    // images, batches; these strips run register-capped at five blocks per SM), else 8 (halo
    // (8+3)/8) where that gives eight warps per SM; on smaller levels a warp's TY + 3 row steps are
    // the latency of the whole iteration, so there strips of two or one row trade redundant halo
    // work for a short chain.  (Measured: 32 beats 8 from 1280x960 up, 31.4 vs 32.9 us per
    // iteration at 1280x960 and 148 vs 196 us at 3840x2160; 8 wins at 640x480, 2 at 320x240.)
    if (const int f = forced_rows_per_warp()) return f;
    const long sms = 152;
    if (strip_rows / 32 >= 8L * sms) return 32;
    const int cand[3] = {8, 2, 1};
    for (int t : cand)
        if (strip_rows / t >= 8L * sms) return t;
    return 1;
}

int admm_fused_tile_h(Geom g) { return admm_fused_rows_per_warp((long)((g.W + roll::SW - 1) / roll::SW) * g.H); }

int admm_fused_blocks(Geom g, int ty) {
    const int th = ty > 0 ? ty : admm_fused_tile_h(g);
    return ((g.W + roll::SW - 1) / roll::SW) * ((g.H + th * roll::WARPS - 1) / (th * roll::WARPS));
}

void launch_admm_fused(const IterArgs &a, int prec, int prec_flow, cudaStream_t s) {
    const int ty = a.tile_h > 0 ? a.tile_h : admm_fused_tile_h(a.g);
    if (prec == PREC_F32) roll_launch_f32(a, ty, s);
    else if (prec == PREC_F16) roll_launch_f16(a, ty, prec_flow == PREC_F32, s);
    else roll_launch_bf16(a, ty, prec_flow == PREC_F32, s);
}

}  // namespace tvl1
