// k_admm_roll.cu -- launch policy of the row-streaming ADMM kernel (k_admm_roll.cuh): strip
// height per level and storage-type dispatch.
#include "k_admm_roll.cuh"

namespace tvl1 {

int admm_fused_strip_w() { return roll::SW; }
int admm_fused_warps() { return roll::WARPS; }

int admm_fused_rows_per_warp(long strip_rows, bool storage16) {
    // rows per warp: 8 (halo (8+3)/8) where that still gives at least ten warps per SM; on smaller
    // levels a warp's TY + 3 row steps are the latency of the whole iteration, so there strips of
    // two rows (at least eight warps per SM) or one row trade redundant halo work for a short
    // chain.  With 16-bit storage, launches of at least 16 warps per SM even at 32 rows (batches,
    // very large images) take 32 (halo (32+3)/32, the register-capped kernel).  Measured per
    // iteration (FP32, single pairs): 320x240 4.0 us at 2 rows; 640x480 (9 warps per SM at 8 rows)
    // 7.98 at 2 against 8.27 at 8; 1024x436 (13 per SM) 10.7 at 2 against 9.7 at 8; 1280x960 24.3
    // at 8 vs 31.6 at 32; 3840x2160 143 vs 149; a 64-pair batch 288 vs 304 in FP32 but 331 vs 285
    // with BF16 duals.
    const long sms = 152;
    if (storage16 && strip_rows / 32 >= 16L * sms) return 32;
    if (strip_rows / 8 >= 10L * sms) return 8;
    if (strip_rows / 2 >= 8L * sms) return 2;
    return 1;
}

int admm_fused_tile_h(Geom g, bool storage16) {
    return admm_fused_rows_per_warp((long)((g.W + roll::SW - 1) / roll::SW) * g.H, storage16);
}

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
