// k_admm_roll.cuh -- fused engine of the ADMM inner iteration (Sec. 3.1.1), row-streaming form:
// one kernel per iteration of rpADMMI / pADMM (eq. rpADMMI), rpADMMII (eq. rpADMMII) or the
// beta = 0 model (eq. Zach-pADMM), reading one state buffer and writing the other.
//
// Each warp owns a strip of 32 consecutive columns and walks down TY + 3 rows of it.  Lane l holds
// column c0 + l; the 29 lanes 2..30 produce output, lanes 0, 1 and 31 supply the stencil halo
// (neighbouring strips overlap by 3 columns).
// The rows stream through registers: each lane keeps the two rows being finished and the two
// rows below them already in flight (loads issued two steps ahead; zeros outside the image), so a
// warp keeps 26 loads outstanding.  Per row step the warp
//   1. takes the next row of p1 p2 q11 q12 q21 q22 s Ix Iy It (storage T) and w u v (storage TF)
//      and issues the loads of the row two steps ahead;
//   2. forms div y^k on that row (west neighbours by shuffle, north from the previous step);
//   3. forms y^{k+1} = P[y^k + (1/a) grad(div y^k) + (1/a)(grad Lambda / c - grad(A s))] on the
//      row above (east neighbours by shuffle, south values from the new row);
//   4. on that row forms div y^{k+1} (west by shuffle, north from the step before),
//      s^{k+1} = P_s[...] with the old multipliers, Lambda^{k+1} and the squared constraint
//      residual, and stores the state.
// No block barrier: values move between lanes by shuffle and between rows in registers.  Every
// state element is read once and written once per iteration apart from the strip halo
// (32/29 in x, (TY+3)/TY in y), which hits L2.
// Batched form: warp w of block b works on the strip tiles[b] (pair, strip column, row group) of
// pair pairs[tiles[b].pair]; the single-pair form maps the grid onto one pair's strips.
//
// The templates are instantiated per storage type in k_admm_roll_{f32,f16,bf16}.cu so that the
// three translation units compile in parallel; the launch policy is in k_admm_roll.cu.
#pragma once
#include <math.h>

#include "k_admm_math.cuh"
#include "tvl1_device.cuh"

namespace tvl1 {

// Per storage type: launches k_admm_roll with TY rows per warp (TY in 1, 2, 8, 32).
void roll_launch_f32(const IterArgs &a, int ty, cudaStream_t s);
void roll_launch_f16(const IterArgs &a, int ty, bool flow32, cudaStream_t s);
void roll_launch_bf16(const IterArgs &a, int ty, bool flow32, cudaStream_t s);

namespace roll {

constexpr int WARPS = 4;          // warps per block, stacked vertically (one strip each)
constexpr int SW = 29;            // output columns per strip
constexpr unsigned FULL = 0xffffffffu;

// The values of one row at this lane's column.
struct Row {
    float p1, p2, q11, q12, q21, q22, s, w, u, v, ix, iy, it;
};

// Loads row i of this lane's column: src holds the planes p1 p2 q11 q12 q21 q22 s Ix Iy It
// (storage T) and w u v (storage TF); zeros outside the image.
template <typename T, typename TF, bool HAS_W, bool INT>
__device__ __forceinline__ void load_row(Row &R, const void *const *src, int i, int c, int H, int W, int P) {
    const bool ok = INT || (i >= 0 && i < H && c >= 0 && c < W);
    const size_t o = ok ? (size_t)i * P + c : 0;
    R.p1 = (HAS_W && ok) ? ldT<T>(src[0], o) : 0.f;
    R.p2 = (HAS_W && ok) ? ldT<T>(src[1], o) : 0.f;
    R.q11 = ok ? ldT<T>(src[2], o) : 0.f;
    R.q12 = ok ? ldT<T>(src[3], o) : 0.f;
    R.q21 = ok ? ldT<T>(src[4], o) : 0.f;
    R.q22 = ok ? ldT<T>(src[5], o) : 0.f;
    R.s = ok ? ldT<T>(src[6], o) : 0.f;
    R.ix = ok ? ldT<T>(src[7], o) : 0.f;
    R.iy = ok ? ldT<T>(src[8], o) : 0.f;
    R.it = ok ? ldT<T>(src[9], o) : 0.f;
    R.w = (HAS_W && ok) ? ldT<TF>(src[10], o) : 0.f;
    R.u = ok ? ldT<TF>(src[11], o) : 0.f;
    R.v = ok ? ldT<TF>(src[12], o) : 0.f;
}

#ifndef ROLL_RUNTIME_UNROLL  // unroll of the run-time row loop: the four-row register rotation
#define ROLL_RUNTIME_UNROLL 4
#endif

// One warp's strip: TY output rows of the 29 output columns starting at c0 + 2 (TY = 0: `ny` rows,
// a run-time count).  INT: the strip and its halo lie strictly inside the image, so every boundary
// test folds away.  skp: the warp's step coefficients when the caller has them already (else they
// are formed here, after the first rows' loads are in flight).  Returns this lane's sum of squared
// constraint residuals of its output pixels (FP32; the block or warp sum is FP64).
template <typename T, typename TF, bool HAS_W, int VARIANT, int TY, bool INT>
__device__ __forceinline__ float strip(const void *const *src, void *const *dst, int H, int W, int P, int c0, int y0,
                                       int lane, const Coefs &K, const float *msp, int ny = 0,
                                       const StepK *skp = nullptr) {
    const int c = c0 + lane;                   // this lane's column
    const bool out_lane = lane >= 2 && lane < 2 + SW && (INT || c < W);
    const bool ex = INT || c < W - 1, wx = INT || c > 0;   // east / west neighbour inside the image
    // rows i-1 (prev) and i (cur) in registers, rows i+1 (n1) and i+2 (n2) in flight.  A run-time
    // row count unrolls by the four-row register rotation only (a short loop body that stays in
    // the instruction cache).
    const int ty = TY > 0 ? TY : ny;
    const int NROWS = ty + 3;
    constexpr int UNROLL = TY == 0 ? ROLL_RUNTIME_UNROLL : (TY <= 8 ? TY + 3 : 4);
    Row prev{}, cur{}, n1{}, n2{};
    float dp_prev = 0.f, dq1_prev = 0.f, dq2_prev = 0.f;   // div y^k on row i-1
    float six_prev = 0.f, siy_prev = 0.f;                  // (s Ix, s Iy) on row i-1
    // y^{k+1} on the row above the one being finished (north neighbours of the div)
    float yp2_n = 0.f, yq12_n = 0.f, yq22_n = 0.f;
    float res = 0.f;

    load_row<T, TF, HAS_W, INT>(n1, src, y0 - 2, c, H, W, P);
    load_row<T, TF, HAS_W, INT>(n2, src, y0 - 1, c, H, W, P);
    // a~ (one device scalar of the warp) and the step coefficients after the first rows' loads
    // are in flight, so their latencies overlap
    const StepK SK = skp ? *skp : step_coefs(K, a_tilde_of(K, msp), c_of(K, msp));
#pragma unroll UNROLL
    for (int k = 0; k < NROWS; ++k) {
        const int i = y0 - 2 + k;                 // row entering the window
        prev = cur;
        cur = n1;
        n1 = n2;
        if (k + 2 < NROWS) load_row<T, TF, HAS_W, INT>(n2, src, i + 2, c, H, W, P);
        if (!INT && i >= H + 1) break;            // uniform: nothing left below the image
        // ---- div y^k on row i
        const bool rin = INT || (i >= 0 && i < H), ey = INT || i < H - 1, ny = INT || i > 0;
        const float p1w = __shfl_up_sync(FULL, cur.p1, 1), q11w = __shfl_up_sync(FULL, cur.q11, 1);
        const float q21w = __shfl_up_sync(FULL, cur.q21, 1);
        float dp = 0.f, dq1 = 0.f, dq2 = 0.f;
        if (rin && (INT || (c >= 0 && c < W))) {
            if (HAS_W) dp = div2(ex ? cur.p1 : 0.f, wx ? p1w : 0.f, ey ? cur.p2 : 0.f, ny ? prev.p2 : 0.f);
            dq1 = div2(ex ? cur.q11 : 0.f, wx ? q11w : 0.f, ey ? cur.q12 : 0.f, ny ? prev.q12 : 0.f);
            dq2 = div2(ex ? cur.q21 : 0.f, wx ? q21w : 0.f, ey ? cur.q22 : 0.f, ny ? prev.q22 : 0.f);
        }
        // rounded products (never fused into the differences below), as in the resident engine
        const float six_cur = __fmul_rn(cur.s, cur.ix), siy_cur = __fmul_rn(cur.s, cur.iy);
        // ---- y^{k+1} on row i-1 (south = row i, east = lane + 1)
        const int im = i - 1;
        const bool pin = INT || (im >= 0 && im < H && c >= 0 && c < W);
        const bool hy = INT || im < H - 1;
        const float dpE = __shfl_down_sync(FULL, dp_prev, 1), dq1E = __shfl_down_sync(FULL, dq1_prev, 1);
        const float dq2E = __shfl_down_sync(FULL, dq2_prev, 1);
        const float sE = __shfl_down_sync(FULL, prev.s, 1), wE = __shfl_down_sync(FULL, prev.w, 1);
        const float uE = __shfl_down_sync(FULL, prev.u, 1), vE = __shfl_down_sync(FULL, prev.v, 1);
        const float sixE = __shfl_down_sync(FULL, six_prev, 1);
        const float siyE = __shfl_down_sync(FULL, siy_prev, 1);
        float np1 = 0.f, np2 = 0.f, nq11 = 0.f, nq12 = 0.f, nq21 = 0.f, nq22 = 0.f;
        if (pin) {
            if (HAS_W) {
                const float s0 = prev.s;
                const float gdx = ex ? dpE - dp_prev : 0.f, gdy = hy ? dp - dp_prev : 0.f;
                const float wx_ = ex ? wE - prev.w : 0.f, wy_ = hy ? cur.w - prev.w : 0.f;
                const float sx_ = ex ? sE - s0 : 0.f, sy_ = hy ? cur.s - s0 : 0.f;
                y_update_p(prev.p1, prev.p2, gdx, gdy, wx_, wy_, sx_, sy_, SK, np1, np2);
            }
            const float sixx = ex ? sixE - six_prev : 0.f, sixy = hy ? six_cur - six_prev : 0.f;
            const float siyx = ex ? siyE - siy_prev : 0.f, siyy = hy ? siy_cur - siy_prev : 0.f;
            const float g1x = ex ? dq1E - dq1_prev : 0.f, g1y = hy ? dq1 - dq1_prev : 0.f;
            const float g2x = ex ? dq2E - dq2_prev : 0.f, g2y = hy ? dq2 - dq2_prev : 0.f;
            const float ux = ex ? uE - prev.u : 0.f, uy = hy ? cur.u - prev.u : 0.f;
            const float vx = ex ? vE - prev.v : 0.f, vy = hy ? cur.v - prev.v : 0.f;
            y_update_q(prev.q11, prev.q12, prev.q21, prev.q22, g1x, g1y, g2x, g2y, ux, uy, vx, vy, sixx, sixy, siyx,
                       siyy, SK, nq11, nq12, nq21, nq22);
        }
        // ---- finish row i-1: div y^{k+1}, s, multipliers, residual, stores
        const float np1W = __shfl_up_sync(FULL, np1, 1), nq11W = __shfl_up_sync(FULL, nq11, 1);
        const float nq21W = __shfl_up_sync(FULL, nq21, 1);
        if (pin && out_lane && im >= y0 && im < y0 + ty) {
            const bool nyy = INT || im > 0;
            float dpn = 0.f;
            if (HAS_W) dpn = div2(ex ? np1 : 0.f, wx ? np1W : 0.f, hy ? np2 : 0.f, nyy ? yp2_n : 0.f);
            const float dq1n = div2(ex ? nq11 : 0.f, wx ? nq11W : 0.f, hy ? nq12 : 0.f, nyy ? yq12_n : 0.f);
            const float dq2n = div2(ex ? nq21 : 0.f, wx ? nq21W : 0.f, hy ? nq22 : 0.f, nyy ? yq22_n : 0.f);
            float w = prev.w, u = prev.u, v = prev.v, s_new;
            res += finish_pixel<HAS_W, VARIANT>(prev.ix, prev.iy, prev.it, prev.s, w, u, v, dpn, dq1n, dq2n, SK, s_new);
            const size_t o = (size_t)im * P + c;
            if (HAS_W) {
                stT<T>(dst[F_P1], o, np1);
                stT<T>(dst[F_P2], o, np2);
                stT<TF>(dst[F_W], o, w);
            }
            stT<T>(dst[F_Q11], o, nq11);
            stT<T>(dst[F_Q12], o, nq12);
            stT<T>(dst[F_Q21], o, nq21);
            stT<T>(dst[F_Q22], o, nq22);
            stT<T>(dst[F_S], o, s_new);
            stT<TF>(dst[F_U], o, u);
            stT<TF>(dst[F_V], o, v);
        }
        yp2_n = np2;
        yq12_n = nq12;
        yq22_n = nq22;
        dp_prev = dp;
        dq1_prev = dq1;
        dq2_prev = dq2;
        six_prev = six_cur;
        siy_prev = siy_cur;
    }
    return res;
}

// The whole iteration for one block's strips (the body of both kernel entries below).
template <typename T, typename TF, bool HAS_W, int VARIANT, int TY>
__device__ __forceinline__ void roll_block(const IterArgs &A) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // ---- which strip: geometry in plain scalars, one 16-byte load per mode
    int H, W, P, sx, sy;
    const void *src[13];   // p1 p2 q11 q12 q21 q22 s Ix Iy It w u v
    void *dst[10];
    const float *msp;
    const int *donep;
    {
        const int order[10] = {F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22, F_S, F_W, F_U, F_V};
        // src slots: 0..6 <- p1..s, 10..12 <- w u v (order[7..9]), 7, 8, 9 <- Ix, Iy, It
        if (A.tiles) {
            const int4 tr = reinterpret_cast<const int4 *>(A.tiles)[blockIdx.x];
            const PairIter *pp = A.pairs + tr.x;
            const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
            H = gq.x;
            W = gq.y;
            P = gq.z;
            sx = tr.y;
            sy = tr.z * WARPS + wid;
            const Fields *in = pp->buf + A.parity, *out = pp->buf + (A.parity ^ 1);
#pragma unroll
            for (int k = 0; k < 10; ++k) src[k < 7 ? k : k + 3] = in->f[order[k]];
#pragma unroll
            for (int k = 0; k < 10; ++k) dst[k] = out->f[k];
            msp = pp->ms_max;
            donep = pp->done;
            src[7] = pp->Ix;
            src[8] = pp->Iy;
            src[9] = pp->It;
        } else {
            H = A.g.H;
            W = A.g.W;
            P = A.g.pitch;
            sx = blockIdx.x;
            sy = blockIdx.y * WARPS + wid;
#pragma unroll
            for (int k = 0; k < 10; ++k) src[k < 7 ? k : k + 3] = A.in.f[order[k]];
#pragma unroll
            for (int k = 0; k < 10; ++k) dst[k] = A.out.f[k];
            msp = A.ms_max;
            donep = A.done;
            src[7] = A.Ix;
            src[8] = A.Iy;
            src[9] = A.It;
        }
    }
    if (donep && *donep) return;  // uniform per block: the pair's warp met its stopping test

    const int c0 = sx * SW - 2;                // first column of the strip
    const int y0 = sy * TY;                    // first output row of the strip
    // interior strip: columns c0 .. c0+31 and rows y0-2 .. y0+TY all away from the image border
    const bool interior = c0 >= 1 && c0 + 32 <= W - 1 && y0 >= 2 && y0 + TY <= H - 2;
    const float res = interior ? strip<T, TF, HAS_W, VARIANT, TY, true>(src, dst, H, W, P, c0, y0, lane, A.k, msp)
                               : strip<T, TF, HAS_W, VARIANT, TY, false>(src, dst, H, W, P, c0, y0, lane, A.k, msp);
    if (A.partials) {
        const double tot = block_sum((double)res, red);
        if (threadIdx.x == 0) A.partials[blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

// Strips of 1, 2 and 8 rows: the compiler's own register budget for 128-thread blocks (at most 128
// registers, four blocks per SM).  Asking for one block per SM instead let the 8-row strips take
// 203 registers, half the resident warps, and measured 40% slower per iteration at 640x480.
template <typename T, typename TF, bool HAS_W, int VARIANT, int TY>
__global__ void __launch_bounds__(WARPS * 32) k_admm_roll(IterArgs A) {
    roll_block<T, TF, HAS_W, VARIANT, TY>(A);
}

// 32-row strips run in many waves (large images, batches): capping their registers at five
// 128-thread blocks per SM (96 registers) raises the resident warps from 16 to 20 per SM and
// measured 17-26% faster (a 12-16 byte spill in the beta > 0 variants included).  The shorter
// strips' fully unrolled chains spill heavily under such a cap.
#ifndef ROLL_TY32_MIN_BLOCKS
#define ROLL_TY32_MIN_BLOCKS 5
#endif
template <typename T, typename TF, bool HAS_W, int VARIANT>
__global__ void __launch_bounds__(WARPS * 32, ROLL_TY32_MIN_BLOCKS) k_admm_roll32(IterArgs A) {
    roll_block<T, TF, HAS_W, VARIANT, 32>(A);
}

template <typename T, typename TF, bool HAS_W, int VARIANT, int TY> void launch_t(const IterArgs &a, cudaStream_t s) {
    dim3 grid = a.tiles ? dim3(a.ntiles)
                        : dim3((a.g.W + SW - 1) / SW, (a.g.H + TY * WARPS - 1) / (TY * WARPS));
    if constexpr (TY == 32) k_admm_roll32<T, TF, HAS_W, VARIANT><<<grid, dim3(32 * WARPS), 0, s>>>(a);
    else k_admm_roll<T, TF, HAS_W, VARIANT, TY><<<grid, dim3(32 * WARPS), 0, s>>>(a);
}

template <typename T, typename TF, bool HAS_W, int VARIANT> void launch_ty(const IterArgs &a, int ty, cudaStream_t s) {
    switch (ty) {
    case 1: launch_t<T, TF, HAS_W, VARIANT, 1>(a, s); break;
    case 2: launch_t<T, TF, HAS_W, VARIANT, 2>(a, s); break;
    case 8: launch_t<T, TF, HAS_W, VARIANT, 8>(a, s); break;
    default: launch_t<T, TF, HAS_W, VARIANT, 32>(a, s); break;
    }
}

template <typename T, typename TF> void launch_m(const IterArgs &a, int ty, cudaStream_t s) {
    const bool has_w = a.k.beta != 0.f;
    if (a.k.method == 1) {
        if (a.k.a_tilde_mode == 1) {
            if (has_w) launch_ty<T, TF, true, 3>(a, ty, s);
            else launch_ty<T, TF, false, 3>(a, ty, s);
        } else {
            if (has_w) launch_ty<T, TF, true, 1>(a, ty, s);
            else launch_ty<T, TF, false, 1>(a, ty, s);
        }
    } else {
        if (a.k.a_tilde_mode == 1) {
            if (has_w) launch_ty<T, TF, true, 2>(a, ty, s);
            else launch_ty<T, TF, false, 2>(a, ty, s);
        } else {
            if (has_w) launch_ty<T, TF, true, 0>(a, ty, s);
            else launch_ty<T, TF, false, 0>(a, ty, s);
        }
    }
}

}  // namespace roll
}  // namespace tvl1
