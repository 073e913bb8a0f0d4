// k_pdr_math.cuh -- the per-pixel arithmetic of one pDR iteration (Sec. 3.1.2, eq. pDR with the
// red-black symmetric Gauss-Seidel preconditioner), shared by the per-kernel engine (k_pdr.cu) and
// the level-resident engine (k_resident.cu).  Explicit FMAs, so both round alike.
#pragma once
#include <math.h>

namespace tvl1 {

// b = Xbar + sigma div ybar (one component).
__device__ __forceinline__ float pdr_rhs(float xbar, float div, float sigma) { return fmaf(sigma, div, xbar); }

// One Gauss-Seidel update of (1 + st n) x - st sum_nb x_nb = b at a pixel with n in-domain
// neighbours whose values sum (west, east, north, south, in that order) to acc.
__device__ __forceinline__ float pdr_gs(float b, float acc, int n, float st) {
    return fmaf(st, acc, b) / fmaf(st, (float)n, 1.f);
}

__device__ __forceinline__ float pdr_ball_scale(float n2) { return n2 > 1.f ? rsqrtf(n2) : 1.f; }

// Xbar^{k+1} = Xbar + prox_{sigma F}(2 X^{k+1} - Xbar) - X^{k+1} at one pixel (x = X^{k+1},
// xb = Xbar^k, updated in place; w components ignored without HAS_W).  prox_{sigma F}: the
// three-case L1 resolvent (eq. resolvent) with e = (beta, Ix, Iy).
template <bool HAS_W>
__device__ __forceinline__ void pdr_xbar(const float x[3], float xb[3], float ix, float iy, float it, float beta,
                                         float lam, float sg) {
    float zw = HAS_W ? 2.f * x[0] - xb[0] : 0.f;
    float zu = 2.f * x[1] - xb[1], zv = 2.f * x[2] - xb[2];
    const float e2 = fmaf(iy, iy, fmaf(ix, ix, beta * beta));
    const float rho = fmaf(iy, zv, fmaf(ix, zu, HAS_W ? fmaf(beta, zw, it) : it));
    const float sl = sg * lam * e2;
    float t;
    if (e2 <= 0.f) t = 0.f;
    else if (rho < -sl) t = sg * lam;
    else if (rho > sl) t = -sg * lam;
    else t = -rho / e2;
    if (HAS_W) zw = fmaf(t, beta, zw);
    zu = fmaf(t, ix, zu);
    zv = fmaf(t, iy, zv);
    if (HAS_W) xb[0] = (xb[0] + zw) - x[0];
    xb[1] = (xb[1] + zu) - x[1];
    xb[2] = (xb[2] + zv) - x[2];
}

// ybar^{k+1} = P(ybar + 2 tau grad X^{k+1}) - tau grad X^{k+1} at one pixel; g: forward
// differences (d_x w, d_y w, d_x u, d_y u, d_x v, d_y v) of X^{k+1}; P_p on p, the joint P_q on q.
template <bool HAS_W>
__device__ __forceinline__ void pdr_ybar(const float y[6], const float g[6], float tau, float out[6]) {
    const float t2 = 2.f * tau;
    if (HAS_W) {
        const float a1 = fmaf(t2, g[0], y[0]), a2 = fmaf(t2, g[1], y[1]);
        const float f = pdr_ball_scale(fmaf(a1, a1, a2 * a2));
        out[0] = fmaf(-tau, g[0], a1 * f);
        out[1] = fmaf(-tau, g[1], a2 * f);
    } else {
        out[0] = out[1] = 0.f;
    }
    const float b11 = fmaf(t2, g[2], y[2]), b12 = fmaf(t2, g[3], y[3]);
    const float b21 = fmaf(t2, g[4], y[4]), b22 = fmaf(t2, g[5], y[5]);
    const float f = pdr_ball_scale(fmaf(b11, b11, fmaf(b12, b12, fmaf(b21, b21, b22 * b22))));
    out[2] = fmaf(-tau, g[2], b11 * f);
    out[3] = fmaf(-tau, g[3], b12 * f);
    out[4] = fmaf(-tau, g[4], b21 * f);
    out[5] = fmaf(-tau, g[5], b22 * f);
}

}  // namespace tvl1
