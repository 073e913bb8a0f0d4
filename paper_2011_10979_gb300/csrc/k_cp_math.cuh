// k_cp_math.cuh -- the per-pixel arithmetic of one ALG1 iteration (Sec. 4: Chambolle-Pock with
// constant steps on eq. primal-dual:optical:o), shared by the one-kernel-per-iteration engine
// (k_cp.cu) and the level-resident engine (k_resident.cu).  Explicit FMAs, so both round alike.
#pragma once
#include <math.h>

namespace tvl1 {

// 1 / max(1, sqrt(n2)): the scale of the projection onto the unit ball.
__device__ __forceinline__ float cp_ball_scale(float n2) { return n2 > 1.f ? rsqrtf(n2) : 1.f; }

// Dual step at one pixel: y' = P(y + tau grad Xbar), with the forward differences of Xbar
// (g[0..5] = d_x wbar, d_y wbar, d_x ubar, d_y ubar, d_x vbar, d_y vbar; zeros at the border).
// P_p on (p1, p2), the joint P_q on (q11, q12, q21, q22).  y and out: p1 p2 q11 q12 q21 q22.
template <bool HAS_W>
__device__ __forceinline__ void cp_dual(const float y[6], const float g[6], float tau, float out[6]) {
    if (HAS_W) {
        const float t1 = fmaf(tau, g[0], y[0]), t2 = fmaf(tau, g[1], y[1]);
        const float f = cp_ball_scale(fmaf(t1, t1, t2 * t2));
        out[0] = t1 * f;
        out[1] = t2 * f;
    } else {
        out[0] = out[1] = 0.f;
    }
    const float t11 = fmaf(tau, g[2], y[2]), t12 = fmaf(tau, g[3], y[3]);
    const float t21 = fmaf(tau, g[4], y[4]), t22 = fmaf(tau, g[5], y[5]);
    const float f = cp_ball_scale(fmaf(t11, t11, fmaf(t12, t12, fmaf(t21, t21, t22 * t22))));
    out[2] = t11 * f;
    out[3] = t12 * f;
    out[4] = t21 * f;
    out[5] = t22 * f;
}

// Primal step at one pixel: X' = prox_{sigma F}(X + sigma div y') with F = lambda |rho|,
// rho(Z) = It + beta Z_w + Ix Z_u + Iy Z_v: Z + t e, e = (beta, Ix, Iy), t from the three cases
// of rho(Z) against sigma lambda |e|^2 (eq. resolvent).  dv: div y' for (p, q1, q2).  Returns X'
// in x[0..2] (w u v) and the squared step |X' - X|^2.
template <bool HAS_W>
__device__ __forceinline__ float cp_primal(float x[3], const float dv[3], float ix, float iy, float it, float beta,
                                           float lam, float sg) {
    const float xw = HAS_W ? x[0] : 0.f, xu = x[1], xv = x[2];
    float zw = HAS_W ? fmaf(sg, dv[0], xw) : 0.f;
    float zu = fmaf(sg, dv[1], xu), zv = fmaf(sg, dv[2], xv);
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
    const float dw = zw - xw, du = zu - xu, dd = zv - xv;
    x[0] = zw;
    x[1] = zu;
    x[2] = zv;
    return fmaf(dd, dd, fmaf(du, du, dw * dw));
}

}  // namespace tvl1
