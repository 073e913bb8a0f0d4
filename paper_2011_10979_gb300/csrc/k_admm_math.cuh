// k_admm_math.cuh -- the per-pixel arithmetic of one ADMM iteration (Sec. 3.1.1), shared by the
// row-streaming kernel (k_admm_roll.cuh) and the level-resident kernel (k_resident.cu).
// Every product-sum is an explicit fmaf, so both kernels round every pixel alike (FP32).
#pragma once
#include <math.h>

#include "tvl1_internal.h"

namespace tvl1 {

// Step constants of one warp (c: the step of the iteration, c_of): 1/a, 1/c, beta, 1/a~, 1/(a~ c), c, lambda, rho, 1 - rho, r c, and
// whether a~ is the per-pixel diagonal a~_ij = M_s(ij) instead of one value per warp.
struct StepK {
    float inv_a, inv_c, beta, inv_at, inv_atc, cc, lam, rho, omr, rc;
    int per_pixel;
};

__device__ __forceinline__ StepK step_coefs(const Coefs &K, float at, float c) {
    StepK s;
    s.inv_a = 1.f / K.a;
    s.inv_c = 1.f / c;
    s.beta = K.beta;
    s.inv_at = 1.f / at;
    s.inv_atc = 1.f / (at * c);
    s.cc = c;
    s.lam = K.lambda;
    s.rho = K.rho;
    s.omr = 1.f - K.rho;
    s.rc = K.r * c;
    s.per_pixel = K.a_tilde_mode == 1;
    return s;
}

// Divergence (div = -grad^*, forward differences with Neumann boundary) of a 2-vector field at
// one pixel from its own components x, y and the west x / north y neighbours; terms outside the
// image are passed as 0 by the caller.
__device__ __forceinline__ float div2(float x, float xw, float y, float yn) { return ((x - xw) + y) - yn; }

// 1 / max(1, sqrt(n2)) for n2 >= 0: the scale of the projection onto the unit ball (P_p, P_q).
// rsqrtf carries at most 2 ulp of error; the factor is exactly 1 inside the ball.
__device__ __forceinline__ float ball_scale(float n2) { return n2 > 1.f ? rsqrtf(n2) : 1.f; }

// p^{k+1} = P_p[p^k + (1/a)(grad div p^k + grad w / c - beta grad s)] from the forward differences
// (gd*: of div p^k, w*: of w, s*: of s).
__device__ __forceinline__ void y_update_p(float p1, float p2, float gdx, float gdy, float wx, float wy, float sx,
                                           float sy, const StepK &K, float &np1, float &np2) {
    const float a1 = fmaf(fmaf(-K.beta, sx, fmaf(wx, K.inv_c, gdx)), K.inv_a, p1);
    const float a2 = fmaf(fmaf(-K.beta, sy, fmaf(wy, K.inv_c, gdy)), K.inv_a, p2);
    const float f = ball_scale(fmaf(a1, a1, a2 * a2));
    np1 = a1 * f;
    np2 = a2 * f;
}

// q^{k+1} = P_q[q^k + (1/a)(grad div q^k + grad (u, v) / c - grad (s Ix, s Iy))], the joint
// projection of (q1, q2) onto the unit ball of R^4.
__device__ __forceinline__ void y_update_q(float q11, float q12, float q21, float q22, float g1x, float g1y,
                                           float g2x, float g2y, float ux, float uy, float vx, float vy, float sixx,
                                           float sixy, float siyx, float siyy, const StepK &K, float &nq11,
                                           float &nq12, float &nq21, float &nq22) {
    const float b11 = fmaf(fmaf(ux, K.inv_c, g1x) - sixx, K.inv_a, q11);
    const float b12 = fmaf(fmaf(uy, K.inv_c, g1y) - sixy, K.inv_a, q12);
    const float b21 = fmaf(fmaf(vx, K.inv_c, g2x) - siyx, K.inv_a, q21);
    const float b22 = fmaf(fmaf(vy, K.inv_c, g2y) - siyy, K.inv_a, q22);
    const float f = ball_scale(fmaf(b11, b11, fmaf(b12, b12, fmaf(b21, b21, b22 * b22))));
    nq11 = b11 * f;
    nq12 = b12 * f;
    nq21 = b21 * f;
    nq22 = b22 * f;
}

// The s-step and the multiplier step at one pixel, given div y^{k+1} there (dpn, dq1n, dq2n):
//   s^{k+1} = P_s[(1 - M_s / a~) s^k + (l + c t) / (a~ c)]            (VARIANT 0: rpADMMI / pADMM)
//   s^{k+1} = P_s[(1 - rho M_s / a~) s^k + (l + c rho t) / (a~ c)]    (VARIANT 1: rpADMMII)
// with M_s = beta^2 + Ix^2 + Iy^2, l = It + Ix u + Iy v + beta w, t = Ix dq1n + Iy dq2n + beta dpn;
// With the per-pixel preconditioner a~ is M_s at the pixel (floored at 1e-12): M_s is diagonal,
// so the s-block proximal matrix c(diag(a~) - M_s) stays positive semidefinite;
// then Lambda = (w, u, v) -= r c (A s^{k+1} - div y^{k+1}) (VARIANT 0) or
// Lambda -= c (A s^{k+1} - rho div y^{k+1} - (1 - rho) A s^k) (VARIANT 1), A s = (beta, Ix, Iy) s.
// VARIANT bit 0: rpADMMII; bit 1: the per-pixel a~ (a compile-time choice, so the one-launch-per-
// iteration kernel carries no branch for it).
// Updates w, u, v in place, returns s^{k+1} in s_new and the squared constraint residual
// |A s^{k+1} - div y^{k+1}|^2.
template <bool HAS_W, int VARIANT>
__device__ __forceinline__ float finish_pixel(float ix, float iy, float it, float s_old, float &w, float &u, float &v,
                                              float dpn, float dq1n, float dq2n, const StepK &K, float &s_new) {
    const float beta = K.beta;
    const float ms = fmaf(iy, iy, fmaf(ix, ix, beta * beta));
    const float lin0 = fmaf(iy, v, fmaf(ix, u, it));
    const float lin = HAS_W ? fmaf(beta, w, lin0) : lin0;
    const float divt0 = fmaf(iy, dq2n, ix * dq1n);
    const float divt = HAS_W ? fmaf(beta, dpn, divt0) : divt0;
    float inv_at = K.inv_at, inv_atc = K.inv_atc;
    if (VARIANT & 2) {
        const float at = fmaxf(ms, 1e-12f);
        inv_at = __frcp_rn(at);
        inv_atc = __frcp_rn(at * K.cc);
    }
    float s;
    if ((VARIANT & 1) == 0) s = fmaf(fmaf(K.cc, divt, lin), inv_atc, fmaf(-ms, inv_at, 1.f) * s_old);
    else s = fmaf(fmaf(K.cc * K.rho, divt, lin), inv_atc, fmaf(-K.rho * ms, inv_at, 1.f) * s_old);
    s = fminf(fmaxf(s, -K.lam), K.lam);  // P_s: projection onto |s| <= lambda
    s_new = s;
    const float cw = HAS_W ? fmaf(beta, s, -dpn) : 0.f;
    const float cu = fmaf(ix, s, -dq1n), cv = fmaf(iy, s, -dq2n);
    if ((VARIANT & 1) == 0) {
        if (HAS_W) w = fmaf(-K.rc, cw, w);
        u = fmaf(-K.rc, cu, u);
        v = fmaf(-K.rc, cv, v);
    } else {
        if (HAS_W) w = fmaf(-K.cc, fmaf(-K.omr * beta, s_old, fmaf(-K.rho, dpn, beta * s)), w);
        u = fmaf(-K.cc, fmaf(-K.omr * ix, s_old, fmaf(-K.rho, dq1n, ix * s)), u);
        v = fmaf(-K.cc, fmaf(-K.omr * iy, s_old, fmaf(-K.rho, dq2n, iy * s)), v);
    }
    return fmaf(cv, cv, fmaf(cu, cu, cw * cw));
}

}  // namespace tvl1
