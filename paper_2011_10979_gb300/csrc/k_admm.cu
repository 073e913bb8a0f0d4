// k_admm.cu -- inner iteration of the preconditioned ADMM solvers of Sec. 3.1.1:
//   rpADMMI (eq. rpADMMI; pADMM for r = 1), rpADMMII (eq. rpADMMII) and the beta = 0 model
//   (Zach-pADMM, eq. Zach-pADMM, with w and p absent).
// With grad^* = -div, the y-update reads  p <- P_p[p + (1/a) grad(div p) + (1/a)(grad w / c - beta grad s)],
// q_k likewise with grad(u or v)/c - grad(s I_x or s I_y) and the joint projection P_q; the s-update
// uses the old multipliers and the new duals; the multipliers then take the constraint
// A s + B y = (beta s - div p, I_x s - div q1, I_y s - div q2).
//
// This file holds the plain engine -- one kernel per operator (div, y-update, div, s/multiplier
// update) in FP32, in place; the fused engine is k_admm_roll.cuh.
#include <math.h>

#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

// ------------------------------------------------------------------------------ plain engine
constexpr int PX = 32, PY = 8;

__device__ __forceinline__ float divergence(const float *a, const float *b, int i, int j, int H, int W, int P) {
    const size_t o = (size_t)i * P + j;
    float d = 0.f;
    if (j < W - 1) d += a[o];
    if (j > 0) d -= a[o - 1];
    if (i < H - 1) d += b[o];
    if (i > 0) d -= b[o - P];
    return d;
}

// div p, div q1, div q2 into tmp planes 0..2
__global__ void k_div3(IterArgs A, float *dp, float *dq1, float *dq2, bool has_w) {
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    if (i >= H || j >= W) return;
    const size_t o = (size_t)i * P + j;
    auto F = [&](int f) { return (const float *)A.in.f[f]; };
    dp[o] = has_w ? divergence(F(F_P1), F(F_P2), i, j, H, W, P) : 0.f;
    dq1[o] = divergence(F(F_Q11), F(F_Q12), i, j, H, W, P);
    dq2[o] = divergence(F(F_Q21), F(F_Q22), i, j, H, W, P);
}

__global__ void k_yupdate_plain(IterArgs A, const float *dp, const float *dq1, const float *dq2, bool has_w) {
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    if (i >= H || j >= W) return;
    const size_t o = (size_t)i * P + j;
    const bool hx = j < W - 1, hy = i < H - 1;
    auto F = [&](int f) { return (float *)A.in.f[f]; };
    auto gx = [&](const float *f) { return hx ? f[o + 1] - f[o] : 0.f; };
    auto gy = [&](const float *f) { return hy ? f[o + P] - f[o] : 0.f; };
    const float *s = F(F_S), *Ix = (const float *)A.Ix, *Iy = (const float *)A.Iy;
    const float inv_a = 1.f / A.k.a, inv_c = 1.f / c_of(A.k, A.ms_max), beta = A.k.beta;
    if (has_w) {
        float p1 = F(F_P1)[o] + gx(dp) * inv_a + (gx(F(F_W)) * inv_c - beta * gx(s)) * inv_a;
        float p2 = F(F_P2)[o] + gy(dp) * inv_a + (gy(F(F_W)) * inv_c - beta * gy(s)) * inv_a;
        const float f = fmaxf(1.f, sqrtf(p1 * p1 + p2 * p2));
        F(F_P1)[o] = p1 / f;
        F(F_P2)[o] = p2 / f;
    }
    const float sixx = hx ? s[o + 1] * Ix[o + 1] - s[o] * Ix[o] : 0.f;
    const float sixy = hy ? s[o + P] * Ix[o + P] - s[o] * Ix[o] : 0.f;
    const float siyx = hx ? s[o + 1] * Iy[o + 1] - s[o] * Iy[o] : 0.f;
    const float siyy = hy ? s[o + P] * Iy[o + P] - s[o] * Iy[o] : 0.f;
    float q11 = F(F_Q11)[o] + gx(dq1) * inv_a + (gx(F(F_U)) * inv_c - sixx) * inv_a;
    float q12 = F(F_Q12)[o] + gy(dq1) * inv_a + (gy(F(F_U)) * inv_c - sixy) * inv_a;
    float q21 = F(F_Q21)[o] + gx(dq2) * inv_a + (gx(F(F_V)) * inv_c - siyx) * inv_a;
    float q22 = F(F_Q22)[o] + gy(dq2) * inv_a + (gy(F(F_V)) * inv_c - siyy) * inv_a;
    const float f = fmaxf(1.f, sqrtf(q11 * q11 + q12 * q12 + q21 * q21 + q22 * q22));
    F(F_Q11)[o] = q11 / f;
    F(F_Q12)[o] = q12 / f;
    F(F_Q21)[o] = q21 / f;
    F(F_Q22)[o] = q22 / f;
}

__global__ void k_supdate_plain(IterArgs A, const float *dp, const float *dq1, const float *dq2, bool has_w) {
    __shared__ double red[32];
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    double res = 0.0;
    if (i < H && j < W) {
        const size_t o = (size_t)i * P + j;
        auto F = [&](int f) { return (float *)A.in.f[f]; };
        const float ix = ((const float *)A.Ix)[o], iy = ((const float *)A.Iy)[o], it = ((const float *)A.It)[o];
        const float beta = A.k.beta, c = c_of(A.k, A.ms_max), lam = A.k.lambda, rho = A.k.rho;
        const float s_old = F(F_S)[o];
        float w = has_w ? F(F_W)[o] : 0.f, u = F(F_U)[o], v = F(F_V)[o];
        const float ms = beta * beta + ix * ix + iy * iy;
        // a~: one value per warp, or the per-pixel diagonal a~_ij = M_s(ij)
        const float at = A.k.a_tilde_mode == 1 ? fmaxf(ms, 1e-12f) : a_tilde_of(A.k, A.ms_max);
        const float lin = it + ix * u + iy * v + (has_w ? beta * w : 0.f);
        const float divt = ix * dq1[o] + iy * dq2[o] + (has_w ? beta * dp[o] : 0.f);
        float s_new;
        if (A.k.method == 1) s_new = (1.f - rho * ms / at) * s_old + (lin + c * rho * divt) / (at * c);
        else s_new = (1.f - ms / at) * s_old + (lin + c * divt) / (at * c);
        s_new = fminf(fmaxf(s_new, -lam), lam);
        const float cw = has_w ? beta * s_new - dp[o] : 0.f, cu = ix * s_new - dq1[o], cv = iy * s_new - dq2[o];
        if (A.k.method == 1) {
            if (has_w) w -= c * (beta * s_new - rho * dp[o] - (1.f - rho) * beta * s_old);
            u -= c * (ix * s_new - rho * dq1[o] - (1.f - rho) * ix * s_old);
            v -= c * (iy * s_new - rho * dq2[o] - (1.f - rho) * iy * s_old);
        } else {
            const float rc = A.k.r * c;
            if (has_w) w -= rc * cw;
            u -= rc * cu;
            v -= rc * cv;
        }
        F(F_S)[o] = s_new;
        if (has_w) F(F_W)[o] = w;
        F(F_U)[o] = u;
        F(F_V)[o] = v;
        res = (double)cw * cw + (double)cu * cu + (double)cv * cv;
    }
    if (A.partials) {
        const double tot = block_sum(res, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) A.partials[block_linear_id()] = tot;
    }
}

}  // namespace

int admm_plain_blocks(Geom g) { return ((g.W + PX - 1) / PX) * ((g.H + PY - 1) / PY); }

void launch_admm_plain(const IterArgs &a, cudaStream_t s) {
    const bool has_w = a.k.beta != 0.f;
    const size_t plane = (size_t)a.g.H * a.g.pitch;
    float *dp = a.tmp, *dq1 = a.tmp + plane, *dq2 = a.tmp + 2 * plane;
    dim3 grid((a.g.W + PX - 1) / PX, (a.g.H + PY - 1) / PY), blk(PX, PY);
    IterArgs b = a;
    b.partials = nullptr;
    k_div3<<<grid, blk, 0, s>>>(b, dp, dq1, dq2, has_w);
    k_yupdate_plain<<<grid, blk, 0, s>>>(b, dp, dq1, dq2, has_w);
    k_div3<<<grid, blk, 0, s>>>(b, dp, dq1, dq2, has_w);
    k_supdate_plain<<<grid, blk, 0, s>>>(a, dp, dq1, dq2, has_w);
}

}  // namespace tvl1
