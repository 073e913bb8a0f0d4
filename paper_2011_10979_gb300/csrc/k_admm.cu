// k_admm.cu -- inner iteration of the preconditioned ADMM solvers of Sec. 3.1.1:
//   rpADMMI (eq. rpADMMI; pADMM for r = 1), rpADMMII (eq. rpADMMII) and the beta = 0 model
//   (Zach-pADMM, eq. Zach-pADMM, with w and p absent).
// With grad^* = -div, the y-update reads  p <- P_p[p + (1/a) grad(div p) + (1/a)(grad w / c - beta grad s)],
// q_k likewise with grad(u or v)/c - grad(s I_x or s I_y) and the joint projection P_q; the s-update
// uses the old multipliers and the new duals; the multipliers then take the constraint
// A s + B y = (beta s - div p, I_x s - div q1, I_y s - div q2).
//
// Two engines:
//  * fused: one kernel per iteration.  A 32 x 16 tile with a (2 left/top, 1 right/bottom) halo of
//    all iterated fields is staged in shared memory; div y^k is formed on the tile + 1 ring,
//    y^{k+1} on the tile + 1 left/top ring, then div y^{k+1}, s^{k+1} and the multipliers on the
//    tile.  Reads one state buffer and writes the other (ping-pong), so every HBM/L2 byte of
//    state is read once and written once per iteration, apart from the halo.
//  * plain: one kernel per operator (div, y-update, div, s/multiplier update) in FP32, in place.
#include <math.h>

#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

// ------------------------------------------------------------------------------ fused engine
constexpr int TX = 32, TY = 16;          // output tile
constexpr int BX = 32, BY = 8;           // threads; each thread owns two tile rows
constexpr int RX = TX + 3, RY = TY + 3;  // staged region: cols [-2, TX+1), rows [-2, TY+1)
constexpr int DX = TX + 2, DY = TY + 2;  // div y^k region: cols [-1, TX+1), rows [-1, TY+1)
constexpr int NS = 12;                   // staged fields
// staged field slots
enum { S_P1 = 0, S_P2, S_Q11, S_Q12, S_Q21, S_Q22, S_S, S_W, S_U, S_V, S_IX, S_IY };
constexpr size_t FUSED_SMEM = sizeof(float) * (NS * RY * RX + 3 * DY * DX);

template <typename T, bool HAS_W, int VARIANT>
__global__ void __launch_bounds__(BX *BY) k_admm_fused(IterArgs A) {
    if (A.done && *A.done) return;
    extern __shared__ float sm[];
    float *S = sm;
    float *D = sm + NS * RY * RX;
    __shared__ double red[32];

    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * BX + threadIdx.x;
    auto s_at = [&](int f, int r, int c) -> float & { return S[f * RY * RX + (r + 2) * RX + (c + 2)]; };
    auto d_at = [&](int f, int r, int c) -> float & { return D[f * DY * DX + (r + 1) * DX + (c + 1)]; };

    // ---- stage the region (zeros outside the image)
    const void *src[NS] = {A.in.f[F_P1], A.in.f[F_P2], A.in.f[F_Q11], A.in.f[F_Q12], A.in.f[F_Q21], A.in.f[F_Q22],
                           A.in.f[F_S],  A.in.f[F_W],  A.in.f[F_U],   A.in.f[F_V],   A.Ix,          A.Iy};
    for (int k = tid; k < RY * RX; k += BX * BY) {
        const int r = k / RX, c = k - r * RX;
        const int gi = y0 + r - 2, gj = x0 + c - 2;
        const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
        const size_t o = in ? (size_t)gi * P + gj : 0;
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const bool used = HAS_W || (f != S_P1 && f != S_P2 && f != S_W);
            S[f * RY * RX + k] = (in && used) ? ldT<T>(src[f], o) : 0.f;
        }
    }
    __syncthreads();

    // ---- div y^k on rows [-1, TY+1) x cols [-1, TX+1)
    for (int k = tid; k < DY * DX; k += BX * BY) {
        const int r = k / DX - 1, c = k % DX - 1;
        const int gi = y0 + r, gj = x0 + c;
        const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            float d = 0.f;
            if (in && (HAS_W || t > 0)) {
                const int fa = 2 * t, fb = 2 * t + 1;  // (p1,p2), (q11,q12), (q21,q22)
                if (gj < W - 1) d += s_at(fa, r, c);
                if (gj > 0) d -= s_at(fa, r, c - 1);
                if (gi < H - 1) d += s_at(fb, r, c);
                if (gi > 0) d -= s_at(fb, r - 1, c);
            }
            D[t * DY * DX + k] = d;
        }
    }
    __syncthreads();

    // ---- y^{k+1} on rows [-1, TY) x cols [-1, TX), in place in the staged p/q slots
    const float inv_a = 1.f / A.k.a, inv_c = 1.f / A.k.c, beta = A.k.beta;
    for (int k = tid; k < (TY + 1) * (TX + 1); k += BX * BY) {
        const int r = k / (TX + 1) - 1, c = k % (TX + 1) - 1;
        const int gi = y0 + r, gj = x0 + c;
        if (gi < 0 || gi >= H || gj < 0 || gj >= W) continue;
        const bool hx = gj < W - 1, hy = gi < H - 1;
        const float s0 = s_at(S_S, r, c);
        const float sE = s_at(S_S, r, c + 1), sS = s_at(S_S, r + 1, c);
        if (HAS_W) {
            const float gdx = hx ? d_at(0, r, c + 1) - d_at(0, r, c) : 0.f;
            const float gdy = hy ? d_at(0, r + 1, c) - d_at(0, r, c) : 0.f;
            const float wx = hx ? s_at(S_W, r, c + 1) - s_at(S_W, r, c) : 0.f;
            const float wy = hy ? s_at(S_W, r + 1, c) - s_at(S_W, r, c) : 0.f;
            const float sx = hx ? sE - s0 : 0.f, sy = hy ? sS - s0 : 0.f;
            float p1 = s_at(S_P1, r, c) + gdx * inv_a + (wx * inv_c - beta * sx) * inv_a;
            float p2 = s_at(S_P2, r, c) + gdy * inv_a + (wy * inv_c - beta * sy) * inv_a;
            const float f = fmaxf(1.f, sqrtf(p1 * p1 + p2 * p2));
            s_at(S_P1, r, c) = p1 / f;
            s_at(S_P2, r, c) = p2 / f;
        }
        const float ix0 = s_at(S_IX, r, c), iy0 = s_at(S_IY, r, c);
        const float sixx = hx ? sE * s_at(S_IX, r, c + 1) - s0 * ix0 : 0.f;
        const float sixy = hy ? sS * s_at(S_IX, r + 1, c) - s0 * ix0 : 0.f;
        const float siyx = hx ? sE * s_at(S_IY, r, c + 1) - s0 * iy0 : 0.f;
        const float siyy = hy ? sS * s_at(S_IY, r + 1, c) - s0 * iy0 : 0.f;
        const float g1x = hx ? d_at(1, r, c + 1) - d_at(1, r, c) : 0.f;
        const float g1y = hy ? d_at(1, r + 1, c) - d_at(1, r, c) : 0.f;
        const float g2x = hx ? d_at(2, r, c + 1) - d_at(2, r, c) : 0.f;
        const float g2y = hy ? d_at(2, r + 1, c) - d_at(2, r, c) : 0.f;
        const float ux = hx ? s_at(S_U, r, c + 1) - s_at(S_U, r, c) : 0.f;
        const float uy = hy ? s_at(S_U, r + 1, c) - s_at(S_U, r, c) : 0.f;
        const float vx = hx ? s_at(S_V, r, c + 1) - s_at(S_V, r, c) : 0.f;
        const float vy = hy ? s_at(S_V, r + 1, c) - s_at(S_V, r, c) : 0.f;
        float q11 = s_at(S_Q11, r, c) + g1x * inv_a + (ux * inv_c - sixx) * inv_a;
        float q12 = s_at(S_Q12, r, c) + g1y * inv_a + (uy * inv_c - sixy) * inv_a;
        float q21 = s_at(S_Q21, r, c) + g2x * inv_a + (vx * inv_c - siyx) * inv_a;
        float q22 = s_at(S_Q22, r, c) + g2y * inv_a + (vy * inv_c - siyy) * inv_a;
        const float f = fmaxf(1.f, sqrtf(q11 * q11 + q12 * q12 + q21 * q21 + q22 * q22));
        s_at(S_Q11, r, c) = q11 / f;
        s_at(S_Q12, r, c) = q12 / f;
        s_at(S_Q21, r, c) = q21 / f;
        s_at(S_Q22, r, c) = q22 / f;
    }
    __syncthreads();

    // ---- s^{k+1} and the multipliers on the tile
    const float at = a_tilde_of(A.k, A.ms_max);
    const float inv_at = 1.f / at, inv_atc = 1.f / (at * A.k.c), c = A.k.c, lam = A.k.lambda;
    const float rho = A.k.rho, rc = A.k.r * A.k.c;
    double res = 0.0;
#pragma unroll
    for (int m = 0; m < TY / BY; ++m) {
        const int r = threadIdx.y + m * BY, cc = threadIdx.x;
        const int gi = y0 + r, gj = x0 + cc;
        if (gi >= H || gj >= W) continue;
        const size_t o = (size_t)gi * P + gj;
        float dp = 0.f;
        if (HAS_W) {
            if (gj < W - 1) dp += s_at(S_P1, r, cc);
            if (gj > 0) dp -= s_at(S_P1, r, cc - 1);
            if (gi < H - 1) dp += s_at(S_P2, r, cc);
            if (gi > 0) dp -= s_at(S_P2, r - 1, cc);
        }
        float dq1 = 0.f, dq2 = 0.f;
        if (gj < W - 1) { dq1 += s_at(S_Q11, r, cc); dq2 += s_at(S_Q21, r, cc); }
        if (gj > 0) { dq1 -= s_at(S_Q11, r, cc - 1); dq2 -= s_at(S_Q21, r, cc - 1); }
        if (gi < H - 1) { dq1 += s_at(S_Q12, r, cc); dq2 += s_at(S_Q22, r, cc); }
        if (gi > 0) { dq1 -= s_at(S_Q12, r - 1, cc); dq2 -= s_at(S_Q22, r - 1, cc); }
        const float ix = s_at(S_IX, r, cc), iy = s_at(S_IY, r, cc), it = ldT<T>(A.It, o);
        const float s_old = s_at(S_S, r, cc);
        float w = HAS_W ? s_at(S_W, r, cc) : 0.f, u = s_at(S_U, r, cc), v = s_at(S_V, r, cc);
        const float ms = beta * beta + ix * ix + iy * iy;
        const float lin = it + ix * u + iy * v + (HAS_W ? beta * w : 0.f);
        const float divt = ix * dq1 + iy * dq2 + (HAS_W ? beta * dp : 0.f);
        float s_new;
        if (VARIANT == 0) s_new = (1.f - ms * inv_at) * s_old + (lin + c * divt) * inv_atc;
        else s_new = (1.f - rho * ms * inv_at) * s_old + (lin + c * rho * divt) * inv_atc;
        s_new = fminf(fmaxf(s_new, -lam), lam);  // P_s: projection onto |s| <= lambda
        const float cw = HAS_W ? beta * s_new - dp : 0.f;
        const float cu = ix * s_new - dq1, cv = iy * s_new - dq2;
        if (VARIANT == 0) {
            if (HAS_W) w -= rc * cw;
            u -= rc * cu;
            v -= rc * cv;
        } else {
            if (HAS_W) w -= c * (beta * s_new - rho * dp - (1.f - rho) * beta * s_old);
            u -= c * (ix * s_new - rho * dq1 - (1.f - rho) * ix * s_old);
            v -= c * (iy * s_new - rho * dq2 - (1.f - rho) * iy * s_old);
        }
        res += (double)cw * cw + (double)cu * cu + (double)cv * cv;
        if (HAS_W) {
            stT<T>(A.out.f[F_P1], o, s_at(S_P1, r, cc));
            stT<T>(A.out.f[F_P2], o, s_at(S_P2, r, cc));
            stT<T>(A.out.f[F_W], o, w);
        }
        stT<T>(A.out.f[F_Q11], o, s_at(S_Q11, r, cc));
        stT<T>(A.out.f[F_Q12], o, s_at(S_Q12, r, cc));
        stT<T>(A.out.f[F_Q21], o, s_at(S_Q21, r, cc));
        stT<T>(A.out.f[F_Q22], o, s_at(S_Q22, r, cc));
        stT<T>(A.out.f[F_S], o, s_new);
        stT<T>(A.out.f[F_U], o, u);
        stT<T>(A.out.f[F_V], o, v);
    }
    if (A.partials) {
        const double tot = block_sum(res, red);
        if (tid == 0) A.partials[block_linear_id()] = tot;
    }
}

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
    const float inv_a = 1.f / A.k.a, inv_c = 1.f / A.k.c, beta = A.k.beta;
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
        const float beta = A.k.beta, c = A.k.c, lam = A.k.lambda, rho = A.k.rho;
        const float at = a_tilde_of(A.k, A.ms_max);
        const float s_old = F(F_S)[o];
        float w = has_w ? F(F_W)[o] : 0.f, u = F(F_U)[o], v = F(F_V)[o];
        const float ms = beta * beta + ix * ix + iy * iy;
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

template <typename T>
__global__ void k_admm_residual(Fields f, const T *Ix, const T *Iy, Geom g, float beta, double *partials) {
    __shared__ double red[32];
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    const int H = g.H, W = g.W, P = g.pitch;
    const bool has_w = beta != 0.f;
    double res = 0.0;
    if (i < H && j < W) {
        const size_t o = (size_t)i * P + j;
        auto L = [&](int fi, int di, int dj) { return ldT<T>(f.f[fi], (size_t)(i + di) * P + (j + dj)); };
        auto dv = [&](int fa, int fb) {
            float d = 0.f;
            if (j < W - 1) d += L(fa, 0, 0);
            if (j > 0) d -= L(fa, 0, -1);
            if (i < H - 1) d += L(fb, 0, 0);
            if (i > 0) d -= L(fb, -1, 0);
            return d;
        };
        const float s = ldT<T>(f.f[F_S], o), ix = Store<T>::ld(Ix + o), iy = Store<T>::ld(Iy + o);
        const float cw = has_w ? beta * s - dv(F_P1, F_P2) : 0.f;
        const float cu = ix * s - dv(F_Q11, F_Q12), cv = iy * s - dv(F_Q21, F_Q22);
        res = (double)cw * cw + (double)cu * cu + (double)cv * cv;
    }
    const double tot = block_sum(res, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[block_linear_id()] = tot;
}

static_assert(FUSED_SMEM <= 48 * 1024, "fused ADMM tile must fit the default dynamic shared memory");

template <typename T, bool HAS_W, int VARIANT> void launch_fused_t(const IterArgs &a, cudaStream_t s) {
    dim3 grid((a.g.W + TX - 1) / TX, (a.g.H + TY - 1) / TY);
    k_admm_fused<T, HAS_W, VARIANT><<<grid, dim3(BX, BY), FUSED_SMEM, s>>>(a);
}

}  // namespace

int admm_fused_blocks(Geom g) { return ((g.W + TX - 1) / TX) * ((g.H + TY - 1) / TY); }
int admm_plain_blocks(Geom g) { return ((g.W + PX - 1) / PX) * ((g.H + PY - 1) / PY); }

void launch_admm_fused(const IterArgs &a, int prec, cudaStream_t s) {
    const bool has_w = a.k.beta != 0.f;
    TVL1_DISPATCH_PREC(prec, T, {
        if (a.k.method == 1) {
            if (has_w) launch_fused_t<T, true, 1>(a, s);
            else launch_fused_t<T, false, 1>(a, s);
        } else {
            if (has_w) launch_fused_t<T, true, 0>(a, s);
            else launch_fused_t<T, false, 0>(a, s);
        }
    });
}

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

void launch_admm_residual(const Fields &f, const void *Ix, const void *Iy, Geom g, float beta, int prec,
                          double *partials, cudaStream_t s) {
    dim3 grid((g.W + PX - 1) / PX, (g.H + PY - 1) / PY), blk(PX, PY);
    TVL1_DISPATCH_PREC(prec, T,
                       k_admm_residual<T><<<grid, blk, 0, s>>>(f, (const T *)Ix, (const T *)Iy, g, beta, partials));
}

}  // namespace tvl1
