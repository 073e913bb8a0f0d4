// k_adapt.cu -- opt-in residual balancing of the ADMM step c (an extension of Sec. 3.1.1; the
// paper keeps c fixed).  Prop. 3.1's conditions bound only a and a~ (eq. stepsize:constraint), so
// every c > 0 keeps both proximal metrics c(aI - grad grad^*) and c(a~ - M_s) positive
// semidefinite; the multipliers (w, u, v) are stored unscaled, so changing c needs no rescaling.
//
// After an iteration k -> k+1 of eq. (aug:pre1:vector) the optimality conditions of its two
// subproblems leave, beside the constraint residual r = A s + B y, the dual residual
//   d_y = c (B^*A (s^{k+1} - s^k) - (a I - B^*B)(y^{k+1} - y^k)),
//   d_s = c (M_s - a~)(s^{k+1} - s^k),
// with B^*A ds = (grad(beta ds), grad(Ix ds), grad(Iy ds)) and B^*B dy = -grad div dy per
// component.  The balancing rule doubles c when ||r|| > 10 ||d|| and halves it when
// ||d|| > 10 ||r|| (residual balancing, He, Yang and Wang 2000).  k_adapt_residuals forms both
// squared norms (FP32 per pixel, FP64 block sums), k_adapt_update sums the blocks in a fixed order
// and rescales the device copy of c that the iteration kernels read.
#include <math.h>

#include "tvl1_device.cuh"

namespace tvl1 {
namespace {

constexpr int ADAPT_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(ADAPT_THREADS) k_adapt_residuals(AdaptArgs A) {
    __shared__ double sh[32];
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    const float c = c_of(A.k, A.ms_max), a = A.k.a, beta = A.k.beta;
    const float at_warp = a_tilde_of(A.k, A.ms_max);
    auto cur = [&](int f, int i, int j) { return ldT<T>(A.cur.f[f], (size_t)i * P + j); };
    auto dl = [&](int f, int i, int j) { return cur(f, i, j) - ldT<T>(A.prev.f[f], (size_t)i * P + j); };
    auto ix = [&](int i, int j) { return ldT<T>(A.Ix, (size_t)i * P + j); };
    auto iy = [&](int i, int j) { return ldT<T>(A.Iy, (size_t)i * P + j); };
    // discrete divergence (Sec. 2.2) of a 2-vector field given by an accessor of its components
    auto divg = [&](auto fx, auto fy, int i, int j) {
        float v = 0.f;
        if (j < W - 1) v += fx(i, j);
        if (j > 0) v -= fx(i, j - 1);
        if (i < H - 1) v += fy(i, j);
        if (i > 0) v -= fy(i - 1, j);
        return v;
    };
    double r2 = 0.0, d2 = 0.0;
    const long long n = (long long)H * W;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / W), j = (int)(q % W);
        const bool hx = j < W - 1, hy = i < H - 1;
        // constraint residual A s + B y at the new state
        const float s = cur(F_S, i, j), ixo = ix(i, j), iyo = iy(i, j);
        auto c1 = [&](int f) { return [&, f](int ii, int jj) { return cur(f, ii, jj); }; };
        auto d1 = [&](int f) { return [&, f](int ii, int jj) { return dl(f, ii, jj); }; };
        const float ru = ixo * s - divg(c1(F_Q11), c1(F_Q12), i, j);
        const float rv = iyo * s - divg(c1(F_Q21), c1(F_Q22), i, j);
        float rr = ru * ru + rv * rv;
        // dual residual; the forward difference of a product field g at (i, j)
        const float ds = dl(F_S, i, j);
        auto gxp = [&](auto g) { return hx ? g(i, j + 1) - g(i, j) : 0.f; };
        auto gyp = [&](auto g) { return hy ? g(i + 1, j) - g(i, j) : 0.f; };
        auto dsix = [&](int ii, int jj) { return ix(ii, jj) * dl(F_S, ii, jj); };
        auto dsiy = [&](int ii, int jj) { return iy(ii, jj) * dl(F_S, ii, jj); };
        auto ddq1 = [&](int ii, int jj) { return divg(d1(F_Q11), d1(F_Q12), ii, jj); };
        auto ddq2 = [&](int ii, int jj) { return divg(d1(F_Q21), d1(F_Q22), ii, jj); };
        const float e11 = c * (gxp(dsix) - a * dl(F_Q11, i, j) - gxp(ddq1));
        const float e12 = c * (gyp(dsix) - a * dl(F_Q12, i, j) - gyp(ddq1));
        const float e21 = c * (gxp(dsiy) - a * dl(F_Q21, i, j) - gxp(ddq2));
        const float e22 = c * (gyp(dsiy) - a * dl(F_Q22, i, j) - gyp(ddq2));
        float dd = e11 * e11 + e12 * e12 + e21 * e21 + e22 * e22;
        if (A.has_w) {
            const float rw = beta * s - divg(c1(F_P1), c1(F_P2), i, j);
            rr += rw * rw;
            auto dsb = [&](int ii, int jj) { return beta * dl(F_S, ii, jj); };
            auto ddp = [&](int ii, int jj) { return divg(d1(F_P1), d1(F_P2), ii, jj); };
            const float e1 = c * (gxp(dsb) - a * dl(F_P1, i, j) - gxp(ddp));
            const float e2 = c * (gyp(dsb) - a * dl(F_P2, i, j) - gyp(ddp));
            dd += e1 * e1 + e2 * e2;
        }
        const float ms = beta * beta + ixo * ixo + iyo * iyo;
        const float at = A.k.a_tilde_mode == 1 ? fmaxf(ms, 1e-12f) : at_warp;
        const float es = c * (ms - at) * ds;
        dd += es * es;
        r2 += rr;
        d2 += dd;
    }
    r2 = block_sum(r2, sh);
    __syncthreads();
    d2 = block_sum(d2, sh);
    if (threadIdx.x == 0) {
        A.part_r[blockIdx.x] = r2;
        A.part_d[blockIdx.x] = d2;
    }
}

// pDR (Sec. 3.1.2 leaves sigma and tau free; the balancing moves their ratio with sigma tau fixed, so
// T = I - sigma tau Laplace and its SRBGS preconditioner stay the same): the squared changes of the
// primal block X = (w, u, v) and of the dual block ybar over the step prev -> cur.
template <typename T, typename TF>
__global__ void __launch_bounds__(ADAPT_THREADS) k_adapt_pdr_residuals(AdaptArgs A) {
    __shared__ double sh[32];
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    double x2 = 0.0, y2 = 0.0;
    const long long n = (long long)H * W;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const size_t o = (size_t)(q / W) * P + (size_t)(q % W);
        float xx = 0.f, yy = 0.f;
#pragma unroll
        for (int f = F_W; f <= F_V; ++f) {
            if (f == F_W && !A.has_w) continue;
            const float e = ldT<TF>(A.cur.f[f], o) - ldT<TF>(A.prev.f[f], o);
            xx = fmaf(e, e, xx);
        }
#pragma unroll
        for (int f = F_P1; f <= F_Q22; ++f) {
            if ((f == F_P1 || f == F_P2) && !A.has_w) continue;
            const float e = ldT<T>(A.cur.f[f], o) - ldT<T>(A.prev.f[f], o);
            yy = fmaf(e, e, yy);
        }
        x2 += xx;
        y2 += yy;
    }
    x2 = block_sum(x2, sh);
    __syncthreads();
    y2 = block_sum(y2, sh);
    if (threadIdx.x == 0) {
        A.part_r[blockIdx.x] = x2;
        A.part_d[blockIdx.x] = y2;
    }
}

__global__ void __launch_bounds__(ADAPT_THREADS) k_adapt_update(AdaptArgs A, int nb) {
    __shared__ double sh[32];
    double r2 = 0.0, d2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        r2 += A.part_r[b];
        d2 += A.part_d[b];
    }
    r2 = block_sum(r2, sh);
    __syncthreads();
    d2 = block_sum(d2, sh);
    if (threadIdx.x == 0) {
        float *c = A.c;
        double r = sqrt(r2), d = sqrt(d2);
        if (A.pdr) {  // primal change per unit sigma against dual change per unit tau; *c is theta
            r /= (double)(A.k.sigma * *c);
            d /= (double)(A.k.tau / *c);
        }
        if (r > 10.0 * d) *c = *c * 2.f;
        else if (d > 10.0 * r) *c = *c * 0.5f;
    }
}

__global__ void k_c_init(float *c, float c0) { *c = c0; }

}  // namespace

int adapt_blocks(Geom g) {
    const long long n = (long long)g.H * g.W;
    const long long b = (n + ADAPT_THREADS - 1) / ADAPT_THREADS;
    return (int)(b < ADAPT_MAX_BLOCKS ? b : ADAPT_MAX_BLOCKS);
}

void launch_adapt_c(const AdaptArgs &a, int prec, int prec_flow, cudaStream_t s) {
    const int nb = adapt_blocks(a.g);
    if (a.pdr) {
        TVL1_DISPATCH_PREC(prec, T, TVL1_DISPATCH_PREC(prec_flow, TF, k_adapt_pdr_residuals<T, TF><<<nb, ADAPT_THREADS, 0, s>>>(a)));
    } else {
        TVL1_DISPATCH_PREC(prec, T, k_adapt_residuals<T><<<nb, ADAPT_THREADS, 0, s>>>(a));
    }
    k_adapt_update<<<1, ADAPT_THREADS, 0, s>>>(a, nb);
}

void launch_c_init(float *c, float c0, cudaStream_t s) { k_c_init<<<1, 1, 0, s>>>(c, c0); }

}  // namespace tvl1
