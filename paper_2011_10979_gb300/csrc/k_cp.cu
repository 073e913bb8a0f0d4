// k_cp.cu -- ALG1, the comparison solver of Sec. 4: the first-order primal-dual method of
// Chambolle and Pock with constant steps (theta = 1) on the saddle-point form
// eq. (primal-dual:optical:o), K = (grad w, grad u, grad v), F = lambda ||rho(w, d)||_1:
//   y^{k+1}    = P(y^k + tau grad Xbar^k)                 (P_p on p, the joint P_q on q)
//   X^{k+1}    = prox_{sigma F}(X^k + sigma div y^{k+1})   (three-case L1 resolvent, eq. resolvent)
//   Xbar^{k+1} = 2 X^{k+1} - X^k
// with the steps tau (dual) and sigma = 1 / (8 tau) (primal).  One fused kernel per iteration
// reads one state buffer and writes the other.  A pixel needs y^{k+1} at itself and at its west
// and north neighbours; each thread projects those three dual vectors itself (the neighbours'
// own threads compute the same values), so the kernel needs no shared memory and no barrier
// except the residual's block sum.  Residual: ||X^{k+1} - X^k||^2 (FP64 block partials).
// Batched form: blockIdx.z selects pair pairs[z], which reads buf[parity] and writes
// buf[parity ^ 1]; its partials occupy cp_blocks(args.g) slots from z * cp_blocks(args.g).
#include <math.h>

#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

constexpr int PX = 32, PY = 8;

// 1 / max(1, sqrt(n2)): the scale of the projection onto the unit ball.
__device__ __forceinline__ float ball_scale_cp(float n2) { return n2 > 1.f ? rsqrtf(n2) : 1.f; }

template <typename T, typename TF, bool HAS_W>
__global__ void __launch_bounds__(PX *PY) k_cp(IterArgs A) {
    __shared__ double red[32];
    int H, W, P;
    Fields in, out;
    const void *Ixp, *Iyp, *Itp;
    const int *donep;
    if (A.pairs) {
        const PairIter *pp = A.pairs + blockIdx.z;
        const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
        H = gq.x;
        W = gq.y;
        P = gq.z;
        in = pp->buf[A.parity];
        out = pp->buf[A.parity ^ 1];
        Ixp = pp->Ix;
        Iyp = pp->Iy;
        Itp = pp->It;
        donep = pp->done;
    } else {
        H = A.g.H;
        W = A.g.W;
        P = A.g.pitch;
        in = A.in;
        out = A.out;
        Ixp = A.Ix;
        Iyp = A.Iy;
        Itp = A.It;
        donep = A.done;
    }
    if (donep && *donep) return;  // uniform per block: the pair's warp met its stopping test
    const float tau = A.k.cp_tau, sg = A.k.cp_sigma, beta = A.k.beta, lam = A.k.lambda;
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    float res = 0.f;
    if (i < H && j < W) {
        // y^{k+1} at pixel (a, b): the projected dual ascent step from grad Xbar^k
        auto dual = [&](int a, int b, float y[6]) {
            const size_t o = (size_t)a * P + b;
            const bool hx = b < W - 1, hy = a < H - 1;
            auto gx = [&](int f) { return hx ? ldT<TF>(in.f[f], o + 1) - ldT<TF>(in.f[f], o) : 0.f; };
            auto gy = [&](int f) { return hy ? ldT<TF>(in.f[f], o + P) - ldT<TF>(in.f[f], o) : 0.f; };
            if (HAS_W) {
                const float t1 = fmaf(tau, gx(F_WB), ldT<T>(in.f[F_P1], o));
                const float t2 = fmaf(tau, gy(F_WB), ldT<T>(in.f[F_P2], o));
                const float f = ball_scale_cp(fmaf(t1, t1, t2 * t2));
                y[0] = t1 * f;
                y[1] = t2 * f;
            } else {
                y[0] = y[1] = 0.f;
            }
            const float t11 = fmaf(tau, gx(F_UB), ldT<T>(in.f[F_Q11], o));
            const float t12 = fmaf(tau, gy(F_UB), ldT<T>(in.f[F_Q12], o));
            const float t21 = fmaf(tau, gx(F_VB), ldT<T>(in.f[F_Q21], o));
            const float t22 = fmaf(tau, gy(F_VB), ldT<T>(in.f[F_Q22], o));
            const float f = ball_scale_cp(fmaf(t11, t11, fmaf(t12, t12, fmaf(t21, t21, t22 * t22))));
            y[2] = t11 * f;
            y[3] = t12 * f;
            y[4] = t21 * f;
            y[5] = t22 * f;
        };
        float y0[6], yw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, yn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        dual(i, j, y0);
        if (j > 0) dual(i, j - 1, yw);
        if (i > 0) dual(i - 1, j, yn);
        const bool ex = j < W - 1, ey = i < H - 1;
        // div y^{k+1} = -K^* y^{k+1} (forward differences, Neumann)
        auto dv = [&](int cx, int cy) { return (((ex ? y0[cx] : 0.f) - yw[cx]) + (ey ? y0[cy] : 0.f)) - yn[cy]; };
        const size_t o = (size_t)i * P + j;
        const float xw = HAS_W ? ldT<TF>(in.f[F_W], o) : 0.f;
        const float xu = ldT<TF>(in.f[F_U], o), xv = ldT<TF>(in.f[F_V], o);
        float zw = HAS_W ? fmaf(sg, dv(0, 1), xw) : 0.f;
        float zu = fmaf(sg, dv(2, 3), xu), zv = fmaf(sg, dv(4, 5), xv);
        // prox_{sigma F}: X = Z + t e with e = (beta, Ix, Iy), three cases of rho(Z) against sigma lambda |e|^2
        const float ix = ldT<T>(Ixp, o), iy = ldT<T>(Iyp, o), it = ldT<T>(Itp, o);
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
        if (HAS_W) {
            stT<T>(out.f[F_P1], o, y0[0]);
            stT<T>(out.f[F_P2], o, y0[1]);
            stT<TF>(out.f[F_W], o, zw);
            stT<TF>(out.f[F_WB], o, 2.f * zw - xw);
        }
        stT<T>(out.f[F_Q11], o, y0[2]);
        stT<T>(out.f[F_Q12], o, y0[3]);
        stT<T>(out.f[F_Q21], o, y0[4]);
        stT<T>(out.f[F_Q22], o, y0[5]);
        stT<TF>(out.f[F_U], o, zu);
        stT<TF>(out.f[F_V], o, zv);
        stT<TF>(out.f[F_UB], o, 2.f * zu - xu);
        stT<TF>(out.f[F_VB], o, 2.f * zv - xv);
        const float dw = zw - xw, du = zu - xu, dd = zv - xv;
        res = fmaf(dd, dd, fmaf(du, du, dw * dw));
    }
    if (A.partials) {
        const double tot = block_sum((double)res, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) A.partials[block_linear_id()] = tot;
    }
}

template <typename T, typename TF> void launch_t(const IterArgs &a, cudaStream_t s) {
    dim3 grid((a.g.W + PX - 1) / PX, (a.g.H + PY - 1) / PY, a.pairs ? a.ntiles : 1), blk(PX, PY);
    if (a.k.beta != 0.f) k_cp<T, TF, true><<<grid, blk, 0, s>>>(a);
    else k_cp<T, TF, false><<<grid, blk, 0, s>>>(a);
}

}  // namespace

int cp_blocks(Geom g) { return ((g.W + PX - 1) / PX) * ((g.H + PY - 1) / PY); }

void launch_cp(const IterArgs &a, int prec, int prec_flow, cudaStream_t s) {
    if (prec == PREC_F32) launch_t<float, float>(a, s);
    else if (prec == PREC_F16 && prec_flow == PREC_F32) launch_t<__half, float>(a, s);
    else if (prec == PREC_F16) launch_t<__half, __half>(a, s);
    else if (prec_flow == PREC_F32) launch_t<__nv_bfloat16, float>(a, s);
    else launch_t<__nv_bfloat16, __nv_bfloat16>(a, s);
}

}  // namespace tvl1
