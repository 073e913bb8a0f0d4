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
// Batched form: slice z of the grid works on pair k = plist[z] (the level's pairs that are not on
// the level-resident engine), which reads buf[parity] and writes buf[parity ^ 1]; its partials
// occupy cp_blocks(args.g) slots from k * cp_blocks(args.g).
// Storage: the dual y is kept in the flow fields' type TF, like X and Xbar (FP32 under fp32_flow):
// it moves by constant steps tau = 0.1, which an 8-bit mantissa would round away; only the
// linearisation data is stored in T.
#include <math.h>

#include "k_cp_math.cuh"
#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

// Blocks of 32 columns by PY rows: 4, 8 (the default) or 16, the autotuner's choice.  The height is
// a template parameter with launch bounds of its own: a run-time height under one 512-thread bound
// measured 37% slower per iteration at 640x480 (12.4 against 9.0 us).
constexpr int PX = 32, PY_DEFAULT = 8;

template <typename T, typename TF, bool HAS_W, int PY>
__global__ void __launch_bounds__(PX *PY) k_cp(IterArgs A) {
    __shared__ double red[32];
    int H, W, P;
    Fields in, out;
    const void *Ixp, *Iyp, *Itp;
    const int *donep;
    int pair = 0;
    if (A.pairs) {
        pair = A.plist[blockIdx.z];
        const PairIter *pp = A.pairs + pair;
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
            float y0[6], g[6];
            y0[0] = HAS_W ? ldT<TF>(in.f[F_P1], o) : 0.f;
            y0[1] = HAS_W ? ldT<TF>(in.f[F_P2], o) : 0.f;
            y0[2] = ldT<TF>(in.f[F_Q11], o);
            y0[3] = ldT<TF>(in.f[F_Q12], o);
            y0[4] = ldT<TF>(in.f[F_Q21], o);
            y0[5] = ldT<TF>(in.f[F_Q22], o);
            g[0] = HAS_W ? gx(F_WB) : 0.f;
            g[1] = HAS_W ? gy(F_WB) : 0.f;
            g[2] = gx(F_UB);
            g[3] = gy(F_UB);
            g[4] = gx(F_VB);
            g[5] = gy(F_VB);
            cp_dual<HAS_W>(y0, g, tau, y);
        };
        float y0[6], yw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, yn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        dual(i, j, y0);
        if (j > 0) dual(i, j - 1, yw);
        if (i > 0) dual(i - 1, j, yn);
        const bool ex = j < W - 1, ey = i < H - 1;
        // div y^{k+1} = -K^* y^{k+1} (forward differences, Neumann)
        auto dv = [&](int cx, int cy) { return (((ex ? y0[cx] : 0.f) - yw[cx]) + (ey ? y0[cy] : 0.f)) - yn[cy]; };
        const size_t o = (size_t)i * P + j;
        float x[3] = {HAS_W ? ldT<TF>(in.f[F_W], o) : 0.f, ldT<TF>(in.f[F_U], o), ldT<TF>(in.f[F_V], o)};
        const float xold[3] = {x[0], x[1], x[2]};
        const float d3[3] = {HAS_W ? dv(0, 1) : 0.f, dv(2, 3), dv(4, 5)};
        res = cp_primal<HAS_W>(x, d3, ldT<T>(Ixp, o), ldT<T>(Iyp, o), ldT<T>(Itp, o), beta, lam, sg);
        if (HAS_W) {
            stT<TF>(out.f[F_P1], o, y0[0]);
            stT<TF>(out.f[F_P2], o, y0[1]);
            stT<TF>(out.f[F_W], o, x[0]);
            stT<TF>(out.f[F_WB], o, 2.f * x[0] - xold[0]);
        }
        stT<TF>(out.f[F_Q11], o, y0[2]);
        stT<TF>(out.f[F_Q12], o, y0[3]);
        stT<TF>(out.f[F_Q21], o, y0[4]);
        stT<TF>(out.f[F_Q22], o, y0[5]);
        stT<TF>(out.f[F_U], o, x[1]);
        stT<TF>(out.f[F_V], o, x[2]);
        stT<TF>(out.f[F_UB], o, 2.f * x[1] - xold[1]);
        stT<TF>(out.f[F_VB], o, 2.f * x[2] - xold[2]);
    }
    if (A.partials) {
        const double tot = block_sum((double)res, red);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            A.partials[(size_t)pair * gridDim.x * gridDim.y + blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

int block_rows(int tile_h) { return (tile_h == 4 || tile_h == 16) ? tile_h : PY_DEFAULT; }

template <typename T, typename TF, int PY> void launch_py(const IterArgs &a, cudaStream_t s) {
    dim3 grid((a.g.W + PX - 1) / PX, (a.g.H + PY - 1) / PY, a.pairs ? a.ntiles : 1), blk(PX, PY);
    if (a.k.beta != 0.f) k_cp<T, TF, true, PY><<<grid, blk, 0, s>>>(a);
    else k_cp<T, TF, false, PY><<<grid, blk, 0, s>>>(a);
}

template <typename T, typename TF> void launch_t(const IterArgs &a, cudaStream_t s) {
    switch (block_rows(a.tile_h)) {
    case 4: launch_py<T, TF, 4>(a, s); break;
    case 16: launch_py<T, TF, 16>(a, s); break;
    default: launch_py<T, TF, 8>(a, s); break;
    }
}

}  // namespace

int cp_blocks(Geom g, int tile_h) {
    const int py = block_rows(tile_h);
    return ((g.W + PX - 1) / PX) * ((g.H + py - 1) / py);
}

void launch_cp(const IterArgs &a, int prec, int prec_flow, cudaStream_t s) {
    if (prec == PREC_F32) launch_t<float, float>(a, s);
    else if (prec == PREC_F16 && prec_flow == PREC_F32) launch_t<__half, float>(a, s);
    else if (prec == PREC_F16) launch_t<__half, __half>(a, s);
    else if (prec_flow == PREC_F32) launch_t<__nv_bfloat16, float>(a, s);
    else launch_t<__nv_bfloat16, __nv_bfloat16>(a, s);
}

}  // namespace tvl1
