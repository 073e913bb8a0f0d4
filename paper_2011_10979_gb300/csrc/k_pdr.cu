// k_pdr.cu -- preconditioned Douglas-Rachford iteration of Sec. 3.1.2, eq. (pDR) for the flow
// model, for each primal component X_c in (w, u, v) with its barred dual ybar_c:
//   b = Xbar + sigma div ybar;  X^{k+1} = SRBGS^n(T, b, X^k) with T = I - sigma tau Laplace
//   (Neumann); Xbar^{k+1} = Xbar + prox_{sigma F}(2X^{k+1} - Xbar) - X^{k+1} with the three-case
//   resolvent eq. (resolvent); ybar^{k+1} = P(ybar + 2 tau grad X^{k+1}) - tau grad X^{k+1}.
// A red-black Gauss-Seidel half-sweep updates one colour from the other colour's values only, so
// it is data-parallel and in place.  One symmetric sweep is red, black, black, red; the repeated
// black half-sweep recomputes identical values, so the fused engine runs red (black red)^n, the
// plain engine the literal sequence.  Both give bitwise identical results.  The fused engine takes
// 2n + 1 launches per iteration: the right-hand side with the first red half-sweep, the half-sweeps
// between, and the last red half-sweep with the Xbar / ybar updates.
#include <math.h>

#include <mutex>
#include <type_traits>

#include "k_pdr_math.cuh"
#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

// Blocks of 32 columns by blockDim.y rows: 4, 8 (the default) or 16, the autotuner's choice.
constexpr int PX = 32, PY_DEFAULT = 8;

int block_rows(int tile_h) { return (tile_h == 4 || tile_h == 16) ? tile_h : PY_DEFAULT; }

// The planes one block works on: the single pair of the launch, or in a batch the pair
// plist[blockIdx.z] (the level's pairs not on the level-resident engine; all pairs if plist is
// NULL).  Partial sums go to slot pair * (blocks per slice) + block within the slice.
struct PView {
    Geom g;
    Fields f;
    const void *Ix, *Iy, *It;
    float *tmp;
    const int *done;
    int pair;
};

__device__ __forceinline__ PView view_of(const IterArgs &A) {
    // geometry in plain scalars from one 16-byte load per mode (as in k_admm_roll.cuh)
    PView v;
    v.pair = 0;
    if (A.pairs) {
        v.pair = A.plist ? A.plist[blockIdx.z] : (int)blockIdx.z;
        const PairIter *pp = A.pairs + v.pair;
        const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
        v.g.H = gq.x;
        v.g.W = gq.y;
        v.g.pitch = gq.z;
        v.f = pp->buf[A.parity];
        v.Ix = pp->Ix;
        v.Iy = pp->Iy;
        v.It = pp->It;
        v.tmp = pp->tmp;
        v.done = pp->done;
    } else {
        v.g.H = A.g.H;
        v.g.W = A.g.W;
        v.g.pitch = A.g.pitch;
        v.f = A.in;
        v.Ix = A.Ix;
        v.Iy = A.Iy;
        v.It = A.It;
        v.tmp = A.tmp;
        v.done = A.done;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ float div_at(const void *a, const void *b, int i, int j, int H, int W, int P) {
    const size_t o = (size_t)i * P + j;
    return (((j < W - 1 ? ldT<T>(a, o) : 0.f) - (j > 0 ? ldT<T>(a, o - 1) : 0.f)) + (i < H - 1 ? ldT<T>(b, o) : 0.f)) -
           (i > 0 ? ldT<T>(b, o - P) : 0.f);
}

__device__ __forceinline__ size_t partial_slot(const PView &V) {
    return (size_t)V.pair * gridDim.x * gridDim.y + blockIdx.x + gridDim.x * blockIdx.y;
}

// b_c = Xbar_c + sigma div ybar_c, and a copy of X^k for the residual (FP32 planes in tmp).
template <typename T, typename TF, bool HAS_W>
__global__ void k_pdr_b(IterArgs A) {
    const PView V = view_of(A);
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
    const int H = V.g.H, W = V.g.W, P = V.g.pitch;
    if (i >= H || j >= W) return;
    if (V.done && *V.done) return;
    float *tmp = V.tmp;
    const size_t o = (size_t)i * P + j, plane = (size_t)H * P;
    const int X[3] = {F_W, F_U, F_V}, XB[3] = {F_WB, F_UB, F_VB};
    const int Y1[3] = {F_P1, F_Q11, F_Q21}, Y2[3] = {F_P2, F_Q12, F_Q22};
#pragma unroll
    for (int c = HAS_W ? 0 : 1; c < 3; ++c) {
        tmp[c * plane + o] = pdr_rhs(ldT<TF>(V.f.f[XB[c]], o), div_at<T>(V.f.f[Y1[c]], V.f.f[Y2[c]], i, j, H, W, P), A.k.sigma);
        tmp[(3 + c) * plane + o] = ldT<TF>(V.f.f[X[c]], o);
    }
}

// The Gauss-Seidel update of component c at pixel (a, b) from b (tmp plane c) and the current X of
// its in-domain neighbours (west, east, north, south), rounded to the flow storage type as a store
// and a load would round it.
template <typename TF>
__device__ __forceinline__ float gs_value(const PView &V, const float *tmp, size_t plane, int c, int a, int b,
                                          float st) {
    const int H = V.g.H, W = V.g.W, P = V.g.pitch;
    const int X[3] = {F_W, F_U, F_V};
    const void *x = V.f.f[X[c]];
    const size_t o = (size_t)a * P + b;
    float acc = 0.f;
    int nb = 0;
    if (b > 0) { acc += ldT<TF>(x, o - 1); ++nb; }
    if (b < W - 1) { acc += ldT<TF>(x, o + 1); ++nb; }
    if (a > 0) { acc += ldT<TF>(x, o - P); ++nb; }
    if (a < H - 1) { acc += ldT<TF>(x, o + P); ++nb; }
    return storage_round<TF>(pdr_gs(tmp[c * plane + o], acc, nb, st));
}

// Fused engine, first kernel of an iteration: b = Xbar + sigma div ybar and X^k at every pixel,
// then the red half-sweep at the red pixels (a red update reads only its own b and the black
// neighbours, which this kernel does not write).
template <typename T, typename TF, bool HAS_W>
__global__ void k_pdr_b_red(IterArgs A) {
    const PView V = view_of(A);
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
    const int H = V.g.H, W = V.g.W, P = V.g.pitch;
    if (i >= H || j >= W) return;
    if (V.done && *V.done) return;
    float *tmp = V.tmp;
    const size_t o = (size_t)i * P + j, plane = (size_t)H * P;
    const int X[3] = {F_W, F_U, F_V}, XB[3] = {F_WB, F_UB, F_VB};
    const int Y1[3] = {F_P1, F_Q11, F_Q21}, Y2[3] = {F_P2, F_Q12, F_Q22};
#pragma unroll
    for (int c = HAS_W ? 0 : 1; c < 3; ++c) {
        tmp[c * plane + o] = pdr_rhs(ldT<TF>(V.f.f[XB[c]], o), div_at<T>(V.f.f[Y1[c]], V.f.f[Y2[c]], i, j, H, W, P), A.k.sigma);
        tmp[(3 + c) * plane + o] = ldT<TF>(V.f.f[X[c]], o);
    }
    if (((i + j) & 1) == 0) {
        const float st = A.k.sigma * A.k.tau;
#pragma unroll
        for (int c = HAS_W ? 0 : 1; c < 3; ++c) stT<TF>(V.f.f[X[c]], o, gs_value<TF>(V, tmp, plane, c, i, j, st));
    }
}

// Fused engine, last kernel of an iteration: the final red half-sweep and the Xbar / ybar updates.
// X^{k+1} at a red pixel is its red update (black neighbours final); a black pixel's east and south
// neighbours are red, so its thread recomputes their updates (the same value their own threads
// store) instead of waiting for them.  This kernel writes only red pixels' X and reads only black
// pixels' X, so no thread reads a value another thread of it writes.
template <typename T, typename TF, bool HAS_W>
__global__ void k_pdr_red_finish(IterArgs A) {
    __shared__ double red[32];
    const PView V = view_of(A);
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
    const int H = V.g.H, W = V.g.W, P = V.g.pitch;
    if (V.done && *V.done) return;
    const float *tmp = V.tmp;
    double res = 0.0;
    if (i < H && j < W) {
        const size_t o = (size_t)i * P + j, plane = (size_t)H * P;
        const float beta = A.k.beta, lam = A.k.lambda, sg = A.k.sigma, ta = A.k.tau, st = sg * ta;
        const int X[3] = {F_W, F_U, F_V};
        auto xnew = [&](int a, int b, int c) {
            return ((a + b) & 1) == 0 ? gs_value<TF>(V, tmp, plane, c, a, b, st)
                                      : ldT<TF>(V.f.f[X[c]], (size_t)a * P + b);
        };
        const bool hx = j < W - 1, hy = i < H - 1, is_red = ((i + j) & 1) == 0;
        float x[3] = {0.f, 0.f, 0.f}, g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = HAS_W ? 0 : 1; c < 3; ++c) {
            x[c] = xnew(i, j, c);
            g[2 * c] = hx ? xnew(i, j + 1, c) - x[c] : 0.f;
            g[2 * c + 1] = hy ? xnew(i + 1, j, c) - x[c] : 0.f;
        }
        const float ix = ldT<T>(V.Ix, o), iy = ldT<T>(V.Iy, o), it = ldT<T>(V.It, o);
        float xb[3] = {HAS_W ? ldT<TF>(V.f.f[F_WB], o) : 0.f, ldT<TF>(V.f.f[F_UB], o), ldT<TF>(V.f.f[F_VB], o)};
        if (HAS_W) pdr_xbar<true>(x, xb, ix, iy, it, beta, lam, sg);
        else pdr_xbar<false>(x, xb, ix, iy, it, beta, lam, sg);
        const float y[6] = {HAS_W ? ldT<T>(V.f.f[F_P1], o) : 0.f, HAS_W ? ldT<T>(V.f.f[F_P2], o) : 0.f,
                            ldT<T>(V.f.f[F_Q11], o), ldT<T>(V.f.f[F_Q12], o), ldT<T>(V.f.f[F_Q21], o),
                            ldT<T>(V.f.f[F_Q22], o)};
        float yn[6];
        if (HAS_W) pdr_ybar<true>(y, g, ta, yn);
        else pdr_ybar<false>(y, g, ta, yn);
        if (is_red) {
#pragma unroll
            for (int c = HAS_W ? 0 : 1; c < 3; ++c) stT<TF>(V.f.f[X[c]], o, x[c]);
        }
        if (HAS_W) {
            stT<TF>(V.f.f[F_WB], o, xb[0]);
            stT<T>(V.f.f[F_P1], o, yn[0]);
            stT<T>(V.f.f[F_P2], o, yn[1]);
        }
        stT<TF>(V.f.f[F_UB], o, xb[1]);
        stT<TF>(V.f.f[F_VB], o, xb[2]);
        stT<T>(V.f.f[F_Q11], o, yn[2]);
        stT<T>(V.f.f[F_Q12], o, yn[3]);
        stT<T>(V.f.f[F_Q21], o, yn[4]);
        stT<T>(V.f.f[F_Q22], o, yn[5]);
        const float dw = HAS_W ? x[0] - tmp[3 * plane + o] : 0.f;
        const float du = x[1] - tmp[4 * plane + o], dv = x[2] - tmp[5 * plane + o];
        res = (double)dw * dw + (double)du * du + (double)dv * dv;
    }
    if (A.partials) {
        const double tot = block_sum(res, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) A.partials[partial_slot(V)] = tot;
    }
}

// One red (colour 0) or black (colour 1) Gauss-Seidel half-sweep on (1 + st n_ij) x_ij - st sum x_nb = b_ij.
template <typename T, typename TF, bool HAS_W>
__global__ void k_gs_half(IterArgs A, int colour) {
    const PView V = view_of(A);
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
    const int H = V.g.H, W = V.g.W, P = V.g.pitch;
    if (i >= H || j >= W || ((i + j) & 1) != colour) return;
    if (V.done && *V.done) return;
    const float *tmp = V.tmp;
    const size_t o = (size_t)i * P + j, plane = (size_t)H * P;
    const float st = A.k.sigma * A.k.tau;
    const int X[3] = {F_W, F_U, F_V};
#pragma unroll
    for (int c = HAS_W ? 0 : 1; c < 3; ++c) {
        const void *x = V.f.f[X[c]];
        float acc = 0.f;
        int nb = 0;
        if (j > 0) { acc += ldT<TF>(x, o - 1); ++nb; }
        if (j < W - 1) { acc += ldT<TF>(x, o + 1); ++nb; }
        if (i > 0) { acc += ldT<TF>(x, o - P); ++nb; }
        if (i < H - 1) { acc += ldT<TF>(x, o + P); ++nb; }
        stT<TF>(V.f.f[X[c]], o, pdr_gs(tmp[c * plane + o], acc, nb, st));
    }
}

// Xbar update through the L1 resolvent, ybar update, residual partial ||X^{k+1} - X^k||^2.
template <typename T, typename TF, bool HAS_W>
__global__ void k_pdr_finish(IterArgs A) {
    __shared__ double red[32];
    const PView V = view_of(A);
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
    const int H = V.g.H, W = V.g.W, P = V.g.pitch;
    if (V.done && *V.done) return;
    const float *tmp = V.tmp;
    double res = 0.0;
    if (i < H && j < W) {
        const size_t o = (size_t)i * P + j, plane = (size_t)H * P;
        const float beta = A.k.beta, lam = A.k.lambda, sg = A.k.sigma, ta = A.k.tau;
        const float ix = ldT<T>(V.Ix, o), iy = ldT<T>(V.Iy, o), it = ldT<T>(V.It, o);
        const float x[3] = {HAS_W ? ldT<TF>(V.f.f[F_W], o) : 0.f, ldT<TF>(V.f.f[F_U], o), ldT<TF>(V.f.f[F_V], o)};
        float xb[3] = {HAS_W ? ldT<TF>(V.f.f[F_WB], o) : 0.f, ldT<TF>(V.f.f[F_UB], o), ldT<TF>(V.f.f[F_VB], o)};
        if (HAS_W) pdr_xbar<true>(x, xb, ix, iy, it, beta, lam, sg);
        else pdr_xbar<false>(x, xb, ix, iy, it, beta, lam, sg);
        if (HAS_W) stT<TF>(V.f.f[F_WB], o, xb[0]);
        stT<TF>(V.f.f[F_UB], o, xb[1]);
        stT<TF>(V.f.f[F_VB], o, xb[2]);
        const bool hx = j < W - 1, hy = i < H - 1;
        auto gx = [&](int f, float x0) { return hx ? ldT<TF>(V.f.f[f], o + 1) - x0 : 0.f; };
        auto gy = [&](int f, float x0) { return hy ? ldT<TF>(V.f.f[f], o + P) - x0 : 0.f; };
        const float g[6] = {HAS_W ? gx(F_W, x[0]) : 0.f, HAS_W ? gy(F_W, x[0]) : 0.f, gx(F_U, x[1]), gy(F_U, x[1]),
                            gx(F_V, x[2]), gy(F_V, x[2])};
        const float y[6] = {HAS_W ? ldT<T>(V.f.f[F_P1], o) : 0.f, HAS_W ? ldT<T>(V.f.f[F_P2], o) : 0.f,
                            ldT<T>(V.f.f[F_Q11], o), ldT<T>(V.f.f[F_Q12], o), ldT<T>(V.f.f[F_Q21], o),
                            ldT<T>(V.f.f[F_Q22], o)};
        float yn[6];
        if (HAS_W) pdr_ybar<true>(y, g, ta, yn);
        else pdr_ybar<false>(y, g, ta, yn);
        if (HAS_W) {
            stT<T>(V.f.f[F_P1], o, yn[0]);
            stT<T>(V.f.f[F_P2], o, yn[1]);
        }
        stT<T>(V.f.f[F_Q11], o, yn[2]);
        stT<T>(V.f.f[F_Q12], o, yn[3]);
        stT<T>(V.f.f[F_Q21], o, yn[4]);
        stT<T>(V.f.f[F_Q22], o, yn[5]);
        const float dw = HAS_W ? x[0] - tmp[3 * plane + o] : 0.f;
        const float du = x[1] - tmp[4 * plane + o], dv = x[2] - tmp[5 * plane + o];
        res = (double)dw * dw + (double)du * du + (double)dv * dv;
    }
    if (A.partials) {
        const double tot = block_sum(res, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) A.partials[partial_slot(V)] = tot;
    }
}

// ---------------------------------------------------------------- one launch per iteration
// The whole iteration (gs_sweeps = 1: red, black, red) for a TT x TT tile of output pixels in one
// block, reading buffer `in` and writing buffer `out` (ping-pong, so no block reads what another
// writes).  The chain of dependencies fixes the tile's halo: the ybar update needs X^{k+1} one
// pixel east and south; X^{k+1} at a red pixel is its second red update, which needs black values
// one pixel around, which need first red values one more pixel around, which need X^k (the old
// black values) and b one more; b needs ybar one pixel west and north.  So the block stages, in
// a (TT + 7)^2 frame starting 3 pixels above and left of the tile, X^k on the whole frame, ybar on
// offsets -3 .. TT + 2 and Xbar on -2 .. TT + 2, and runs the stages on shrinking squares between
// block barriers: b and the first red half-sweep on -2 .. TT + 2, black on -1 .. TT + 1, the
// second red on 0 .. TT, then the Xbar / ybar updates and the stores on the tile.  Each stage's
// arithmetic and rounding (X rounded to its storage type after every half-sweep, b in FP32) is
// that of the per-kernel engine, so the flows are bitwise equal; the residual's partial sums are
// grouped per tile.
// Tiles of TT x TT output pixels: 32 (512 threads), or 16 (256 threads) on levels with fewer
// 32-pixel tiles than SMs, where the larger tiles would leave most of the GPU idle.
enum { TX0 = 0, TB0 = 3, TY0 = 6, TXB0 = 12, TNPL = 15 };
template <int TT> struct TileShape {
    static constexpr int FS = TT + 7, FN = FS * FS, NT = TT == 32 ? 512 : 256, SMEM = TNPL * FN * 4;
};
int pdr_tile_size(Geom g) { return ((g.W + 31) / 32) * ((g.H + 31) / 32) < 152 ? 16 : 32; }

template <typename T, typename TF, bool HAS_W, int TT>
__global__ void __launch_bounds__(TileShape<TT>::NT) k_pdr_tile(IterArgs A) {
    constexpr int TFS = TileShape<TT>::FS, TFN = TileShape<TT>::FN, TNT = TileShape<TT>::NT;
    extern __shared__ float sm[];
    __shared__ double red[32];
    int H, W, P, pair = 0;
    Fields in, out;
    const void *Ixp, *Iyp, *Itp;
    const int *donep;
    if (A.pairs) {
        pair = A.plist ? A.plist[blockIdx.z] : (int)blockIdx.z;
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
    const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
    if (i0 >= H || j0 >= W) {     // a tile of a smaller pair in a batched launch
        if (A.partials && threadIdx.x == 0)
            A.partials[(size_t)pair * gridDim.x * gridDim.y + blockIdx.x + gridDim.x * blockIdx.y] = 0.0;
        return;
    }
    const int fi = i0 - 3, fj = j0 - 3;   // global coordinates of frame cell (0, 0)
    const int X[3] = {F_W, F_U, F_V}, XB[3] = {F_WB, F_UB, F_VB};
    const int Y1[3] = {F_P1, F_Q11, F_Q21}, Y2[3] = {F_P2, F_Q12, F_Q22};
    float sg, ta;
    pdr_steps(A.k, A.pairs ? A.pairs[pair].ms_max : A.ms_max, sg, ta);
    const float st = sg * ta;
    constexpr int C0 = HAS_W ? 0 : 1;
    auto S = [&](int k) { return sm + k * TFN; };
    // frame cell x at offset (li - 3, lj - 3) from the tile's corner; the loops below visit the
    // cells of a square of offsets [lo, hi] only
    // the cells of the square of offsets [LO, HI] (compile-time bounds: no division at run time)
    auto for_cells = [&](auto LO_, auto HI_, auto &&f) {
        constexpr int lo = decltype(LO_)::value, n = decltype(HI_)::value - lo + 1;
        for (int t = threadIdx.x; t < n * n; t += TNT) {
            const int li = lo + 3 + t / n, lj = lo + 3 + t % n;
            const int i = fi + li, j = fj + lj;
            if (i >= 0 && i < H && j >= 0 && j < W) f(li * TFS + lj, i, j);
        }
    };
    // ---- stage X^k (whole frame), ybar (offsets -3 .. TT + 2), Xbar (-2 .. TT + 2); zeros outside.  All
    // of a thread's loads are issued before its shared-memory stores.
    {
        constexpr int NP = (TFN + TNT - 1) / TNT;
        float v[NP][15];
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const int x = threadIdx.x + r * TNT;
            const int li = x / TFS, lj = x % TFS;
            const int i = fi + li, j = fj + lj;
            const bool ok = x < TFN && i >= 0 && i < H && j >= 0 && j < W;
            const bool oky = ok && li <= TT + 5 && lj <= TT + 5, okb = oky && li >= 1 && lj >= 1;
            const size_t o = ok ? (size_t)i * P + j : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool on = c >= C0;
                v[r][TX0 + c] = (ok && on) ? ldT<TF>(in.f[X[c]], o) : 0.f;
                v[r][TY0 + 2 * c] = (oky && on) ? ldT<T>(in.f[Y1[c]], o) : 0.f;
                v[r][TY0 + 2 * c + 1] = (oky && on) ? ldT<T>(in.f[Y2[c]], o) : 0.f;
                v[r][TXB0 + c] = (okb && on) ? ldT<TF>(in.f[XB[c]], o) : 0.f;
            }
        }
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const int x = threadIdx.x + r * TNT;
            if (x >= TFN) continue;
#pragma unroll
            for (int k = 0; k < 15; ++k)
                if (k < TB0 || k >= TY0) S(k)[x] = v[r][k];
        }
    }
    __syncthreads();
    using I = int;
    // ---- b = Xbar + sigma div ybar on offsets -2 .. TT + 2
    for_cells(std::integral_constant<I, -2>{}, std::integral_constant<I, TT + 2>{}, [&](int x, int i, int j) {
#pragma unroll
        for (int c = C0; c < 3; ++c) {
            const float *a = S(TY0 + 2 * c), *b = S(TY0 + 2 * c + 1);
            const float d = (((j < W - 1 ? a[x] : 0.f) - (j > 0 ? a[x - 1] : 0.f)) + (i < H - 1 ? b[x] : 0.f)) -
                            (i > 0 ? b[x - TFS] : 0.f);
            S(TB0 + c)[x] = pdr_rhs(S(TXB0 + c)[x], d, sg);
        }
    });
    __syncthreads();
    // one Gauss-Seidel update of the pixels of colour `colour` (only those are visited) in the square
    // of offsets [LO, HI], in place, rounded to the flow storage type
    auto half_sweep = [&](auto LO_, auto HI_, int colour) {
        constexpr int lo = decltype(LO_)::value, n = decltype(HI_)::value - lo + 1, hn = (n + 1) / 2;
        for (int t = threadIdx.x; t < n * hn; t += TNT) {
            const int r = t / hn, k = t % hn;
            const int li = lo + 3 + r;
            const int lj = lo + 3 + ((colour ^ (fi + li + fj + lo + 3)) & 1) + 2 * k;
            if (lj > lo + 3 + n - 1) continue;
            const int i = fi + li, j = fj + lj;
            if (!(i >= 0 && i < H && j >= 0 && j < W)) continue;
            const int x = li * TFS + lj;
            const bool hw = j > 0, he = j < W - 1, hn_ = i > 0, hs = i < H - 1;
            const int nb = (int)hw + (int)he + (int)hn_ + (int)hs;
#pragma unroll
            for (int c = C0; c < 3; ++c) {
                const float *xc = S(TX0 + c);
                float acc = 0.f;
                if (hw) acc += xc[x - 1];
                if (he) acc += xc[x + 1];
                if (hn_) acc += xc[x - TFS];
                if (hs) acc += xc[x + TFS];
                S(TX0 + c)[x] = storage_round<TF>(pdr_gs(S(TB0 + c)[x], acc, nb, st));
            }
        }
    };
    half_sweep(std::integral_constant<I, -2>{}, std::integral_constant<I, TT + 2>{}, 0);
    __syncthreads();
    half_sweep(std::integral_constant<I, -1>{}, std::integral_constant<I, TT + 1>{}, 1);
    __syncthreads();
    half_sweep(std::integral_constant<I, 0>{}, std::integral_constant<I, TT>{}, 0);
    __syncthreads();
    // ---- the tile: Xbar and ybar updates, stores, residual ||X^{k+1} - X^k||^2
    double res = 0.0;
    const float beta = A.k.beta, lam = A.k.lambda;
    for_cells(std::integral_constant<I, 0>{}, std::integral_constant<I, TT - 1>{}, [&](int x, int i, int j) {
        const size_t o = (size_t)i * P + j;
        const bool hx = j < W - 1, hy = i < H - 1;
        float xv[3] = {0.f, 0.f, 0.f}, g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = C0; c < 3; ++c) {
            const float *xc = S(TX0 + c);
            xv[c] = xc[x];
            g[2 * c] = hx ? xc[x + 1] - xv[c] : 0.f;
            g[2 * c + 1] = hy ? xc[x + TFS] - xv[c] : 0.f;
        }
        const float ix = ldT<T>(Ixp, o), iy = ldT<T>(Iyp, o), it = ldT<T>(Itp, o);
        float xb[3] = {S(TXB0)[x], S(TXB0 + 1)[x], S(TXB0 + 2)[x]};
        pdr_xbar<HAS_W>(xv, xb, ix, iy, it, beta, lam, sg);
        const float y[6] = {S(TY0)[x], S(TY0 + 1)[x], S(TY0 + 2)[x], S(TY0 + 3)[x], S(TY0 + 4)[x], S(TY0 + 5)[x]};
        float yn[6];
        pdr_ybar<HAS_W>(y, g, ta, yn);
#pragma unroll
        for (int c = C0; c < 3; ++c) {
            stT<TF>(out.f[X[c]], o, xv[c]);
            stT<TF>(out.f[XB[c]], o, xb[c]);
            stT<T>(out.f[Y1[c]], o, yn[2 * c]);
            stT<T>(out.f[Y2[c]], o, yn[2 * c + 1]);
        }
        const float dw = HAS_W ? xv[0] - ldT<TF>(in.f[F_W], o) : 0.f;
        const float du = xv[1] - ldT<TF>(in.f[F_U], o), dv = xv[2] - ldT<TF>(in.f[F_V], o);
        res += (double)dw * dw + (double)du * du + (double)dv * dv;
    });
    if (A.partials) {
        const double tot = block_sum(res, red);
        if (threadIdx.x == 0)
            A.partials[(size_t)pair * gridDim.x * gridDim.y + blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

template <typename T, typename TF, int TT> void launch_pdr_tile_tt(const IterArgs &a, cudaStream_t s) {
    using TS = TileShape<TT>;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_pdr_tile<T, TF, true, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TS::SMEM);
        cudaFuncSetAttribute(k_pdr_tile<T, TF, false, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TS::SMEM);
    });
    dim3 grid((a.g.W + TT - 1) / TT, (a.g.H + TT - 1) / TT, a.pairs ? a.ntiles : 1);
    if (a.k.beta != 0.f) k_pdr_tile<T, TF, true, TT><<<grid, TS::NT, TS::SMEM, s>>>(a);
    else k_pdr_tile<T, TF, false, TT><<<grid, TS::NT, TS::SMEM, s>>>(a);
}

template <typename T, typename TF> void launch_pdr_tile_t(const IterArgs &a, cudaStream_t s) {
    if (pdr_tile_size(a.g) == 16) launch_pdr_tile_tt<T, TF, 16>(a, s);
    else launch_pdr_tile_tt<T, TF, 32>(a, s);
}

template <typename T, typename TF, bool HAS_W> void launch_pdr_w(const IterArgs &a, bool literal, cudaStream_t s) {
    const int py = literal ? PY_DEFAULT : block_rows(a.tile_h);
    dim3 grid((a.g.W + PX - 1) / PX, (a.g.H + py - 1) / py, a.pairs ? a.ntiles : 1), blk(PX, py);
    if (literal) {
        k_pdr_b<T, TF, HAS_W><<<grid, blk, 0, s>>>(a);
        for (int sw = 0; sw < a.k.gs_sweeps; ++sw) {
            k_gs_half<T, TF, HAS_W><<<grid, blk, 0, s>>>(a, 0);
            k_gs_half<T, TF, HAS_W><<<grid, blk, 0, s>>>(a, 1);
            k_gs_half<T, TF, HAS_W><<<grid, blk, 0, s>>>(a, 1);
            k_gs_half<T, TF, HAS_W><<<grid, blk, 0, s>>>(a, 0);
        }
        k_pdr_finish<T, TF, HAS_W><<<grid, blk, 0, s>>>(a);
        return;
    }
    // fused: R (B R)^n in 2n + 1 launches, the first R with the right-hand side, the last with
    // the Xbar / ybar updates
    IterArgs b = a;
    b.partials = nullptr;
    k_pdr_b_red<T, TF, HAS_W><<<grid, blk, 0, s>>>(b);
    for (int sw = 0; sw < a.k.gs_sweeps; ++sw) {
        k_gs_half<T, TF, HAS_W><<<grid, blk, 0, s>>>(b, 1);
        if (sw + 1 < a.k.gs_sweeps) k_gs_half<T, TF, HAS_W><<<grid, blk, 0, s>>>(b, 0);
    }
    k_pdr_red_finish<T, TF, HAS_W><<<grid, blk, 0, s>>>(a);
}

template <typename T, typename TF> void launch_pdr_t(const IterArgs &a, bool literal, cudaStream_t s) {
    if (a.k.beta != 0.f) launch_pdr_w<T, TF, true>(a, literal, s);
    else launch_pdr_w<T, TF, false>(a, literal, s);
}

}  // namespace

int pdr_plain_blocks(Geom g, int tile_h) {
    const int py = block_rows(tile_h);
    return ((g.W + PX - 1) / PX) * ((g.H + py - 1) / py);
}
int pdr_fused_blocks(Geom g) { return pdr_plain_blocks(g); }

void launch_pdr_plain(const IterArgs &a, cudaStream_t s) { launch_pdr_t<float, float>(a, true, s); }

int pdr_tile_blocks(Geom g) {
    const int tt = pdr_tile_size(g);
    return ((g.W + tt - 1) / tt) * ((g.H + tt - 1) / tt);
}

void launch_pdr_fused(const IterArgs &a, int prec, int prec_flow, cudaStream_t s) {
    if (a.pdr_tile) {
        if (prec == PREC_F32) launch_pdr_tile_t<float, float>(a, s);
        else if (prec == PREC_F16 && prec_flow == PREC_F32) launch_pdr_tile_t<__half, float>(a, s);
        else if (prec == PREC_F16) launch_pdr_tile_t<__half, __half>(a, s);
        else if (prec_flow == PREC_F32) launch_pdr_tile_t<__nv_bfloat16, float>(a, s);
        else launch_pdr_tile_t<__nv_bfloat16, __nv_bfloat16>(a, s);
        return;
    }
    if (prec == PREC_F32) launch_pdr_t<float, float>(a, false, s);
    else if (prec == PREC_F16 && prec_flow == PREC_F32) launch_pdr_t<__half, float>(a, false, s);
    else if (prec == PREC_F16) launch_pdr_t<__half, __half>(a, false, s);
    else if (prec_flow == PREC_F32) launch_pdr_t<__nv_bfloat16, float>(a, false, s);
    else launch_pdr_t<__nv_bfloat16, __nv_bfloat16>(a, false, s);
}

}  // namespace tvl1
