// k_cp_tile.cu -- several ALG1 iterations (Sec. 4: Chambolle-Pock with constant steps on
// eq. primal-dual:optical:o) in one launch, for the single-pair levels that run on the
// per-iteration engine (with the stopping test, the tested iterations run on k_cp.cu): each block
// owns a TT x TT tile of output pixels and stages in shared memory what the iterations need
// around it.
//
// One iteration at an output pixel needs y^{k+1} at the pixel and one pixel west and north (the
// divergence in the primal step), and y^{k+1} at a pixel needs Xbar^k there and one pixel east and
// south (the forward differences in the dual step).  NI iterations (2 or 3) chain that NI times,
// so the block stages a (TT + 2 NI)^2 frame starting NI pixels above and left of the tile: y and
// Xbar on the whole frame, X and the data (Ix, Iy, It) without its outermost ring.  Then, between
// block barriers, on squares that shrink by one pixel per iteration: the dual step y^{k+1} in
// place, then the primal step X^{k+1} and Xbar^{k+1} = 2 X^{k+1} - X^k; the last iteration's primal
// step on the tile stores the state and the squared step |X^{k+1} - X^k|^2.
// The per-pixel arithmetic is that of the per-iteration kernel (k_cp_math.cuh), and the state
// between the iterations is rounded to the flow storage type exactly where that kernel's stores
// round it (y^{k+1} when read as y, X and Xbar when written), so NI iterations here are bitwise NI
// launches of k_cp.  The launch reads one state buffer and writes the other; the residual's
// partial sums are those of the last iteration, grouped per tile.
#include <math.h>

#include <mutex>

#include "k_cp_math.cuh"
#include "k_tile_cells.cuh"
#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

enum { CY0 = 0, CX0 = 6, CB0 = 9, CIX = 12, CIY = 13, CIT = 14, CNPL = 15 };
// NI iterations per launch on TT x TT tiles: the frame spans offsets -NI .. TT + NI - 1, FS cells a
// side (FC in all), a plane row FS floats; 512 threads.
template <int TT, int NI> struct CpShape {
    static constexpr int FS = TT + 2 * NI, FC = FS * FS, NT = 512, SMEM = CNPL * FC * 4;
};

template <int N> using CIC = std::integral_constant<int, N>;

template <typename T, typename TF, bool HAS_W, int TT, int NI>
__global__ void __launch_bounds__(CpShape<TT, NI>::NT) k_cp_tile(IterArgs A) {
    using SH = CpShape<TT, NI>;
    constexpr int FS = SH::FS, FC = SH::FC, NT = SH::NT, OFF = NI;
    extern __shared__ float sm[];
    __shared__ double red[32];
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    if (A.done && *A.done) return;
    const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
    const int fi = i0 - OFF, fj = j0 - OFF;  // image coordinates of frame cell (0, 0)
    auto S = [&](int k) { return sm + k * FC; };
    const int YF[6] = {F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22};
    const int XF[3] = {F_W, F_U, F_V}, BF[3] = {F_WB, F_UB, F_VB};
    constexpr int C0 = HAS_W ? 0 : 1;  // first live primal component (w is absent with beta = 0)
    // ---- stage the frame; all of a thread's loads are issued before its shared-memory stores
    {
        constexpr int NP = (FC + NT - 1) / NT;
        float v[NP][CNPL];
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const int x = threadIdx.x + r * NT;
            const int li = x / FS, lj = x % FS;
            const int i = fi + li, j = fj + lj;
            const bool ok = x < FC && i >= 0 && i < H && j >= 0 && j < W;
            const bool ok2 = ok && li >= 1 && lj >= 1 && li <= FS - 2 && lj <= FS - 2;
            const size_t o = ok ? (size_t)i * P + j : 0;
#pragma unroll
            for (int k = 0; k < 6; ++k) v[r][CY0 + k] = ((HAS_W || k >= 2) && ok) ? ldT<TF>(A.in.f[YF[k]], o) : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[r][CB0 + c] = (c >= C0 && ok) ? ldT<TF>(A.in.f[BF[c]], o) : 0.f;
                v[r][CX0 + c] = (c >= C0 && ok2) ? ldT<TF>(A.in.f[XF[c]], o) : 0.f;
            }
            v[r][CIX] = ok2 ? ldT<T>(A.Ix, o) : 0.f;
            v[r][CIY] = ok2 ? ldT<T>(A.Iy, o) : 0.f;
            v[r][CIT] = ok2 ? ldT<T>(A.It, o) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const int x = threadIdx.x + r * NT;
            if (x >= FC) continue;
#pragma unroll
            for (int k = 0; k < CNPL; ++k) S(k)[x] = v[r][k];
        }
    }
    const float tau = A.k.cp_tau, sg = A.k.cp_sigma, beta = A.k.beta, lam = A.k.lambda;
    __syncthreads();
    auto for_cells = [&](auto LO_, auto HI_, auto &&f) {
        tile_cells<TT, FS, OFF, NT, decltype(LO_)::value, decltype(HI_)::value>(fi, fj, H, W, f);
    };
    // ---- the dual step on a square, in place: y^{k+1} = P(y^k + tau grad Xbar^k), y^k as the
    // per-iteration kernel reads it (rounded to the flow storage type)
    auto dual_phase = [&](auto LO_, auto HI_) {
        for_cells(LO_, HI_, [&](int x, int i, int j) {
            const bool hx = j < W - 1, hy = i < H - 1;
            float y0[6], g[6], yn[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) y0[k] = storage_round<TF>(S(CY0 + k)[x]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *b = S(CB0 + c);
                g[2 * c] = hx ? b[x + 1] - b[x] : 0.f;
                g[2 * c + 1] = hy ? b[x + FS] - b[x] : 0.f;
            }
            cp_dual<HAS_W>(y0, g, tau, yn);
#pragma unroll
            for (int k = 0; k < 6; ++k) S(CY0 + k)[x] = yn[k];
        });
    };
    // ---- the primal step at a pixel from the unrounded y^{k+1} (as the per-iteration kernel's own
    // dual steps at the pixel and its west and north neighbours): X^{k+1} in xn, Xbar^{k+1} in bn,
    // returns |X^{k+1} - X^k|^2
    auto primal = [&](int x, int i, int j, float xn[3], float bn[3]) -> float {
        const bool ex = j < W - 1, ey = i < H - 1;
        // div y^{k+1} = -K^* y^{k+1} (forward differences, Neumann)
        auto dv = [&](int cx, int cy) {
            const float yw = j > 0 ? S(CY0 + cx)[x - 1] : 0.f, ynn = i > 0 ? S(CY0 + cy)[x - FS] : 0.f;
            return (((ex ? S(CY0 + cx)[x] : 0.f) - yw) + (ey ? S(CY0 + cy)[x] : 0.f)) - ynn;
        };
        const float d3[3] = {HAS_W ? dv(0, 1) : 0.f, dv(2, 3), dv(4, 5)};
        float xv[3] = {S(CX0)[x], S(CX0 + 1)[x], S(CX0 + 2)[x]};
        const float xold[3] = {xv[0], xv[1], xv[2]};
        const float r = cp_primal<HAS_W>(xv, d3, S(CIX)[x], S(CIY)[x], S(CIT)[x], beta, lam, sg);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xn[c] = xv[c];
            bn[c] = 2.f * xv[c] - xold[c];
        }
        return r;
    };
    // ---- iterations k .. k + NI - 2: an iteration E pixels from the last one takes the dual step
    // on -1 - E .. TT - 1 + E and the primal step on -E .. TT - 1 + E (X and Xbar rounded as stored)
    auto iteration = [&](auto E_) {
        constexpr int e = decltype(E_)::value;
        dual_phase(CIC<-1 - e>{}, CIC<TT - 1 + e>{});
        __syncthreads();
        for_cells(CIC<-e>{}, CIC<TT - 1 + e>{}, [&](int x, int i, int j) {
            float xn[3], bn[3];
            primal(x, i, j, xn, bn);
#pragma unroll
            for (int c = C0; c < 3; ++c) {
                S(CX0 + c)[x] = storage_round<TF>(xn[c]);
                S(CB0 + c)[x] = storage_round<TF>(bn[c]);
            }
        });
        __syncthreads();
    };
    if constexpr (NI >= 3) iteration(CIC<2>{});
    iteration(CIC<1>{});
    // ---- the last iteration: its primal step on the tile stores the state
    dual_phase(CIC<-1>{}, CIC<TT - 1>{});
    __syncthreads();
    float res = 0.f;
    for_cells(CIC<0>{}, CIC<TT - 1>{}, [&](int x, int i, int j) {
        float xn[3], bn[3];
        res += primal(x, i, j, xn, bn);
        const size_t o = (size_t)i * P + j;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (HAS_W || k >= 2) stT<TF>(A.out.f[YF[k]], o, S(CY0 + k)[x]);
#pragma unroll
        for (int c = C0; c < 3; ++c) {
            stT<TF>(A.out.f[XF[c]], o, xn[c]);
            stT<TF>(A.out.f[BF[c]], o, bn[c]);
        }
    });
    if (A.partials) {
        const double tot = block_sum((double)res, red);
        if (threadIdx.x == 0) A.partials[blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

template <typename T, typename TF, bool HAS_W, int TT, int NI> void launch_tt(const IterArgs &a, cudaStream_t s) {
    using SH = CpShape<TT, NI>;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_cp_tile<T, TF, HAS_W, TT, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM);
    });
    dim3 grid((a.g.W + TT - 1) / TT, (a.g.H + TT - 1) / TT);
    k_cp_tile<T, TF, HAS_W, TT, NI><<<grid, SH::NT, SH::SMEM, s>>>(a);
}

template <typename T, typename TF, bool HAS_W> void launch_w(const IterArgs &a, int ni, cudaStream_t s) {
    const bool small = cp_tile_size(a.g) == 16;
    if (ni == 3) {
        if (small) launch_tt<T, TF, HAS_W, 16, 3>(a, s);
        else launch_tt<T, TF, HAS_W, 32, 3>(a, s);
    } else {
        if (small) launch_tt<T, TF, HAS_W, 16, 2>(a, s);
        else launch_tt<T, TF, HAS_W, 32, 2>(a, s);
    }
}

template <typename T, typename TF> void launch_m(const IterArgs &a, int ni, cudaStream_t s) {
    if (a.k.beta != 0.f) launch_w<T, TF, true>(a, ni, s);
    else launch_w<T, TF, false>(a, ni, s);
}

}  // namespace

// 16-pixel tiles where 32-pixel ones would give fewer blocks than SMs.
int cp_tile_size(Geom g) { return ((g.W + 31) / 32) * ((g.H + 31) / 32) < 152 ? 16 : 32; }

int cp_tile_blocks(Geom g) {
    const int tt = cp_tile_size(g);
    return ((g.W + tt - 1) / tt) * ((g.H + tt - 1) / tt);
}

void launch_cp_tile(const IterArgs &a, int ni, int prec, int prec_flow, cudaStream_t s) {
    if (prec == PREC_F32) launch_m<float, float>(a, ni, s);
    else if (prec == PREC_F16 && prec_flow == PREC_F32) launch_m<__half, float>(a, ni, s);
    else if (prec == PREC_F16) launch_m<__half, __half>(a, ni, s);
    else if (prec_flow == PREC_F32) launch_m<__nv_bfloat16, float>(a, ni, s);
    else launch_m<__nv_bfloat16, __nv_bfloat16>(a, ni, s);
}

}  // namespace tvl1
