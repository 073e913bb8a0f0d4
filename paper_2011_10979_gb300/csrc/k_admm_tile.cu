// k_admm_tile.cu -- several ADMM inner iterations (Sec. 3.1.1, eq. rpADMMI / rpADMMII /
// Zach-pADMM) in one launch, for the single-pair levels that run on the per-iteration engines
// (with the stopping test, the tested iterations run on the streaming kernel): each block owns a
// TT x TT tile of output pixels and stages in shared memory what the iterations need around it.
//
// One iteration at an output pixel needs y^{k+1} one pixel west and north (div y^{k+1}), y^{k+1}
// at a pixel needs div y^k, s, Lambda and the data one pixel east and south, and div y^k needs
// y^k one pixel west and north.  NI iterations (2 or 3) chain that NI times, so the block stages a
// (TT + 2 NI + 1)^2 frame starting NI + 1 pixels above and left of the tile: y^k on the whole
// frame, s, Lambda, Ix, Iy without its first row and column, and It where the finishes need it.
// Then, between block barriers, on squares that shrink by one pixel per iteration: div y^k; per
// iteration the y update, then s, Lambda and the next iteration's div y on the region it needs it
// on; the last iteration's finish on the tile stores the state and the squared residual.
// The per-pixel arithmetic is that of the streaming kernel (k_admm_math.cuh), and the state
// between the iterations is rounded to its storage type exactly where the streaming kernel's
// stores round it (y^{k+1} when read as y, s and Lambda when written), so NI iterations here are
// bitwise NI launches of the streaming kernel.  The launch reads one state buffer and writes the
// other; the residual's partial sums are those of the last iteration, grouped per tile.
#include <math.h>

#include <mutex>
#include <type_traits>

#include "k_admm_math.cuh"
#include "k_tile_cells.cuh"
#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

enum { SY0 = 0, SS = 6, SW_ = 7, SU = 8, SV = 9, SIX = 10, SIY = 11, SIT = 12, SDP = 13, NPL = 16 };
// NI iterations per launch on TT x TT tiles: the frame spans offsets -NI - 1 .. TT + NI - 1, FS
// cells a side (FC in all), a plane row FS floats.  512 threads for both tile sizes (measured per
// iteration with 16-pixel tiles, 256 against 512 threads: 2.66 / 2.38 us at 320x240, 2.00 / 1.59
// at 160x120, where the blocks do not fill the GPU and each phase's latency is the bound).
template <int TT, int NI> struct Shape {
    static constexpr int FS = TT + 2 * NI + 1, FC = FS * FS, NT = 512, SMEM = NPL * FC * 4;
};

template <int N> using IC = std::integral_constant<int, N>;

template <typename T, typename TF, bool HAS_W, int VARIANT, int TT, int NI>
__global__ void __launch_bounds__(Shape<TT, NI>::NT) k_admm_tile2(IterArgs A) {
    using SH = Shape<TT, NI>;
    constexpr int FS = SH::FS, FC = SH::FC, NT = SH::NT, OFF = NI + 1;
    extern __shared__ float sm[];
    __shared__ double red[32];
    const int H = A.g.H, W = A.g.W, P = A.g.pitch;
    if (A.done && *A.done) return;
    const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
    const int fi = i0 - OFF, fj = j0 - OFF;  // global coordinates of frame cell (0, 0)
    auto S = [&](int k) { return sm + k * FC; };
    const int YF[6] = {F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22};
    // ---- stage the frame; all of a thread's loads are issued before its shared-memory stores
    {
        constexpr int NP = (FC + NT - 1) / NT;
        float v[NP][13];
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const int x = threadIdx.x + r * NT;
            const int li = x / FS, lj = x % FS;
            const int i = fi + li, j = fj + lj;
            const bool ok = x < FC && i >= 0 && i < H && j >= 0 && j < W;
            const bool ok2 = ok && li >= 1 && lj >= 1;
            const bool ok3 = ok2 && li >= 2 && lj >= 2 && li <= FS - 2 && lj <= FS - 2;
            const size_t o = ok ? (size_t)i * P + j : 0;
#pragma unroll
            for (int k = 0; k < 6; ++k) v[r][k] = ((HAS_W || k >= 2) && ok) ? ldT<T>(A.in.f[YF[k]], o) : 0.f;
            v[r][SS] = ok2 ? ldT<T>(A.in.f[F_S], o) : 0.f;
            v[r][SW_] = (HAS_W && ok2) ? ldT<TF>(A.in.f[F_W], o) : 0.f;
            v[r][SU] = ok2 ? ldT<TF>(A.in.f[F_U], o) : 0.f;
            v[r][SV] = ok2 ? ldT<TF>(A.in.f[F_V], o) : 0.f;
            v[r][SIX] = ok2 ? ldT<T>(A.Ix, o) : 0.f;
            v[r][SIY] = ok2 ? ldT<T>(A.Iy, o) : 0.f;
            v[r][SIT] = ok3 ? ldT<T>(A.It, o) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const int x = threadIdx.x + r * NT;
            if (x >= FC) continue;
#pragma unroll
            for (int k = 0; k < 13; ++k) S(k)[x] = v[r][k];
        }
    }
    const StepK K = step_coefs(A.k, a_tilde_of(A.k, A.ms_max), c_of(A.k, A.ms_max));
    __syncthreads();
    // the in-image cells of the square of offsets [LO, HI], dealt to the threads conflict-free
    // (k_tile_cells.cuh)
    auto for_cells = [&](auto LO_, auto HI_, auto &&f) {
        tile_cells<TT, FS, OFF, NT, decltype(LO_)::value, decltype(HI_)::value>(fi, fj, H, W, f);
    };
    // y as the streaming kernel reads it: the stored value, rounded to the storage type
    auto Y = [&](int k, int x) { return storage_round<T>(S(SY0 + k)[x]); };
    // ---- div y at a pixel (from y rounded to storage), stored for the next y phase
    auto div_store = [&](int x, int i, int j) {
        const bool ex = j < W - 1, wx = j > 0, ey = i < H - 1, ny = i > 0;
        float dp = 0.f;
        if (HAS_W) dp = div2(ex ? Y(0, x) : 0.f, wx ? Y(0, x - 1) : 0.f, ey ? Y(1, x) : 0.f, ny ? Y(1, x - FS) : 0.f);
        S(SDP)[x] = dp;
        S(SDP + 1)[x] = div2(ex ? Y(2, x) : 0.f, wx ? Y(2, x - 1) : 0.f, ey ? Y(3, x) : 0.f, ny ? Y(3, x - FS) : 0.f);
        S(SDP + 2)[x] = div2(ex ? Y(4, x) : 0.f, wx ? Y(4, x - 1) : 0.f, ey ? Y(5, x) : 0.f, ny ? Y(5, x - FS) : 0.f);
    };
    // ---- y^{k+1} on a square, in place (only the pixel itself reads its y here)
    auto y_phase = [&](auto LO_, auto HI_) {
        for_cells(LO_, HI_, [&](int x, int i, int j) {
            const bool ex = j < W - 1, hy = i < H - 1;
            auto east = [&](int k) { return S(k)[x + 1]; };
            auto south = [&](int k) { return S(k)[x + FS]; };
            const float s0 = S(SS)[x], ix0 = S(SIX)[x], iy0 = S(SIY)[x];
            const float sE = ex ? east(SS) : 0.f, sS = hy ? south(SS) : 0.f;
            if (HAS_W) {
                const float d0 = S(SDP)[x], w0 = S(SW_)[x];
                const float gdx = ex ? east(SDP) - d0 : 0.f, gdy = hy ? south(SDP) - d0 : 0.f;
                const float wx_ = ex ? east(SW_) - w0 : 0.f, wy_ = hy ? south(SW_) - w0 : 0.f;
                const float sx_ = ex ? sE - s0 : 0.f, sy_ = hy ? sS - s0 : 0.f;
                float np1, np2;
                y_update_p(Y(0, x), Y(1, x), gdx, gdy, wx_, wy_, sx_, sy_, K, np1, np2);
                S(SY0)[x] = np1;
                S(SY0 + 1)[x] = np2;
            }
            // rounded products (never fused into the differences), as in the streaming kernel
            const float six0 = __fmul_rn(s0, ix0), siy0 = __fmul_rn(s0, iy0);
            const float sixx = ex ? __fmul_rn(sE, east(SIX)) - six0 : 0.f;
            const float sixy = hy ? __fmul_rn(sS, south(SIX)) - six0 : 0.f;
            const float siyx = ex ? __fmul_rn(sE, east(SIY)) - siy0 : 0.f;
            const float siyy = hy ? __fmul_rn(sS, south(SIY)) - siy0 : 0.f;
            const float d1 = S(SDP + 1)[x], d2 = S(SDP + 2)[x];
            const float g1x = ex ? east(SDP + 1) - d1 : 0.f, g1y = hy ? south(SDP + 1) - d1 : 0.f;
            const float g2x = ex ? east(SDP + 2) - d2 : 0.f, g2y = hy ? south(SDP + 2) - d2 : 0.f;
            const float u0 = S(SU)[x], v0 = S(SV)[x];
            const float ux = ex ? east(SU) - u0 : 0.f, uy = hy ? south(SU) - u0 : 0.f;
            const float vx = ex ? east(SV) - v0 : 0.f, vy = hy ? south(SV) - v0 : 0.f;
            float nq11, nq12, nq21, nq22;
            y_update_q(Y(2, x), Y(3, x), Y(4, x), Y(5, x), g1x, g1y, g2x, g2y, ux, uy, vx, vy, sixx, sixy, siyx,
                       siyy, K, nq11, nq12, nq21, nq22);
            S(SY0 + 2)[x] = nq11;
            S(SY0 + 3)[x] = nq12;
            S(SY0 + 4)[x] = nq21;
            S(SY0 + 5)[x] = nq22;
        });
    };
    // div y^{k+1} at a pixel from the unrounded y^{k+1} (as the streaming kernel's finish)
    auto div_new = [&](int x, int i, int j, float &dpn, float &dq1n, float &dq2n) {
        const bool ex = j < W - 1, wx = j > 0, hy = i < H - 1, nyy = i > 0;
        dpn = 0.f;
        if (HAS_W)
            dpn = div2(ex ? S(SY0)[x] : 0.f, wx ? S(SY0)[x - 1] : 0.f, hy ? S(SY0 + 1)[x] : 0.f,
                       nyy ? S(SY0 + 1)[x - FS] : 0.f);
        dq1n = div2(ex ? S(SY0 + 2)[x] : 0.f, wx ? S(SY0 + 2)[x - 1] : 0.f, hy ? S(SY0 + 3)[x] : 0.f,
                    nyy ? S(SY0 + 3)[x - FS] : 0.f);
        dq2n = div2(ex ? S(SY0 + 4)[x] : 0.f, wx ? S(SY0 + 4)[x - 1] : 0.f, hy ? S(SY0 + 5)[x] : 0.f,
                    nyy ? S(SY0 + 5)[x - FS] : 0.f);
    };
    // ---- iterations k .. k + NI - 2: an iteration E pixels from the last one computes y on
    // -1 - E .. TT - 1 + E, then on -E .. TT - 1 + E s and Lambda (rounded as stored; only the
    // pixel itself reads them in that phase) and, for the next iteration, div y^{k+1} -- the
    // region the next iteration needs it on, so no phase of its own.  The first iteration's div y^k
    // comes from the staged y.
    for_cells(IC<-NI>{}, IC<TT + NI - 1>{}, div_store);
    __syncthreads();
    auto iteration = [&](auto E_) {
        constexpr int e = decltype(E_)::value;
        y_phase(IC<-1 - e>{}, IC<TT - 1 + e>{});
        __syncthreads();
        for_cells(IC<-e>{}, IC<TT - 1 + e>{}, [&](int x, int i, int j) {
            float dpn, dq1n, dq2n, s_new;
            div_new(x, i, j, dpn, dq1n, dq2n);
            float w = S(SW_)[x], u = S(SU)[x], v = S(SV)[x];
            finish_pixel<HAS_W, VARIANT>(S(SIX)[x], S(SIY)[x], S(SIT)[x], S(SS)[x], w, u, v, dpn, dq1n, dq2n, K,
                                         s_new);
            S(SS)[x] = storage_round<T>(s_new);
            if (HAS_W) S(SW_)[x] = storage_round<TF>(w);
            S(SU)[x] = storage_round<TF>(u);
            S(SV)[x] = storage_round<TF>(v);
            if (std::is_same<T, float>::value) {  // y as stored is y: the finish's div is the next one
                S(SDP)[x] = dpn;
                S(SDP + 1)[x] = dq1n;
                S(SDP + 2)[x] = dq2n;
            } else {
                div_store(x, i, j);
            }
        });
        __syncthreads();
    };
    if constexpr (NI >= 3) iteration(IC<2>{});
    iteration(IC<1>{});
    // ---- the last iteration: its finish on the tile stores the state
    y_phase(IC<-1>{}, IC<TT - 1>{});
    __syncthreads();
    float res = 0.f;
    for_cells(IC<0>{}, IC<TT - 1>{}, [&](int x, int i, int j) {
        float dpn, dq1n, dq2n, s_new;
        div_new(x, i, j, dpn, dq1n, dq2n);
        float w = S(SW_)[x], u = S(SU)[x], v = S(SV)[x];
        res += finish_pixel<HAS_W, VARIANT>(S(SIX)[x], S(SIY)[x], S(SIT)[x], S(SS)[x], w, u, v, dpn, dq1n, dq2n, K,
                                            s_new);
        const size_t o = (size_t)i * P + j;
        if (HAS_W) {
            stT<T>(A.out.f[F_P1], o, S(SY0)[x]);
            stT<T>(A.out.f[F_P2], o, S(SY0 + 1)[x]);
            stT<TF>(A.out.f[F_W], o, w);
        }
        stT<T>(A.out.f[F_Q11], o, S(SY0 + 2)[x]);
        stT<T>(A.out.f[F_Q12], o, S(SY0 + 3)[x]);
        stT<T>(A.out.f[F_Q21], o, S(SY0 + 4)[x]);
        stT<T>(A.out.f[F_Q22], o, S(SY0 + 5)[x]);
        stT<T>(A.out.f[F_S], o, s_new);
        stT<TF>(A.out.f[F_U], o, u);
        stT<TF>(A.out.f[F_V], o, v);
    });
    if (A.partials) {
        const double tot = block_sum((double)res, red);
        if (threadIdx.x == 0) A.partials[blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

template <typename T, typename TF, bool HAS_W, int VARIANT, int TT, int NI>
void launch_tt(const IterArgs &a, cudaStream_t s) {
    using SH = Shape<TT, NI>;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_admm_tile2<T, TF, HAS_W, VARIANT, TT, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SH::SMEM);
    });
    dim3 grid((a.g.W + TT - 1) / TT, (a.g.H + TT - 1) / TT);
    k_admm_tile2<T, TF, HAS_W, VARIANT, TT, NI><<<grid, SH::NT, SH::SMEM, s>>>(a);
}

template <typename T, typename TF, bool HAS_W, int VARIANT> void launch_v(const IterArgs &a, int ni, cudaStream_t s) {
    const bool small = admm_tile2_size(a.g) == 16;
    if (ni == 3) {
        if (small) launch_tt<T, TF, HAS_W, VARIANT, 16, 3>(a, s);
        else launch_tt<T, TF, HAS_W, VARIANT, 32, 3>(a, s);
    } else {
        if (small) launch_tt<T, TF, HAS_W, VARIANT, 16, 2>(a, s);
        else launch_tt<T, TF, HAS_W, VARIANT, 32, 2>(a, s);
    }
}

template <typename T, typename TF> void launch_m(const IterArgs &a, int ni, cudaStream_t s) {
    const bool has_w = a.k.beta != 0.f;
    const int variant = (a.k.method == 1 ? 1 : 0) | (a.k.a_tilde_mode == 1 ? 2 : 0);
    switch (variant) {
    case 0: return has_w ? launch_v<T, TF, true, 0>(a, ni, s) : launch_v<T, TF, false, 0>(a, ni, s);
    case 1: return has_w ? launch_v<T, TF, true, 1>(a, ni, s) : launch_v<T, TF, false, 1>(a, ni, s);
    case 2: return has_w ? launch_v<T, TF, true, 2>(a, ni, s) : launch_v<T, TF, false, 2>(a, ni, s);
    default: return has_w ? launch_v<T, TF, true, 3>(a, ni, s) : launch_v<T, TF, false, 3>(a, ni, s);
    }
}

}  // namespace

// 16-pixel tiles where 32-pixel ones would give fewer blocks than SMs.
int admm_tile2_size(Geom g) { return ((g.W + 31) / 32) * ((g.H + 31) / 32) < 152 ? 16 : 32; }

int admm_tile2_blocks(Geom g) {
    const int tt = admm_tile2_size(g);
    return ((g.W + tt - 1) / tt) * ((g.H + tt - 1) / tt);
}

void launch_admm_tile2(const IterArgs &a, int ni, int prec, int prec_flow, cudaStream_t s) {
    if (prec == PREC_F32) launch_m<float, float>(a, ni, s);
    else if (prec == PREC_F16 && prec_flow == PREC_F32) launch_m<__half, float>(a, ni, s);
    else if (prec == PREC_F16) launch_m<__half, __half>(a, ni, s);
    else if (prec_flow == PREC_F32) launch_m<__nv_bfloat16, float>(a, ni, s);
    else launch_m<__nv_bfloat16, __nv_bfloat16>(a, ni, s);
}

}  // namespace tvl1
