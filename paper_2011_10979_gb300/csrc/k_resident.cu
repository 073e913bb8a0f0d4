// k_resident.cu -- level-resident engines of the ADMM inner iteration (Sec. 3.1.1) and of ALG1 (Sec. 4):
// one thread-block cluster per pair keeps a whole pyramid level in shared memory and runs every
// inner iteration of one warp (eq. rpADMMI / rpADMMII / Zach-pADMM, with the stopping test of
// Sec. 4) in a single launch.  Coarse levels are far too small to fill the GPU, so the per-launch
// latency of the streaming engine (k_admm_roll.cuh), not bandwidth, bounds them there.
//
// Layout: CTA r of a cluster of NC owns the band of rows [r * rpc, min(H, (r + 1) * rpc)),
// rpc = ceil(H / NC), as 16 FP32 planes in shared memory: the duals p1 p2 q11 q12 q21 q22 s, the
// multipliers w u v, the data Ix Iy It and div y (p, q1, q2), each with one ghost row above and
// below the band.  A CTA writes the boundary rows its neighbours need straight into their ghost
// rows (distributed shared memory stores, which do not stall the writer); the cluster barrier that
// ends each phase publishes them, so every read in the phases is a local shared-memory read.  The
// storage precision of the state only matters on entry and exit; inside, everything is FP32.
//
// One iteration is two phases separated by cluster barriers:
//   A. y^{k+1} at the band's pixels from y^k, div y^k, s, Lambda (east and south neighbours);
//      written in place (no other pixel reads y in this phase); the last band row of p2, q12, q22
//      goes to the south CTA's north ghost row;
//   B. div y^{k+1} (west and north neighbours of y^{k+1}), then s^{k+1} and Lambda^{k+1}, all
//      pointwise, with the squared constraint residual on checking iterations; the first band row
//      of s, w, u, v and div y goes to the north CTA's south ghost row.
// A ghost row written in one phase is read only in the other, across a barrier.
// With 16-bit storage the state is rounded to the storage type exactly where the streaming
// engine's per-iteration stores round it (y^k on entry to phase A, s and Lambda when stored,
// div y^k taken from the rounded y), so both engines give bitwise the same results in every
// storage precision.
// Every 10th iteration (tolerance > 0) and on the final iteration of the last warp the CTAs'
// FP64 residual partials are summed by every CTA in rank order, so all CTAs take the same stop
// decision.  The per-pixel arithmetic is that of the streaming engine (k_admm_math.cuh).
#include <cooperative_groups.h>
#include <math.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <type_traits>

#include "k_admm_math.cuh"
#include "k_cp_math.cuh"
#include "k_pdr_math.cuh"
#include "tvl1_device.cuh"

namespace cg = cooperative_groups;

namespace tvl1 {

namespace {

constexpr int RT = 512;      // threads per CTA
constexpr int NPL = 16;      // FP32 shared planes per pixel
enum { S_P1, S_P2, S_Q11, S_Q12, S_Q21, S_Q22, S_S, S_W, S_U, S_V, S_IX, S_IY, S_IT, S_DP, S_DQ1, S_DQ2 };
// the state fields in shared-plane order (S_P1 .. S_V)
__constant__ int kField[10] = {F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22, F_S, F_W, F_U, F_V};

// Calls f(x, li, j) for this thread's pixels of the band: flat index x = tid + m * RT over
// nrow x W (local row li, column j), stepped incrementally so no division runs per pixel.
template <typename F>
__device__ __forceinline__ void for_band(int npx, int W, int di, int dj, F &&f) {
    int li = threadIdx.x / W, j = threadIdx.x - (threadIdx.x / W) * W;
    for (int x = threadIdx.x; x < npx; x += RT) {
        f(x, li, j);
        li += di;
        j += dj;
        if (j >= W) {
            j -= W;
            ++li;
        }
    }
}

// The stopping test of one cluster.  end_iteration() ends phase B of an iteration: on checking
// (every 10th, tolerance > 0) and final iterations each CTA publishes its FP64 residual partial,
// the cluster barrier that ends the phase follows, and every CTA sums the partials in rank order
// (the same bits on every CTA), so the stop decision is uniform over the cluster.
struct ClusterStop {
    double *red;          // block-sum scratch (32 doubles, shared)
    double *part, *total; // this CTA's partial and the broadcast total (shared)
    double *res_check, *res_final;
    int *done;
    long long *iters;
    double rows, tol;
    int rank, nc, run = 0;
    bool have_tot = false;
    double last_tot = 0.0;

    __device__ bool end_iteration(cg::cluster_group &cl, int it, float res, bool check, bool fin) {
        if (check || fin) {  // uniform over the cluster
            const double b = block_sum((double)res, red);
            if (threadIdx.x == 0) *part = b;
        }
        cl.sync();
        run = it + 1;
        if (!(check || fin)) return false;
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int r = 0; r < nc; ++r) tot += *cl.map_shared_rank(part, r);
            *total = tot;
        }
        __syncthreads();
        last_tot = *total;
        have_tot = true;
        if (!check) return false;
        if (rank == 0 && threadIdx.x == 0) *res_check = last_tot;
        if (tol > 0.0 && sqrt(last_tot / rows) < tol) {
            if (rank == 0 && threadIdx.x == 0) *done = 1;
            return true;
        }
        return false;
    }

    // after the loop: the warp's iteration count and (last warp) the final residual
    __device__ void finish(bool final_res) const {
        if (rank == 0 && threadIdx.x == 0) {
            *iters += run;
            if (final_res && have_tot) *res_final = last_tot;
        }
    }
};

template <typename T, typename TF, bool HAS_W, int VARIANT>
__global__ void __launch_bounds__(RT, 1) k_admm_resident(ResArgs A) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[32];
    __shared__ double part;   // this CTA's residual partial of the current checking iteration
    __shared__ double total;  // the cluster's sum, broadcast inside the CTA
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), NC = (int)cl.num_blocks();

    // ---- the pair: geometry in plain scalars, one 16-byte load in batched mode
    int H, W, P;
    const void *in[10], *dat[3];
    void *out[10];
    const float *msp;
    double *res_check, *res_final;
    int *donep;
    long long *itersp;
    double rows;
    if (A.pairs) {
        const int q = A.list[blockIdx.x / NC];
        const PairIter *pp = A.pairs + q;
        const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
        H = gq.x;
        W = gq.y;
        P = gq.z;
        const Fields *fi = pp->buf + A.parity_in, *fo = pp->buf + A.parity_out;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            in[k] = fi->f[kField[k]];
            out[k] = fo->f[kField[k]];
        }
        dat[0] = pp->Ix;
        dat[1] = pp->Iy;
        dat[2] = pp->It;
        msp = pp->ms_max;
        const PairScalars *ps = A.scal + q;
        res_check = ps->res_check;
        res_final = ps->res_final;
        donep = ps->done;
        itersp = ps->iters;
        rows = ps->rows;
    } else {
        H = A.g.H;
        W = A.g.W;
        P = A.g.pitch;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            in[k] = A.in.f[kField[k]];
            out[k] = A.out.f[kField[k]];
        }
        dat[0] = A.Ix;
        dat[1] = A.Iy;
        dat[2] = A.It;
        msp = A.ms_max;
        res_check = A.sc.res_check;
        res_final = A.sc.res_final;
        donep = A.sc.done;
        itersp = A.sc.iters;
        rows = A.sc.rows;
    }
    const int rpc = (H + NC - 1) / NC;
    const int r0 = rank * rpc, r1 = min(H, r0 + rpc);
    const int nrow = max(0, r1 - r0), npx = nrow * W;
    const int PL = (rpc + 2) * W;                 // shared plane stride: ghost row, rpc rows, ghost row
    const int di = RT / W, dj = RT - (RT / W) * W;
    // plane k of the band at S + k * PL (local row li at li * W); local row -1 is the north ghost row
    // (the last row of the CTA above), local row rpc the south ghost row (the first row of the CTA
    // below).  The neighbours write their boundary rows into these ghost rows themselves.
    float *const S = sm + W;
    // this CTA's ghost rows as seen by its neighbours: the north CTA's south ghost row and the south
    // CTA's north ghost row (nullptr where that neighbour has no rows next to this band)
    float *const Gn = (rank > 0 && nrow > 0) ? cl.map_shared_rank(sm, rank - 1) + W + rpc * W : nullptr;
    float *const Gs = (rank + 1 < NC && r1 < H) ? cl.map_shared_rank(sm, rank + 1) : nullptr;
    // pushes of one pixel's plane-k value: first band row -> north CTA, last band row -> south CTA
    auto push_n = [&](int k, int li, int j, float v) {
        if (li == 0 && Gn) Gn[k * PL + j] = v;
    };
    auto push_s = [&](int k, int li, int j, float v) {
        if (li == nrow - 1 && Gs) Gs[k * PL + j] = v;
    };

    // ---- load the band (storage precision -> FP32)
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        const size_t o = (size_t)(r0 + li) * P + j;
        float y[7];
#pragma unroll
        for (int k = S_P1; k <= S_S; ++k) {
            y[k] = (HAS_W || k >= S_Q11) ? ldT<T>(in[k], o) : 0.f;
            S[k * PL + x] = y[k];
        }
        const float w = HAS_W ? ldT<TF>(in[7], o) : 0.f, u = ldT<TF>(in[8], o), v = ldT<TF>(in[9], o);
        const float ix = ldT<T>(dat[0], o), iy = ldT<T>(dat[1], o);
        S[S_W * PL + x] = w;
        S[S_U * PL + x] = u;
        S[S_V * PL + x] = v;
        S[S_IX * PL + x] = ix;
        S[S_IY * PL + x] = iy;
        S[S_IT * PL + x] = ldT<T>(dat[2], o);
        push_s(S_P2, li, j, y[S_P2]);
        push_s(S_Q12, li, j, y[S_Q12]);
        push_s(S_Q22, li, j, y[S_Q22]);
        push_n(S_S, li, j, y[S_S]);
        push_n(S_W, li, j, w);
        push_n(S_U, li, j, u);
        push_n(S_V, li, j, v);
        push_n(S_IX, li, j, ix);
        push_n(S_IY, li, j, iy);
    });
    const StepK K = step_coefs(A.k, a_tilde_of(A.k, msp), c_of(A.k, msp));
    cl.sync();

    // div y at the band's pixels from y (west neighbour; north neighbour, for the first band row
    // from the north ghost row)
    auto div_at = [&](int x, int li, int j, float &dp, float &dq1, float &dq2) {
        const int i = r0 + li;
        const bool ex = j < W - 1, wx = j > 0, ey = i < H - 1, ny = i > 0;
        dp = 0.f;
        if (HAS_W)
            dp = div2(ex ? S[S_P1 * PL + x] : 0.f, wx ? S[S_P1 * PL + x - 1] : 0.f, ey ? S[S_P2 * PL + x] : 0.f,
                      ny ? S[S_P2 * PL + x - W] : 0.f);
        dq1 = div2(ex ? S[S_Q11 * PL + x] : 0.f, wx ? S[S_Q11 * PL + x - 1] : 0.f, ey ? S[S_Q12 * PL + x] : 0.f,
                   ny ? S[S_Q12 * PL + x - W] : 0.f);
        dq2 = div2(ex ? S[S_Q21 * PL + x] : 0.f, wx ? S[S_Q21 * PL + x - 1] : 0.f, ey ? S[S_Q22 * PL + x] : 0.f,
                   ny ? S[S_Q22 * PL + x - W] : 0.f);
    };
    // the same from y rounded to the storage type
    auto div_at_r = [&](int x, int li, int j, float &dp, float &dq1, float &dq2) {
        const int i = r0 + li;
        const bool ex = j < W - 1, wx = j > 0, ey = i < H - 1, ny = i > 0;
        auto R = [&](int k, int o) { return storage_round<T>(S[k * PL + o]); };
        dp = 0.f;
        if (HAS_W) dp = div2(ex ? R(S_P1, x) : 0.f, wx ? R(S_P1, x - 1) : 0.f, ey ? R(S_P2, x) : 0.f, ny ? R(S_P2, x - W) : 0.f);
        dq1 = div2(ex ? R(S_Q11, x) : 0.f, wx ? R(S_Q11, x - 1) : 0.f, ey ? R(S_Q12, x) : 0.f, ny ? R(S_Q12, x - W) : 0.f);
        dq2 = div2(ex ? R(S_Q21, x) : 0.f, wx ? R(S_Q21, x - 1) : 0.f, ey ? R(S_Q22, x) : 0.f, ny ? R(S_Q22, x - W) : 0.f);
    };
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        float dp, dq1, dq2;
        div_at(x, li, j, dp, dq1, dq2);
        S[S_DP * PL + x] = dp;
        S[S_DQ1 * PL + x] = dq1;
        S[S_DQ2 * PL + x] = dq2;
        push_n(S_DP, li, j, dp);
        push_n(S_DQ1, li, j, dq1);
        push_n(S_DQ2, li, j, dq2);
    });
    cl.sync();

    ClusterStop stop{red, &part, &total, res_check, res_final, donep, itersp, rows, A.tol, rank, NC};
    for (int it = 0; it < A.iters; ++it) {
        // ---- phase A: y^{k+1} (south neighbours of the last band row from the south ghost row)
        for_band(npx, W, di, dj, [&](int x, int li, int j) {
            const int i = r0 + li;
            const bool ex = j < W - 1, hy = i < H - 1;
            auto south = [&](int k) -> float { return S[k * PL + x + W]; };
            auto east = [&](int k) -> float { return S[k * PL + x + 1]; };
            const float s0 = S[S_S * PL + x], ix0 = S[S_IX * PL + x], iy0 = S[S_IY * PL + x];
            const float sE = ex ? east(S_S) : 0.f, sS = hy ? south(S_S) : 0.f;
            if (HAS_W) {
                const float d0 = S[S_DP * PL + x], w0 = S[S_W * PL + x];
                const float gdx = ex ? east(S_DP) - d0 : 0.f, gdy = hy ? south(S_DP) - d0 : 0.f;
                const float wx_ = ex ? east(S_W) - w0 : 0.f, wy_ = hy ? south(S_W) - w0 : 0.f;
                const float sx_ = ex ? sE - s0 : 0.f, sy_ = hy ? sS - s0 : 0.f;
                float np1, np2;
                y_update_p(storage_round<T>(S[S_P1 * PL + x]), storage_round<T>(S[S_P2 * PL + x]), gdx, gdy, wx_, wy_,
                           sx_, sy_, K, np1, np2);
                S[S_P1 * PL + x] = np1;
                S[S_P2 * PL + x] = np2;
                push_s(S_P2, li, j, np2);
            }
            // rounded products (never fused into the differences), as in the streaming engine
            const float six0 = __fmul_rn(s0, ix0), siy0 = __fmul_rn(s0, iy0);
            const float sixx = ex ? __fmul_rn(sE, east(S_IX)) - six0 : 0.f;
            const float sixy = hy ? __fmul_rn(sS, south(S_IX)) - six0 : 0.f;
            const float siyx = ex ? __fmul_rn(sE, east(S_IY)) - siy0 : 0.f;
            const float siyy = hy ? __fmul_rn(sS, south(S_IY)) - siy0 : 0.f;
            const float d1 = S[S_DQ1 * PL + x], d2 = S[S_DQ2 * PL + x];
            const float g1x = ex ? east(S_DQ1) - d1 : 0.f, g1y = hy ? south(S_DQ1) - d1 : 0.f;
            const float g2x = ex ? east(S_DQ2) - d2 : 0.f, g2y = hy ? south(S_DQ2) - d2 : 0.f;
            const float u0 = S[S_U * PL + x], v0 = S[S_V * PL + x];
            const float ux = ex ? east(S_U) - u0 : 0.f, uy = hy ? south(S_U) - u0 : 0.f;
            const float vx = ex ? east(S_V) - v0 : 0.f, vy = hy ? south(S_V) - v0 : 0.f;
            float nq11, nq12, nq21, nq22;
            y_update_q(storage_round<T>(S[S_Q11 * PL + x]), storage_round<T>(S[S_Q12 * PL + x]),
                       storage_round<T>(S[S_Q21 * PL + x]), storage_round<T>(S[S_Q22 * PL + x]), g1x, g1y, g2x, g2y,
                       ux, uy, vx, vy, sixx, sixy, siyx, siyy, K, nq11, nq12, nq21, nq22);
            S[S_Q11 * PL + x] = nq11;
            S[S_Q12 * PL + x] = nq12;
            S[S_Q21 * PL + x] = nq21;
            S[S_Q22 * PL + x] = nq22;
            push_s(S_Q12, li, j, nq12);
            push_s(S_Q22, li, j, nq22);
        });
        cl.sync();
        // ---- phase B: div y^{k+1}, s^{k+1}, Lambda^{k+1}
        const bool check = A.check && (it + 1) % 10 == 0;
        const bool fin = A.final_res && it == A.iters - 1;
        float res = 0.f;
        for_band(npx, W, di, dj, [&](int x, int li, int j) {
            float dpn, dq1n, dq2n;
            div_at(x, li, j, dpn, dq1n, dq2n);
            float w = S[S_W * PL + x], u = S[S_U * PL + x], v = S[S_V * PL + x], s_new;
            res += K.per_pixel  // uniform over the launch
                       ? finish_pixel<HAS_W, VARIANT | 2>(S[S_IX * PL + x], S[S_IY * PL + x], S[S_IT * PL + x],
                                                          S[S_S * PL + x], w, u, v, dpn, dq1n, dq2n, K, s_new)
                       : finish_pixel<HAS_W, VARIANT>(S[S_IX * PL + x], S[S_IY * PL + x], S[S_IT * PL + x],
                                                      S[S_S * PL + x], w, u, v, dpn, dq1n, dq2n, K, s_new);
            s_new = storage_round<T>(s_new);
            w = storage_round<TF>(w);
            u = storage_round<TF>(u);
            v = storage_round<TF>(v);
            // div y^{k+1} as the next iteration sees it: from y^{k+1} rounded to storage
            if (!std::is_same<T, float>::value) div_at_r(x, li, j, dpn, dq1n, dq2n);
            S[S_S * PL + x] = s_new;
            if (HAS_W) S[S_W * PL + x] = w;
            S[S_U * PL + x] = u;
            S[S_V * PL + x] = v;
            S[S_DP * PL + x] = dpn;
            S[S_DQ1 * PL + x] = dq1n;
            S[S_DQ2 * PL + x] = dq2n;
            push_n(S_S, li, j, s_new);
            if (HAS_W) push_n(S_W, li, j, w);
            push_n(S_U, li, j, u);
            push_n(S_V, li, j, v);
            push_n(S_DP, li, j, dpn);
            push_n(S_DQ1, li, j, dq1n);
            push_n(S_DQ2, li, j, dq2n);
        });
        if (stop.end_iteration(cl, it, res, check, fin)) break;
    }
    stop.finish(A.final_res);

    // ---- store the band (FP32 -> storage precision)
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        const size_t o = (size_t)(r0 + li) * P + j;
#pragma unroll
        for (int k = S_P1; k <= S_S; ++k)
            if (HAS_W || k >= S_Q11) stT<T>(out[k], o, S[k * PL + x]);
        if (HAS_W) stT<TF>(out[7], o, S[S_W * PL + x]);
        stT<TF>(out[8], o, S[S_U * PL + x]);
        stT<TF>(out[9], o, S[S_V * PL + x]);
    });
    cl.sync();  // no CTA leaves while another may still read its shared memory
}


// ---------------------------------------------------------------------------------- ALG1
// The same band layout for ALG1 (Sec. 4, Chambolle-Pock): planes y (p1 p2 q11 q12 q21 q22),
// X (w u v), Xbar (wb ub vb), data (Ix Iy It).  Phase A: y' = P(y + tau grad Xbar) (east and
// south neighbours of Xbar; the last band row of p2, q12, q22 goes to the south CTA's north ghost
// row).  Phase B: X' = prox(X + sigma div y') (west and north neighbours of y'), Xbar' = 2X' - X,
// |X' - X|^2 (the first band row of Xbar' goes to the north CTA's south ghost row).  The state is
// rounded to the storage type where the one-kernel-per-iteration engine's stores round it; y, X
// and Xbar are all kept in the flow fields' type TF (k_cp.cu).
enum { C_P1, C_P2, C_Q11, C_Q12, C_Q21, C_Q22, C_W, C_U, C_V, C_WB, C_UB, C_VB, C_IX, C_IY, C_IT };
__constant__ int kFieldCP[12] = {F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22, F_W, F_U, F_V, F_WB, F_UB, F_VB};

template <typename T, typename TF, bool HAS_W>
__global__ void __launch_bounds__(RT, 1) k_cp_resident(ResArgs A) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[32];
    __shared__ double part, total;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), NC = (int)cl.num_blocks();

    int H, W, P;
    const void *in[12], *dat[3];
    void *out[12];
    double *res_check, *res_final;
    int *donep;
    long long *itersp;
    double rows;
    if (A.pairs) {
        const int q = A.list[blockIdx.x / NC];
        const PairIter *pp = A.pairs + q;
        const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
        H = gq.x;
        W = gq.y;
        P = gq.z;
        const Fields *fi = pp->buf + A.parity_in, *fo = pp->buf + A.parity_out;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            in[k] = fi->f[kFieldCP[k]];
            out[k] = fo->f[kFieldCP[k]];
        }
        dat[0] = pp->Ix;
        dat[1] = pp->Iy;
        dat[2] = pp->It;
        const PairScalars *ps = A.scal + q;
        res_check = ps->res_check;
        res_final = ps->res_final;
        donep = ps->done;
        itersp = ps->iters;
        rows = ps->rows;
    } else {
        H = A.g.H;
        W = A.g.W;
        P = A.g.pitch;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            in[k] = A.in.f[kFieldCP[k]];
            out[k] = A.out.f[kFieldCP[k]];
        }
        dat[0] = A.Ix;
        dat[1] = A.Iy;
        dat[2] = A.It;
        res_check = A.sc.res_check;
        res_final = A.sc.res_final;
        donep = A.sc.done;
        itersp = A.sc.iters;
        rows = A.sc.rows;
    }
    const int rpc = (H + NC - 1) / NC;
    const int r0 = rank * rpc, r1 = min(H, r0 + rpc);
    const int nrow = max(0, r1 - r0), npx = nrow * W;
    const int PL = (rpc + 2) * W;
    const int di = RT / W, dj = RT - (RT / W) * W;
    float *const S = sm + W;
    float *const Gn = (rank > 0 && nrow > 0) ? cl.map_shared_rank(sm, rank - 1) + W + rpc * W : nullptr;
    float *const Gs = (rank + 1 < NC && r1 < H) ? cl.map_shared_rank(sm, rank + 1) : nullptr;
    auto push_n = [&](int k, int li, int j, float v) {
        if (li == 0 && Gn) Gn[k * PL + j] = v;
    };
    auto push_s = [&](int k, int li, int j, float v) {
        if (li == nrow - 1 && Gs) Gs[k * PL + j] = v;
    };
    const float tau = A.k.cp_tau, sg = A.k.cp_sigma, beta = A.k.beta, lam = A.k.lambda;

    // ---- load the band; the first row of Xbar goes to the north CTA (its south ghost row)
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        const size_t o = (size_t)(r0 + li) * P + j;
#pragma unroll
        for (int k = C_P1; k <= C_Q22; ++k) S[k * PL + x] = (HAS_W || k >= C_Q11) ? ldT<TF>(in[k], o) : 0.f;
#pragma unroll
        for (int k = C_W; k <= C_VB; ++k) {
            const float v = (HAS_W || (k != C_W && k != C_WB)) ? ldT<TF>(in[k], o) : 0.f;
            S[k * PL + x] = v;
            if (k >= C_WB) push_n(k, li, j, v);
        }
        S[C_IX * PL + x] = ldT<T>(dat[0], o);
        S[C_IY * PL + x] = ldT<T>(dat[1], o);
        S[C_IT * PL + x] = ldT<T>(dat[2], o);
    });
    cl.sync();

    ClusterStop stop{red, &part, &total, res_check, res_final, donep, itersp, rows, A.tol, rank, NC};
    for (int it = 0; it < A.iters; ++it) {
        // ---- phase A: y' = P(y + tau grad Xbar)
        for_band(npx, W, di, dj, [&](int x, int li, int j) {
            const int i = r0 + li;
            const bool hx = j < W - 1, hy = i < H - 1;
            auto gx = [&](int k) { return hx ? S[k * PL + x + 1] - S[k * PL + x] : 0.f; };
            auto gy = [&](int k) { return hy ? S[k * PL + x + W] - S[k * PL + x] : 0.f; };
            float y[6], g[6], yn[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) y[k] = (HAS_W || k >= 2) ? storage_round<TF>(S[k * PL + x]) : 0.f;
            g[0] = HAS_W ? gx(C_WB) : 0.f;
            g[1] = HAS_W ? gy(C_WB) : 0.f;
            g[2] = gx(C_UB);
            g[3] = gy(C_UB);
            g[4] = gx(C_VB);
            g[5] = gy(C_VB);
            cp_dual<HAS_W>(y, g, tau, yn);
#pragma unroll
            for (int k = 0; k < 6; ++k) S[k * PL + x] = yn[k];
            push_s(C_P2, li, j, yn[1]);
            push_s(C_Q12, li, j, yn[3]);
            push_s(C_Q22, li, j, yn[5]);
        });
        cl.sync();
        // ---- phase B: X' = prox(X + sigma div y'), Xbar' = 2X' - X
        const bool check = A.check && (it + 1) % 10 == 0;
        const bool fin = A.final_res && it == A.iters - 1;
        float res = 0.f;
        for_band(npx, W, di, dj, [&](int x, int li, int j) {
            const int i = r0 + li;
            const bool ex = j < W - 1, ey = i < H - 1, wx = j > 0, ny = i > 0;
            auto dv = [&](int cx, int cy) {
                return (((ex ? S[cx * PL + x] : 0.f) - (wx ? S[cx * PL + x - 1] : 0.f)) + (ey ? S[cy * PL + x] : 0.f)) -
                       (ny ? S[cy * PL + x - W] : 0.f);
            };
            float xv[3] = {HAS_W ? S[C_W * PL + x] : 0.f, S[C_U * PL + x], S[C_V * PL + x]};
            const float xold[3] = {xv[0], xv[1], xv[2]};
            const float d3[3] = {HAS_W ? dv(C_P1, C_P2) : 0.f, dv(C_Q11, C_Q12), dv(C_Q21, C_Q22)};
            res += cp_primal<HAS_W>(xv, d3, S[C_IX * PL + x], S[C_IY * PL + x], S[C_IT * PL + x], beta, lam, sg);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!HAS_W && c == 0) continue;
                const float xb = storage_round<TF>(2.f * xv[c] - xold[c]);
                S[(C_W + c) * PL + x] = storage_round<TF>(xv[c]);
                S[(C_WB + c) * PL + x] = xb;
                push_n(C_WB + c, li, j, xb);
            }
        });
        if (stop.end_iteration(cl, it, res, check, fin)) break;
    }
    stop.finish(A.final_res);

    // ---- store the band
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        const size_t o = (size_t)(r0 + li) * P + j;
#pragma unroll
        for (int k = C_P1; k <= C_Q22; ++k)
            if (HAS_W || k >= C_Q11) stT<TF>(out[k], o, S[k * PL + x]);
#pragma unroll
        for (int k = C_W; k <= C_VB; ++k)
            if (HAS_W || (k != C_W && k != C_WB)) stT<TF>(out[k], o, S[k * PL + x]);
    });
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------------- pDR
// The band layout for pDR (Sec. 3.1.2): planes X (w u v), Xbar, ybar (p1 p2 q11 q12 q21 q22), the
// data, the right-hand side b and X^k (for the residual): 21 planes.  Per iteration:
//   1. b = Xbar + sigma div ybar and X^k at every band pixel, then the red Gauss-Seidel update at
//      the red ones (it reads only its own b and black neighbours, which this phase leaves alone);
//   2. n times: black half-sweep, red half-sweep (the fused engine's R (B R)^n);
//   3. Xbar and ybar updates (east and south neighbours of X^{k+1}) and |X^{k+1} - X^k|^2.
// Each half-sweep writes the updated pixels of the first / last band row into the neighbours'
// ghost rows; within a half-sweep a CTA reads only the other colour of its ghost rows, which no
// CTA writes in that half-sweep.  The last band row of ybar goes to the south CTA after step 3.
// The state is rounded to the storage type where the per-kernel engine's stores round it.
enum { D_W, D_U, D_V, D_WB, D_UB, D_VB, D_P1, D_P2, D_Q11, D_Q12, D_Q21, D_Q22, D_IX, D_IY, D_IT, D_B, D_O = D_B + 3 };
constexpr int NPL_PDR = D_O + 3;
__constant__ int kFieldPDR[12] = {F_W, F_U, F_V, F_WB, F_UB, F_VB, F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22};

template <typename T, typename TF, bool HAS_W>
__global__ void __launch_bounds__(RT, 1) k_pdr_resident(ResArgs A) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[32];
    __shared__ double part, total;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), NC = (int)cl.num_blocks();

    int H, W, P;
    const void *in[12], *dat[3];
    void *out[12];
    double *res_check, *res_final;
    int *donep;
    long long *itersp;
    double rows;
    if (A.pairs) {
        const int q = A.list[blockIdx.x / NC];
        const PairIter *pp = A.pairs + q;
        const int4 gq = *reinterpret_cast<const int4 *>(&pp->g);
        H = gq.x;
        W = gq.y;
        P = gq.z;
        const Fields *fi = pp->buf + A.parity_in, *fo = pp->buf + A.parity_out;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            in[k] = fi->f[kFieldPDR[k]];
            out[k] = fo->f[kFieldPDR[k]];
        }
        dat[0] = pp->Ix;
        dat[1] = pp->Iy;
        dat[2] = pp->It;
        const PairScalars *ps = A.scal + q;
        res_check = ps->res_check;
        res_final = ps->res_final;
        donep = ps->done;
        itersp = ps->iters;
        rows = ps->rows;
    } else {
        H = A.g.H;
        W = A.g.W;
        P = A.g.pitch;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            in[k] = A.in.f[kFieldPDR[k]];
            out[k] = A.out.f[kFieldPDR[k]];
        }
        dat[0] = A.Ix;
        dat[1] = A.Iy;
        dat[2] = A.It;
        res_check = A.sc.res_check;
        res_final = A.sc.res_final;
        donep = A.sc.done;
        itersp = A.sc.iters;
        rows = A.sc.rows;
    }
    const int rpc = (H + NC - 1) / NC;
    const int r0 = rank * rpc, r1 = min(H, r0 + rpc);
    const int nrow = max(0, r1 - r0), npx = nrow * W;
    const int PL = (rpc + 2) * W;
    const int di = RT / W, dj = RT - (RT / W) * W;
    float *const S = sm + W;
    float *const Gn = (rank > 0 && nrow > 0) ? cl.map_shared_rank(sm, rank - 1) + W + rpc * W : nullptr;
    float *const Gs = (rank + 1 < NC && r1 < H) ? cl.map_shared_rank(sm, rank + 1) : nullptr;
    auto push_n = [&](int k, int li, int j, float v) {
        if (li == 0 && Gn) Gn[k * PL + j] = v;
    };
    auto push_s = [&](int k, int li, int j, float v) {
        if (li == nrow - 1 && Gs) Gs[k * PL + j] = v;
    };
    float sg, ta;
    pdr_steps(A.k, A.pairs ? A.pairs[A.list[blockIdx.x / NC]].ms_max : A.ms_max, sg, ta);
    const float st = sg * ta, beta = A.k.beta, lam = A.k.lambda;
    const int c0 = HAS_W ? 0 : 1;

    // ---- load the band; boundary rows of X to both neighbours, the last row of ybar to the south
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        const size_t o = (size_t)(r0 + li) * P + j;
#pragma unroll
        for (int k = D_W; k <= D_VB; ++k) {
            const float v = (HAS_W || (k != D_W && k != D_WB)) ? ldT<TF>(in[k], o) : 0.f;
            S[k * PL + x] = v;
            if (k <= D_V) {
                push_n(k, li, j, v);
                push_s(k, li, j, v);
            }
        }
#pragma unroll
        for (int k = D_P1; k <= D_Q22; ++k) {
            const float v = (HAS_W || k >= D_Q11) ? ldT<T>(in[k], o) : 0.f;
            S[k * PL + x] = v;
            if (k == D_P2 || k == D_Q12 || k == D_Q22) push_s(k, li, j, v);
        }
        S[D_IX * PL + x] = ldT<T>(dat[0], o);
        S[D_IY * PL + x] = ldT<T>(dat[1], o);
        S[D_IT * PL + x] = ldT<T>(dat[2], o);
    });
    cl.sync();

    // one Gauss-Seidel update of the pixel's X (all components), stored rounded and pushed
    auto gs_pixel = [&](int x, int li, int j) {
        const int i = r0 + li;
        const bool hw = j > 0, he = j < W - 1, hn = i > 0, hs = i < H - 1;
        const int nb = (int)hw + (int)he + (int)hn + (int)hs;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c < c0) continue;
            const float *Xc = S + (D_W + c) * PL;
            float acc = 0.f;
            if (hw) acc += Xc[x - 1];
            if (he) acc += Xc[x + 1];
            if (hn) acc += Xc[x - W];
            if (hs) acc += Xc[x + W];
            const float v = storage_round<TF>(pdr_gs(S[(D_B + c) * PL + x], acc, nb, st));
            S[(D_W + c) * PL + x] = v;
            push_n(D_W + c, li, j, v);
            push_s(D_W + c, li, j, v);
        }
    };
    ClusterStop stop{red, &part, &total, res_check, res_final, donep, itersp, rows, A.tol, rank, NC};
    for (int it = 0; it < A.iters; ++it) {
        // ---- 1. b = Xbar + sigma div ybar, X^k, and the red half-sweep
        for_band(npx, W, di, dj, [&](int x, int li, int j) {
            const int i = r0 + li;
            const bool ex = j < W - 1, wx = j > 0, ey = i < H - 1, ny = i > 0;
            const int Y1[3] = {D_P1, D_Q11, D_Q21}, Y2[3] = {D_P2, D_Q12, D_Q22};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c < c0) continue;
                const float *a = S + Y1[c] * PL, *b = S + Y2[c] * PL;
                const float dv = (((ex ? a[x] : 0.f) - (wx ? a[x - 1] : 0.f)) + (ey ? b[x] : 0.f)) - (ny ? b[x - W] : 0.f);
                S[(D_B + c) * PL + x] = pdr_rhs(S[(D_WB + c) * PL + x], dv, sg);
                S[(D_O + c) * PL + x] = S[(D_W + c) * PL + x];
            }
            if (((i + j) & 1) == 0) gs_pixel(x, li, j);
        });
        cl.sync();
        // ---- 2. (black, red)^n
        for (int sw = 0; sw < A.k.gs_sweeps; ++sw) {
            for (int colour = 1; colour >= 0; --colour) {
                for_band(npx, W, di, dj, [&](int x, int li, int j) {
                    if (((r0 + li + j) & 1) == colour) gs_pixel(x, li, j);
                });
                cl.sync();
            }
        }
        // ---- 3. Xbar, ybar, residual
        const bool check = A.check && (it + 1) % 10 == 0;
        const bool fin = A.final_res && it == A.iters - 1;
        float res = 0.f;
        for_band(npx, W, di, dj, [&](int x, int li, int j) {
            const int i = r0 + li;
            const bool hx = j < W - 1, hy = i < H - 1;
            const float xv[3] = {HAS_W ? S[D_W * PL + x] : 0.f, S[D_U * PL + x], S[D_V * PL + x]};
            float xb[3] = {HAS_W ? S[D_WB * PL + x] : 0.f, S[D_UB * PL + x], S[D_VB * PL + x]};
            pdr_xbar<HAS_W>(xv, xb, S[D_IX * PL + x], S[D_IY * PL + x], S[D_IT * PL + x], beta, lam, sg);
            float g[6], y[6], yn[6];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *Xc = S + (D_W + c) * PL;
                g[2 * c] = (HAS_W || c > 0) && hx ? Xc[x + 1] - xv[c] : 0.f;
                g[2 * c + 1] = (HAS_W || c > 0) && hy ? Xc[x + W] - xv[c] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) y[k] = (HAS_W || k >= 2) ? S[(D_P1 + k) * PL + x] : 0.f;
            pdr_ybar<HAS_W>(y, g, ta, yn);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c < c0) continue;
                S[(D_WB + c) * PL + x] = storage_round<TF>(xb[c]);
                const float d = xv[c] - S[(D_O + c) * PL + x];
                res = fmaf(d, d, res);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (!HAS_W && k < 2) continue;
                const float v = storage_round<T>(yn[k]);
                S[(D_P1 + k) * PL + x] = v;
                if (k == 1 || k == 3 || k == 5) push_s(D_P1 + k, li, j, v);
            }
        });
        if (stop.end_iteration(cl, it, res, check, fin)) break;
    }
    stop.finish(A.final_res);

    // ---- store the band
    for_band(npx, W, di, dj, [&](int x, int li, int j) {
        const size_t o = (size_t)(r0 + li) * P + j;
#pragma unroll
        for (int k = D_W; k <= D_VB; ++k)
            if (HAS_W || (k != D_W && k != D_WB)) stT<TF>(out[k], o, S[k * PL + x]);
#pragma unroll
        for (int k = D_P1; k <= D_Q22; ++k)
            if (HAS_W || k >= D_Q11) stT<T>(out[k], o, S[k * PL + x]);
    });
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

constexpr size_t SMEM_MAX = 200 * 1024;  // dynamic shared memory a CTA may use for its band

// The function attributes every launch of one kernel instance needs, set once per instance and
// process: the dynamic shared-memory ceiling at SMEM_MAX (not at one launch's own size -- a
// CUDA graph node captured with a larger band than a later launch would otherwise find the
// function's ceiling lowered beneath it) and, for 16-CTA clusters, the non-portable size.  All
// instances share one function-pointer type, so the record is keyed by the pointer itself.
template <typename K> cudaError_t prepare_kernel(K kern) {
    static std::mutex mu;
    static std::map<const void *, cudaError_t> done;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = done.find((const void *)kern);
    if (it != done.end()) return it->second;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    done[(const void *)kern] = r;
    return r;
}

template <typename K>
cudaError_t launch_cluster(K kern, const ResArgs &a, int nclusters, int nc, size_t smem, cudaStream_t s) {
    if (smem > SMEM_MAX || nclusters < 1 || nc < 1) return cudaErrorInvalidValue;
    cudaError_t e = prepare_kernel(kern);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nclusters * nc);   // a whole number of clusters
    cfg.blockDim = dim3(RT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T, typename TF>
cudaError_t launch_m(const ResArgs &a, int nclusters, int nc, size_t smem, cudaStream_t s) {
    const bool has_w = a.k.beta != 0.f;
    auto go = [&](auto kern) { return launch_cluster(kern, a, nclusters, nc, smem, s); };
    if (a.k.method == 3) return has_w ? go(k_cp_resident<T, TF, true>) : go(k_cp_resident<T, TF, false>);
    if (a.k.method == 2) return has_w ? go(k_pdr_resident<T, TF, true>) : go(k_pdr_resident<T, TF, false>);
    if (a.k.method == 1) return has_w ? go(k_admm_resident<T, TF, true, 1>) : go(k_admm_resident<T, TF, false, 1>);
    return has_w ? go(k_admm_resident<T, TF, true, 0>) : go(k_admm_resident<T, TF, false, 0>);
}

// The cluster size and how many such clusters the device runs at once, for a launch with a full
// band of shared memory (one CTA per SM): 16 CTAs (a non-portable size) where the device
// schedules at least one such cluster, else 8, else none (the resident engine is then off).
// cudaOccupancyMaxActiveClusters counts what the GPC layout allows, which is fewer than
// SMs / cluster size when a GPC cannot hold a whole 16-CTA cluster.  Queried once, with one
// instance of the kernels: every instance launches 512 threads with at most 128 registers and a
// band of up to SMEM_MAX bytes, so all share the same one-CTA-per-SM occupancy.
struct ClusterCaps {
    int nc = 0, active = 0;
};

ClusterCaps query_cluster() {
    ClusterCaps c;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return c;
    }
    auto kern = k_admm_resident<float, float, true, 0>;
    if (prepare_kernel(kern) != cudaSuccess) {
        cudaGetLastError();
        return c;
    }
    for (int nc : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nc);
        cfg.blockDim = dim3(RT);
        cfg.dynamicSmemBytes = SMEM_MAX;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = nc;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        if (n > 0) {
            c.nc = nc;
            c.active = n;
            return c;
        }
    }
    return c;
}

const ClusterCaps &cluster_caps() {
    static const ClusterCaps c = query_cluster();
    return c;
}

// Largest level (pixels) the default engine runs resident: above it one cluster's 16 SMs
// compute an iteration more slowly than a streaming kernel spread over the whole GPU.
constexpr long RESIDENT_MAX_PX = 32000;

}  // namespace

int admm_resident_cluster() { return cluster_caps().nc; }

int admm_resident_max_clusters() { return cluster_caps().active; }

size_t admm_resident_smem(Geom g, int method, int nc) {
    if (nc <= 0) nc = admm_resident_cluster();
    if (nc <= 0) return SIZE_MAX;
    const size_t rpc = (size_t)((g.H + nc - 1) / nc);
    return (rpc + 2) * (size_t)g.W * (method == 2 ? NPL_PDR : NPL) * sizeof(float);
}

bool admm_resident_fits(Geom g, int method) {
    return admm_resident_cluster() > 0 && g.H >= 1 && g.W >= 1 && admm_resident_smem(g, method, 0) <= SMEM_MAX;
}

int admm_resident_nc(Geom, int) { return admm_resident_cluster(); }

// pDR's per-kernel engine takes 2n + 1 launches per iteration, so its resident form wins at every
// size that fits (with one sweep the runtime compares against the one-launch tile kernel
// instead); the ADMM methods and ALG1 (one launch per iteration) only up to RESIDENT_MAX_PX.
bool admm_resident_preferred(Geom g, int method) { return method == 2 || (long)g.H * g.W <= RESIDENT_MAX_PX; }

cudaError_t launch_admm_resident(const ResArgs &a, int nclusters, int nc, size_t smem, int prec, int prec_flow,
                                 cudaStream_t s) {
    if (prec == PREC_F32) return launch_m<float, float>(a, nclusters, nc, smem, s);
    if (prec == PREC_F16)
        return prec_flow == PREC_F32 ? launch_m<__half, float>(a, nclusters, nc, smem, s)
                                     : launch_m<__half, __half>(a, nclusters, nc, smem, s);
    return prec_flow == PREC_F32 ? launch_m<__nv_bfloat16, float>(a, nclusters, nc, smem, s)
                                 : launch_m<__nv_bfloat16, __nv_bfloat16>(a, nclusters, nc, smem, s);
}

}  // namespace tvl1
