// k_reduce.cu -- FP64 reductions on the device: the residual behind the stopping test (the
// paper proves convergence, Props. 3.1/3.2, but gives no stopping rule; the library stops a
// warp's inner loop when the normalised residual drops below tol, tested every 10 iterations),
// the primal energy of eq. (l1:finite) and the dual value <It, s> of eq. (dual:l1:flow:cons).
// Partial sums are formed per block with warp shuffles and summed in a fixed order, so the
// results are deterministic.
#include <math.h>

#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

constexpr int PX = 32, PY = 8;

__global__ void k_reduce_check(const double *partials, int n, double *out, double rows, double tol, int *done,
                               long long *iters_counter, int add_iters) {
    __shared__ double red[32];
    if (done && *done) return;  // the warp already stopped: keep the residual of the stop
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partials[k];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) {
        out[0] = tot;
        if (iters_counter) *iters_counter += add_iters;
        if (tol > 0.0 && done && sqrt(tot / rows) < tol) *done = 1;
    }
}

__global__ void k_sum(const double *partials, int n, double *out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partials[k];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) out[0] = tot;
}

__global__ void k_count_iters(long long *counter, const int *done, int n) {
    if (!(done && *done)) *counter += n;
}

// One block per pair: the stopping test (final = 0) or the final residual (final = 1).  A pair
// that stopped keeps the residual of its stopping test.
__global__ void k_reduce_check_batched(const double *partials, const PairScalars *ps, double tol, int add_iters,
                                       int final) {
    __shared__ double red[32];
    const PairScalars P = ps[blockIdx.x];
    if (P.resident) return;  // the level-resident engine keeps this pair's scalars itself
    const bool stopped = P.done && *P.done;
    if (stopped && !final) return;
    if (stopped) {
        if (threadIdx.x == 0) *P.res_final = *P.res_check;
        return;
    }
    double v = 0.0;
    for (int k = P.part_begin + threadIdx.x; k < P.part_end; k += blockDim.x) v += partials[k];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) {
        if (final) {
            *P.res_final = tot;
        } else {
            *P.res_check = tot;
            if (P.iters) *P.iters += add_iters;
            if (tol > 0.0 && sqrt(tot / P.rows) < tol) *P.done = 1;
        }
    }
}

__global__ void k_count_iters_batched(const PairScalars *ps, int npairs, int n, bool use_done) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    const PairScalars P = ps[k];
    if (!P.resident && !(use_done && P.done && *P.done)) *P.iters += n;
}

template <typename T, typename TF>
__global__ void k_energy(Fields f, const T *Ix, const T *Iy, const T *It, Geom g, float beta, float lambda,
                         double *pe, double *pd) {
    __shared__ double red[32];
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    const int H = g.H, W = g.W, P = g.pitch;
    const bool has_w = beta != 0.f && f.f[F_W];
    double e = 0.0, d = 0.0;
    if (i < H && j < W) {
        const size_t o = (size_t)i * P + j;
        const bool hx = j < W - 1, hy = i < H - 1;
        auto L = [&](int fi, size_t off) { return is_flow_field(fi) ? ldT<TF>(f.f[fi], off) : ldT<T>(f.f[fi], off); };
        const float u = L(F_U, o), v = L(F_V, o);
        const float ux = hx ? L(F_U, o + 1) - u : 0.f, uy = hy ? L(F_U, o + P) - u : 0.f;
        const float vx = hx ? L(F_V, o + 1) - v : 0.f, vy = hy ? L(F_V, o + P) - v : 0.f;
        e = sqrt((double)ux * ux + (double)uy * uy + (double)vx * vx + (double)vy * vy);
        float rho = Store<T>::ld(Ix + o) * u + Store<T>::ld(Iy + o) * v + Store<T>::ld(It + o);
        if (has_w) {
            const float w = L(F_W, o);
            rho += beta * w;
            const float wx = hx ? L(F_W, o + 1) - w : 0.f, wy = hy ? L(F_W, o + P) - w : 0.f;
            e += sqrt((double)wx * wx + (double)wy * wy);
        }
        e += (double)lambda * fabs((double)rho);
        if (f.f[F_S]) d = (double)Store<T>::ld(It + o) * (double)L(F_S, o);
    }
    const double te = block_sum(e, red);
    __syncthreads();
    const double td = block_sum(d, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        pe[block_linear_id()] = te;
        pd[block_linear_id()] = td;
    }
}

template <typename T, typename TF>
__global__ void k_parity_fix(Fields from, Fields to, Geom g, const int *done, int want_done) {
    if (((done && *done) ? 1 : 0) != want_done) return;
    const int j = blockIdx.x * PX + threadIdx.x, i = blockIdx.y * PY + threadIdx.y;
    if (i >= g.H || j >= g.W) return;
    const size_t o = (size_t)i * g.pitch + j;
    for (int k = 0; k < NFIELDS; ++k) {
        if (!(from.f[k] && to.f[k])) continue;
        if (is_flow_field(k)) reinterpret_cast<TF *>(to.f[k])[o] = reinterpret_cast<const TF *>(from.f[k])[o];
        else reinterpret_cast<T *>(to.f[k])[o] = reinterpret_cast<const T *>(from.f[k])[o];
    }
}

}  // namespace

void launch_reduce_check(const double *partials, int n, double *out, double rows, double tol, int *done,
                         long long *iters_counter, int add_iters, cudaStream_t s) {
    k_reduce_check<<<1, 1024, 0, s>>>(partials, n, out, rows, tol, done, iters_counter, add_iters);
}

void launch_sum(const double *partials, int n, double *out, cudaStream_t s) { k_sum<<<1, 1024, 0, s>>>(partials, n, out); }

void launch_count_iters(long long *counter, const int *done, int n, cudaStream_t s) {
    k_count_iters<<<1, 1, 0, s>>>(counter, done, n);
}

void launch_reduce_check_batched(const double *partials, const PairScalars *ps, int npairs, double tol,
                                 int add_iters, int final, cudaStream_t s) {
    if (npairs > 0) k_reduce_check_batched<<<npairs, 256, 0, s>>>(partials, ps, tol, add_iters, final);
}

void launch_count_iters_batched(const PairScalars *ps, int npairs, int n, bool use_done, cudaStream_t s) {
    if (npairs > 0) k_count_iters_batched<<<(npairs + 127) / 128, 128, 0, s>>>(ps, npairs, n, use_done);
}

int energy_blocks(Geom g) { return ((g.W + PX - 1) / PX) * ((g.H + PY - 1) / PY); }

void launch_energy(const Fields &f, const void *Ix, const void *Iy, const void *It, Geom g, float beta, float lambda,
                   int prec, int prec_flow, double *pe, double *pd, cudaStream_t s) {
    dim3 grid((g.W + PX - 1) / PX, (g.H + PY - 1) / PY), blk(PX, PY);
    TVL1_DISPATCH_PREC(prec, T, TVL1_DISPATCH_PREC(prec_flow, TF,
                       k_energy<T, TF><<<grid, blk, 0, s>>>(f, (const T *)Ix, (const T *)Iy, (const T *)It, g, beta,
                                                            lambda, pe, pd)));
}

void launch_parity_fix(const Fields &from, const Fields &to, Geom g, int prec, int prec_flow, const int *done,
                       int want_done, cudaStream_t s) {
    dim3 grid((g.W + PX - 1) / PX, (g.H + PY - 1) / PY), blk(PX, PY);
    TVL1_DISPATCH_PREC(prec, T, TVL1_DISPATCH_PREC(prec_flow, TF,
                       k_parity_fix<T, TF><<<grid, blk, 0, s>>>(from, to, g, done, want_done)));
}

}  // namespace tvl1
