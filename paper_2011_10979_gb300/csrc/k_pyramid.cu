// k_pyramid.cu -- coarse-to-fine machinery (Sec. 4: "standard coarse-to-fine framework ...
// multiscale pyramid" with warping; the paper gives no details, the readings are stated at
// each kernel): Gaussian pre-smoothing + resampling, level transfer of the fields, derivative
// images, warping + linearisation with the per-warp max of M_s, and precision conversion.
#include <math.h>

#include "tvl1_device.cuh"

namespace tvl1 {

namespace {

constexpr int B2X = 32, B2Y = 8;

__device__ __forceinline__ int reflect_index(int k, int n) {
    // half-sample symmetric extension for any integer k: period 2n, mirrored halves
    const int period = 2 * n;
    int m = k % period;
    if (m < 0) m += period;
    return m < n ? m : period - 1 - m;
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// Bilinear value of plane f (H x W, pitch P) at (x, y) inside [0, W-1] x [0, H-1].
template <typename T>
__device__ __forceinline__ float bilinear(const T *f, int H, int W, int P, float x, float y) {
    const float xf = floorf(x), yf = floorf(y);
    const int x0 = (int)xf, y0 = (int)yf;
    const float fx = x - xf, fy = y - yf;
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    const float a = Store<T>::ld(f + (size_t)y0 * P + x0), b = Store<T>::ld(f + (size_t)y0 * P + x1);
    const float c = Store<T>::ld(f + (size_t)y1 * P + x0), d = Store<T>::ld(f + (size_t)y1 * P + x1);
    const float top = (1.f - fx) * a + fx * b;
    const float bot = (1.f - fx) * c + fx * d;
    return (1.f - fy) * top + fy * bot;
}

// Sample position j + d clamped to [0, n-1], as integer part and fraction, in FP64: j + d and
// its fraction are exact there for any FP32 displacement d.
__device__ __forceinline__ void split_pos_f64(int j, float d, int n, int &x0, double &fx) {
    const double xs = (double)j + (double)d;
    if (!(xs > 0.0)) {              // also catches NaN
        x0 = 0;
        fx = 0.0;
    } else if (xs >= (double)(n - 1)) {
        x0 = n - 1;
        fx = 0.0;
    } else {
        const double fl = floor(xs);
        x0 = (int)fl;
        fx = xs - fl;
    }
}

// Bilinear value of an FP32 plane (H x W, pitch P) at (x0 + fx, y0 + fy) in FP64 arithmetic (the
// four samples are exact in FP64).
__device__ __forceinline__ double bilinear_split_f64(const float *f, int H, int W, int P, int x0, double fx, int y0,
                                                     double fy) {
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    const double a = __ldg(f + (size_t)y0 * P + x0), b = __ldg(f + (size_t)y0 * P + x1);
    const double c = __ldg(f + (size_t)y1 * P + x0), d = __ldg(f + (size_t)y1 * P + x1);
    const double top = (1.0 - fx) * a + fx * b;
    const double bot = (1.0 - fx) * c + fx * d;
    return (1.0 - fy) * top + fy * bot;
}

// Separable Gaussian, first along rows (x), then along columns (y); half-sample symmetric border.
__global__ void k_blur_rows(const float *__restrict__ in, float *__restrict__ out, Geom g, GaussTaps t) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= g.H || j >= g.W) return;
    const float *row = in + (size_t)i * g.pitch;
    float acc = 0.f;
    for (int k = -t.R; k <= t.R; ++k) acc += t.w[k + t.R] * __ldg(row + reflect_index(j + k, g.W));
    out[(size_t)i * g.pitch + j] = acc;
}

__global__ void k_blur_cols(const float *__restrict__ in, float *__restrict__ out, Geom g, GaussTaps t) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= g.H || j >= g.W) return;
    float acc = 0.f;
    for (int k = -t.R; k <= t.R; ++k) acc += t.w[k + t.R] * __ldg(in + (size_t)reflect_index(i + k, g.H) * g.pitch + j);
    out[(size_t)i * g.pitch + j] = acc;
}

// Coarse pixel centre (j + 0.5) maps to fine x = (j + 0.5) * Wf / Wc - 0.5, clamped.
__global__ void k_resample(const float *__restrict__ fine, Geom gf, float *__restrict__ coarse, Geom gc) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= gc.H || j >= gc.W) return;
    const float sx = (float)gf.W / (float)gc.W, sy = (float)gf.H / (float)gc.H;
    const float x = clampf((j + 0.5f) * sx - 0.5f, 0.f, (float)(gf.W - 1));
    const float y = clampf((i + 0.5f) * sy - 0.5f, 0.f, (float)(gf.H - 1));
    coarse[(size_t)i * gc.pitch + j] = bilinear<float>(fine, gf.H, gf.W, gf.pitch, x, y);
}

// Level transfer: fine pixel centre maps to coarse x = (j + 0.5) * Wc / Wf - 0.5, clamped.
template <typename T>
__global__ void k_upsample(const T *__restrict__ coarse, Geom gc, T *__restrict__ fine, Geom gf, float scale) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= gf.H || j >= gf.W) return;
    const float sx = (float)gc.W / (float)gf.W, sy = (float)gc.H / (float)gf.H;
    const float x = clampf((j + 0.5f) * sx - 0.5f, 0.f, (float)(gc.W - 1));
    const float y = clampf((i + 0.5f) * sy - 0.5f, 0.f, (float)(gc.H - 1));
    Store<T>::st(fine + (size_t)i * gf.pitch + j, scale * bilinear<T>(coarse, gc.H, gc.W, gc.pitch, x, y));
}

// Central differences with clamped neighbour indices.
__global__ void k_derivatives(const float *__restrict__ I, Geom g, float *__restrict__ Ix, float *__restrict__ Iy) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= g.H || j >= g.W) return;
    const int jl = max(j - 1, 0), jr = min(j + 1, g.W - 1), iu = max(i - 1, 0), id = min(i + 1, g.H - 1);
    const size_t o = (size_t)i * g.pitch + j;
    Ix[o] = 0.5f * (__ldg(I + (size_t)i * g.pitch + jr) - __ldg(I + (size_t)i * g.pitch + jl));
    Iy[o] = 0.5f * (__ldg(I + (size_t)id * g.pitch + j) - __ldg(I + (size_t)iu * g.pitch + j));
}

// Warp I1 and its derivatives to (x + u0, y + v0) (clamped), linearise around d0:
// It = I1w - I0 - Ix u0 - Iy v0, so that rho(w, d) = Ix u + Iy v + beta w + It.
// The block max of M_s = beta^2 + Ix^2 + Iy^2 (of the stored, rounded values) raises *ms_max.
// The interpolation and It run in FP64 and are rounded once, when stored: It is a small difference
// of terms up to |grad I| |d0|, and the L1 data term puts the flow of weakly textured pixels on the
// line Ix u + Iy v + It = 0, so an FP32 It moved those pixels by up to a few 1e-3 px over a whole
// schedule (measured against the FP64 oracle).  The kernel runs once per warp; FP64 costs little.
template <typename T, typename TF>
__global__ void k_warp(const float *__restrict__ I0, const float *__restrict__ I1, const float *__restrict__ I1x,
                       const float *__restrict__ I1y, const TF *__restrict__ u0, const TF *__restrict__ v0, Geom g,
                       float beta, T *__restrict__ Ix, T *__restrict__ Iy, T *__restrict__ It, float *ms_max) {
    __shared__ float red[B2X * B2Y / 32];
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    float ms = 0.f;
    if (i < g.H && j < g.W) {
        const size_t o = (size_t)i * g.pitch + j;
        const float uu = Store<TF>::ld(u0 + o), vv = Store<TF>::ld(v0 + o);
        int x0, y0;
        double fx, fy;
        split_pos_f64(j, uu, g.W, x0, fx);
        split_pos_f64(i, vv, g.H, y0, fy);
        const double w1 = bilinear_split_f64(I1, g.H, g.W, g.pitch, x0, fx, y0, fy);
        const double gx = bilinear_split_f64(I1x, g.H, g.W, g.pitch, x0, fx, y0, fy);
        const double gy = bilinear_split_f64(I1y, g.H, g.W, g.pitch, x0, fx, y0, fy);
        Store<T>::st(Ix + o, (float)gx);
        Store<T>::st(Iy + o, (float)gy);
        Store<T>::st(It + o, (float)(w1 - (double)__ldg(I0 + o) - gx * (double)uu - gy * (double)vv));
        const float gxr = Store<T>::ld(Ix + o), gyr = Store<T>::ld(Iy + o);
        ms = beta * beta + gxr * gxr + gyr * gyr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ms = fmaxf(ms, __shfl_down_sync(0xffffffffu, ms, o));
    const int tid = threadIdx.y * B2X + threadIdx.x;
    if ((tid & 31) == 0) red[tid >> 5] = ms;
    __syncthreads();
    if (tid == 0) {
        float m = red[0];
        for (int k = 1; k < B2X * B2Y / 32; ++k) m = fmaxf(m, red[k]);
        // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<unsigned int *>(ms_max), __float_as_uint(m));
    }
}

template <typename S, typename D>
__global__ void k_convert(const S *__restrict__ src, D *__restrict__ dst, Geom g) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= g.H || j >= g.W) return;
    const size_t o = (size_t)i * g.pitch + j;
    Store<D>::st(dst + o, Store<S>::ld(src + o));
}

template <typename T>
__global__ void k_fill(T *__restrict__ dst, Geom g, float value) {
    const int j = blockIdx.x * B2X + threadIdx.x, i = blockIdx.y * B2Y + threadIdx.y;
    if (i >= g.H || j >= g.W) return;
    Store<T>::st(dst + (size_t)i * g.pitch + j, value);
}

dim3 grid2(int H, int W) { return dim3((W + B2X - 1) / B2X, (H + B2Y - 1) / B2Y); }

}  // namespace

GaussTaps gauss_taps(float eta) {
    GaussTaps t{};
    const double sg = 0.6 * sqrt(1.0 / ((double)eta * (double)eta) - 1.0);
    t.R = (int)ceil(3.0 * sg);
    if (t.R > MAX_GAUSS_R) {
        t.R = -1;
        return t;
    }
    double w[2 * MAX_GAUSS_R + 1], sum = 0.0;
    for (int k = -t.R; k <= t.R; ++k) {
        w[k + t.R] = sg > 0.0 ? exp(-(double)(k * k) / (2.0 * sg * sg)) : 1.0;
        sum += w[k + t.R];
    }
    for (int k = 0; k <= 2 * t.R; ++k) t.w[k] = (float)(w[k] / sum);
    return t;
}

void launch_pyr_down(const float *fine, Geom gf, float *coarse, Geom gc, const GaussTaps &taps, float *scratch,
                     cudaStream_t s) {
    // scratch holds two Hf x pitch planes: rows-blurred and fully blurred
    float *t1 = scratch, *t2 = scratch + (size_t)gf.H * gf.pitch;
    k_blur_rows<<<grid2(gf.H, gf.W), dim3(B2X, B2Y), 0, s>>>(fine, t1, gf, taps);
    k_blur_cols<<<grid2(gf.H, gf.W), dim3(B2X, B2Y), 0, s>>>(t1, t2, gf, taps);
    k_resample<<<grid2(gc.H, gc.W), dim3(B2X, B2Y), 0, s>>>(t2, gf, coarse, gc);
}

void launch_upsample(const void *coarse, Geom gc, void *fine, Geom gf, float scale, int prec, cudaStream_t s) {
    TVL1_DISPATCH_PREC(prec, T,
                       k_upsample<T><<<grid2(gf.H, gf.W), dim3(B2X, B2Y), 0, s>>>(
                           (const T *)coarse, gc, (T *)fine, gf, scale));
}

void launch_upsample_f32(const float *coarse, Geom gc, float *fine, Geom gf, float scale, cudaStream_t s) {
    k_upsample<float><<<grid2(gf.H, gf.W), dim3(B2X, B2Y), 0, s>>>(coarse, gc, fine, gf, scale);
}

void launch_derivatives(const float *I, Geom g, float *Ix, float *Iy, cudaStream_t s) {
    k_derivatives<<<grid2(g.H, g.W), dim3(B2X, B2Y), 0, s>>>(I, g, Ix, Iy);
}

void launch_warp(const float *I0, const float *I1, const float *I1x, const float *I1y, const void *u0,
                 const void *v0, Geom g, float beta, void *Ix, void *Iy, void *It, float *ms_max, int prec,
                 int prec_flow, cudaStream_t s) {
    TVL1_DISPATCH_PREC(prec, T, TVL1_DISPATCH_PREC(prec_flow, TF,
                       k_warp<T, TF><<<grid2(g.H, g.W), dim3(B2X, B2Y), 0, s>>>(
                           I0, I1, I1x, I1y, (const TF *)u0, (const TF *)v0, g, beta, (T *)Ix, (T *)Iy, (T *)It,
                           ms_max)));
}

void launch_convert(const void *const *src, int src_prec, void *const *dst, int dst_prec, int nplanes, Geom g,
                    cudaStream_t s) {
    for (int k = 0; k < nplanes; ++k) {
        if (!src[k] || !dst[k]) continue;
        TVL1_DISPATCH_PREC(src_prec, S,
                           TVL1_DISPATCH_PREC(dst_prec, D,
                                              k_convert<S, D><<<grid2(g.H, g.W), dim3(B2X, B2Y), 0, s>>>(
                                                  (const S *)src[k], (D *)dst[k], g)));
    }
}

void launch_fill(void *const *dst, int prec, int nplanes, Geom g, float value, cudaStream_t s) {
    for (int k = 0; k < nplanes; ++k) {
        if (!dst[k]) continue;
        TVL1_DISPATCH_PREC(prec, T, k_fill<T><<<grid2(g.H, g.W), dim3(B2X, B2Y), 0, s>>>((T *)dst[k], g, value));
    }
}

void launch_copy_planes(const void *const *src, void *const *dst, int nplanes, Geom g, int prec, cudaStream_t s) {
    launch_convert(src, prec, dst, prec, nplanes, g, s);
}

}  // namespace tvl1
