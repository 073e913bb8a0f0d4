// tvl1_device.cuh -- device helpers: storage conversions and reductions.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tvl1_internal.h"

namespace tvl1 {

template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// x rounded to storage type T and back: the value a store of x followed by a load yields.
template <typename T> __device__ __forceinline__ float storage_round(float x) {
    T t;
    Store<T>::st(&t, x);
    return Store<T>::ld(&t);
}

template <typename T> __device__ __forceinline__ float ldT(const void *base, size_t off) {
    return Store<T>::ld(reinterpret_cast<const T *>(base) + off);
}
template <typename T> __device__ __forceinline__ void stT(void *base, size_t off, float v) {
    Store<T>::st(reinterpret_cast<T *>(base) + off, v);
}

// Sum of one double per thread over the block (blockDim.x*blockDim.y*blockDim.z <= 1024,
// multiple of 32).  The result is valid in thread 0.  Fixed order: deterministic.
__device__ __forceinline__ double block_sum(double v, double *sh /* >= 32 doubles */) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = tid < (nthr >> 5) ? sh[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

__device__ __forceinline__ int block_linear_id() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }

// a~ of the current warp: a fixed value or max M_s (Prop. 3.1: a~ = ||M_s||), at least 1e-12.
__device__ __forceinline__ float a_tilde_of(const Coefs &k, const float *ms_max) {
    if (k.a_tilde_fixed > 0.f) return k.a_tilde_fixed;
    float m = ms_max ? *ms_max : 0.f;
    return m > 1e-12f ? m : 1e-12f;
}

// The ADMM step c of the current iteration: the parameter, or with an adaptive step the value the
// solve keeps on the device directly before the pair's ms_max.
__device__ __forceinline__ float c_of(const Coefs &k, const float *ms_max) { return k.c_dev ? ms_max[-1] : k.c; }

// pDR's steps: sigma and tau of the parameters, or with adaptive steps (sigma theta, tau / theta)
// with the factor theta (a power of two, so sigma tau stays bitwise the same) kept on the device in
// the same slot as the adaptive ADMM step.
__device__ __forceinline__ void pdr_steps(const Coefs &k, const float *ms_max, float &sg, float &ta) {
    if (k.c_dev) {
        const float th = ms_max[-1];
        sg = k.sigma * th;
        ta = k.tau / th;
    } else {
        sg = k.sigma;
        ta = k.tau;
    }
}

}  // namespace tvl1

#define TVL1_DISPATCH_PREC(prec, T, ...)                         \
    do {                                                          \
        if ((prec) == tvl1::PREC_F32) {                           \
            using T = float;                                      \
            __VA_ARGS__;                                          \
        } else if ((prec) == tvl1::PREC_F16) {                    \
            using T = __half;                                     \
            __VA_ARGS__;                                          \
        } else {                                                  \
            using T = __nv_bfloat16;                              \
            __VA_ARGS__;                                          \
        }                                                         \
    } while (0)
