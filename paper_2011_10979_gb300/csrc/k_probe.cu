// k_probe.cu -- bandwidth probe of the L2 cache for the roofline of the L2-resident pyramid levels
// (a 640 x 480 level's iteration moves 28 MB, which stays in the 129 MB L2 between iterations).
// One launch streams a working set of `bytes` (half read, half written) `passes` times: every
// thread copies the same 16-byte words on every pass, loading with the L2-only cache hint, so the
// passes after the first are served by L2 and the launch overhead is spread over all of them.
#include <cuda_runtime.h>

#include <string>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"

namespace tvl1 {
namespace {

__global__ void k_l2_stream(const float4 *__restrict__ src, float4 *__restrict__ dst, size_t n4, int passes) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 v = __ldcg(src + i);
            v.x += 1.f;  // keeps the copy from being folded across passes
            dst[i] = v;
        }
}

}  // namespace
}  // namespace tvl1

extern "C" of_status of_l2_bandwidth(size_t bytes, int passes, double *gbps) {
    using namespace tvl1;
    if (!gbps || passes < 1 || bytes < 4096) {
        tvl1_set_error("of_l2_bandwidth: bad arguments");
        return OF_EINVAL;
    }
    const size_t half = bytes / 2 / 16 * 16, n4 = half / 16;
    int dev = 0, sms = 0;
    char *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&buf, 2 * half);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, 2 * half);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        const float4 *src = (const float4 *)buf;
        float4 *dst = (float4 *)(buf + half);
        const dim3 grid((unsigned)sms * 8), block(256);
        k_l2_stream<<<grid, block>>>(src, dst, n4, 2);  // warm: the working set into L2
        cudaEventRecord(e0);
        k_l2_stream<<<grid, block>>>(src, dst, n4, passes);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) {
        tvl1_set_error((std::string("of_l2_bandwidth: ") + cudaGetErrorString(e)).c_str());
        return OF_ECUDA;
    }
    *gbps = 2.0 * (double)half * passes / (ms * 1e-3) / 1e9;
    return OF_OK;
}
