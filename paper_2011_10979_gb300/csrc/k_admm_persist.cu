// k_admm_persist.cu -- launch of the persistent ADMM engine (k_admm_persist.cuh): the instance
// for the storage types and method, its co-resident capacity, and the launch itself.
#include "tvl1_internal.h"

namespace tvl1 {

// Instances per storage type (k_admm_persist_{f32,f16,bf16}.cu, compiled in parallel).
void *persist_kernel_f32(const Coefs &k);
void *persist_kernel_f16(const Coefs &k, bool flow32);
void *persist_kernel_bf16(const Coefs &k, bool flow32);

namespace {

void *kernel_for(const Coefs &k, int prec, int prec_flow) {
    if (prec == PREC_F32) return persist_kernel_f32(k);
    if (prec == PREC_F16) return persist_kernel_f16(k, prec_flow == PREC_F32);
    return persist_kernel_bf16(k, prec_flow == PREC_F32);
}

constexpr int THREADS = 128;  // admm_fused_warps() warps of 32 lanes

}  // namespace

int persist_capacity(const Coefs &k, int prec, int prec_flow) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kernel_for(k, prec, prec_flow), THREADS, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

cudaError_t launch_admm_persist(const PersistArgs &a, int prec, int prec_flow, cudaStream_t s) {
    if (a.nwarps < 1) return cudaSuccess;
    void *args[] = {(void *)&a};
    const unsigned blocks = (unsigned)((a.nwarps + THREADS / 32 - 1) / (THREADS / 32));
    return cudaLaunchKernel(kernel_for(a.k, prec, prec_flow), dim3(blocks), dim3(THREADS), args, 0, s);
}

}  // namespace tvl1
