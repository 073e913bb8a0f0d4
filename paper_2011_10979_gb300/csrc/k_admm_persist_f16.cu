// k_admm_persist_f16.cu -- FP16-storage instances of the persistent ADMM engine
// (k_admm_persist.cuh): duals and data in FP16, multipliers in FP32 or FP16.
#include "k_admm_persist.cuh"

namespace tvl1 {

void *persist_kernel_f16(const Coefs &k, bool flow32) {
    return flow32 ? persist::instance<__half, float>(k) : persist::instance<__half, __half>(k);
}

}  // namespace tvl1
