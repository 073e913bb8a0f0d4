// k_admm_persist_bf16.cu -- BF16-storage instances of the persistent ADMM engine
// (k_admm_persist.cuh): duals and data in BF16, multipliers in FP32 or BF16.
#include "k_admm_persist.cuh"

namespace tvl1 {

void *persist_kernel_bf16(const Coefs &k, bool flow32) {
    return flow32 ? persist::instance<__nv_bfloat16, float>(k) : persist::instance<__nv_bfloat16, __nv_bfloat16>(k);
}

}  // namespace tvl1
