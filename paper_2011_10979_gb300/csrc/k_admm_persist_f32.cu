// k_admm_persist_f32.cu -- FP32 instances of the persistent ADMM engine (k_admm_persist.cuh).
#include "k_admm_persist.cuh"

namespace tvl1 {

void *persist_kernel_f32(const Coefs &k) { return persist::instance<float, float>(k); }

}  // namespace tvl1
