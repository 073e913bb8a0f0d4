// k_admm_roll_f32.cu -- FP32 instantiations of the row-streaming ADMM kernel (k_admm_roll.cuh).
#include "k_admm_roll.cuh"

namespace tvl1 {

void roll_launch_f32(const IterArgs &a, int ty, cudaStream_t s) { roll::launch_m<float, float>(a, ty, s); }

}  // namespace tvl1
