// k_admm_roll_f16.cu -- FP16-storage instantiations of the row-streaming ADMM kernel
// (k_admm_roll.cuh): duals and linearisation data in FP16, multipliers in FP32 or FP16.
#include "k_admm_roll.cuh"

namespace tvl1 {

void roll_launch_f16(const IterArgs &a, int ty, bool flow32, cudaStream_t s) {
    if (flow32) roll::launch_m<__half, float>(a, ty, s);
    else roll::launch_m<__half, __half>(a, ty, s);
}

}  // namespace tvl1
