// k_admm_roll_bf16.cu -- BF16-storage instantiations of the row-streaming ADMM kernel
// (k_admm_roll.cuh): duals and linearisation data in BF16, multipliers in FP32 or BF16.
#include "k_admm_roll.cuh"

namespace tvl1 {

void roll_launch_bf16(const IterArgs &a, int ty, bool flow32, cudaStream_t s) {
    if (flow32) roll::launch_m<__nv_bfloat16, float>(a, ty, s);
    else roll::launch_m<__nv_bfloat16, __nv_bfloat16>(a, ty, s);
}

}  // namespace tvl1
