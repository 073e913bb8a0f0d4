// tvl1_noalloc.cu -- allocation-free form of the fused ADMM iteration entry point.
//
// Some callers cannot allocate device memory: they run under an allocator they do not control,
// inside regions where cudaMalloc would synchronise the device or is not allowed, or inside a
// runtime that owns every device byte.  For them of_admm_iterate_noalloc takes its scratch (the
// second ping-pong state buffer, FP64 partial sums and the stop flag) from one static device
// array defined here instead of from a caller-provided buffer.  The array is part of the
// library's device image, so every GPU that loads the library holds its 32 MiB until the
// process exits.
#include <mutex>
#include <string>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code `g_noalloc_scratch` names a host-side stand-in, not device memory: its device
// address is looked up once per device (with that device current) and cached here.  The cache
// assumes the device's primary context, which the CUDA runtime uses, and no cudaDeviceReset
// between calls (a reset unloads the module and so the array).
std::mutex g_mu;
void *g_scratch_ptr[MAX_DEVICES] = {};

}  // namespace

extern "C" of_status of_admm_iterate_noalloc(of_fields f, const float *Ix, const float *Iy, const float *It, int H,
                                             int W, int pitch, float a_tilde, const of_params *params, int iters,
                                             double *res2, void *stream) {
    if (!params) {
        tvl1_set_error("of_admm_iterate_noalloc: params is NULL");
        return OF_EINVAL;
    }
    const size_t need = of_fields_bytes(H, pitch);
    if (need == 0 || need > NOALLOC_SCRATCH_BYTES) {
        tvl1_set_error(("of_admm_iterate_noalloc: fields of " + std::to_string(H) + " rows x pitch " +
                        std::to_string(pitch) + " need " + std::to_string(need) +
                        " bytes of scratch, more than the static 32 MiB (use of_admm_iterate)")
                           .c_str());
        return OF_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        tvl1_set_error(("of_admm_iterate_noalloc: cudaGetDevice: " + std::string(cudaGetErrorString(e))).c_str());
        return OF_ECUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        tvl1_set_error(("of_admm_iterate_noalloc: device " + std::to_string(dev) + " is beyond the " +
                        std::to_string(MAX_DEVICES) + " devices this entry point keeps an address for")
                           .c_str());
        return OF_EINVAL;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                tvl1_set_error(("of_admm_iterate_noalloc: cudaGetSymbolAddress: " +
                                std::string(cudaGetErrorString(e))).c_str());
                return OF_ECUDA;
            }
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    of_params p = *params;
    p.engine = OF_ENGINE_FUSED;
    // of_admm_iterate clears the stop flag, counters and zero-routed planes it uses, then runs
    // the fused kernel with `scratch` as its second state buffer.
    return of_admm_iterate(f, Ix, Iy, It, H, W, pitch, a_tilde, &p, iters, scratch, res2, stream);
}
