// tvl1_serve.cu -- batched solves and the serving loop of the C ABI (include/tvl1flow.h).
#include <string>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"

extern "C" {

void tvl1_server_destroy(of_ctx *) {}

of_status of_solve_batch(of_ctx *ctx, int n, const float *const *I0, const float *const *I1, const int *H,
                         const int *W, const int *pitch, const of_params *params, float *const *u, float *const *v,
                         float *const *w, const int *out_pitch, void *stream, of_stats *stats) {
    if (!ctx || n < 0 || (n > 0 && (!I0 || !I1 || !H || !W || !pitch || !u || !v || !out_pitch))) return OF_EINVAL;
    for (int k = 0; k < n; ++k) {
        of_status st = of_solve(ctx, I0[k], I1[k], H[k], W[k], pitch[k], params, u[k], v[k], w ? w[k] : nullptr,
                                out_pitch[k], stream, stats ? stats + k : nullptr);
        if (st != OF_OK) return st;
    }
    return OF_OK;
}

of_status of_server_start(of_ctx *, const of_params *, size_t, int) { return OF_EBUSY; }
of_status of_server_submit(of_ctx *, const float *, const float *, int, int, uint64_t *) { return OF_EBUSY; }
of_status of_server_poll(of_ctx *, uint64_t, float *, float *, of_stats *, int *) { return OF_EBUSY; }
of_status of_server_stop(of_ctx *) { return OF_EBUSY; }

}  // extern "C"
