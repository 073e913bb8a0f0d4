// tvl1_internal.h -- internal declarations shared by the kernel translation units and the host
// runtime of the GB300 TV-L1 library.  Not part of the public C ABI (include/tvl1flow.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tvl1 {

// Storage precision of the iterated fields and linearisation data; arithmetic is always FP32.
enum Prec { PREC_F32 = 0, PREC_F16 = 1, PREC_BF16 = 2 };

inline size_t prec_bytes(int prec) { return prec == PREC_F32 ? 4 : 2; }

// Field indices of a state buffer (13 planes).  ADMM: multipliers (w, u, v) and duals
// p = (p1, p2), q1 = (q11, q12), q2 = (q21, q22), s.  pDR: X = (w, u, v), ybar = (p, q),
// Xbar = (wb, ub, vb).
enum Field { F_W = 0, F_U, F_V, F_P1, F_P2, F_Q11, F_Q12, F_Q21, F_Q22, F_S, F_WB, F_UB, F_VB, NFIELDS };

// One pair at one pyramid level: planes are H x W with row pitch `pitch` elements.
struct Geom {
    int H, W, pitch;
};

// The 13 planes of one state buffer (element type given by the precision).
struct Fields {
    void *f[NFIELDS];
};

struct Coefs {
    float lambda, beta, c, a, r, rho, sigma, tau;
    float a_tilde_fixed;  // > 0: used as a~; otherwise a~ = max(ms_max, 1e-12)
    int method;           // 0 rpADMMI, 1 rpADMMII, 2 pDR
    int gs_sweeps;
};

// Per-iteration launch arguments of the ADMM / pDR engines.
struct IterArgs {
    Geom g;
    Coefs k;
    Fields in, out;                // fused engine: ping-pong buffers; plain engine: in == out
    const void *Ix, *Iy, *It;      // linearisation data (same precision as the fields)
    const float *ms_max;           // device max M_s of the current warp
    double *partials;              // per-block residual partial sums, or nullptr
    const int *done;               // early-exit flag of the current warp, or nullptr
    float *tmp;                    // FP32 scratch planes (H x pitch each) for engines that need them
};

// ---------------------------------------------------------------- pyramid / warp (k_pyramid.cu)
constexpr int MAX_GAUSS_R = 16;
struct GaussTaps {
    float w[2 * MAX_GAUSS_R + 1];
    int R;
};
GaussTaps gauss_taps(float eta);
void launch_pyr_down(const float *fine, Geom gf, float *coarse, Geom gc, const GaussTaps &taps,
                     float *scratch, cudaStream_t s);
void launch_upsample(const void *coarse, Geom gc, void *fine, Geom gf, float scale, int prec, cudaStream_t s);
void launch_upsample_f32(const float *coarse, Geom gc, float *fine, Geom gf, float scale, cudaStream_t s);
void launch_derivatives(const float *I, Geom g, float *Ix, float *Iy, cudaStream_t s);
// u0, v0 and the outputs Ix, Iy, It in precision `prec`; ms_max raised with atomicMax.
void launch_warp(const float *I0, const float *I1, const float *I1x, const float *I1y, const void *u0,
                 const void *v0, Geom g, float beta, void *Ix, void *Iy, void *It, float *ms_max,
                 int prec, cudaStream_t s);
// Element-wise precision conversion of `nplanes` planes (same geometry).
void launch_convert(const void *const *src, int src_prec, void *const *dst, int dst_prec, int nplanes,
                    Geom g, cudaStream_t s);
void launch_fill(void *const *dst, int prec, int nplanes, Geom g, float value, cudaStream_t s);
void launch_copy_planes(const void *const *src, void *const *dst, int nplanes, Geom g, int prec, cudaStream_t s);

// ---------------------------------------------------------------- ADMM (k_admm.cu)
// Fused engine: one kernel per iteration, reads args.in, writes args.out.
int admm_fused_blocks(Geom g);
void launch_admm_fused(const IterArgs &a, int prec, cudaStream_t s);
// Plain engine (FP32): one kernel per operator, in place on args.in; args.tmp: 3 FP32 planes.
int admm_plain_blocks(Geom g);
void launch_admm_plain(const IterArgs &a, cudaStream_t s);
// ||A s + B y||^2 partials of a state (for stats), per block.
void launch_admm_residual(const Fields &f, const void *Ix, const void *Iy, Geom g, float beta, int prec,
                          double *partials, cudaStream_t s);

// ---------------------------------------------------------------- pDR (k_pdr.cu)
// Both pDR engines work in place on args.in; args.tmp: 6 FP32 planes (b for w, u, v and X^k).
int pdr_fused_blocks(Geom g);
void launch_pdr_fused(const IterArgs &a, int prec, cudaStream_t s);
int pdr_plain_blocks(Geom g);
void launch_pdr_plain(const IterArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- reductions (k_reduce.cu)
// Sums `n` partials in a fixed order into out[0]; if tol > 0 and the normalised residual
// sqrt(sum / rows) < tol, sets *done = 1.  iters_counter (nullable) += add_iters while not done.
void launch_reduce_check(const double *partials, int n, double *out, double rows, double tol, int *done,
                         long long *iters_counter, int add_iters, cudaStream_t s);
int energy_blocks(Geom g);
void launch_energy(const Fields &f, const void *Ix, const void *Iy, const void *It, Geom g, float beta,
                   float lambda, int prec, double *partials_e, double *partials_d, cudaStream_t s);
void launch_sum(const double *partials, int n, double *out, cudaStream_t s);
// Adds `n` to *counter unless *done is set.
void launch_count_iters(long long *counter, const int *done, int n, cudaStream_t s);
// Ping-pong parity repair: copies every non-NULL plane of `from` to `to` when the stop flag
// state ((done && *done) ? 1 : 0) equals `want_done`.
void launch_parity_fix(const Fields &from, const Fields &to, Geom g, int prec, const int *done, int want_done,
                       cudaStream_t s);

}  // namespace tvl1

// ---------------------------------------------------------------- runtime hooks (tvl1_api.cu)
struct of_ctx;
// Enqueues one solve on `s` without synchronising: host->device copy of I0/I1 (host pointers,
// dense, pinned for asynchronous copies), the cached graph of the schedule, device->host copy of
// u/v (dense, level params->out_level).  Validates and grows the context arena first.
int tvl1_solve_async(of_ctx *ctx, const float *I0, const float *I1, int H, int W, const void *params,
                     float *u, float *v, cudaStream_t s);
// Device bytes the context currently holds (arena).
size_t tvl1_ctx_bytes(of_ctx *ctx);
// Sets the thread-local error message returned by of_last_error.
void tvl1_set_error(const char *msg);
