/*
 * tvl1flow.h -- C ABI of the GB300 TV-L1 optical-flow library.
 *
 * The library solves the illumination-invariant isotropic TV-L1 optical-flow model
 *     min_{w,u,v} ||grad w||_1 + ||grad (u,v)||_1 + lambda ||Ix u + Iy v + beta w + It||_1
 * (Sun, Tai & Yuan, "Variational Image Motion Estimation by Accelerated Dual Optimization",
 * Sec. 1 eq. (l1:optical:flow) and Sec. 2.2 eq. (l1:finite)) with the paper's preconditioned
 * dual solvers -- rpADMMI / pADMM and rpADMMII (Sec. 3.1.1), Zach-pADMM (beta = 0, Sec.
 * 3.1.1) and pDR with red-black symmetric Gauss-Seidel preconditioning (Sec. 3.1.2) -- inside
 * a coarse-to-fine pyramid with bilinear warping (Sec. 4).  All arithmetic runs in CUDA kernels
 * for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point:
 *  - Images and fields are single-channel, row-major, H rows x W columns, with a row pitch
 *    `pitch` given in ELEMENTS (pitch >= W).  x runs along columns, y along rows.
 *  - Flow sign: I1(x + u, y + v) ~ I0(x, y); u is horizontal (+columns), v vertical (+rows).
 *  - Unless a name ends in `_host`, every array pointer is a DEVICE pointer owned by the caller.
 *    The library never frees or retains caller memory after a call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls are
 *    stream-ordered and return after enqueueing, except where a stats pointer is given or the
 *    name ends in `_host`: those synchronise the stream before returning.
 *  - Errors are returned as of_status, never by aborting; of_last_error() gives the message of
 *    the last non-OK status on the calling thread.
 *  - An of_ctx may be used by one host thread at a time.
 */
#ifndef TVL1FLOW_H
#define TVL1FLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct of_ctx of_ctx;

/* Largest image side the whole-solve entry points and the serving loop accept (H and W each); the
 * kernels' grids and the arena's offsets are sized for it. */
#define OF_MAX_SIDE 32768

typedef enum {
    OF_OK = 0,
    OF_EINVAL = 1,    /* invalid argument (sizes, pitches, parameters, NULL pointers) */
    OF_ENOMEM = 2,    /* the device arena would exceed the context's HBM budget, or cudaMalloc failed */
    OF_ECUDA = 3,     /* a CUDA runtime call failed (message names it) */
    OF_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    OF_ENUMERIC = 5,  /* non-finite residual or energy (NaN/Inf input or parameters); reported
                         by the calls that wait for the solve (a stats pointer given, or a
                         `_host` entry point); the other calls return after enqueueing */
    OF_EBUSY = 6      /* the serving loop is not running / queue full */
} of_status;

typedef enum {
    OF_PADMM_I = 0,   /* rpADMMI, Sec. 3.1.1 eq. (rpADMMI); r = 1 is pADMM; beta = 0 is Zach-pADMM */
    OF_PADMM_II = 1,  /* rpADMMII, Sec. 3.1.1 eq. (rpADMMII) */
    OF_PDR = 2,       /* pDR, Sec. 3.1.2 eq. (pDR) with SRBGS preconditioner */
    OF_CP = 3         /* ALG1, the comparison solver of Sec. 4: the primal-dual method of
                         Chambolle and Pock with constant steps cp_tau (dual), cp_sigma (primal) */
} of_method;

typedef enum { OF_PREC_FP32 = 0, OF_PREC_FP16 = 1, OF_PREC_BF16 = 2 } of_precision;

typedef enum {
    OF_ENGINE_FUSED = 0,    /* default: small levels (those the level-resident launch runs faster)
                               run all inner iterations of a warp in one level-resident launch of
                               a thread-block cluster; the others one fused streaming kernel per
                               inner iteration.  Both give bitwise the same flow. */
    OF_ENGINE_PLAIN = 1,    /* one kernel per operator, FP32 only: the plain reference GPU path */
    OF_ENGINE_STREAM = 2,   /* the fused streaming kernel on every level */
    OF_ENGINE_RESIDENT = 3, /* the level-resident launch on every level that fits one cluster's
                               shared memory, the streaming kernel on the others */
    OF_ENGINE_PERSISTENT = 4 /* ADMM methods: levels that the default engine does not run
                               level-resident run every inner iteration of a warp in one
                               persistent launch over all pairs of the level, whose warps
                               synchronise with their neighbours through device counters
                               (bounded waits: OF_ETIMEOUT if one runs out); pDR and ALG1 as
                               OF_ENGINE_FUSED.  Bitwise the same flow as the other fused
                               engines. */
} of_engine;

/* Solver parameters.  Defaults (of_default_params) are the paper's Sec. 4 settings. */
typedef struct {
    int method;          /* of_method */
    float lambda;        /* data weight lambda, |s| <= lambda (eq. ofc-dual)                  */
    float beta;          /* illumination weight beta (eq. l1:optical:flow); 0 = beta = 0 model  */
    float c;             /* ADMM penalty / step c (Sec. 4: 0.05)                               */
    float a;             /* y-block preconditioner a, 1/a <= 1/||grad grad^*|| (Prop. 3.1: 8)    */
    float a_tilde;       /* s-block preconditioner a~; <= 0 means ||M_s|| = max M_s per warp    */
    float r;             /* rpADMMI relaxation r in (0, (1+sqrt 5)/2) (Sec. 4: 1 or 1.618)       */
    float rho;           /* rpADMMII relaxation rho in (0, 2) (Sec. 4: 1.9)                     */
    float sigma, tau;    /* pDR step sizes (Sec. 4: 2 and 0.4)                                  */
    int gs_sweeps;       /* symmetric red-black Gauss-Seidel sweeps per pDR iteration (>= 1)    */
    float eta;           /* pyramid scale factor in (0, 1)                                      */
    int levels;          /* pyramid levels (1 = no pyramid), 1..16                              */
    int warps;           /* warps (re-linearisations) per level, >= 1                          */
    int iters;           /* inner iterations per warp, >= 0                                     */
    double tol;          /* > 0: a warp's inner loop stops once the residual < tol, tested
                            every 10 iterations; 0 = fixed schedule                            */
    int precision;       /* of_precision: storage of the iterated fields; arithmetic is FP32   */
    int fp32_last_warp;  /* 1: the finest level's last warp runs with FP32 storage             */
    int fp32_flow;       /* 1: with 16-bit storage, keep the flow and illumination fields
                            (w, u, v; pDR also its barred copies; ALG1 its barred copies
                            and its dual y, which moves by constant cp_tau steps) in FP32
                            and store only the other dual fields and the linearisation
                            data in 16 bits                                                  */
    int engine;          /* of_engine                                                           */
    int out_level;       /* stop after this pyramid level and return its flow (0 = finest)     */
    float cp_tau;        /* ALG1 dual step (Sec. 4: 0.1)                                        */
    float cp_sigma;      /* ALG1 primal step; Sec. 4's garbled rule read as 1 / (8 cp_tau) = 1.25 */
    int a_tilde_mode;    /* ADMM s-block preconditioner: 0 = one a~ per warp (a_tilde, or
                            ||M_s|| = max M_s, Prop. 3.1); 1 = the per-pixel diagonal
                            a~_ij = max(M_s(ij), 1e-12), which keeps c(diag(a~) - M_s) positive
                            semidefinite because M_s is diagonal (an extension, not in the paper) */
    int rows_per_warp;   /* ADMM methods: strip height of the fused streaming kernel (rows each
                            warp finishes per inner iteration; the strip is 29 columns wide):
                            0 = chosen per level from the level's size by the built-in rule;
                            1, 2, 8 or 32 = that height on every streamed level.
                            pDR with gs_sweeps > 1 and ALG1: block height of their per-iteration
                            kernels (blocks of 32 columns): 0 = 8; 4, 8 or 16 = that height
                            (pDR with one sweep runs one kernel of fixed 32 x 32 tiles per
                            iteration and ignores it).
                            -1 = autotuned: the first solve of a layout on a context times every
                            height on each level that runs those kernels (a few iterations of the
                            real launch on the arena, after a device synchronisation) and keeps
                            the fastest for that context.  The flow does not depend on it (the
                            per-pixel arithmetic is the same); only the grouping of the
                            residual's partial sums changes, so the residual (and a stopping
                            decision taken on it) can differ in the last FP32 digits.  Used by
                            of_solve and of_solve_batch; the step-level entry points and the
                            serving loop use the built-in choice.                             */
    int c_adapt_iters;   /* ADMM methods and pDR, opt-in (an extension, not in the paper): 0 =
                            the fixed steps of Sec. 4.  K > 0 (a multiple of 10): in the first
                            warp of every pyramid level, after each 10th of its first K inner
                            iterations, the steps are rebalanced.  ADMM: c, by residual balancing:
                            with r the constraint residual ||A s + B y|| and d the dual residual
                            of the preconditioned ADMM, c(B^*A ds - (a I - B^*B) dy,
                            (M_s - a~) ds) (ds, dy: the change of s and y over the iteration), c
                            is doubled when r > 10 d and halved when d > 10 r.  pDR (one
                            Gauss-Seidel sweep): sigma -> theta sigma, tau -> tau / theta with
                            sigma tau (so T and its preconditioner) unchanged; theta is doubled
                            when ||X^{k+1} - X^k|| / sigma > 10 ||ybar^{k+1} - ybar^k|| / tau and
                            halved in the opposite case.  After those K iterations the steps are
                            frozen for the rest of the level (its fixed-step convergence, Props.
                            3.1 and 3.2, applies from there on); the next finer level starts its
                            window from them.  The stopping test (tol) starts after the window.
                            Single pairs (of_solve, of_solve_host, n = 1) on the fused engines
                            only: OF_EINVAL for ALG1, pDR with more sweeps, the plain engine,
                            batches, the serving loop and the step-level entry points.          */
} of_params;

typedef struct {
    long long iters_run; /* inner iterations executed over the whole schedule                   */
    double residual;     /* last residual: ||A s + B y|| / sqrt(rows) (ADMM) or
                            ||X^{k+1} - X^k|| / sqrt(rows) (pDR, ALG1), on the output level    */
    double energy;       /* primal energy eq. (l1:finite) at the output level's last linearisation */
    double dual_value;   /* <It, s> (eq. dual:l1:flow:cons); NaN for pDR and ALG1               */
    float ms;            /* device time of the solve in milliseconds                            */
    float c;             /* the step at the end of the solve: ADMM c, pDR sigma (params->c,
                            params->sigma unless c_adapt_iters)                                   */
} of_stats;

/* Fills p with the paper's Sec. 4 settings: pADMM (r = 1), c = 0.05, a = 8, a~ = max M_s,
 * rho = 1.9, sigma = 2, tau = 0.4, beta = 0.05, one SRBGS sweep; lambda = 0.05; eta = 0.5,
 * 3 levels, 5 warps, 50 iterations; FP32, fused engine; with 16-bit storage, the last warp
 * and the flow fields in FP32; the built-in strip heights (rows_per_warp = 0); fixed c
 * (c_adapt_iters = 0). */
void of_default_params(of_params *p);

/* Creates a context on CUDA device `device`.  The context owns one device arena that grows on
 * demand up to `hbm_budget_bytes` (0 = 80% of the device's memory).  OF_EINVAL for a bad
 * device, OF_ECUDA if the device cannot be used. */
of_status of_create(of_ctx **out, int device, size_t hbm_budget_bytes);

/* Releases the context, its arena and its cached CUDA graphs.  NULL is a no-op. */
void of_destroy(of_ctx *ctx);

/* Message of the last non-OK status returned on this thread (never NULL). */
const char *of_last_error(of_ctx *ctx);

/* Bytes of device arena a solve of an H x W pair with these parameters needs. */
size_t of_arena_bytes(int H, int W, const of_params *params);

/* Number of kernel launches one of_solve of an H x W pair with these parameters makes (the
 * kernel nodes of its CUDA graph; captures the graph if it is not cached yet).  Returns -1 on
 * error (message in of_last_error). */
long long of_solve_kernel_count(of_ctx *ctx, int H, int W, const of_params *params);

/* Strip heights of the fused streaming ADMM kernel (pDR, ALG1: block heights of their
 * per-iteration kernels) in a solve of n pairs of sizes H[k] x W[k] (n = 1: of_solve; n > 1:
 * of_solve_batch) with these parameters: rows[l] for l in [0, params->levels) is the height used on
 * pyramid level l, 0 where no pair of that level runs on those kernels (a level-resident or
 * persistent launch, pDR's one-launch tile kernel, the plain engine, or a level below out_level).  With params->rows_per_warp = -1 it runs the autotuner first if this layout is not
 * tuned on the context yet (allocating the arena and launching kernels; the device is
 * synchronised).  `rows` is caller-owned host memory of params->levels ints.  OF_EINVAL for bad
 * arguments, OF_ENOMEM / OF_ECUDA as for of_solve_batch. */
of_status of_rows_per_warp(of_ctx *ctx, int n, const int *H, const int *W, const of_params *params, int *rows);

/* Capacity of the level-resident engine on the current CUDA device: *cluster_ctas receives the
 * CTAs per thread-block cluster it launches (16, or 8 where the device cannot schedule 16 CTAs
 * with a full band of shared memory, or 0 when it can schedule neither, which turns the engine
 * off: every level then runs on the streaming kernels), *max_active how many such clusters the
 * device runs at once (cudaOccupancyMaxActiveClusters, which follows the GPC layout and can be
 * fewer than SMs / cluster_ctas).  A batch runs a level's small pairs on the resident engine only
 * when they fit in one such wave of clusters; otherwise they join the streaming work-list.
 * Queried once per process.  OF_EINVAL for NULL pointers. */
of_status of_resident_clusters(int *cluster_ctas, int *max_active);

/* Self-test of the bounded device-side waits of the persistent engine (OF_ENGINE_PERSISTENT):
 * runs `iters` pADMM iterations of that engine on zero-filled fields of one H x W level (it
 * allocates and frees its own device buffers, on the current device and the legacy stream),
 * with segment `withhold` of the launch never publishing its progress (-1: none) and every wait
 * bounded by wait_ms milliseconds.  *timed_out receives 1 when a wait ran out -- the launch then
 * ended early with its error flag set, and the device stays usable -- else 0.  *segments
 * (optional) receives the launch's segment count.  OF_EINVAL for bad arguments, OF_ECUDA when a
 * CUDA call fails. */
of_status of_persistent_selftest(int H, int W, int iters, int withhold, double wait_ms, int *timed_out,
                                 int *segments);

/* Bandwidth of the L2 cache for a working set of `bytes` (half read, half written, FP32 words):
 * one kernel streams the set `passes` times, loading with the L2-only cache hint, after one warm
 * launch; *gbps receives (read + written bytes) / time.  It is the roofline denominator of the
 * pyramid levels whose state stays in L2 between inner iterations (a working set under the
 * 129 MB L2).  Allocates and frees its buffers; synchronises the device.  OF_EINVAL for
 * bytes < 4096 or passes < 1, OF_ECUDA when a CUDA call fails. */
of_status of_l2_bandwidth(size_t bytes, int passes, double *gbps);

/* Solves one pair (whole schedule: pyramid, levels, warps, inner iterations; Sec. 3-4).
 * I0, I1: H x W FP32 images (device, pitch `pitch`), 1 <= H, W <= OF_MAX_SIDE (else OF_EINVAL).
 * u, v (and w unless NULL): outputs of size
 * H_l x W_l at level params->out_level, FP32, pitch `out_pitch` (>= W_l).  stats: optional; if
 * given the call synchronises `stream` and fills it.  The first call for a new (H, W, params)
 * captures a CUDA graph that later calls replay. */
of_status of_solve(of_ctx *ctx, const float *I0, const float *I1, int H, int W, int pitch,
                   const of_params *params, float *u, float *v, float *w, int out_pitch,
                   void *stream, of_stats *stats);

/* As of_solve, but I0, I1, u, v, w are HOST pointers (dense, pitch = W resp. W_l); the
 * host<->device copies run on `stream` inside the call, which returns after they finish. */
of_status of_solve_host(of_ctx *ctx, const float *I0, const float *I1, int H, int W,
                        const of_params *params, float *u, float *v, float *w,
                        void *stream, of_stats *stats);

/* Solves n independent pairs of possibly different sizes with one set of parameters.  Arrays
 * of n device pointers / sizes; pitches in elements; w may be NULL (or entries NULL).  Pairs
 * are processed together per pyramid level so that every launch covers all pairs.  stats: NULL
 * or n entries (then the call synchronises).  Results equal n separate of_solve calls. */
of_status of_solve_batch(of_ctx *ctx, int n, const float *const *I0, const float *const *I1,
                         const int *H, const int *W, const int *pitch, const of_params *params,
                         float *const *u, float *const *v, float *const *w, const int *out_pitch,
                         void *stream, of_stats *stats);

/* ---------------------------------------------------------------------------------------
 * Step-level entry points: one row of the solver each, on caller-provided FP32 planes.  They
 * exist so that each step can be checked on its own; of_solve chains the same kernels.
 * All planes: device, H x W, pitch `pitch` elements unless stated.
 * --------------------------------------------------------------------------------------- */

/* Pyramid step (Sec. 4, reading: Gaussian pre-smoothing with sigma_g = 0.6 sqrt(eta^-2 - 1),
 * radius ceil(3 sigma_g), half-sample symmetric border, then bilinear sampling at pixel
 * centres).  fine: Hf x Wf (pitch pf) -> coarse: Hc x Wc (pitch pc).  scratch: >= Hf*pf floats. */
of_status of_pyr_down(const float *fine, int Hf, int Wf, int pf, float *coarse, int Hc, int Wc,
                      int pc, float eta, float *scratch, void *stream);

/* Level transfer (Sec. 4 reading): bilinear upsampling of a field from Hc x Wc (pitch pc) to
 * Hf x Wf (pitch pf), multiplied by `scale` (W_f/W_c for u, H_f/H_c for v, 1 for w). */
of_status of_upsample(const float *coarse, int Hc, int Wc, int pc, float *fine, int Hf, int Wf,
                      int pf, float scale, void *stream);

/* Derivative images of I (Sec. 1 optical-flow constraint; reading: central differences with
 * clamped indices). */
of_status of_derivatives(const float *I, int H, int W, int pitch, float *Ix, float *Iy, void *stream);

/* Warping and linearisation around d0 = (u0, v0): Ix, Iy = I1x, I1y sampled bilinearly at
 * (x + u0, y + v0) clamped to the image, It = I1(x + d0) - I0 - Ix u0 - Iy v0, computed in FP64
 * and rounded once to the stored type (Sec. 1: rho(d) = grad I^T d + I_t; reading: its
 * linearisation around d0 inside Sec. 4's coarse-to-fine warping, bilinear sampling).  ms_max: device
 * pointer to one float that receives max(beta^2 + Ix^2 + Iy^2) (it must hold 0 or a smaller
 * non-negative value on entry; the kernel raises it). */
of_status of_warp_linearise(const float *I0, const float *I1, const float *I1x, const float *I1y,
                            const float *u0, const float *v0, int H, int W, int pitch, float beta,
                            float *Ix, float *Iy, float *It, float *ms_max, void *stream);

/* Pointers to the iterated fields of one pair at one level (FP32 planes, shared pitch).
 * ADMM: multipliers (w, u, v) and duals p = (p1, p2), q1 = (q11, q12), q2 = (q21, q22), s.
 * pDR: X = (w, u, v), Xbar = (wb, ub, vb), ybar = (p, q); s unused.
 * Components ending in 1 are x-components.  w, p1, p2, wb may be NULL when beta = 0. */
typedef struct {
    float *w, *u, *v, *p1, *p2, *q11, *q12, *q21, *q22, *s, *wb, *ub, *vb;
} of_fields;

/* `iters` inner iterations of rpADMMI / rpADMMII (params->method 0 or 1) at a fixed
 * linearisation (Sec. 3.1.1), in place on `f`.  a_tilde > 0 is used as given.  The stopping
 * rule params->tol applies.  res2: optional host pointer, receives ||A s + B y||^2 after the
 * last iteration (synchronises).  Uses params->engine: PLAIN, or the fused streaming kernel
 * (FUSED and STREAM alike: this call has no level-resident form); the fused kernel
 * needs `scratch`, a device buffer of >= of_fields_bytes(H, pitch) bytes (NULL for PLAIN). */
of_status of_admm_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H,
                          int W, int pitch, float a_tilde, const of_params *params, int iters,
                          void *scratch, double *res2, void *stream);

/* Allocation-free form of of_admm_iterate with the fused engine.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory at all -- code running under a
 * host allocator they do not control, inside a region where cudaMalloc would synchronise or is
 * forbidden, or embedded in a runtime that owns every device byte.  Instead of a caller-provided
 * `scratch` it uses one library-owned static device array of 32 MiB (every GPU that loads the
 * library holds it until the process exits), so fields with of_fields_bytes(H, pitch) > 32 MiB
 * are rejected with OF_EINVAL (640 x 480 FP32 fits).  The caller still passes every field and
 * the linearisation data.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream capture.  The
 * cached address belongs to the device's primary context (the CUDA runtime's): a cudaDeviceReset
 * after the first call, or a different current context, is not supported.  It calls
 * no cudaMalloc/cudaFree.  All calls on a device share its one array, which keeps the last call's
 * contents; each call clears what must start at zero, but two calls that overlap on the same GPU
 * (e.g. issued on different streams) race on it: serialise them.  Arguments, results and errors
 * are those of
 * of_admm_iterate with params->engine forced to OF_ENGINE_FUSED. */
of_status of_admm_iterate_noalloc(of_fields f, const float *Ix, const float *Iy, const float *It, int H,
                                  int W, int pitch, float a_tilde, const of_params *params, int iters,
                                  double *res2, void *stream);

/* `iters` pDR iterations (Sec. 3.1.2) in place on `f`; res2: optional host pointer receiving
 * ||X^{k+1} - X^k||^2 of the last iteration.  scratch as for of_admm_iterate. */
of_status of_pdr_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H,
                         int W, int pitch, const of_params *params, int iters, void *scratch,
                         double *res2, void *stream);

/* `iters` ALG1 iterations (Sec. 4; params->method OF_CP) in place on `f`: w u v hold X, wb ub
 * vb the extrapolated point Xbar, p and q the dual y (s unused).  res2: optional host pointer
 * receiving ||X^{k+1} - X^k||^2 of the last iteration.  scratch as for of_admm_iterate (the
 * kernel reads one plane set and writes the other). */
of_status of_cp_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H,
                        int W, int pitch, const of_params *params, int iters, void *scratch,
                        double *res2, void *stream);

/* Scratch bytes the fused engines of the calls above need for an H-row plane set. */
size_t of_fields_bytes(int H, int pitch);

/* Primal energy eq. (l1:finite) and dual value <It, s> (eq. dual:l1:flow:cons) of FP32 fields,
 * accumulated in FP64 on the device; results to host pointers (synchronises).  w and s may be
 * NULL (then beta*w and the dual value are skipped / NaN). */
of_status of_energy(const float *w, const float *u, const float *v, const float *s,
                    const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                    float beta, float lambda, double *energy, double *dual_value, void *stream);

/* ---------------------------------------------------------------------------------------
 * Serving loop (continuous batching of requests of different sizes; no counterpart in the
 * paper, which solves one pair at a time).
 * --------------------------------------------------------------------------------------- */

/* Starts the serving loop on the context with fixed parameters.  Requests are admitted while
 * their arena bytes fit in `hbm_budget` (0 = the context budget) and at most `max_active` are
 * on the device at once.  The loop runs on its own host thread and CUDA stream. */
of_status of_server_start(of_ctx *ctx, const of_params *params, size_t hbm_budget, int max_active);

/* Queues one request; I0, I1 are HOST float images (dense, pitch W) copied before return.
 * *req_id receives the request id. */
of_status of_server_submit(of_ctx *ctx, const float *I0, const float *I1, int H, int W, uint64_t *req_id);

/* Polls a request.  *done = 1 when finished; then u, v (host, H x W dense, may be NULL) are
 * filled, stats filled (may be NULL; ms = submit-to-finish latency), and the request retired. */
of_status of_server_poll(of_ctx *ctx, uint64_t req_id, float *u, float *v, of_stats *stats, int *done);

/* Stops the loop after the requests in flight finish; unfinished queued requests are dropped. */
of_status of_server_stop(of_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TVL1FLOW_H */
