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
    float cp_tau, cp_sigma;  // ALG1 dual and primal steps
    int a_tilde_mode;     // 0: a~ per warp; 1: per-pixel a~_ij = max(M_s(ij), 1e-12)
    int method;           // 0 rpADMMI, 1 rpADMMII, 2 pDR, 3 ALG1
    int gs_sweeps;
    int c_dev;            // 1: c is the adapted value the solve keeps on the device, read at
                          // ms_max[-1] (Misc::c_cur); 0: c above
};

// One pair at one level, for the batched (work-list) form of the fused engines: both ping-pong
// state buffers, the linearisation data and the pair's device scalars.
struct __align__(16) PairIter {
    Geom g;  // read on the device as one 16-byte load (H, W, pitch, padding)
    int pad_;
    Fields buf[2];
    const void *Ix, *Iy, *It;
    const float *ms_max;
    const int *done;
    float *tmp;  // the pair's FP32 scratch planes (pDR engine)
};

// Device scalars of one pair in a batch, for the batched reductions: the partial sums of the
// pair are partials[part_begin, part_end); rows normalises the residual.
struct PairScalars {
    double *res_check, *res_final;
    int *done;
    long long *iters;
    int part_begin, part_end;
    double rows;
    int resident, pad_;  // resident: this pair's level runs on the level-resident engine
    int *timeout;        // set when a bounded device-side wait of the pair's launch ran out
};

// One work-list entry of a batched launch: pair index, tile column, tile row.
struct TileRef {
    int pair, tx, ty, pad;
};

// Per-iteration launch arguments of the ADMM / pDR engines.
struct IterArgs {
    Geom g{};
    Coefs k{};
    Fields in{}, out{};            // fused engine: ping-pong buffers; plain engine: in == out
    const void *Ix = nullptr, *Iy = nullptr, *It = nullptr;  // linearisation data (field precision)
    const float *ms_max = nullptr; // device max M_s of the current warp
    double *partials = nullptr;    // per-block residual partial sums, or nullptr
    const int *done = nullptr;     // early-exit flag of the current warp, or nullptr
    float *tmp = nullptr;          // FP32 scratch planes (H x pitch each) for engines that need them
    // batched form (fused ADMM engine): when `tiles` is set, block b works on tiles[b] of pair
    // pairs[tiles[b].pair], reads buf[parity] and writes buf[parity ^ 1]; g/in/out/Ix/Iy/It/
    // ms_max/done above are ignored.  tile_h is the tile height the work-list was built for; in
    // the single-pair form a positive tile_h sets the strip height (0: the built-in rule).
    const PairIter *pairs = nullptr;
    const TileRef *tiles = nullptr;
    int ntiles = 0, parity = 0, tile_h = 0;
    // ALG1 batched form: slice z of the grid works on pair plist[z] (the pairs of the level not on
    // the level-resident engine); its partials start at plist[z] * cp_blocks(g)
    const int *plist = nullptr;
    // pDR, gs_sweeps = 1: the one-launch tile kernel, reading `in` and writing `out` (batched:
    // buf[parity] -> buf[parity ^ 1]); 0: the per-kernel engine, in place in `in`
    int pdr_tile = 0;
};

// Geometry of the fused ADMM engine: each warp owns a strip of admm_fused_strip_w() output
// columns and TY rows (TY = 1, 2, 8 or 32, chosen per level by admm_fused_tile_h); a block stacks
// admm_fused_warps() strips vertically.  A work-list entry (pair, tx, ty) is the block covering
// columns [tx * strip_w, ...) and rows [ty * warps * TY, ...).
// The built-in rule; storage16: the duals are stored in 16 bits.  The FP32 rule never takes a
// greater height than the 16-bit one, so admm_fused_blocks(g) bounds the blocks of both.
int admm_fused_tile_h(Geom g, bool storage16 = false);
int admm_fused_rows_per_warp(long strip_rows, bool storage16 = false);   // strip_rows: sum over pairs of strips x rows
int admm_fused_strip_w();
int admm_fused_warps();

// Level-resident engine of the ADMM methods, pDR and ALG1 (k_resident.cu): one thread-block cluster per pair keeps
// a whole level in shared memory and runs all inner iterations of one warp in one launch, with
// the stopping test, the iteration count, res_check / res_final and the done flag handled inside
// (the scalars of PairScalars).  Reads the state from `in` (buf[parity_in]) and writes the final
// state to `out` (buf[parity_out]); in may equal out.
struct ResArgs {
    Coefs k{};
    // single pair (pairs == nullptr)
    Geom g{};
    Fields in{}, out{};
    const void *Ix = nullptr, *Iy = nullptr, *It = nullptr;
    const float *ms_max = nullptr;
    PairScalars sc{};
    // batched: cluster c works on pair list[c] of pairs[] with the scalars scal[list[c]]
    const PairIter *pairs = nullptr;
    const PairScalars *scal = nullptr;
    const int *list = nullptr;
    int parity_in = 0, parity_out = 0;
    int iters = 0, check = 0, final_res = 0;
    double tol = 0.0;
};
// Persistent engine of the ADMM methods (k_admm_persist.cuh): one launch per warp of a level runs
// every inner iteration.  A segment is strip sx (admm_fused_strip_w() output columns) by row band
// t of m (rows [t H / m, (t + 1) H / m)) of pair `pair`; a pair's segments are numbered
// t * S + sx from its first one, S = its strip count, and every band has at least two rows
// unless m = 1.
struct __align__(16) PSeg {
    int pair, sx, t, m;
};
struct PersistArgs {
    Coefs k{};
    const PairIter *pairs = nullptr;    // per pair: geometry, both state buffers, data, a~, stop flag
    const PairScalars *scal = nullptr;  // per pair: part_begin/part_end = its segment range
    const PSeg *segs = nullptr;
    const int *woff = nullptr, *wseg = nullptr;  // warp w holds segments wseg[woff[w] .. woff[w + 1])
    int nwarps = 0;
    unsigned *flags = nullptr;          // per segment: iterations finished in this launch (zeroed before)
    unsigned *pbar = nullptr;           // per pair: stopping-test arrivals in this launch (zeroed before)
    double *partials = nullptr;         // per segment: FP64 residual partial
    int parity = 0, iters = 0, check = 0, final_res = 0;
    double tol = 0.0;
    long long wait_ns = 2000000000LL;   // bound of every device-side wait
    int withhold = -1;                  // self-test: this segment never publishes its counter
};
// Co-resident blocks (of admm_fused_warps() warps) of the persistent instance for these storage
// types and method, over the whole device.
int persist_capacity(const Coefs &k, int prec, int prec_flow);
cudaError_t launch_admm_persist(const PersistArgs &a, int prec, int prec_flow, cudaStream_t s);

int admm_resident_cluster();           // CTAs per cluster: 16 where the device schedules it, else 8, else 0 (off)
int admm_resident_max_clusters();      // such clusters the device runs at once (cudaOccupancyMaxActiveClusters)
// dynamic shared memory of one CTA for this level in a cluster of nc CTAs (0: the largest cluster)
size_t admm_resident_smem(Geom g, int method, int nc);
bool admm_resident_fits(Geom g, int method);    // whether a level of this geometry fits one cluster
int admm_resident_nc(Geom g, int method);       // the cluster size a level of this geometry runs with
bool admm_resident_preferred(Geom g, int method);  // whether the resident launch is the faster engine
// nclusters clusters of nc CTAs (one per pair), each with smem bytes of dynamic shared memory
cudaError_t launch_admm_resident(const ResArgs &a, int nclusters, int nc, size_t smem, int prec, int prec_flow,
                                 cudaStream_t s);

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
// u0, v0 in precision `prec_flow`, the outputs Ix, Iy, It in `prec`; ms_max raised with atomicMax.
void launch_warp(const float *I0, const float *I1, const float *I1x, const float *I1y, const void *u0,
                 const void *v0, Geom g, float beta, void *Ix, void *Iy, void *It, float *ms_max,
                 int prec, int prec_flow, cudaStream_t s);
// Element-wise precision conversion of `nplanes` planes (same geometry).
void launch_convert(const void *const *src, int src_prec, void *const *dst, int dst_prec, int nplanes,
                    Geom g, cudaStream_t s);
void launch_fill(void *const *dst, int prec, int nplanes, Geom g, float value, cudaStream_t s);
void launch_copy_planes(const void *const *src, void *const *dst, int nplanes, Geom g, int prec, cudaStream_t s);

// ---------------------------------------------------------------- ADMM (k_admm.cu)
// Fused engine: one kernel per iteration, reads args.in, writes args.out.  The multipliers
// (w, u, v) are stored in `prec_flow`, every other field and the linearisation data in `prec`.
// Blocks of one single-pair launch with strip height ty (0: the built-in rule for g); with
// ty = 1 the most any height launches.
int admm_fused_blocks(Geom g, int ty = 0);
void launch_admm_fused(const IterArgs &a, int prec, int prec_flow, cudaStream_t s);
// Plain engine (FP32): one kernel per operator, in place on args.in; args.tmp: 3 FP32 planes.
int admm_plain_blocks(Geom g);
void launch_admm_plain(const IterArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- pDR (k_pdr.cu)
// Both pDR engines work in place on args.in; args.tmp: 6 FP32 planes (b for w, u, v and X^k).
// Batched form (args.pairs set, args.ntiles = number of pairs, args.g = the largest pair's
// geometry): blockIdx.z selects the pair, its planes are pairs[z].buf[0] and pairs[z].tmp, and
// its partials occupy pdr_plain_blocks(args.g) slots starting at z * pdr_plain_blocks(args.g).
int pdr_fused_blocks(Geom g);
// Blocks of the pDR and ALG1 per-iteration kernels: 32 columns by tile_h rows (4, 8 or 16; any
// other value means 8).  PARTIAL_ROWS_MIN is the smallest height, which launches the most blocks.
constexpr int PARTIAL_ROWS_MIN = 4;
// X and Xbar (w u v wb ub vb) in `prec_flow`, ybar and the data in `prec`.
void launch_pdr_fused(const IterArgs &a, int prec, int prec_flow, cudaStream_t s);
int pdr_plain_blocks(Geom g, int tile_h = 8);
// Blocks of the one-launch pDR tile kernel (32 x 32 output pixels each) on geometry g.
int pdr_tile_blocks(Geom g);
void launch_pdr_plain(const IterArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- ALG1 (k_cp.cu)
// One fused kernel per iteration, reads args.in and writes args.out (ping-pong).  Batched form
// as the pDR engines (blockIdx.z = pair, args.g = the largest geometry, parity selects buffers).
// For both, args.tile_h is the block height (see pdr_plain_blocks).
int cp_blocks(Geom g, int tile_h = 8);
void launch_cp(const IterArgs &a, int prec, int prec_flow, cudaStream_t s);

// ---------------------------------------------------------------- reductions (k_reduce.cu)
// Sums `n` partials in a fixed order into out[0]; if tol > 0 and the normalised residual
// sqrt(sum / rows) < tol, sets *done = 1.  iters_counter (nullable) += add_iters while not done.
void launch_reduce_check(const double *partials, int n, double *out, double rows, double tol, int *done,
                         long long *iters_counter, int add_iters, cudaStream_t s);
int energy_blocks(Geom g);
void launch_energy(const Fields &f, const void *Ix, const void *Iy, const void *It, Geom g, float beta,
                   float lambda, int prec, int prec_flow, double *partials_e, double *partials_d, cudaStream_t s);
void launch_sum(const double *partials, int n, double *out, cudaStream_t s);
// Adds `n` to *counter unless *done is set.
void launch_count_iters(long long *counter, const int *done, int n, cudaStream_t s);
// Batched forms over `npairs` pairs (one block per pair): the stopping test on each pair's
// partials (final = 0) or the final residual sum (final = 1, into res_final), and the counter.
void launch_reduce_check_batched(const double *partials, const PairScalars *ps, int npairs, double tol,
                                 int add_iters, int final, cudaStream_t s);
void launch_count_iters_batched(const PairScalars *ps, int npairs, int n, bool use_done, cudaStream_t s);
// Ping-pong parity repair: copies every non-NULL plane of `from` to `to` when the stop flag
// state ((done && *done) ? 1 : 0) equals `want_done`.
void launch_parity_fix(const Fields &from, const Fields &to, Geom g, int prec, int prec_flow, const int *done,
                       int want_done, cudaStream_t s);

// ---------------------------------------------------------------- several iterations per launch (k_admm_tile.cu, k_cp_tile.cu)
// Single pair: ni (2 or 3) consecutive iterations of the fused ADMM engine (ALG1: of k_cp) in one
// launch over TT x TT tiles (*_tile_size: 32, or 16 on small levels), reading a.in and writing
// a.out, bitwise ni launches of the one-iteration kernel; partials (of the last iteration) in
// *_tile_blocks(a.g) slots.
int admm_tile2_size(Geom g);
int admm_tile2_blocks(Geom g);
void launch_admm_tile2(const IterArgs &a, int ni, int prec, int prec_flow, cudaStream_t s);
int cp_tile_size(Geom g);
int cp_tile_blocks(Geom g);
void launch_cp_tile(const IterArgs &a, int ni, int prec, int prec_flow, cudaStream_t s);

// ---------------------------------------------------------------- adaptive ADMM step (k_adapt.cu)
// Residual balancing of c after one ADMM iteration prev -> cur (both state buffers intact): the
// constraint residual ||A s + B y|| and the dual residual of the preconditioned ADMM, summed over
// adapt_blocks(g) blocks into part_r / part_d, then c doubled (||r|| > 10 ||d||) or halved
// (||d|| > 10 ||r||) in place.  Duals and data in `prec`.  pDR (a.pdr): the same rule on
// ||X^{k+1} - X^k|| / sigma and ||ybar^{k+1} - ybar^k|| / tau, rescaling theta.
constexpr int ADAPT_MAX_BLOCKS = 1216;
struct AdaptArgs {
    Geom g{};
    Coefs k{};        // k.c_dev = 1: c is read at ms_max[-1] (== c below)
    Fields prev{}, cur{};
    const void *Ix = nullptr, *Iy = nullptr;
    const float *ms_max = nullptr;
    float *c = nullptr;
    double *part_r = nullptr, *part_d = nullptr;  // adapt_blocks(g) slots each
    int has_w = 0;
    int pdr = 0;      // pDR: *c is theta (sigma theta, tau / theta); the changes of X and ybar
};
int adapt_blocks(Geom g);
void launch_adapt_c(const AdaptArgs &a, int prec, int prec_flow, cudaStream_t s);
// *c = c0 (one thread): the adapted step starts from the parameter at the start of a solve.
void launch_c_init(float *c, float c0, cudaStream_t s);

// Whether field k is a flow/illumination plane (w u v wb ub vb), stored in the flow precision.
__host__ __device__ inline bool is_flow_field(int k) { return k == F_W || k == F_U || k == F_V || k == F_WB || k == F_UB || k == F_VB; }

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
