// tvl1_api.cu -- host runtime and C ABI of the GB300 TV-L1 optical-flow library
// (include/tvl1flow.h).  It plans the per-pair device arena, enqueues the whole coarse-to-fine
// schedule (pyramid, levels, warps, inner iterations; Sec. 3-4 of the paper) as kernels on a
// stream, captures it once per (size, parameters) into a CUDA graph and replays the graph on
// later calls.  No arithmetic of the method runs on the host.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"
#include "tvl1_plan.h"

namespace tvl1 {

Plan make_plan(int H, int W, const of_params *p) {
    Plan pl;
    pl.L = p->levels;
    pl.out_level = p->out_level;
    pl.prec = p->precision;
    pl.pflow = (p->precision != PREC_F32 && p->fp32_flow) ? PREC_F32 : p->precision;
    pl.use32_last = p->precision != PREC_F32 && p->fp32_last_warp && p->out_level == 0;
    pl.H[0] = H;
    pl.W[0] = W;
    for (int l = 1; l < pl.L; ++l) {
        pl.H[l] = level_size(pl.H[l - 1], p->eta);
        pl.W[l] = level_size(pl.W[l - 1], p->eta);
    }
    for (int l = 0; l < pl.L; ++l) pl.P[l] = pitch_of(pl.W[l]);
    const size_t n0 = (size_t)pl.H[0] * pl.P[0];
    pl.plane32 = align_up(n0 * 4, 256);
    pl.planeT = align_up(n0 * prec_bytes(pl.prec), 256);
    pl.planeS = align_up(n0 * std::max(prec_bytes(pl.prec), prec_bytes(pl.pflow)), 256);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes, 256);
        return o;
    };
    for (int l = 0; l < pl.L; ++l) {
        const size_t b = align_up((size_t)pl.H[l] * pl.P[l] * 4, 256);
        pl.img0[l] = take(b);
        pl.img1[l] = take(b);
    }
    pl.I1x = take(pl.plane32);
    pl.I1y = take(pl.plane32);
    pl.blur = take(2 * pl.plane32);
    pl.stA = take(NFIELDS * pl.planeS);
    pl.stB = take(NFIELDS * pl.planeS);
    pl.data = take(3 * pl.planeT);
    if (pl.use32_last) {
        pl.stA32 = take(NFIELDS * pl.plane32);
        pl.stB32 = take(NFIELDS * pl.plane32);
        pl.data32 = take(3 * pl.plane32);
    } else {
        pl.stA32 = pl.stB32 = pl.data32 = 0;
    }
    pl.tmp = take(6 * pl.plane32);
    // partial-sum slots: the most blocks any engine launches on any level (the streaming engine's
    // strip height changes with the level, so a coarser level can need more blocks; a height set
    // in the parameters or by the autotuner can be the lowest, 1, which launches the most)
    int mb = 1;
    for (int l = 0; l < pl.L; ++l) {
        const Geom g{pl.H[l], pl.W[l], pl.P[l]};
        mb = std::max({mb, admm_fused_blocks(g, p->rows_per_warp != 0 ? 1 : 0), admm_plain_blocks(g),
                       pdr_plain_blocks(g, PARTIAL_ROWS_MIN), cp_blocks(g, PARTIAL_ROWS_MIN), energy_blocks(g),
                       adapt_blocks(g), admm_tile2_blocks(g), pdr_tile_blocks(g), cp_tile_blocks(g)});
    }
    pl.max_blocks = mb;
    pl.partials = take(3 * (size_t)mb * sizeof(double));
    pl.misc = take(sizeof(Misc));
    const size_t nout = (size_t)pl.H[pl.out_level] * pl.P[pl.out_level];
    pl.out = take(3 * nout * 4);
    pl.total = off;
    return pl;
}

Coefs coefs_of(const of_params *p) {
    Coefs k;
    k.lambda = p->lambda;
    k.beta = p->beta;
    k.c = p->c;
    k.a = p->a;
    k.r = p->method == OF_PADMM_I ? p->r : 1.f;
    k.rho = p->rho;
    k.sigma = p->sigma;
    k.tau = p->tau;
    k.a_tilde_fixed = p->a_tilde;
    k.cp_tau = p->cp_tau;
    k.cp_sigma = p->cp_sigma;
    k.a_tilde_mode = p->a_tilde_mode;
    k.method = p->method;
    k.gs_sweeps = p->gs_sweeps;
    k.c_dev = p->c_adapt_iters > 0 ? 1 : 0;
    return k;
}

Fields fields_at(char *base, size_t plane) {
    Fields f;
    for (int k = 0; k < NFIELDS; ++k) f.f[k] = base + (size_t)k * plane;
    return f;
}

}  // namespace tvl1

using namespace tvl1;

namespace {

thread_local std::string g_err = "no error";

of_status fail(of_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define OF_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(OF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

of_status validate(const of_params *p, int H, int W) {
    if (!p) return fail(OF_EINVAL, "params is NULL");
    if (H < 1 || W < 1 || H > OF_MAX_SIDE || W > OF_MAX_SIDE)
        return fail(OF_EINVAL, "image sizes must lie in [1, " + std::to_string(OF_MAX_SIDE) + "]");
    if (p->method < 0 || p->method > 3) return fail(OF_EINVAL, "unknown method");
    if (!(p->lambda > 0.f) || !isfinite(p->lambda)) return fail(OF_EINVAL, "lambda must be > 0");
    if (!(p->beta >= 0.f) || !isfinite(p->beta)) return fail(OF_EINVAL, "beta must be >= 0");
    if (p->method == OF_CP) {
        if (!(p->cp_tau > 0.f) || !(p->cp_sigma > 0.f) || !isfinite(p->cp_tau) || !isfinite(p->cp_sigma))
            return fail(OF_EINVAL, "cp_tau and cp_sigma must be > 0");
        if (p->engine == OF_ENGINE_PLAIN) return fail(OF_EINVAL, "ALG1 has one (fused) engine");
    } else if (p->method != OF_PDR) {
        if (!(p->c > 0.f) || !isfinite(p->c)) return fail(OF_EINVAL, "c must be > 0");
        if (!(p->a > 0.f) || !isfinite(p->a)) return fail(OF_EINVAL, "a must be > 0");
        if (!isfinite(p->a_tilde)) return fail(OF_EINVAL, "a_tilde must be finite");
        if (p->method == OF_PADMM_I && !(p->r > 0.f && p->r < 1.6181f))
            return fail(OF_EINVAL, "r must lie in (0, (1+sqrt 5)/2)");
        if (p->method == OF_PADMM_II && !(p->rho > 0.f && p->rho < 2.f)) return fail(OF_EINVAL, "rho must lie in (0, 2)");
    } else {
        if (!(p->sigma > 0.f) || !(p->tau > 0.f) || !isfinite(p->sigma) || !isfinite(p->tau))
            return fail(OF_EINVAL, "sigma and tau must be > 0");
        if (p->gs_sweeps < 1 || p->gs_sweeps > 64) return fail(OF_EINVAL, "gs_sweeps must lie in [1, 64]");
    }
    if (!(p->eta > 0.f && p->eta < 1.f)) return fail(OF_EINVAL, "eta must lie in (0, 1)");
    if (gauss_taps(p->eta).R < 0) return fail(OF_EINVAL, "eta too small for the pre-smoothing kernel");
    if (p->levels < 1 || p->levels > MAX_LEVELS) return fail(OF_EINVAL, "levels must lie in [1, 16]");
    if (p->warps < 1) return fail(OF_EINVAL, "warps must be >= 1");
    if (p->iters < 0) return fail(OF_EINVAL, "iters must be >= 0");
    if (!(p->tol >= 0.0) || !isfinite(p->tol)) return fail(OF_EINVAL, "tol must be >= 0");
    if (p->precision < 0 || p->precision > 2) return fail(OF_EINVAL, "unknown precision");
    if (p->engine < 0 || p->engine > 4) return fail(OF_EINVAL, "unknown engine");
    if (p->a_tilde_mode < 0 || p->a_tilde_mode > 1) return fail(OF_EINVAL, "a_tilde_mode must be 0 or 1");
    if (p->method == OF_PDR || p->method == OF_CP) {
        if (p->rows_per_warp != -1 && p->rows_per_warp != 0 && p->rows_per_warp != 4 && p->rows_per_warp != 8 &&
            p->rows_per_warp != 16)
            return fail(OF_EINVAL, "rows_per_warp of pDR and ALG1 (their block height) must be -1 (autotune), 0, 4, 8 "
                                   "or 16");
    } else if (p->rows_per_warp != -1 && p->rows_per_warp != 0 && p->rows_per_warp != 1 && p->rows_per_warp != 2 &&
               p->rows_per_warp != 8 && p->rows_per_warp != 32) {
        return fail(OF_EINVAL, "rows_per_warp must be -1 (autotune), 0 (built-in rule), 1, 2, 8 or 32");
    }
    if (p->engine == OF_ENGINE_PLAIN && p->precision != OF_PREC_FP32)
        return fail(OF_EINVAL, "the plain engine runs in FP32 only");
    if (p->out_level < 0 || p->out_level >= p->levels) return fail(OF_EINVAL, "out_level must lie in [0, levels)");
    if (p->c_adapt_iters < 0 || p->c_adapt_iters % 10 != 0)
        return fail(OF_EINVAL, "c_adapt_iters must be 0 or a positive multiple of 10");
    if (p->c_adapt_iters > 0 && p->method == OF_CP)
        return fail(OF_EINVAL, "c_adapt_iters applies to the ADMM methods and pDR only");
    if (p->c_adapt_iters > 0 && p->method == OF_PDR && p->gs_sweeps != 1)
        return fail(OF_EINVAL, "c_adapt_iters with pDR needs one Gauss-Seidel sweep (its one-launch kernel)");
    if (p->c_adapt_iters > 0 && p->engine == OF_ENGINE_PLAIN)
        return fail(OF_EINVAL, "c_adapt_iters needs a fused engine (the plain engine iterates in place)");
    return OF_OK;
}

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

}  // namespace

struct of_ctx {
    int device = 0;
    size_t budget = 0;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::map<std::string, GraphEntry> graphs;
    // the batch layout whose launch tables the arena holds (graphs of other layouts re-upload)
    std::string tables_key;
    // autotuned strip heights of the streaming ADMM kernel, per level workload (tune_key)
    std::map<std::string, int> tuned;
    // serving loop state (tvl1_serve.cu)
    void *server = nullptr;
};

namespace {

void drop_graphs(of_ctx *ctx) {
    for (auto &kv : ctx->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    ctx->graphs.clear();
    ctx->tables_key.clear();
}

of_status ensure_arena(of_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->arena_bytes) return OF_OK;
    if (bytes > ctx->budget)
        return fail(OF_ENOMEM, "arena of " + std::to_string(bytes) + " bytes exceeds the HBM budget of " +
                                   std::to_string(ctx->budget));
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    if (ctx->arena) cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(OF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    ctx->arena = (char *)p;
    ctx->arena_bytes = bytes;
    return OF_OK;
}



// Enqueues the whole schedule of one pair on `s` (arena pointers only: graph-capturable).
// A batch of n pairs solved with one set of parameters.  Pair k owns the arena region
// [base[k], base[k] + pl[k].total).  For n > 1 the arena also holds the tables of the batched
// launches: per level the PairIter descriptors of all pairs (storage-precision buffers and, on
// level 0 with the FP32 last warp, the FP32 buffers), the fused-ADMM tile work-list and the
// per-pair scalars of the batched reductions, plus one partial-sum array shared by the batch.
struct Batch {
    int n = 0, L = 0, out_level = 0;
    std::vector<Plan> pl;
    std::vector<size_t> base;
    size_t pairs_off[MAX_LEVELS][2] = {}, tiles_off[MAX_LEVELS] = {}, scal_off[MAX_LEVELS] = {};
    // strip height of the streaming ADMM kernel per level (a single pair: 0 = the built-in rule)
    // and, batched, the size of the level's tile work-list for it
    int ntiles[MAX_LEVELS] = {}, tile_h[MAX_LEVELS] = {};
    Geom gmax[MAX_LEVELS] = {};
    // level-resident pairs per level: flags, count, device list offset, shared memory per CTA
    std::vector<char> res[MAX_LEVELS];
    int nres[MAX_LEVELS] = {};
    size_t reslist_off[MAX_LEVELS] = {}, res_smem[MAX_LEVELS] = {};
    int res_nc[MAX_LEVELS] = {};  // CTAs per cluster of the level's resident launch
    // the other pairs, for the one-slice-per-pair batched kernels (ALG1)
    size_t streamlist_off[MAX_LEVELS] = {};
    size_t partials = 0, table_off = 0, table_bytes = 0, total = 0;
    // persistent ADMM engine per level (any n): the segment plan and the offsets (in the table
    // region) of its segments, warp lists, per-pair scalars, counters and partial sums
    bool pers[MAX_LEVELS] = {};
    std::vector<PSeg> psegs[MAX_LEVELS];
    std::vector<int> pwoff[MAX_LEVELS], pwseg[MAX_LEVELS], pbegin[MAX_LEVELS], pend[MAX_LEVELS];
    int pnwarps[MAX_LEVELS] = {};
    size_t pseg_off[MAX_LEVELS] = {}, pwoff_off[MAX_LEVELS] = {}, pwseg_off[MAX_LEVELS] = {},
           pscal_off[MAX_LEVELS] = {}, pctr_off[MAX_LEVELS] = {}, ppart_off[MAX_LEVELS] = {};
    std::string key;
};


// Whether a level of geometry g runs its inner iterations on the level-resident engine: the level
// fits one cluster's shared memory and, with the default engine, is small enough for the resident
// launch to beat the per-iteration kernels (all methods have a resident form).
// pDR with one symmetric Gauss-Seidel sweep on the fused engines runs its non-resident levels on
// the one-launch tile kernel (ping-pong buffers); more sweeps, the plain engine and the
// stage-by-stage solver use the per-kernel engine (in place).
bool pdr_tile_of(const of_params *p) {
    return p->method == OF_PDR && p->engine != OF_ENGINE_PLAIN && p->gs_sweeps == 1;
}

// Levels up to this many pixels run pDR level-resident when its one-launch tile kernel is the
// alternative (measured per iteration, resident against tile kernel: 2.3 / 4.0 us at 40x30,
// 2.7 / 4.3 at 80x60, 4.3 / 4.3 at 120x90, 6.0 / 4.4 at 160x120).
constexpr long PDR_TILE_RESIDENT_MAX_PX = 12000;

// Whether a single pair's streamed ADMM level runs several iterations per launch (k_admm_tile.cu):
// the built-in strip rule (a pinned or autotuned height asks for the row-streaming kernel), at any
// size.  Measured per iteration against the row-streaming kernel (2-row strips at 640x480 and
// below, 8-row above): 320x240 2.34 against 3.99 us, 640x480 5.41 against 7.98, 1024x436 7.82
// against 9.27, 1920x1080 35.2 against 39.9 (DRAM-bound: the state is read and written once per
// three iterations); 1242x375 9.40 against 9.27 and 960x540 9.92 against 9.63 are the exceptions,
// within 3%.
// Iterations per launch (the last launch of a warp may run 2, or 1).  Measured per iteration at
// 640x480 / 320x240: 7.86 / 3.21 us with 2, 6.72 / 2.78 with 3, 7.13 / 3.01 with 4 (a 41 x 41
// frame: 64 registers and 108 KB of shared memory per block, and a third more halo work).
constexpr int TILE_ITERS = 3;

bool admm_tile2_of(const of_params *p, bool batched, Geom) {
    return !batched && (p->method == OF_PADMM_I || p->method == OF_PADMM_II) && p->rows_per_warp == 0 &&
           (p->engine == OF_ENGINE_FUSED || p->engine == OF_ENGINE_STREAM);
}

// Whether a single pair's streamed ALG1 level runs several iterations per launch (k_cp_tile.cu):
// the built-in block height (a pinned or autotuned one asks for the one-iteration kernel k_cp).
bool cp_tile_of(const of_params *p, bool batched) {
    return !batched && p->method == OF_CP && p->rows_per_warp == 0 &&
           (p->engine == OF_ENGINE_FUSED || p->engine == OF_ENGINE_STREAM);
}

// Levels up to this many pixels run ALG1 level-resident when its tile kernel is the alternative
// (measured per iteration, resident against tile kernel: 1.03 / 1.21 us at 40x30, 1.21 / 1.29 at
// 80x60, 1.79 / 1.29 at 120x90, 2.41 / 1.32 at 160x120).
constexpr long CP_TILE_RESIDENT_MAX_PX = 6000;

// Levels up to this many pixels run the ADMM methods level-resident when the several-iterations
// tile kernel is the alternative (measured per iteration, resident against tile kernel: 1.04 /
// 1.51 us at 40x30, 1.34 / 1.58 at 80x60, 1.93 / 1.58 at 120x90, 2.67 / 1.61 at 160x120); against
// the row-streaming kernel the resident launch wins up to 32,000 px.
constexpr long TILE_RESIDENT_MAX_PX = 7000;

bool use_resident(const of_params *p, Geom g, bool batched = false) {
    if (!admm_resident_fits(g, p->method)) return false;
    if (p->engine == OF_ENGINE_RESIDENT) return true;
    if (p->engine != OF_ENGINE_FUSED && p->engine != OF_ENGINE_PERSISTENT) return false;
    if (pdr_tile_of(p)) return (long)g.H * g.W <= PDR_TILE_RESIDENT_MAX_PX;
    if (admm_tile2_of(p, batched, g)) return (long)g.H * g.W <= TILE_RESIDENT_MAX_PX;
    if (cp_tile_of(p, batched)) return (long)g.H * g.W <= CP_TILE_RESIDENT_MAX_PX;
    return admm_resident_preferred(g, p->method);
}

// Tiles of level l's work-list (the pairs not on the level-resident engine) with strip height ty.
int batch_tiles(const Batch &B, int l, int ty) {
    const int rows = ty * admm_fused_warps(), SWD = admm_fused_strip_w();
    int nt = 0;
    for (int k = 0; k < B.n; ++k) {
        if (B.res[l][k]) continue;
        const Geom g = geom_of(B.pl[k], l);
        nt += ((g.W + SWD - 1) / SWD) * ((g.H + rows - 1) / rows);
    }
    return nt;
}

// The block height of the pDR and ALG1 per-iteration kernels before any tuning: the parameters'
// height (4, 8 or 16), else 8; 0 for the ADMM methods, whose levels take a strip height instead.
int block_height_of(const of_params *p) {
    if (p->method != OF_PDR && p->method != OF_CP) return 0;
    return (p->rows_per_warp == 4 || p->rows_per_warp == 16) ? p->rows_per_warp : 8;
}

// Segments of one level for the persistent engine.  gs: per pair its level geometry, H = 0 for a
// pair that is not on the engine at this level; max_warps: the warps one wave of the launch holds.
// Every segment gets about the same number of rows (at least two, unless its pair has fewer than
// four); a single pair is cut into as many segments as there are warps, a batch into segments of
// the batch's mean rows per warp.  When there are more segments than warps, each goes, longest
// first, to the warp with the fewest rows so far.
struct PersistPlan {
    std::vector<PSeg> segs;
    std::vector<int> woff, wseg, pbegin, pend;
    int nwarps = 0;
};

PersistPlan plan_persist(const std::vector<Geom> &gs, int max_warps) {
    PersistPlan pp;
    const int n = (int)gs.size(), SWD = admm_fused_strip_w();
    pp.pbegin.assign(n, 0);
    pp.pend.assign(n, 0);
    double R = 0.0;
    int active = 0;
    for (const Geom &g : gs)
        if (g.H > 0) {
            R += (double)((g.W + SWD - 1) / SWD) * g.H;
            ++active;
        }
    if (active == 0 || max_warps < 1) return pp;
    const double L = std::max(2.0, R / max_warps);  // rows per segment
    auto rows_of = [&](const PSeg &sg) {
        const int h = gs[sg.pair].H;
        return (int)((long long)(sg.t + 1) * h / sg.m - (long long)sg.t * h / sg.m);
    };
    for (int k = 0; k < n; ++k) {
        const Geom g = gs[k];
        pp.pbegin[k] = (int)pp.segs.size();
        if (g.H > 0) {
            const int S = (g.W + SWD - 1) / SWD;
            int m = active == 1 ? max_warps / S : (int)std::lround(g.H / L);
            m = std::max(1, std::min(m, std::max(1, g.H / 2)));
            for (int t = 0; t < m; ++t)
                for (int sx = 0; sx < S; ++sx) pp.segs.push_back(PSeg{k, sx, t, m});
        }
        pp.pend[k] = (int)pp.segs.size();
    }
    const int N = (int)pp.segs.size();
    std::vector<std::vector<int>> lists;
    if (N <= max_warps) {
        lists.resize(N);
        for (int q = 0; q < N; ++q) lists[q].push_back(q);
    } else {
        lists.resize(max_warps);
        std::vector<int> order(N);
        for (int q = 0; q < N; ++q) order[q] = q;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return rows_of(pp.segs[a]) > rows_of(pp.segs[b]); });
        std::vector<std::pair<long long, int>> heap;  // (rows so far, warp), min-heap
        for (int w = 0; w < max_warps; ++w) heap.push_back({0, w});
        auto cmp = [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) { return a > b; };
        std::make_heap(heap.begin(), heap.end(), cmp);
        for (int q : order) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto &top = heap.back();
            lists[top.second].push_back(q);
            top.first += rows_of(pp.segs[q]) + 3;   // a segment's row steps: its rows and the halo
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
        for (auto &l : lists) std::sort(l.begin(), l.end());
    }
    pp.nwarps = (int)lists.size();
    pp.woff.push_back(0);
    for (auto &l : lists) {
        for (int q : l) pp.wseg.push_back(q);
        pp.woff.push_back((int)pp.wseg.size());
    }
    return pp;
}

// Whether level l of this layout runs its inner iterations on the persistent engine (ADMM
// methods, engine OF_ENGINE_PERSISTENT, a pair left to the per-iteration kernels).
bool pers_level(const Batch &B, const of_params *p, int l) {
    if (p->engine != OF_ENGINE_PERSISTENT || p->iters < 1) return false;
    if (p->method != OF_PADMM_I && p->method != OF_PADMM_II) return false;
    if (l < B.out_level) return false;
    for (int k = 0; k < B.n; ++k)
        if (B.n > 1 ? !B.res[l][k] : !use_resident(p, geom_of(B.pl[0], l))) return true;
    return false;
}

// Warps one wave of the persistent launch holds for this layout's kernel instances (the FP32
// instance too where the finest level's last warp switches to FP32 storage).
int persist_warps(const Batch &B, const of_params *p) {
    const Coefs k = coefs_of(p);
    int cap = persist_capacity(k, B.pl[0].prec, B.pl[0].pflow);
    if (B.pl[0].use32_last) cap = std::min(cap, persist_capacity(k, PREC_F32, PREC_F32));
    if (cap <= 0) cap = 152 * 3;  // no device to ask (sizing only): a full GB300
    return cap * admm_fused_warps();
}

Batch make_batch(int n, const int *H, const int *W, const of_params *p) {
    Batch B;
    B.n = n;
    B.L = p->levels;
    B.out_level = p->out_level;
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        B.pl.push_back(make_plan(H[k], W[k], p));
        B.base.push_back(off);
        off += align_up(B.pl.back().total, 256);
    }
    B.key.append((const char *)&n, sizeof(int));
    for (int k = 0; k < n; ++k) {
        B.key.append((const char *)&H[k], sizeof(int));
        B.key.append((const char *)&W[k], sizeof(int));
    }
    of_params q;
    memset(&q, 0, sizeof(q));
    q = *p;
    B.key.append((const char *)&q, sizeof(q));
    if (n > 1) {
        size_t t = 0, maxpart = 1;
        const int SWD = admm_fused_strip_w();
        for (int l = 0; l < B.L; ++l) {
            long strip_rows = 0;
            Geom gm{0, 0, 0};
            // the level-resident engine takes this level's eligible pairs only when all their
            // clusters run at once; otherwise one work-list launch per iteration serves them better
            B.res[l].assign(n, 0);
            int elig = 0;
            for (int k = 0; k < n; ++k) elig += use_resident(p, geom_of(B.pl[k], l), true) ? 1 : 0;
            const bool take = elig > 0 && elig <= admm_resident_max_clusters();
            for (int k = 0; k < n; ++k) {
                const Geom g = geom_of(B.pl[k], l);
                if (g.H > gm.H) gm.H = g.H;
                if (g.W > gm.W) gm.W = g.W;
                if (take && use_resident(p, g, true)) {
                    B.res[l][k] = 1;
                    ++B.nres[l];
                    B.res_nc[l] = std::max(B.res_nc[l], admm_resident_nc(g, p->method));
                    continue;
                }
                strip_rows += (long)((g.W + SWD - 1) / SWD) * g.H;
            }
            // one cluster size for the launch: the largest any of its pairs asks for (a larger
            // cluster only shrinks a pair's band)
            for (int k = 0; k < n; ++k)
                if (B.res[l][k])
                    B.res_smem[l] = std::max(B.res_smem[l], admm_resident_smem(geom_of(B.pl[k], l), p->method, B.res_nc[l]));
            gm.pitch = pitch_of(gm.W);
            B.gmax[l] = gm;
            B.tile_h[l] = block_height_of(p) ? block_height_of(p)
                          : p->rows_per_warp > 0 ? p->rows_per_warp
                                                 : admm_fused_rows_per_warp(strip_rows, p->precision != OF_PREC_FP32);
            B.ntiles[l] = batch_tiles(B, l, B.tile_h[l]);
            // room for the longest work-list (height 1) when the autotuner will try every height
            const bool admm = p->method == OF_PADMM_I || p->method == OF_PADMM_II;
            const int nt = (admm && p->rows_per_warp == -1) ? batch_tiles(B, l, 1) : B.ntiles[l];
            B.pairs_off[l][0] = t;
            t += align_up(sizeof(PairIter) * n, 256);
            B.pairs_off[l][1] = t;
            t += align_up(sizeof(PairIter) * n, 256);
            B.tiles_off[l] = t;
            t += align_up(sizeof(TileRef) * nt, 256);
            B.scal_off[l] = t;
            t += align_up(sizeof(PairScalars) * n, 256);
            B.reslist_off[l] = t;
            t += align_up(sizeof(int) * n, 256);
            B.streamlist_off[l] = t;
            t += align_up(sizeof(int) * n, 256);
            const size_t np = std::max({(size_t)nt, (size_t)n * pdr_plain_blocks(gm, PARTIAL_ROWS_MIN),
                                        (size_t)n * cp_blocks(gm, PARTIAL_ROWS_MIN)});
            maxpart = std::max(maxpart, np);
        }
        B.table_bytes = t;
        B.partials = maxpart;  // slots for now; an offset once the tables are laid out
    } else {
        for (int l = 0; l < B.L; ++l)
            B.tile_h[l] = block_height_of(p)      ? block_height_of(p)
                          : p->rows_per_warp > 0  ? p->rows_per_warp
                          : p->rows_per_warp == 0 ? admm_fused_tile_h(geom_of(B.pl[0], l), p->precision != OF_PREC_FP32)
                                                  : 0;  // set by the autotuner
    }
    // persistent engine tables (any n; a single pair also needs its PairIter descriptors)
    size_t t = B.table_bytes;
    int maxw = 0;
    for (int l = 0; l < B.L; ++l) {
        B.pers[l] = pers_level(B, p, l);
        if (!B.pers[l]) continue;
        if (maxw == 0) maxw = persist_warps(B, p);
        std::vector<Geom> gs(n);
        for (int k = 0; k < n; ++k) {
            const Geom g = geom_of(B.pl[k], l);
            const bool on = n > 1 ? !B.res[l][k] : !use_resident(p, g);
            gs[k] = on ? g : Geom{0, 0, 0};
        }
        PersistPlan pp = plan_persist(gs, maxw);
        const size_t N = pp.segs.size();
        if (n == 1) {
            B.pairs_off[l][0] = t;
            t += align_up(sizeof(PairIter), 256);
            B.pairs_off[l][1] = t;
            t += align_up(sizeof(PairIter), 256);
        }
        B.pseg_off[l] = t;
        t += align_up(sizeof(PSeg) * N, 256);
        B.pwoff_off[l] = t;
        t += align_up(sizeof(int) * (pp.nwarps + 1), 256);
        B.pwseg_off[l] = t;
        t += align_up(sizeof(int) * N, 256);
        B.pscal_off[l] = t;
        t += align_up(sizeof(PairScalars) * n, 256);
        B.pctr_off[l] = t;
        t += align_up(sizeof(unsigned) * (N + n), 256);
        B.ppart_off[l] = t;
        t += align_up(sizeof(double) * N, 256);
        B.psegs[l] = std::move(pp.segs);
        B.pwoff[l] = std::move(pp.woff);
        B.pwseg[l] = std::move(pp.wseg);
        B.pbegin[l] = std::move(pp.pbegin);
        B.pend[l] = std::move(pp.pend);
        B.pnwarps[l] = pp.nwarps;
    }
    B.table_bytes = t;
    if (t > 0) {
        B.table_off = off;
        off += align_up(t, 256);
    }
    if (n > 1) {
        const size_t maxpart = B.partials;
        B.partials = off;
        off += align_up(maxpart * sizeof(double), 256);
    }
    B.total = off;
    return B;
}

// Writes the batched-launch tables (absolute device pointers into the current arena).
of_status upload_tables(of_ctx *ctx, const Batch &B, const of_params *p) {
    if (B.table_bytes == 0) return OF_OK;
    std::vector<char> img(B.table_bytes, 0);
    const bool pdr = p->method == OF_PDR, cp = p->method == OF_CP;
    const bool xb = pdr || cp;  // one grid slice per pair (pDR, ALG1) instead of a tile work-list
    // the descriptors of pair k at level l, for its storage-precision and its FP32 buffers
    auto pair_iter = [&](PairIter *pi0, PairIter *pi1, int k, int l) {
        const Plan &pl = B.pl[k];
        char *A = ctx->arena + B.base[k];
        Misc *misc = (Misc *)(A + pl.misc);
        for (int v = 0; v < 2; ++v) {
            PairIter &P = v ? pi1[k] : pi0[k];
            P.g = geom_of(pl, l);
            if (v == 0) {
                P.buf[0] = fields_at(A + pl.stA, pl.planeS);
                P.buf[1] = fields_at(A + pl.stB, pl.planeS);
                P.Ix = A + pl.data;
                P.Iy = A + pl.data + pl.planeT;
                P.It = A + pl.data + 2 * pl.planeT;
            } else {
                P.buf[0] = fields_at(A + pl.stA32, pl.plane32);
                P.buf[1] = fields_at(A + pl.stB32, pl.plane32);
                P.Ix = A + pl.data32;
                P.Iy = A + pl.data32 + pl.plane32;
                P.It = A + pl.data32 + 2 * pl.plane32;
            }
            P.ms_max = &misc->ms_max;
            P.done = p->tol > 0.0 ? &misc->done : nullptr;
            P.tmp = (float *)(A + pl.tmp);
        }
    };
    auto scalars = [&](PairScalars &ps, int k, int l) {
        Misc *misc = (Misc *)(ctx->arena + B.base[k] + B.pl[k].misc);
        const Geom g = geom_of(B.pl[k], l);
        ps.res_check = &misc->res_check;
        ps.res_final = &misc->res_final;
        ps.done = &misc->done;
        ps.iters = &misc->iters;
        ps.rows = (double)g.H * g.W * (p->beta != 0.f ? 3.0 : 2.0);
        ps.timeout = &misc->timeout;
    };
    for (int l = 0; l < B.L && B.n > 1; ++l) {
        PairIter *pi0 = (PairIter *)(img.data() + B.pairs_off[l][0]);
        PairIter *pi1 = (PairIter *)(img.data() + B.pairs_off[l][1]);
        TileRef *tr = (TileRef *)(img.data() + B.tiles_off[l]);
        PairScalars *ps = (PairScalars *)(img.data() + B.scal_off[l]);
        int *rl = (int *)(img.data() + B.reslist_off[l]);
        int *sl = (int *)(img.data() + B.streamlist_off[l]);
        int t = 0, r = 0, ns = 0;
        const int G = cp                ? cp_blocks(B.gmax[l], B.tile_h[l])
                      : pdr_tile_of(p) ? pdr_tile_blocks(B.gmax[l])
                                       : pdr_plain_blocks(B.gmax[l], B.tile_h[l]);
        for (int k = 0; k < B.n; ++k) {
            const Geom g = geom_of(B.pl[k], l);
            pair_iter(pi0, pi1, k, l);
            const int rows = B.tile_h[l] * admm_fused_warps(), SWD = admm_fused_strip_w();
            const int t0 = t;
            if (B.res[l][k]) rl[r++] = k;
            else sl[ns++] = k;
            if (!B.res[l][k])
                for (int ty = 0; ty < (g.H + rows - 1) / rows; ++ty)
                    for (int tx = 0; tx < (g.W + SWD - 1) / SWD; ++tx) tr[t++] = TileRef{k, tx, ty, 0};
            scalars(ps[k], k, l);
            ps[k].part_begin = xb ? k * G : t0;
            ps[k].part_end = xb ? (k + 1) * G : t;
            ps[k].resident = B.res[l][k];
        }
    }
    // persistent engine: segments, warp lists and per-pair scalars over the segment ranges
    for (int l = 0; l < B.L; ++l) {
        if (!B.pers[l]) continue;
        if (B.n == 1)
            pair_iter((PairIter *)(img.data() + B.pairs_off[l][0]), (PairIter *)(img.data() + B.pairs_off[l][1]), 0, l);
        memcpy(img.data() + B.pseg_off[l], B.psegs[l].data(), sizeof(PSeg) * B.psegs[l].size());
        memcpy(img.data() + B.pwoff_off[l], B.pwoff[l].data(), sizeof(int) * B.pwoff[l].size());
        memcpy(img.data() + B.pwseg_off[l], B.pwseg[l].data(), sizeof(int) * B.pwseg[l].size());
        PairScalars *ps = (PairScalars *)(img.data() + B.pscal_off[l]);
        for (int k = 0; k < B.n; ++k) {
            scalars(ps[k], k, l);
            ps[k].part_begin = B.pbegin[l][k];
            ps[k].part_end = B.pend[l][k];
            ps[k].resident = B.pbegin[l][k] == B.pend[l][k];  // not on this engine: skipped by the reductions
        }
    }
    // work already queued on any stream may still read another layout's tables in this region
    OF_CUDA(cudaDeviceSynchronize());
    OF_CUDA(cudaMemcpy(ctx->arena + B.table_off, img.data(), img.size(), cudaMemcpyHostToDevice));
    ctx->tables_key = B.key;
    return OF_OK;
}

// Enqueues the whole schedule of every pair of the batch on `s` (arena pointers only: graph-
// capturable).  Per pair: pyramid, level transfer, derivatives, warping, reductions.  The inner
// iterations of all pairs go in one launch per iteration (a single pair: its own grid).
void enqueue_solve(of_ctx *ctx, const Batch &B, const of_params *p, cudaStream_t s) {
    const int n = B.n;
    const bool batched = n > 1;
    const bool has_w = p->beta != 0.f;
    const bool pdr = p->method == OF_PDR, cp = p->method == OF_CP;
    const bool plain = p->engine == OF_ENGINE_PLAIN;
    const bool pdr_tile = pdr_tile_of(p);
    // ADMM fused engines, ALG1 and the one-launch pDR kernel read one buffer and write the other
    const bool pingpong = (!pdr && !plain) || pdr_tile;
    const GaussTaps taps = gauss_taps(p->eta);
    auto blocks_of = [&](Geom g, int l) {
        return pdr ? (pdr_tile ? pdr_tile_blocks(g) : pdr_plain_blocks(g, plain ? 0 : B.tile_h[l]))
                   : cp ? cp_blocks(g, B.tile_h[l]) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g, B.tile_h[l]));
    };
    const Coefs k = coefs_of(p);
    const int L = B.L;
    double *bpart = batched ? (double *)(ctx->arena + B.partials) : nullptr;

    struct PairCtx {
        char *A;
        const Plan *pl;
        Misc *misc;
        double *partials;
        Fields buf[2], buf32[2];
        const void *data[3], *data32[3];
    };
    std::vector<PairCtx> pc(n);
    for (int q = 0; q < n; ++q) {
        PairCtx &c = pc[q];
        const Plan &pl = B.pl[q];
        c.pl = &pl;
        c.A = ctx->arena + B.base[q];
        c.misc = (Misc *)(c.A + pl.misc);
        c.partials = (double *)(c.A + pl.partials);
        c.buf[0] = fields_at(c.A + pl.stA, pl.planeS);
        c.buf[1] = fields_at(c.A + pl.stB, pl.planeS);
        c.buf32[0] = fields_at(c.A + pl.stA32, pl.plane32);
        c.buf32[1] = fields_at(c.A + pl.stB32, pl.plane32);
        for (int d = 0; d < 3; ++d) {
            c.data[d] = c.A + pl.data + d * pl.planeT;
            c.data32[d] = c.A + pl.data32 + d * pl.plane32;
        }
        cudaMemsetAsync(c.misc, 0, sizeof(Misc), s);
        if (p->c_adapt_iters > 0) launch_c_init(&c.misc->c_cur, pdr ? 1.f : p->c, s);  // pDR: theta
        for (int l = 1; l < L; ++l) {
            launch_pyr_down((float *)(c.A + pl.img0[l - 1]), geom_of(pl, l - 1), (float *)(c.A + pl.img0[l]),
                            geom_of(pl, l), taps, (float *)(c.A + pl.blur), s);
            launch_pyr_down((float *)(c.A + pl.img1[l - 1]), geom_of(pl, l - 1), (float *)(c.A + pl.img1[l]),
                            geom_of(pl, l), taps, (float *)(c.A + pl.blur), s);
        }
    }

    int cur = 0, prec = B.pl[0].prec, pflow = B.pl[0].pflow;
    bool in32 = false;  // the FP32 last-warp buffers are in use
    auto bufs_of = [&](const PairCtx &c) { return in32 ? c.buf32 : c.buf; };
    auto data_of = [&](const PairCtx &c) { return in32 ? c.data32 : c.data; };

    for (int l = L - 1; l >= B.out_level; --l) {
        for (int q = 0; q < n; ++q) {
            const PairCtx &c = pc[q];
            const Plan &pl = *c.pl;
            const Geom g = geom_of(pl, l);
            const Fields *bf = bufs_of(c);
            if (l == L - 1) {
                launch_fill(bf[cur].f + F_W, pflow, 3, g, 0.f, s);
            } else {
                const Geom gc = geom_of(pl, l + 1);
                const int nxt = cur ^ 1;
                launch_upsample(bf[cur].f[F_W], gc, bf[nxt].f[F_W], g, 1.f, pflow, s);
                launch_upsample(bf[cur].f[F_U], gc, bf[nxt].f[F_U], g, (float)g.W / (float)gc.W, pflow, s);
                launch_upsample(bf[cur].f[F_V], gc, bf[nxt].f[F_V], g, (float)g.H / (float)gc.H, pflow, s);
            }
            const int now = l == L - 1 ? cur : cur ^ 1;
            // duals p, q, s restart at 0 (ALG1 keeps its dual in the flow fields' type)
            launch_fill(bf[now].f + F_P1, cp ? pflow : prec, F_S - F_P1 + 1, g, 0.f, s);
            if (!has_w) launch_fill(bf[now].f + F_W, pflow, 1, g, 0.f, s);
            if (pdr || cp) {  // pDR: Xbar = X; ALG1: the extrapolated point starts at X
                const void *src[3] = {bf[now].f[F_W], bf[now].f[F_U], bf[now].f[F_V]};
                void *dst[3] = {bf[now].f[F_WB], bf[now].f[F_UB], bf[now].f[F_VB]};
                launch_copy_planes(src, dst, 3, g, pflow, s);
            }
            launch_derivatives((float *)(c.A + pl.img1[l]), g, (float *)(c.A + pl.I1x), (float *)(c.A + pl.I1y), s);
        }
        if (l != L - 1) cur ^= 1;
        for (int wp = 0; wp < p->warps; ++wp) {
            const bool last_warp = (l == B.out_level) && (wp == p->warps - 1);
            const bool switch32 = B.pl[0].use32_last && l == 0 && wp == p->warps - 1;
            for (int q = 0; q < n; ++q) {
                const PairCtx &c = pc[q];
                const Plan &pl = *c.pl;
                const Geom g = geom_of(pl, l);
                if (switch32) {
                    // precision policy: the finest level's last warp runs with FP32 storage
                    launch_convert(c.buf[cur].f + F_W, pflow, c.buf32[0].f + F_W, PREC_F32, 3, g, s);
                    launch_convert(c.buf[cur].f + F_P1, cp ? pflow : prec, c.buf32[0].f + F_P1, PREC_F32,
                                   F_S - F_P1 + 1, g, s);
                    launch_convert(c.buf[cur].f + F_WB, pflow, c.buf32[0].f + F_WB, PREC_F32, 3, g, s);
                }
                const Fields *bf = switch32 ? c.buf32 : bufs_of(c);
                const int cc = switch32 ? 0 : cur;
                const void *const *dat = switch32 ? c.data32 : data_of(c);
                const int pw = switch32 ? PREC_F32 : prec, pwf = switch32 ? PREC_F32 : pflow;
                cudaMemsetAsync(&c.misc->ms_max, 0, sizeof(float) + sizeof(int), s);  // ms_max and done
                launch_warp((float *)(c.A + pl.img0[l]), (float *)(c.A + pl.img1[l]), (float *)(c.A + pl.I1x),
                            (float *)(c.A + pl.I1y), bf[cc].f[F_U], bf[cc].f[F_V], g, p->beta, (void *)dat[0],
                            (void *)dat[1], (void *)dat[2], &c.misc->ms_max, pw, pwf, s);
            }
            if (switch32) {
                in32 = true;
                cur = 0;
                prec = PREC_F32;
                pflow = PREC_F32;
            }
            const int start = cur;
            // adaptive steps (single pair; ADMM: c, pDR: sigma and tau with sigma tau fixed): the
            // level's first warp runs its first c_adapt_iters iterations one per-iteration launch
            // each (streaming kernel, pDR tile kernel) and rebalances after every 10th; the level's
            // engine then runs the other `rest` iterations with the steps frozen
            const int kw = (p->c_adapt_iters > 0 && wp == 0) ? std::min(p->c_adapt_iters, p->iters) : 0;
            const int rest = p->iters - kw;
            if (kw > 0) {
                const PairCtx &c = pc[0];
                const Geom g = geom_of(*c.pl, l);
                const Fields *bf = bufs_of(c);
                const void *const *dat = data_of(c);
                const int mb = c.pl->max_blocks;
                for (int it = 0; it < kw; ++it) {
                    const bool final_it = last_warp && rest == 0 && it == kw - 1;
                    IterArgs a{};
                    a.k = k;
                    a.g = g;
                    a.in = bf[(start + it) & 1];
                    a.out = bf[(start + it + 1) & 1];
                    a.Ix = dat[0];
                    a.Iy = dat[1];
                    a.It = dat[2];
                    a.ms_max = &c.misc->ms_max;
                    a.partials = final_it ? c.partials : nullptr;
                    a.tile_h = B.tile_h[l];
                    if (pdr) {
                        a.pdr_tile = 1;
                        launch_pdr_fused(a, prec, pflow, s);
                    } else {
                        launch_admm_fused(a, prec, pflow, s);
                    }
                    if (final_it) launch_sum(c.partials, blocks_of(g, l), &c.misc->res_final, s);
                    if ((it + 1) % 10 == 0) {
                        AdaptArgs d{};
                        d.g = g;
                        d.k = k;
                        d.prev = a.in;
                        d.cur = a.out;
                        d.Ix = dat[0];
                        d.Iy = dat[1];
                        d.ms_max = &c.misc->ms_max;
                        d.c = &c.misc->c_cur;
                        d.part_r = c.partials + mb;
                        d.part_d = c.partials + 2 * mb;
                        d.has_w = has_w;
                        d.pdr = pdr;
                        launch_adapt_c(d, prec, pflow, s);
                    }
                }
                launch_count_iters(&c.misc->iters, nullptr, kw, s);
            }
            const int start2 = (start + kw) & 1;  // where the level's engine picks the state up
            // level-resident engine: the single pair, or the batch's resident pairs, in one launch
            const bool res1 = !batched && use_resident(p, geom_of(*pc[0].pl, l));
            const bool resb = batched && B.nres[l] > 0;
            if (rest > 0 && (res1 || resb)) {
                ResArgs r{};
                r.k = k;
                r.iters = rest;
                r.check = p->tol > 0.0;
                r.final_res = last_warp;
                r.tol = p->tol;
                r.parity_in = start2;
                r.parity_out = pingpong ? (start2 + rest) & 1 : start2;  // pDR works in place
                if (res1) {
                    const PairCtx &c = pc[0];
                    const Geom g = geom_of(*c.pl, l);
                    const Fields *bf = bufs_of(c);
                    const void *const *dat = data_of(c);
                    r.g = g;
                    r.in = bf[r.parity_in];
                    r.out = bf[r.parity_out];
                    r.Ix = dat[0];
                    r.Iy = dat[1];
                    r.It = dat[2];
                    r.ms_max = &c.misc->ms_max;
                    r.sc.res_check = &c.misc->res_check;
                    r.sc.res_final = &c.misc->res_final;
                    r.sc.done = &c.misc->done;
                    r.sc.iters = &c.misc->iters;
                    r.sc.rows = (double)g.H * g.W * (has_w ? 3.0 : 2.0);
                    r.sc.resident = 1;
                    const int nc = admm_resident_nc(g, p->method);
                    launch_admm_resident(r, 1, nc, admm_resident_smem(g, p->method, nc), prec, pflow, s);
                } else {
                    r.pairs = (const PairIter *)(ctx->arena + B.table_off + B.pairs_off[l][in32 ? 1 : 0]);
                    r.scal = (const PairScalars *)(ctx->arena + B.table_off + B.scal_off[l]);
                    r.list = (const int *)(ctx->arena + B.table_off + B.reslist_off[l]);
                    launch_admm_resident(r, B.nres[l], B.res_nc[l], B.res_smem[l], prec, pflow, s);
                }
            }
            // persistent engine: every inner iteration of the level's other pairs in one launch
            const bool persl = B.pers[l];
            char *T = ctx->arena + B.table_off;
            if (persl && rest > 0) {
                const int N = (int)B.psegs[l].size();
                cudaMemsetAsync(T + B.pctr_off[l], 0, sizeof(unsigned) * (N + n), s);
                PersistArgs a{};
                a.k = k;
                a.pairs = (const PairIter *)(T + B.pairs_off[l][in32 ? 1 : 0]);
                a.scal = (const PairScalars *)(T + B.pscal_off[l]);
                a.segs = (const PSeg *)(T + B.pseg_off[l]);
                a.woff = (const int *)(T + B.pwoff_off[l]);
                a.wseg = (const int *)(T + B.pwseg_off[l]);
                a.nwarps = B.pnwarps[l];
                a.flags = (unsigned *)(T + B.pctr_off[l]);
                a.pbar = a.flags + N;
                a.partials = (double *)(T + B.ppart_off[l]);
                a.parity = start2;
                a.iters = rest;
                a.check = p->tol > 0.0;
                a.final_res = last_warp;
                a.tol = p->tol;
                launch_admm_persist(a, prec, pflow, s);
            }
            // pairs left for one launch per iteration: the tile work-list (ADMM), all pairs (pDR),
            // the non-resident pairs (ALG1)
            const bool streamed = !persl && (batched ? ((cp || pdr) ? B.nres[l] < n : B.ntiles[l] > 0) : !res1);
            // single pair, ADMM or ALG1, the built-in strip rule or block height: several iterations
            // per launch (k_admm_tile.cu, k_cp_tile.cu).  With the
            // stopping test every ten iterations run as launches of 3, 3, 3 and 1: the tested state
            // is a single-iteration launch's (its residual partials), an even number of launches
            // leaves it in bufs[start2] as on the one-launch-per-iteration path, and the warp's last
            // launch is a single iteration too, so the final residual sums the same partials
            // whether or not the test stopped the warp.
            const bool tile2 = streamed && (admm_tile2_of(p, batched, geom_of(*pc[0].pl, l)) || cp_tile_of(p, batched));
            int par = start2, last_nb = 0;  // the several-iterations path's buffer parity and last block count
            for (int it = 0, step = 1; streamed && it < rest; it += step) {
                step = 1;
                if (tile2) {
                    step = std::min(TILE_ITERS, rest - it);
                    if (p->tol > 0.0) {
                        step = std::min(step, 10 - it % 10);
                        if (step > 1 && it + step == rest) --step;
                    }
                }
                const bool check = p->tol > 0.0 && (it + step) % 10 == 0;
                const bool final_it = last_warp && it + step == rest;
                IterArgs a{};
                a.k = k;
                if (!batched) {
                    const PairCtx &c = pc[0];
                    const Geom g = geom_of(*c.pl, l);
                    const Fields *bf = bufs_of(c);
                    const void *const *dat = data_of(c);
                    a.g = g;
                    a.in = bf[tile2 ? par : pingpong ? (start2 + it) & 1 : start2];
                    a.out = bf[tile2 ? par ^ 1 : pingpong ? (start2 + it + 1) & 1 : start2];
                    par ^= 1;
                    a.Ix = dat[0];
                    a.Iy = dat[1];
                    a.It = dat[2];
                    a.ms_max = &c.misc->ms_max;
                    a.partials = (check || final_it) ? c.partials : nullptr;
                    a.done = p->tol > 0.0 ? &c.misc->done : nullptr;
                    a.tmp = (float *)(c.A + c.pl->tmp);
                    a.tile_h = B.tile_h[l];
                    a.pdr_tile = pdr_tile;
                    if (pdr) {
                        if (plain) launch_pdr_plain(a, s);
                        else launch_pdr_fused(a, prec, pflow, s);
                    } else if (cp) {
                        if (step > 1) {
                            launch_cp_tile(a, step, prec, pflow, s);
                            last_nb = cp_tile_blocks(g);
                        } else {
                            launch_cp(a, prec, pflow, s);
                            last_nb = blocks_of(g, l);
                        }
                    } else if (step > 1) {
                        launch_admm_tile2(a, step, prec, pflow, s);
                        last_nb = admm_tile2_blocks(g);
                    } else {
                        if (plain) launch_admm_plain(a, s);
                        else launch_admm_fused(a, prec, pflow, s);
                        last_nb = blocks_of(g, l);
                    }
                    if (check) {
                        const int nb = step > 1 ? (cp ? cp_tile_blocks(g) : admm_tile2_blocks(g)) : blocks_of(g, l);
                        const double rows = (double)g.H * g.W * (has_w ? 3.0 : 2.0);
                        launch_reduce_check(c.partials, nb, &c.misc->res_check, rows, p->tol, &c.misc->done,
                                            &c.misc->iters, 10, s);
                    }
                } else {
                    a.pairs = (const PairIter *)(ctx->arena + B.table_off + B.pairs_off[l][in32 ? 1 : 0]);
                    a.partials = (check || final_it) ? bpart : nullptr;
                    if (pdr) {
                        a.g = B.gmax[l];
                        a.ntiles = n - B.nres[l];
                        a.plist = (const int *)(ctx->arena + B.table_off + B.streamlist_off[l]);
                        a.parity = pdr_tile ? (start2 + it) & 1 : start2;
                        a.tile_h = B.tile_h[l];
                        a.pdr_tile = pdr_tile;
                        launch_pdr_fused(a, prec, pflow, s);
                    } else if (cp) {
                        a.g = B.gmax[l];
                        a.ntiles = n - B.nres[l];
                        a.plist = (const int *)(ctx->arena + B.table_off + B.streamlist_off[l]);
                        a.parity = (start2 + it) & 1;
                        a.tile_h = B.tile_h[l];
                        launch_cp(a, prec, pflow, s);
                    } else {
                        a.tiles = (const TileRef *)(ctx->arena + B.table_off + B.tiles_off[l]);
                        a.ntiles = B.ntiles[l];
                        a.tile_h = B.tile_h[l];
                        a.parity = (start2 + it) & 1;
                        launch_admm_fused(a, prec, pflow, s);
                    }
                    if (check)
                        launch_reduce_check_batched(bpart, (const PairScalars *)(ctx->arena + B.table_off + B.scal_off[l]),
                                                    n, p->tol, 10, 0, s);
                }
            }
            const PairScalars *ps = batched ? (const PairScalars *)(ctx->arena + B.table_off + B.scal_off[l]) : nullptr;
            if (batched) {
                launch_count_iters_batched(ps, n, p->tol > 0.0 ? rest % 10 : rest, p->tol > 0.0, s);
            } else if (!res1) {
                Misc *m = pc[0].misc;
                if (p->tol > 0.0) launch_count_iters(&m->iters, &m->done, rest % 10, s);
                else launch_count_iters(&m->iters, nullptr, rest, s);
            }
            if (pingpong) {
                const int fin = tile2 ? par : (start + p->iters) & 1;
                if (p->tol > 0.0 && (tile2 ? par != start2 : (rest & 1)))
                    for (int q = 0; q < n; ++q)
                        if (!(res1 || (batched && B.res[l][q])))  // the resident engine writes buf[fin] itself
                            launch_parity_fix(bufs_of(pc[q])[start2], bufs_of(pc[q])[fin], geom_of(*pc[q].pl, l),
                                              cp ? pflow : prec, pflow, &pc[q].misc->done, 1, s);
                cur = fin;
            }
            if (last_warp && rest > 0 && !res1) {
                if (persl) {
                    double *pp = (double *)(T + B.ppart_off[l]);
                    if (batched)
                        launch_reduce_check_batched(pp, (const PairScalars *)(T + B.pscal_off[l]), n, 0.0, 0, 1, s);
                    else
                        launch_sum(pp, (int)B.psegs[l].size(), &pc[0].misc->res_final, s);
                } else if (batched) {
                    launch_reduce_check_batched(bpart, ps, n, 0.0, 0, 1, s);
                } else {
                    const Geom g = geom_of(*pc[0].pl, l);
                    launch_sum(pc[0].partials, tile2 ? last_nb : blocks_of(g, l), &pc[0].misc->res_final, s);
                }
            }
        }
        if (l == B.out_level) {
            for (int q = 0; q < n; ++q) {
                const PairCtx &c = pc[q];
                const Plan &pl = *c.pl;
                const Geom g = geom_of(pl, l);
                const int mb = pl.max_blocks;
                double *pe = c.partials + mb, *pd = c.partials + 2 * mb;
                Fields fe = bufs_of(c)[cur];
                if (pdr || cp) fe.f[F_S] = nullptr;
                if (!has_w) fe.f[F_W] = nullptr;
                const void *const *dat = data_of(c);
                launch_energy(fe, dat[0], dat[1], dat[2], g, p->beta, p->lambda, prec, pflow, pe, pd, s);
                launch_sum(pe, energy_blocks(g), &c.misc->energy, s);
                launch_sum(pd, energy_blocks(g), &c.misc->dual, s);
                float *out = (float *)(c.A + pl.out);
                const size_t on = (size_t)pl.H[pl.out_level] * pl.P[pl.out_level];
                const void *src[3] = {bufs_of(c)[cur].f[F_U], bufs_of(c)[cur].f[F_V], bufs_of(c)[cur].f[F_W]};
                void *dst[3] = {out, out + on, out + 2 * on};
                launch_convert(src, pflow, dst, PREC_F32, 3, g, s);
            }
        }
    }
}

// ------------------------------------------------------------ autotuner
// Whether level l of layout B runs its inner iterations on a per-iteration kernel with a tunable
// shape: the streaming ADMM kernel (its strip height) or the pDR / ALG1 kernels (their block
// height), for the pairs the level-resident engine does not take.
bool tunable_level(const Batch &B, const of_params *p, int l) {
    if (l < B.out_level || l >= B.L || B.pers[l]) return false;
    if (p->engine == OF_ENGINE_PLAIN || p->iters <= 0) return false;
    if (pdr_tile_of(p)) return false;  // the one-launch pDR kernel has no block height to tune
    if (p->method == OF_PADMM_I || p->method == OF_PADMM_II)
        return B.n > 1 ? B.ntiles[l] > 0 : !use_resident(p, geom_of(B.pl[0], l));
    return B.n > 1 ? B.nres[l] < B.n : !use_resident(p, geom_of(B.pl[0], l));
}

// The strip height (ADMM) or block height (pDR, ALG1) level l runs with (tunable levels only).
int level_rows(const Batch &B, int l) {
    if (B.n > 1 || B.tile_h[l] > 0) return B.tile_h[l];
    return admm_fused_tile_h(geom_of(B.pl[0], l), B.pl[0].prec != PREC_F32);
}

// What the kernel's speed depends on: the kernel instance (method, per-pixel a~, beta > 0,
// storage types), single or batched form, and the geometries of the streamed pairs.
std::string tune_key(const Batch &B, const of_params *p, int l) {
    const int hdr[6] = {p->method, p->a_tilde_mode, p->beta != 0.f ? 1 : 0, B.pl[0].prec, B.pl[0].pflow, B.n > 1 ? 1 : 0};
    std::string k((const char *)hdr, sizeof(hdr));
    for (int q = 0; q < B.n; ++q) {
        if (B.n > 1 && B.res[l][q]) continue;
        const Geom g = geom_of(B.pl[q], l);
        k.append((const char *)&g.H, sizeof(int));
        k.append((const char *)&g.W, sizeof(int));
    }
    return k;
}

// One inner iteration of level l on its per-iteration kernel, as the solve launches it (storage
// precision of the level's main warps; no stop flag, no residual partials).
void launch_level_iteration(of_ctx *ctx, const Batch &B, const of_params *p, int l, int parity, cudaStream_t s) {
    const bool pdr = p->method == OF_PDR, cp = p->method == OF_CP;
    IterArgs a{};
    a.k = coefs_of(p);
    a.k.c_dev = 0;  // timing only: the fixed parameter c, whatever the arena's device scalars hold
    a.tile_h = B.tile_h[l];
    if (B.n == 1) {
        const Plan &pl = B.pl[0];
        char *A = ctx->arena + B.base[0];
        const Fields b0 = fields_at(A + pl.stA, pl.planeS), b1 = fields_at(A + pl.stB, pl.planeS);
        a.g = geom_of(pl, l);
        const bool inplace = pdr && !pdr_tile_of(p);  // the per-kernel pDR engine works in place
        a.in = parity && !inplace ? b1 : b0;
        a.out = inplace ? b0 : (parity ? b0 : b1);
        a.Ix = A + pl.data;
        a.Iy = A + pl.data + pl.planeT;
        a.It = A + pl.data + 2 * pl.planeT;
        a.ms_max = &((Misc *)(A + pl.misc))->ms_max;
        a.tmp = (float *)(A + pl.tmp);
    } else {
        a.pairs = (const PairIter *)(ctx->arena + B.table_off + B.pairs_off[l][0]);
        if (pdr || cp) {
            a.g = B.gmax[l];
            a.ntiles = B.n - B.nres[l];
            a.plist = (const int *)(ctx->arena + B.table_off + B.streamlist_off[l]);
            a.parity = pdr && !pdr_tile_of(p) ? 0 : parity;
        } else {
            a.tiles = (const TileRef *)(ctx->arena + B.table_off + B.tiles_off[l]);
            a.ntiles = B.ntiles[l];
            a.parity = parity;
        }
    }
    a.pdr_tile = pdr_tile_of(p);
    if (pdr) launch_pdr_fused(a, B.pl[0].prec, B.pl[0].pflow, s);
    else if (cp) launch_cp(a, B.pl[0].prec, B.pl[0].pflow, s);
    else launch_admm_fused(a, B.pl[0].prec, B.pl[0].pflow, s);
}

// Times every candidate shape on level l -- the strip heights of the streaming ADMM kernel, or the
// block heights of the pDR / ALG1 kernels -- (2 untimed and 6 timed iterations each, CUDA events
// on the context's own stream) and returns the fastest; ties keep the lower one.
of_status tune_level(of_ctx *ctx, Batch &B, const of_params *p, int l, int *best) {
    static const int cand_admm[4] = {1, 2, 8, 32}, cand_blocks[3] = {4, 8, 16};
    const bool blocks = p->method == OF_PDR || p->method == OF_CP;
    const int *cand = blocks ? cand_blocks : cand_admm;
    const int ncand = blocks ? 3 : 4;
    constexpr int WARM = 2, REPS = 6;
    of_params q = *p;
    q.tol = 0.0;  // tables without stop flags: every timed launch does the full iteration
    ctx->tables_key.clear();  // from here on the arena's tables are the candidates' (also on error)
    if (B.n > 1 && blocks) {  // the pair descriptors of the batched launches (any block height)
        of_status st = upload_tables(ctx, B, &q);
        ctx->tables_key.clear();
        if (st != OF_OK) return st;
    }
    float best_ms = 0.f;
    *best = 0;
    for (int c = 0; c < ncand; ++c) {
        const int ty = cand[c];
        B.tile_h[l] = ty;
        if (B.n > 1 && !blocks) {
            B.ntiles[l] = batch_tiles(B, l, ty);
            of_status st = upload_tables(ctx, B, &q);
            ctx->tables_key.clear();
            if (st != OF_OK) return st;
        }
        for (int it = 0; it < WARM + REPS; ++it) {
            if (it == WARM) OF_CUDA(cudaEventRecord(ctx->ev0, ctx->cap));
            launch_level_iteration(ctx, B, &q, l, it & 1, ctx->cap);
        }
        OF_CUDA(cudaEventRecord(ctx->ev1, ctx->cap));
        OF_CUDA(cudaEventSynchronize(ctx->ev1));
        OF_CUDA(cudaGetLastError());
        float ms = 0.f;
        OF_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        if (*best == 0 || ms < best_ms) {
            best_ms = ms;
            *best = ty;
        }
    }
    return OF_OK;
}

// rows_per_warp = -1: sets B's strip (or block) heights from the context's tuning, timing the
// levels not tuned yet.  The timing launches run on the arena (state and data zeroed first; the solve
// overwrites them) after a device synchronisation, so no queued solve still uses it.
of_status resolve_rows(of_ctx *ctx, Batch &B, const of_params *p) {
    if (p->rows_per_warp != -1) return OF_OK;
    bool ready = false;
    for (int l = B.L - 1; l >= B.out_level; --l) {
        if (!tunable_level(B, p, l)) continue;
        const std::string key = tune_key(B, p, l);
        auto it = ctx->tuned.find(key);
        int ty = 0;
        if (it != ctx->tuned.end()) {
            ty = it->second;
        } else {
            if (!ready) {
                OF_CUDA(cudaDeviceSynchronize());
                for (int q = 0; q < B.n; ++q) {
                    const Plan &pl = B.pl[q];
                    char *A = ctx->arena + B.base[q];
                    OF_CUDA(cudaMemsetAsync(A + pl.stA, 0, NFIELDS * pl.planeS, ctx->cap));
                    OF_CUDA(cudaMemsetAsync(A + pl.stB, 0, NFIELDS * pl.planeS, ctx->cap));
                    OF_CUDA(cudaMemsetAsync(A + pl.data, 0, 3 * pl.planeT, ctx->cap));
                    OF_CUDA(cudaMemsetAsync(A + pl.misc, 0, sizeof(Misc), ctx->cap));
                }
                ready = true;
            }
            of_status st = tune_level(ctx, B, p, l, &ty);
            if (st != OF_OK) return st;
            ctx->tuned[key] = ty;
        }
        B.tile_h[l] = ty;
        if (B.n > 1 && block_height_of(p) == 0) B.ntiles[l] = batch_tiles(B, l, ty);
    }
    return OF_OK;
}

of_status get_graph(of_ctx *ctx, const Batch &B, const of_params *p, cudaGraphExec_t *out, cudaGraph_t *graph_out = nullptr) {
    // a solve lays its data out from the arena's start, over any other layout's tables; one
    // without tables of its own leaves none intact
    if (B.table_bytes == 0) ctx->tables_key.clear();
    auto it = ctx->graphs.find(B.key);
    if (it != ctx->graphs.end()) {
        // a cached graph reads its tables from the arena: restore them if another layout has
        // replaced them since
        if (B.table_bytes > 0 && ctx->tables_key != B.key) {
            of_status st = upload_tables(ctx, B, p);
            if (st != OF_OK) return st;
        }
        *out = it->second.exec;
        if (graph_out) *graph_out = it->second.graph;
        return OF_OK;
    }
    of_status st = upload_tables(ctx, B, p);
    if (st != OF_OK) return st;
    GraphEntry ge;
    OF_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    enqueue_solve(ctx, B, p, ctx->cap);
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &ge.graph);
    if (e != cudaSuccess) return fail(OF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(ge.graph);
        return fail(OF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    ctx->graphs[B.key] = ge;
    *out = ge.exec;
    if (graph_out) *graph_out = ge.graph;
    return OF_OK;
}

of_status read_stats(of_ctx *ctx, const Batch &B, int q, const of_params *p, cudaStream_t s, of_stats *stats) {
    const Plan &pl = B.pl[q];
    Misc m;
    OF_CUDA(cudaMemcpyAsync(&m, ctx->arena + B.base[q] + pl.misc, sizeof(Misc), cudaMemcpyDeviceToHost, s));
    OF_CUDA(cudaStreamSynchronize(s));
    const Geom g{pl.H[pl.out_level], pl.W[pl.out_level], pl.P[pl.out_level]};
    const double rows = (double)g.H * g.W * (p->beta != 0.f ? 3.0 : 2.0);
    stats->iters_run = m.iters;
    stats->residual = p->iters > 0 ? sqrt(m.res_final / rows) : 0.0;
    stats->energy = m.energy;
    stats->dual_value = (p->method == OF_PDR || p->method == OF_CP) ? NAN : m.dual;
    const bool adapt = p->c_adapt_iters > 0;
    stats->c = p->method == OF_PDR ? p->sigma * (adapt ? m.c_cur : 1.f) : adapt ? m.c_cur : p->c;
    if (m.timeout) return fail(OF_ETIMEOUT, "a bounded wait of the persistent engine ran out");
    if (!isfinite(stats->residual) || !isfinite(stats->energy))
        return fail(OF_ENUMERIC, "non-finite residual or energy (NaN/Inf in the inputs or parameters?)");
    return OF_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

void of_default_params(of_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->method = OF_PADMM_I;
    p->lambda = 0.05f;
    p->beta = 0.05f;
    p->c = 0.05f;
    p->a = 8.f;
    p->a_tilde = 0.f;
    p->r = 1.f;
    p->rho = 1.9f;
    p->sigma = 2.f;
    p->tau = 0.4f;
    p->gs_sweeps = 1;
    p->eta = 0.5f;
    p->levels = 3;
    p->warps = 5;
    p->iters = 50;
    p->tol = 0.0;
    p->precision = OF_PREC_FP32;
    p->fp32_last_warp = 1;
    p->fp32_flow = 1;
    p->engine = OF_ENGINE_FUSED;
    p->out_level = 0;
    p->cp_tau = 0.1f;
    p->cp_sigma = 1.25f;
    p->a_tilde_mode = 0;
    p->c_adapt_iters = 0;
}

of_status of_create(of_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(OF_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    OF_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(OF_EINVAL, "no such CUDA device");
    OF_CUDA(cudaSetDevice(device));
    admm_resident_max_clusters();  // device queries run once, outside any stream capture
    of_ctx *ctx = new of_ctx();
    ctx->device = device;
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(OF_ECUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    }
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)tot);
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        delete ctx;
        return fail(OF_ECUDA, "stream/event creation failed");
    }
    *out = ctx;
    return OF_OK;
}

void tvl1_server_destroy(of_ctx *ctx);  // tvl1_serve.cu

void of_destroy(of_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    tvl1_server_destroy(ctx);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

const char *of_last_error(of_ctx *) { return g_err.c_str(); }

size_t of_arena_bytes(int H, int W, const of_params *params) {
    if (validate(params, H, W) != OF_OK) return 0;
    return make_plan(H, W, params).total;
}

long long of_solve_kernel_count(of_ctx *ctx, int H, int W, const of_params *params) {
    if (!ctx) {
        fail(OF_EINVAL, "ctx is NULL");
        return -1;
    }
    if (validate(params, H, W) != OF_OK) return -1;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return -1;
    Batch B = make_batch(1, &H, &W, params);
    if (ensure_arena(ctx, B.total) != OF_OK) return -1;
    if (resolve_rows(ctx, B, params) != OF_OK) return -1;
    cudaGraphExec_t ge;
    cudaGraph_t g;
    if (get_graph(ctx, B, params, &ge, &g) != OF_OK) return -1;
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    long long k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

of_status of_resident_clusters(int *cluster_ctas, int *max_active) {
    if (!cluster_ctas || !max_active) return fail(OF_EINVAL, "of_resident_clusters: NULL pointer");
    *cluster_ctas = admm_resident_cluster();
    *max_active = admm_resident_max_clusters();
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

of_status of_persistent_selftest(int H, int W, int iters, int withhold, double wait_ms, int *timed_out,
                                 int *segments) {
    if (!timed_out || H < 1 || W < 1 || iters < 1 || !(wait_ms > 0.0) || !isfinite(wait_ms))
        return fail(OF_EINVAL, "of_persistent_selftest: bad arguments");
    of_params p;
    of_default_params(&p);
    p.engine = OF_ENGINE_PERSISTENT;
    const Coefs k = coefs_of(&p);
    const int cap = persist_capacity(k, PREC_F32, PREC_F32);
    if (cap <= 0) return fail(OF_ECUDA, "of_persistent_selftest: no occupancy for the persistent kernel");
    const Geom g{H, W, pitch_of(W)};
    PersistPlan pp = plan_persist({g}, cap * admm_fused_warps());
    const int N = (int)pp.segs.size();
    if (withhold >= N) return fail(OF_EINVAL, "of_persistent_selftest: withhold beyond the segment count");
    if (segments) *segments = N;
    // one device block: 2 x 13 state planes, 3 data planes, the pair's scalars and the tables
    const size_t plane = align_up((size_t)g.H * g.pitch * 4, 256);
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += align_up(b, 256);
        return o;
    };
    const size_t o_st = take(2 * NFIELDS * plane), o_dat = take(3 * plane), o_misc = take(sizeof(Misc));
    const size_t o_pi = take(sizeof(PairIter)), o_ps = take(sizeof(PairScalars)), o_seg = take(sizeof(PSeg) * N);
    const size_t o_woff = take(sizeof(int) * pp.woff.size()), o_wseg = take(sizeof(int) * N);
    const size_t o_ctr = take(sizeof(unsigned) * (N + 1)), o_part = take(sizeof(double) * N);
    char *D = nullptr;
    cudaError_t e = cudaMalloc(&D, off);
    if (e != cudaSuccess) return fail(OF_ECUDA, std::string("of_persistent_selftest: cudaMalloc: ") + cudaGetErrorString(e));
    Misc *misc = (Misc *)(D + o_misc);
    PairIter pi{};
    pi.g = g;
    pi.buf[0] = fields_at(D + o_st, plane);
    pi.buf[1] = fields_at(D + o_st + NFIELDS * plane, plane);
    pi.Ix = D + o_dat;
    pi.Iy = D + o_dat + plane;
    pi.It = D + o_dat + 2 * plane;
    pi.ms_max = &misc->ms_max;
    PairScalars ps{};
    ps.res_check = &misc->res_check;
    ps.res_final = &misc->res_final;
    ps.done = &misc->done;
    ps.iters = &misc->iters;
    ps.part_begin = 0;
    ps.part_end = N;
    ps.rows = 3.0 * H * W;
    ps.timeout = &misc->timeout;
    e = cudaMemset(D, 0, off);
    if (e == cudaSuccess) e = cudaMemcpy(D + o_pi, &pi, sizeof(pi), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D + o_ps, &ps, sizeof(ps), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D + o_seg, pp.segs.data(), sizeof(PSeg) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D + o_woff, pp.woff.data(), sizeof(int) * pp.woff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D + o_wseg, pp.wseg.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        PersistArgs a{};
        a.k = k;
        a.pairs = (const PairIter *)(D + o_pi);
        a.scal = (const PairScalars *)(D + o_ps);
        a.segs = (const PSeg *)(D + o_seg);
        a.woff = (const int *)(D + o_woff);
        a.wseg = (const int *)(D + o_wseg);
        a.nwarps = pp.nwarps;
        a.flags = (unsigned *)(D + o_ctr);
        a.pbar = a.flags + N;
        a.partials = (double *)(D + o_part);
        a.iters = iters;
        a.wait_ns = (long long)(wait_ms * 1e6);
        a.withhold = withhold;
        e = launch_admm_persist(a, PREC_F32, PREC_F32, nullptr);
    }
    int to = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&to, &misc->timeout, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(D);
    if (e != cudaSuccess) return fail(OF_ECUDA, std::string("of_persistent_selftest: ") + cudaGetErrorString(e));
    *timed_out = to ? 1 : 0;
    return OF_OK;
}

of_status of_rows_per_warp(of_ctx *ctx, int n, const int *H, const int *W, const of_params *params, int *rows) {
    if (!ctx || !H || !W || !params || !rows || n < 1) return fail(OF_EINVAL, "of_rows_per_warp: NULL argument or n < 1");
    for (int q = 0; q < n; ++q) {
        of_status st = validate(params, H[q], W[q]);
        if (st != OF_OK) return st;
    }
    OF_CUDA(cudaSetDevice(ctx->device));
    Batch B = make_batch(n, H, W, params);
    if (params->rows_per_warp == -1) {
        of_status st = ensure_arena(ctx, B.total);
        if (st != OF_OK) return st;
        st = resolve_rows(ctx, B, params);
        if (st != OF_OK) return st;
    }
    for (int l = 0; l < B.L; ++l) rows[l] = tunable_level(B, params, l) ? level_rows(B, l) : 0;
    return OF_OK;
}

}  // extern "C"

namespace {

// Common body of the whole-solve entry points.  `host`: I0/I1/u/v/w are host pointers (dense)
// and the copies go host<->device; otherwise device pointers with the given pitches.  `sync`:
// wait for the stream before returning.
of_status solve_pairs(of_ctx *ctx, int n, const float *const *I0, const float *const *I1, const int *H, const int *W,
                      const int *pitch, const of_params *params, float *const *u, float *const *v, float *const *w,
                      const int *out_pitch, bool host, void *stream, of_stats *stats, bool sync) {
    if (!ctx) return fail(OF_EINVAL, "ctx is NULL");
    if (n < 1) return fail(OF_EINVAL, "no pairs");
    if (!params) return fail(OF_EINVAL, "params is NULL");
    if (n > 1 && params->engine == OF_ENGINE_PLAIN)
        return fail(OF_EINVAL, "batched solves use the fused engine (the plain engine is single-pair)");
    if (n > 1 && params->c_adapt_iters != 0)
        return fail(OF_EINVAL, "c_adapt_iters is supported for single-pair solves only");
    for (int q = 0; q < n; ++q) {
        of_status st = validate(params, H[q], W[q]);
        if (st != OF_OK) return st;
        if (!I0[q] || !I1[q] || !u[q] || !v[q]) return fail(OF_EINVAL, "NULL image or output pointer");
        if (!host && pitch[q] < W[q]) return fail(OF_EINVAL, "pitch < W");
    }
    OF_CUDA(cudaSetDevice(ctx->device));
    Batch B = make_batch(n, H, W, params);
    for (int q = 0; q < n; ++q)
        if (!host && out_pitch[q] < B.pl[q].W[B.out_level]) return fail(OF_EINVAL, "out_pitch smaller than the output width");
    of_status st = ensure_arena(ctx, B.total);
    if (st != OF_OK) return st;
    st = resolve_rows(ctx, B, params);
    if (st != OF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaGraphExec_t ge;
    st = get_graph(ctx, B, params, &ge);
    if (st != OF_OK) return st;
    const cudaMemcpyKind kin = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int q = 0; q < n; ++q) {
        const Plan &pl = B.pl[q];
        char *A = ctx->arena + B.base[q];
        const size_t sp = (size_t)(host ? W[q] : pitch[q]) * 4;
        OF_CUDA(cudaMemcpy2DAsync(A + pl.img0[0], (size_t)pl.P[0] * 4, I0[q], sp, (size_t)W[q] * 4, H[q], kin, s));
        OF_CUDA(cudaMemcpy2DAsync(A + pl.img1[0], (size_t)pl.P[0] * 4, I1[q], sp, (size_t)W[q] * 4, H[q], kin, s));
    }
    if (stats) OF_CUDA(cudaEventRecord(ctx->ev0, s));
    OF_CUDA(cudaGraphLaunch(ge, s));
    if (stats) OF_CUDA(cudaEventRecord(ctx->ev1, s));
    for (int q = 0; q < n; ++q) {
        const Plan &pl = B.pl[q];
        const int lo = pl.out_level;
        const size_t on = (size_t)pl.H[lo] * pl.P[lo];
        float *out = (float *)(ctx->arena + B.base[q] + pl.out);
        float *dst[3] = {u[q], v[q], w ? w[q] : nullptr};
        const size_t dp = (size_t)(host ? pl.W[lo] : out_pitch[q]) * 4;
        for (int k = 0; k < 3; ++k)
            if (dst[k])
                OF_CUDA(cudaMemcpy2DAsync(dst[k], dp, out + k * on, (size_t)pl.P[lo] * 4, (size_t)pl.W[lo] * 4,
                                          pl.H[lo], kout, s));
    }
    // a call that waits for the solve anyway (stats requested, or the host entry point) also
    // checks the FP64 residual and energy for non-finite values
    if (stats || sync) {
        float ms = 0.f;
        for (int q = 0; q < n; ++q) {
            of_stats local;
            of_stats *out = stats ? stats + q : &local;
            st = read_stats(ctx, B, q, params, s, out);
            if (stats && q == 0) cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            out->ms = ms;
            if (st != OF_OK) return st;
        }
    }
    if (sync) OF_CUDA(cudaStreamSynchronize(s));
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

}  // namespace

extern "C" {

of_status of_solve(of_ctx *ctx, const float *I0, const float *I1, int H, int W, int pitch, const of_params *params,
                   float *u, float *v, float *w, int out_pitch, void *stream, of_stats *stats) {
    return solve_pairs(ctx, 1, &I0, &I1, &H, &W, &pitch, params, &u, &v, &w, &out_pitch, false, stream, stats, false);
}

of_status of_solve_host(of_ctx *ctx, const float *I0, const float *I1, int H, int W, const of_params *params,
                        float *u, float *v, float *w, void *stream, of_stats *stats) {
    return solve_pairs(ctx, 1, &I0, &I1, &H, &W, &W, params, &u, &v, &w, &W, true, stream, stats, true);
}

of_status of_solve_batch(of_ctx *ctx, int n, const float *const *I0, const float *const *I1, const int *H,
                         const int *W, const int *pitch, const of_params *params, float *const *u, float *const *v,
                         float *const *w, const int *out_pitch, void *stream, of_stats *stats) {
    if (n < 0 || (n > 0 && (!I0 || !I1 || !H || !W || !pitch || !u || !v || !out_pitch)))
        return fail(OF_EINVAL, "of_solve_batch: NULL argument or n < 0");
    if (n == 0) return OF_OK;
    return solve_pairs(ctx, n, I0, I1, H, W, pitch, params, u, v, w, out_pitch, false, stream, stats, false);
}

}  // extern "C"

int tvl1_solve_async(of_ctx *ctx, const float *I0, const float *I1, int H, int W, const void *params_v, float *u,
                     float *v, cudaStream_t s) {
    float *w = nullptr;
    return solve_pairs(ctx, 1, &I0, &I1, &H, &W, &W, (const of_params *)params_v, &u, &v, &w, &W, true, (void *)s,
                       nullptr, false);
}

size_t tvl1_ctx_bytes(of_ctx *ctx) { return ctx ? ctx->arena_bytes : 0; }

void tvl1_set_error(const char *msg) { g_err = msg; }

extern "C" {

// ---------------------------------------------------------------- step-level entry points
of_status of_pyr_down(const float *fine, int Hf, int Wf, int pf, float *coarse, int Hc, int Wc, int pc, float eta,
                      float *scratch, void *stream) {
    if (!fine || !coarse || !scratch) return fail(OF_EINVAL, "NULL pointer");
    if (Hf < 1 || Wf < 1 || Hc < 1 || Wc < 1 || pf < Wf || pc < Wc) return fail(OF_EINVAL, "bad sizes or pitches");
    if (!(eta > 0.f && eta < 1.f)) return fail(OF_EINVAL, "eta must lie in (0, 1)");
    GaussTaps t = gauss_taps(eta);
    if (t.R < 0) return fail(OF_EINVAL, "eta too small");
    launch_pyr_down(fine, Geom{Hf, Wf, pf}, coarse, Geom{Hc, Wc, pc}, t, scratch, (cudaStream_t)stream);
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

of_status of_upsample(const float *coarse, int Hc, int Wc, int pc, float *fine, int Hf, int Wf, int pf, float scale,
                      void *stream) {
    if (!fine || !coarse) return fail(OF_EINVAL, "NULL pointer");
    if (Hf < 1 || Wf < 1 || Hc < 1 || Wc < 1 || pf < Wf || pc < Wc) return fail(OF_EINVAL, "bad sizes or pitches");
    launch_upsample_f32(coarse, Geom{Hc, Wc, pc}, fine, Geom{Hf, Wf, pf}, scale, (cudaStream_t)stream);
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

of_status of_derivatives(const float *I, int H, int W, int pitch, float *Ix, float *Iy, void *stream) {
    if (!I || !Ix || !Iy) return fail(OF_EINVAL, "NULL pointer");
    if (H < 1 || W < 1 || pitch < W) return fail(OF_EINVAL, "bad sizes or pitch");
    launch_derivatives(I, Geom{H, W, pitch}, Ix, Iy, (cudaStream_t)stream);
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

of_status of_warp_linearise(const float *I0, const float *I1, const float *I1x, const float *I1y, const float *u0,
                            const float *v0, int H, int W, int pitch, float beta, float *Ix, float *Iy, float *It,
                            float *ms_max, void *stream) {
    if (!I0 || !I1 || !I1x || !I1y || !u0 || !v0 || !Ix || !Iy || !It || !ms_max) return fail(OF_EINVAL, "NULL pointer");
    if (H < 1 || W < 1 || pitch < W) return fail(OF_EINVAL, "bad sizes or pitch");
    launch_warp(I0, I1, I1x, I1y, u0, v0, Geom{H, W, pitch}, beta, Ix, Iy, It, ms_max, PREC_F32, PREC_F32, (cudaStream_t)stream);
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

}  // extern "C"

namespace {

// Partial-sum slots of the step-level scratch for an H-row plane set of pitch `pitch`: the most
// blocks any engine launches at any width W <= pitch.  Every engine's block count grows with W,
// and the fused ADMM kernel launches the most blocks with 1-row strips, whatever strip height the
// built-in rule picks for the actual width.
int fields_partial_slots(int H, int pitch) {
    const Geom g{H, pitch, pitch};
    return std::max({admm_fused_blocks(g, 1), admm_plain_blocks(g), pdr_plain_blocks(g, PARTIAL_ROWS_MIN),
                     cp_blocks(g, PARTIAL_ROWS_MIN)});
}

}  // namespace

extern "C" {

size_t of_fields_bytes(int H, int pitch) {
    if (H < 1 || pitch < 1) return 0;
    const size_t plane = align_up((size_t)H * pitch * 4, 256);
    return (NFIELDS + 6) * plane + align_up((size_t)fields_partial_slots(H, pitch) * sizeof(double), 256) +
           align_up(sizeof(Misc), 256);
}

namespace {

// Step-level iterations of one method family: KIND_ADMM (rpADMMI / rpADMMII), KIND_PDR, KIND_CP.
enum { KIND_ADMM = 0, KIND_PDR = 1, KIND_CP = 2 };

of_status iterate_common(of_fields f, const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                         float a_tilde, const of_params *params, int iters, void *scratch, double *res2, void *stream,
                         int kind) {
    if (!params) return fail(OF_EINVAL, "params is NULL");
    of_status st = validate(params, H, W);
    if (st != OF_OK) return st;
    if (params->c_adapt_iters != 0)
        return fail(OF_EINVAL, "c_adapt_iters applies to whole solves, not to the step-level entry points");
    const int want = params->method == OF_PDR ? KIND_PDR : params->method == OF_CP ? KIND_CP : KIND_ADMM;
    if (want != kind) return fail(OF_EINVAL, "params->method does not match the entry point");
    const bool pdr = kind == KIND_PDR, cp = kind == KIND_CP, xb = pdr || cp;
    if (params->precision != OF_PREC_FP32) return fail(OF_EINVAL, "step-level entry points take FP32 fields");
    if (pitch < W || iters < 0) return fail(OF_EINVAL, "bad pitch or iteration count");
    if (kind == KIND_ADMM && !(a_tilde > 0.f)) return fail(OF_EINVAL, "a_tilde must be > 0");
    const bool has_w = params->beta != 0.f;
    float *need[] = {f.u, f.v, f.q11, f.q12, f.q21, f.q22};
    for (float *x : need)
        if (!x) return fail(OF_EINVAL, "NULL field pointer");
    if (has_w && (!f.w || !f.p1 || !f.p2)) return fail(OF_EINVAL, "beta > 0 needs w, p1, p2");
    if (kind == KIND_ADMM && !f.s) return fail(OF_EINVAL, "ADMM needs s");
    if (xb && (!f.ub || !f.vb || (has_w && !f.wb))) return fail(OF_EINVAL, "pDR and ALG1 need wb, ub, vb");
    if (!Ix || !Iy || !It) return fail(OF_EINVAL, "NULL linearisation data");
    if (!scratch) return fail(OF_EINVAL, "scratch is NULL (size: of_fields_bytes)");
    cudaStream_t s = (cudaStream_t)stream;
    const Geom g{H, W, pitch};
    const size_t plane = align_up((size_t)H * pitch * 4, 256);
    char *S = (char *)scratch;
    Fields user;
    float *uf[NFIELDS] = {f.w, f.u, f.v, f.p1, f.p2, f.q11, f.q12, f.q21, f.q22, f.s, f.wb, f.ub, f.vb};
    for (int k = 0; k < NFIELDS; ++k) user.f[k] = uf[k];
    // the scratch copy of the state (fused ADMM ping-pong).  Planes the caller left NULL are
    // never read or written by the engine in use; both buffers point them at one zeroed
    // scratch plane.
    Fields other = fields_at(S, plane);
    for (int k = 0; k < NFIELDS; ++k)
        if (!user.f[k]) user.f[k] = other.f[k];
    float *tmp = (float *)(S + NFIELDS * plane);
    // the scratch layout depends on (H, pitch) only, as of_fields_bytes does; the engine in use
    // must find room for its partial sums in it
    const int mb = fields_partial_slots(H, pitch);
    const int nb_used = pdr ? pdr_plain_blocks(g)
                            : cp ? cp_blocks(g)
                                 : (params->engine == OF_ENGINE_PLAIN ? admm_plain_blocks(g) : admm_fused_blocks(g));
    if (nb_used > mb) return fail(OF_EINVAL, "internal: partial sums exceed the scratch layout");
    double *partials = (double *)(S + (NFIELDS + 6) * plane);
    Misc *misc = (Misc *)(S + (NFIELDS + 6) * plane + align_up((size_t)mb * sizeof(double), 256));
    OF_CUDA(cudaMemsetAsync(misc, 0, sizeof(Misc), s));
    for (int k = 0; k < NFIELDS; ++k)
        if (!uf[k]) OF_CUDA(cudaMemset2DAsync(user.f[k], (size_t)pitch * 4, 0, (size_t)W * 4, H, s));
    const bool plain = params->engine == OF_ENGINE_PLAIN;
    const bool pingpong = !pdr && !plain;
    Fields bufs[2] = {user, other};
    of_params pp = *params;
    pp.a_tilde = xb ? 1.f : a_tilde;
    const Coefs k = coefs_of(&pp);
    const double rows = (double)H * W * (has_w ? 3.0 : 2.0);
    for (int it = 0; it < iters; ++it) {
        const bool check = params->tol > 0.0 && (it + 1) % 10 == 0;
        IterArgs a{};
        a.g = g;
        a.k = k;
        a.in = bufs[pingpong ? it & 1 : 0];
        a.out = bufs[pingpong ? (it + 1) & 1 : 0];
        a.Ix = Ix;
        a.Iy = Iy;
        a.It = It;
        a.ms_max = nullptr;
        a.partials = (check || it == iters - 1) ? partials : nullptr;
        a.done = params->tol > 0.0 ? &misc->done : nullptr;
        a.tmp = tmp;
        if (pdr) {
            if (plain) launch_pdr_plain(a, s);
            else launch_pdr_fused(a, PREC_F32, PREC_F32, s);
        } else if (cp) {
            launch_cp(a, PREC_F32, PREC_F32, s);
        } else {
            if (plain) launch_admm_plain(a, s);
            else launch_admm_fused(a, PREC_F32, PREC_F32, s);
        }
        const int nb = pdr ? pdr_plain_blocks(g) : cp ? cp_blocks(g) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g));
        if (check) {
            launch_reduce_check(partials, nb, &misc->res_check, rows, params->tol, &misc->done, &misc->iters, 10, s);
        }
    }
    if (pingpong && (iters & 1)) {
        // after an odd number of iterations the result sits in the scratch buffer; an early stop
        // (always after an even count) leaves it in the caller's planes.  Copy back unless stopped.
        Fields from = bufs[1], to = bufs[0];
        for (int q = 0; q < NFIELDS; ++q)
            if (!uf[q]) from.f[q] = to.f[q] = nullptr;
        launch_parity_fix(from, to, g, PREC_F32, PREC_F32, params->tol > 0.0 ? &misc->done : nullptr, 0, s);
    }
    if (res2) {
        const int nb = pdr ? pdr_plain_blocks(g) : cp ? cp_blocks(g) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g));
        if (iters > 0) launch_sum(partials, nb, &misc->res_final, s);
        Misc m;
        OF_CUDA(cudaMemcpyAsync(&m, misc, sizeof(Misc), cudaMemcpyDeviceToHost, s));
        OF_CUDA(cudaStreamSynchronize(s));
        *res2 = params->tol > 0.0 && m.done ? m.res_check : (iters > 0 ? m.res_final : 0.0);
    }
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

}  // namespace

of_status of_admm_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                          float a_tilde, const of_params *params, int iters, void *scratch, double *res2, void *stream) {
    return iterate_common(f, Ix, Iy, It, H, W, pitch, a_tilde, params, iters, scratch, res2, stream, KIND_ADMM);
}

of_status of_pdr_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                         const of_params *params, int iters, void *scratch, double *res2, void *stream) {
    return iterate_common(f, Ix, Iy, It, H, W, pitch, 1.f, params, iters, scratch, res2, stream, KIND_PDR);
}

of_status of_cp_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                        const of_params *params, int iters, void *scratch, double *res2, void *stream) {
    return iterate_common(f, Ix, Iy, It, H, W, pitch, 1.f, params, iters, scratch, res2, stream, KIND_CP);
}

of_status of_energy(const float *w, const float *u, const float *v, const float *s, const float *Ix, const float *Iy,
                    const float *It, int H, int W, int pitch, float beta, float lambda, double *energy,
                    double *dual_value, void *stream) {
    if (!u || !v || !Ix || !Iy || !It || !energy) return fail(OF_EINVAL, "NULL pointer");
    if (H < 1 || W < 1 || pitch < W) return fail(OF_EINVAL, "bad sizes or pitch");
    if (beta != 0.f && !w) return fail(OF_EINVAL, "beta > 0 needs w");
    const Geom g{H, W, pitch};
    const int nb = energy_blocks(g);
    double *buf = nullptr;
    OF_CUDA(cudaMalloc(&buf, (2 * (size_t)nb + 2) * sizeof(double)));
    cudaStream_t st = (cudaStream_t)stream;
    Fields f;
    for (int k = 0; k < NFIELDS; ++k) f.f[k] = nullptr;
    f.f[F_W] = (void *)w;
    f.f[F_U] = (void *)u;
    f.f[F_V] = (void *)v;
    f.f[F_S] = (void *)s;
    launch_energy(f, Ix, Iy, It, g, beta, lambda, PREC_F32, PREC_F32, buf, buf + nb, st);
    launch_sum(buf, nb, buf + 2 * nb, st);
    launch_sum(buf + nb, nb, buf + 2 * nb + 1, st);
    double h[2];
    cudaError_t e = cudaMemcpyAsync(h, buf + 2 * nb, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(OF_ECUDA, std::string("of_energy: ") + cudaGetErrorString(e));
    *energy = h[0];
    if (dual_value) *dual_value = s ? h[1] : NAN;
    return OF_OK;
}

}  // extern "C"
