// tvl1_api.cu -- host runtime and C ABI of the GB300 TV-L1 optical-flow library
// (include/tvl1flow.h).  It plans the per-pair device arena, enqueues the whole coarse-to-fine
// schedule (pyramid, levels, warps, inner iterations; Sec. 3-4 of the paper) as kernels on a
// stream, captures it once per (size, parameters) into a CUDA graph and replays the graph on
// later calls.  No arithmetic of the method runs on the host.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"

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

constexpr int MAX_LEVELS = 16;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int level_size(int n, float eta) {
    int m = (int)floor((double)n * (double)eta + 0.5);
    return m < 1 ? 1 : m;
}

// Row pitch in elements: a multiple of 64 elements (>= 128 bytes for every storage type).
int pitch_of(int W) { return (int)align_up((size_t)W, 64); }

struct Plan {
    int L = 0, out_level = 0, prec = PREC_F32;
    bool use32_last = false;
    int H[MAX_LEVELS], W[MAX_LEVELS], P[MAX_LEVELS];
    size_t plane32 = 0, planeT = 0;  // bytes of one finest-size plane in FP32 / storage precision
    size_t img0[MAX_LEVELS], img1[MAX_LEVELS];
    size_t I1x, I1y, blur, stA, stB, stA32, stB32, data, data32, tmp, partials, misc, out;
    int max_blocks = 0;
    size_t total = 0;
};

// Device scalars at plan.misc.
struct Misc {
    float ms_max;
    int done;
    long long iters;
    double res_check, res_final, energy, dual;
};

of_status validate(const of_params *p, int H, int W) {
    if (!p) return fail(OF_EINVAL, "params is NULL");
    if (H < 1 || W < 1) return fail(OF_EINVAL, "image sizes must be >= 1");
    if (p->method < 0 || p->method > 2) return fail(OF_EINVAL, "unknown method");
    if (!(p->lambda > 0.f) || !isfinite(p->lambda)) return fail(OF_EINVAL, "lambda must be > 0");
    if (!(p->beta >= 0.f) || !isfinite(p->beta)) return fail(OF_EINVAL, "beta must be >= 0");
    if (p->method != OF_PDR) {
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
    if (p->engine < 0 || p->engine > 1) return fail(OF_EINVAL, "unknown engine");
    if (p->engine == OF_ENGINE_PLAIN && p->precision != OF_PREC_FP32)
        return fail(OF_EINVAL, "the plain engine runs in FP32 only");
    if (p->out_level < 0 || p->out_level >= p->levels) return fail(OF_EINVAL, "out_level must lie in [0, levels)");
    return OF_OK;
}

Plan make_plan(int H, int W, const of_params *p) {
    Plan pl;
    pl.L = p->levels;
    pl.out_level = p->out_level;
    pl.prec = p->precision;
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
    pl.stA = take(NFIELDS * pl.planeT);
    pl.stB = take(NFIELDS * pl.planeT);
    pl.data = take(3 * pl.planeT);
    if (pl.use32_last) {
        pl.stA32 = take(NFIELDS * pl.plane32);
        pl.stB32 = take(NFIELDS * pl.plane32);
        pl.data32 = take(3 * pl.plane32);
    } else {
        pl.stA32 = pl.stB32 = pl.data32 = 0;
    }
    pl.tmp = take(6 * pl.plane32);
    Geom g0{pl.H[0], pl.W[0], pl.P[0]};
    int mb = admm_fused_blocks(g0);
    mb = mb > admm_plain_blocks(g0) ? mb : admm_plain_blocks(g0);
    mb = mb > pdr_plain_blocks(g0) ? mb : pdr_plain_blocks(g0);
    mb = mb > energy_blocks(g0) ? mb : energy_blocks(g0);
    pl.max_blocks = mb;
    pl.partials = take(3 * (size_t)mb * sizeof(double));
    pl.misc = take(sizeof(Misc));
    const size_t nout = (size_t)pl.H[pl.out_level] * pl.P[pl.out_level];
    pl.out = take(3 * nout * 4);
    pl.total = off;
    return pl;
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
    k.method = p->method;
    k.gs_sweeps = p->gs_sweeps;
    return k;
}

Fields fields_at(char *base, size_t plane) {
    Fields f;
    for (int k = 0; k < NFIELDS; ++k) f.f[k] = base + (size_t)k * plane;
    return f;
}

// Enqueues the whole schedule of one pair on `s` (arena pointers only: graph-capturable).
void enqueue_solve(of_ctx *ctx, const Plan &pl, const of_params *p, cudaStream_t s) {
    char *A = ctx->arena;
    Misc *misc = (Misc *)(A + pl.misc);
    double *partials = (double *)(A + pl.partials);
    const int mb = pl.max_blocks;
    const bool has_w = p->beta != 0.f;
    const bool pdr = p->method == OF_PDR;
    const bool plain = p->engine == OF_ENGINE_PLAIN;
    const GaussTaps taps = gauss_taps(p->eta);
    const Coefs k = coefs_of(p);
    cudaMemsetAsync(misc, 0, sizeof(Misc), s);

    auto geom = [&](int l) { return Geom{pl.H[l], pl.W[l], pl.P[l]}; };
    for (int l = 1; l < pl.L; ++l) {
        launch_pyr_down((float *)(A + pl.img0[l - 1]), geom(l - 1), (float *)(A + pl.img0[l]), geom(l), taps,
                        (float *)(A + pl.blur), s);
        launch_pyr_down((float *)(A + pl.img1[l - 1]), geom(l - 1), (float *)(A + pl.img1[l]), geom(l), taps,
                        (float *)(A + pl.blur), s);
    }

    Fields buf[2] = {fields_at(A + pl.stA, pl.planeT), fields_at(A + pl.stB, pl.planeT)};
    Fields buf32[2] = {fields_at(A + pl.stA32, pl.plane32), fields_at(A + pl.stB32, pl.plane32)};
    int cur = 0;
    int prec = pl.prec;
    Fields *bufs = buf;
    const void *data[3] = {A + pl.data, A + pl.data + pl.planeT, A + pl.data + 2 * pl.planeT};
    const void *data32[3] = {A + pl.data32, A + pl.data32 + pl.plane32, A + pl.data32 + 2 * pl.plane32};
    Geom last_g = geom(pl.L - 1);

    for (int l = pl.L - 1; l >= pl.out_level; --l) {
        const Geom g = geom(l);
        last_g = g;
        if (l == pl.L - 1) {
            launch_fill(bufs[cur].f, prec, NFIELDS, g, 0.f, s);
        } else {
            const Geom gc = geom(l + 1);
            const int nxt = cur ^ 1;
            launch_upsample(bufs[cur].f[F_W], gc, bufs[nxt].f[F_W], g, 1.f, prec, s);
            launch_upsample(bufs[cur].f[F_U], gc, bufs[nxt].f[F_U], g, (float)g.W / (float)gc.W, prec, s);
            launch_upsample(bufs[cur].f[F_V], gc, bufs[nxt].f[F_V], g, (float)g.H / (float)gc.H, prec, s);
            launch_fill(bufs[nxt].f + F_P1, prec, NFIELDS - F_P1, g, 0.f, s);
            cur = nxt;
        }
        if (!has_w) launch_fill(bufs[cur].f + F_W, prec, 1, g, 0.f, s);
        if (pdr) {
            const void *src[3] = {bufs[cur].f[F_W], bufs[cur].f[F_U], bufs[cur].f[F_V]};
            void *dst[3] = {bufs[cur].f[F_WB], bufs[cur].f[F_UB], bufs[cur].f[F_VB]};
            launch_copy_planes(src, dst, 3, g, prec, s);
        }
        launch_derivatives((float *)(A + pl.img1[l]), g, (float *)(A + pl.I1x), (float *)(A + pl.I1y), s);
        const double rows = (double)g.H * g.W * (has_w ? 3.0 : 2.0);
        for (int wp = 0; wp < p->warps; ++wp) {
            const bool last_warp = (l == pl.out_level) && (wp == p->warps - 1);
            const void *const *dat = data;
            if (pl.use32_last && l == 0 && wp == p->warps - 1) {
                // precision policy: the finest level's last warp runs with FP32 storage
                launch_convert(bufs[cur].f, prec, buf32[0].f, PREC_F32, NFIELDS, g, s);
                bufs = buf32;
                cur = 0;
                prec = PREC_F32;
            }
            if (prec == PREC_F32 && bufs == buf32) dat = data32;
            cudaMemsetAsync(&misc->ms_max, 0, sizeof(float) + sizeof(int), s);  // ms_max and done
            launch_warp((float *)(A + pl.img0[l]), (float *)(A + pl.img1[l]), (float *)(A + pl.I1x),
                        (float *)(A + pl.I1y), bufs[cur].f[F_U], bufs[cur].f[F_V], g, p->beta, (void *)dat[0],
                        (void *)dat[1], (void *)dat[2], &misc->ms_max, prec, s);
            const bool pingpong = !pdr && !plain;
            const int start = cur;
            for (int it = 0; it < p->iters; ++it) {
                const bool check = p->tol > 0.0 && (it + 1) % 10 == 0;
                const bool final_it = last_warp && it == p->iters - 1;
                IterArgs a;
                a.g = g;
                a.k = k;
                a.in = bufs[pingpong ? (start + it) & 1 : start];
                a.out = bufs[pingpong ? (start + it + 1) & 1 : start];
                a.Ix = dat[0];
                a.Iy = dat[1];
                a.It = dat[2];
                a.ms_max = &misc->ms_max;
                a.partials = (check || final_it) ? partials : nullptr;
                a.done = p->tol > 0.0 ? &misc->done : nullptr;
                a.tmp = (float *)(A + pl.tmp);
                if (pdr) {
                    if (plain) launch_pdr_plain(a, s);
                    else launch_pdr_fused(a, prec, s);
                } else {
                    if (plain) launch_admm_plain(a, s);
                    else launch_admm_fused(a, prec, s);
                }
                if (check) {
                    const int nb = pdr ? pdr_plain_blocks(g) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g));
                    launch_reduce_check(partials, nb, &misc->res_check, rows, p->tol, &misc->done, &misc->iters, 10, s);
                }
            }
            if (p->tol > 0.0) launch_count_iters(&misc->iters, &misc->done, p->iters % 10, s);
            else launch_count_iters(&misc->iters, nullptr, p->iters, s);
            if (pingpong) {
                const int fin = (start + p->iters) & 1;
                if (p->tol > 0.0 && (p->iters & 1)) launch_parity_fix(bufs[start], bufs[fin], g, prec, &misc->done, 1, s);
                cur = fin;
            }
            if (last_warp && p->iters > 0) {
                const int nb = pdr ? pdr_plain_blocks(g) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g));
                launch_sum(partials, nb, &misc->res_final, s);
            }
        }
        if (l == pl.out_level) {
            double *pe = partials + mb, *pd = partials + 2 * mb;
            Fields fe = bufs[cur];
            if (pdr) fe.f[F_S] = nullptr;
            if (!has_w) fe.f[F_W] = nullptr;
            const void *const *dat = (prec == PREC_F32 && bufs == buf32) ? data32 : data;
            launch_energy(fe, dat[0], dat[1], dat[2], g, p->beta, p->lambda, prec, pe, pd, s);
            launch_sum(pe, energy_blocks(g), &misc->energy, s);
            launch_sum(pd, energy_blocks(g), &misc->dual, s);
            Geom go = g;
            float *out = (float *)(A + pl.out);
            const size_t on = (size_t)pl.H[pl.out_level] * pl.P[pl.out_level];
            const void *src[3] = {bufs[cur].f[F_U], bufs[cur].f[F_V], bufs[cur].f[F_W]};
            void *dst[3] = {out, out + on, out + 2 * on};
            launch_convert(src, prec, dst, PREC_F32, 3, go, s);
        }
    }
    (void)last_g;
}

std::string plan_key(int H, int W, const of_params *p) {
    of_params q;
    memset(&q, 0, sizeof(q));
    q = *p;
    std::string key((const char *)&H, sizeof(int));
    key.append((const char *)&W, sizeof(int));
    key.append((const char *)&q, sizeof(q));
    return key;
}

of_status get_graph(of_ctx *ctx, const Plan &pl, int H, int W, const of_params *p, cudaGraphExec_t *out) {
    const std::string key = plan_key(H, W, p);
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        *out = it->second.exec;
        return OF_OK;
    }
    GraphEntry ge;
    OF_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    enqueue_solve(ctx, pl, p, ctx->cap);
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &ge.graph);
    if (e != cudaSuccess) return fail(OF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(ge.graph);
        return fail(OF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    ctx->graphs[key] = ge;
    *out = ge.exec;
    return OF_OK;
}

of_status read_stats(of_ctx *ctx, const Plan &pl, const of_params *p, cudaStream_t s, of_stats *stats) {
    Misc m;
    OF_CUDA(cudaMemcpyAsync(&m, ctx->arena + pl.misc, sizeof(Misc), cudaMemcpyDeviceToHost, s));
    OF_CUDA(cudaStreamSynchronize(s));
    const Geom g{pl.H[pl.out_level], pl.W[pl.out_level], pl.P[pl.out_level]};
    const double rows = (double)g.H * g.W * (p->beta != 0.f ? 3.0 : 2.0);
    stats->iters_run = m.iters;
    stats->residual = p->iters > 0 ? sqrt(m.res_final / rows) : 0.0;
    stats->energy = m.energy;
    stats->dual_value = p->method == OF_PDR ? NAN : m.dual;
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
    p->engine = OF_ENGINE_FUSED;
    p->out_level = 0;
}

of_status of_create(of_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(OF_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    OF_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(OF_EINVAL, "no such CUDA device");
    OF_CUDA(cudaSetDevice(device));
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
    const Plan pl = make_plan(H, W, params);
    if (ensure_arena(ctx, pl.total) != OF_OK) return -1;
    cudaGraphExec_t ge;
    if (get_graph(ctx, pl, H, W, params, &ge) != OF_OK) return -1;
    cudaGraph_t g = ctx->graphs[plan_key(H, W, params)].graph;
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

of_status of_solve(of_ctx *ctx, const float *I0, const float *I1, int H, int W, int pitch, const of_params *params,
                   float *u, float *v, float *w, int out_pitch, void *stream, of_stats *stats) {
    if (!ctx) return fail(OF_EINVAL, "ctx is NULL");
    of_status st = validate(params, H, W);
    if (st != OF_OK) return st;
    if (!I0 || !I1 || !u || !v) return fail(OF_EINVAL, "NULL image or output pointer");
    if (pitch < W) return fail(OF_EINVAL, "pitch < W");
    OF_CUDA(cudaSetDevice(ctx->device));
    const Plan pl = make_plan(H, W, params);
    if (out_pitch < pl.W[pl.out_level]) return fail(OF_EINVAL, "out_pitch smaller than the output width");
    st = ensure_arena(ctx, pl.total);
    if (st != OF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaGraphExec_t ge;
    st = get_graph(ctx, pl, H, W, params, &ge);
    if (st != OF_OK) return st;
    char *A = ctx->arena;
    OF_CUDA(cudaMemcpy2DAsync(A + pl.img0[0], (size_t)pl.P[0] * 4, I0, (size_t)pitch * 4, (size_t)W * 4, H,
                              cudaMemcpyDeviceToDevice, s));
    OF_CUDA(cudaMemcpy2DAsync(A + pl.img1[0], (size_t)pl.P[0] * 4, I1, (size_t)pitch * 4, (size_t)W * 4, H,
                              cudaMemcpyDeviceToDevice, s));
    if (stats) OF_CUDA(cudaEventRecord(ctx->ev0, s));
    OF_CUDA(cudaGraphLaunch(ge, s));
    if (stats) OF_CUDA(cudaEventRecord(ctx->ev1, s));
    const int lo = pl.out_level;
    const size_t on = (size_t)pl.H[lo] * pl.P[lo];
    float *out = (float *)(A + pl.out);
    float *dst[3] = {u, v, w};
    for (int k = 0; k < 3; ++k)
        if (dst[k])
            OF_CUDA(cudaMemcpy2DAsync(dst[k], (size_t)out_pitch * 4, out + k * on, (size_t)pl.P[lo] * 4,
                                      (size_t)pl.W[lo] * 4, pl.H[lo], cudaMemcpyDeviceToDevice, s));
    if (stats) {
        st = read_stats(ctx, pl, params, s, stats);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        stats->ms = ms;
        if (st != OF_OK) return st;
    }
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

of_status of_solve_host(of_ctx *ctx, const float *I0, const float *I1, int H, int W, const of_params *params,
                        float *u, float *v, float *w, void *stream, of_stats *stats) {
    if (!ctx) return fail(OF_EINVAL, "ctx is NULL");
    of_status st = validate(params, H, W);
    if (st != OF_OK) return st;
    if (!I0 || !I1 || !u || !v) return fail(OF_EINVAL, "NULL image or output pointer");
    OF_CUDA(cudaSetDevice(ctx->device));
    const Plan pl = make_plan(H, W, params);
    st = ensure_arena(ctx, pl.total);
    if (st != OF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaGraphExec_t ge;
    st = get_graph(ctx, pl, H, W, params, &ge);
    if (st != OF_OK) return st;
    char *A = ctx->arena;
    OF_CUDA(cudaMemcpy2DAsync(A + pl.img0[0], (size_t)pl.P[0] * 4, I0, (size_t)W * 4, (size_t)W * 4, H,
                              cudaMemcpyHostToDevice, s));
    OF_CUDA(cudaMemcpy2DAsync(A + pl.img1[0], (size_t)pl.P[0] * 4, I1, (size_t)W * 4, (size_t)W * 4, H,
                              cudaMemcpyHostToDevice, s));
    if (stats) OF_CUDA(cudaEventRecord(ctx->ev0, s));
    OF_CUDA(cudaGraphLaunch(ge, s));
    if (stats) OF_CUDA(cudaEventRecord(ctx->ev1, s));
    const int lo = pl.out_level;
    const size_t on = (size_t)pl.H[lo] * pl.P[lo];
    float *out = (float *)(A + pl.out);
    float *dst[3] = {u, v, w};
    for (int k = 0; k < 3; ++k)
        if (dst[k])
            OF_CUDA(cudaMemcpy2DAsync(dst[k], (size_t)pl.W[lo] * 4, out + k * on, (size_t)pl.P[lo] * 4,
                                      (size_t)pl.W[lo] * 4, pl.H[lo], cudaMemcpyDeviceToHost, s));
    if (stats) {
        st = read_stats(ctx, pl, params, s, stats);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        stats->ms = ms;
        if (st != OF_OK) return st;
    }
    OF_CUDA(cudaStreamSynchronize(s));
    return OF_OK;
}

}  // extern "C"

int tvl1_solve_async(of_ctx *ctx, const float *I0, const float *I1, int H, int W, const void *params_v, float *u,
                     float *v, cudaStream_t s) {
    const of_params *params = (const of_params *)params_v;
    of_status st = validate(params, H, W);
    if (st != OF_OK) return st;
    OF_CUDA(cudaSetDevice(ctx->device));
    const Plan pl = make_plan(H, W, params);
    st = ensure_arena(ctx, pl.total);
    if (st != OF_OK) return st;
    cudaGraphExec_t ge;
    st = get_graph(ctx, pl, H, W, params, &ge);
    if (st != OF_OK) return st;
    char *A = ctx->arena;
    OF_CUDA(cudaMemcpy2DAsync(A + pl.img0[0], (size_t)pl.P[0] * 4, I0, (size_t)W * 4, (size_t)W * 4, H,
                              cudaMemcpyHostToDevice, s));
    OF_CUDA(cudaMemcpy2DAsync(A + pl.img1[0], (size_t)pl.P[0] * 4, I1, (size_t)W * 4, (size_t)W * 4, H,
                              cudaMemcpyHostToDevice, s));
    OF_CUDA(cudaGraphLaunch(ge, s));
    const int lo = pl.out_level;
    const size_t on = (size_t)pl.H[lo] * pl.P[lo];
    float *out = (float *)(A + pl.out);
    OF_CUDA(cudaMemcpy2DAsync(u, (size_t)pl.W[lo] * 4, out, (size_t)pl.P[lo] * 4, (size_t)pl.W[lo] * 4, pl.H[lo],
                              cudaMemcpyDeviceToHost, s));
    OF_CUDA(cudaMemcpy2DAsync(v, (size_t)pl.W[lo] * 4, out + on, (size_t)pl.P[lo] * 4, (size_t)pl.W[lo] * 4,
                              pl.H[lo], cudaMemcpyDeviceToHost, s));
    return OF_OK;
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
    launch_warp(I0, I1, I1x, I1y, u0, v0, Geom{H, W, pitch}, beta, Ix, Iy, It, ms_max, PREC_F32, (cudaStream_t)stream);
    OF_CUDA(cudaGetLastError());
    return OF_OK;
}

size_t of_fields_bytes(int H, int pitch) {
    if (H < 1 || pitch < 1) return 0;
    const size_t plane = align_up((size_t)H * pitch * 4, 256);
    Geom g{H, pitch, pitch};
    int mb = admm_fused_blocks(g);
    if (admm_plain_blocks(g) > mb) mb = admm_plain_blocks(g);
    if (pdr_plain_blocks(g) > mb) mb = pdr_plain_blocks(g);
    return (NFIELDS + 6) * plane + align_up((size_t)mb * sizeof(double), 256) + align_up(sizeof(Misc), 256);
}

namespace {

of_status iterate_common(of_fields f, const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                         float a_tilde, const of_params *params, int iters, void *scratch, double *res2, void *stream,
                         bool pdr) {
    if (!params) return fail(OF_EINVAL, "params is NULL");
    of_status st = validate(params, H, W);
    if (st != OF_OK) return st;
    if ((params->method == OF_PDR) != pdr) return fail(OF_EINVAL, "params->method does not match the entry point");
    if (params->precision != OF_PREC_FP32) return fail(OF_EINVAL, "step-level entry points take FP32 fields");
    if (pitch < W || iters < 0) return fail(OF_EINVAL, "bad pitch or iteration count");
    if (!pdr && !(a_tilde > 0.f)) return fail(OF_EINVAL, "a_tilde must be > 0");
    const bool has_w = params->beta != 0.f;
    float *need[] = {f.u, f.v, f.q11, f.q12, f.q21, f.q22};
    for (float *x : need)
        if (!x) return fail(OF_EINVAL, "NULL field pointer");
    if (has_w && (!f.w || !f.p1 || !f.p2)) return fail(OF_EINVAL, "beta > 0 needs w, p1, p2");
    if (!pdr && !f.s) return fail(OF_EINVAL, "ADMM needs s");
    if (pdr && (!f.ub || !f.vb || (has_w && !f.wb))) return fail(OF_EINVAL, "pDR needs wb, ub, vb");
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
    int mb = admm_fused_blocks(g);
    if (admm_plain_blocks(g) > mb) mb = admm_plain_blocks(g);
    if (pdr_plain_blocks(g) > mb) mb = pdr_plain_blocks(g);
    double *partials = (double *)(S + (NFIELDS + 6) * plane);
    Misc *misc = (Misc *)(S + (NFIELDS + 6) * plane + align_up((size_t)mb * sizeof(double), 256));
    OF_CUDA(cudaMemsetAsync(misc, 0, sizeof(Misc), s));
    for (int k = 0; k < NFIELDS; ++k)
        if (!uf[k]) OF_CUDA(cudaMemset2DAsync(user.f[k], (size_t)pitch * 4, 0, (size_t)W * 4, H, s));
    const bool plain = params->engine == OF_ENGINE_PLAIN;
    const bool pingpong = !pdr && !plain;
    Fields bufs[2] = {user, other};
    of_params pp = *params;
    pp.a_tilde = pdr ? 1.f : a_tilde;
    const Coefs k = coefs_of(&pp);
    const double rows = (double)H * W * (has_w ? 3.0 : 2.0);
    for (int it = 0; it < iters; ++it) {
        const bool check = params->tol > 0.0 && (it + 1) % 10 == 0;
        IterArgs a;
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
            else launch_pdr_fused(a, PREC_F32, s);
        } else {
            if (plain) launch_admm_plain(a, s);
            else launch_admm_fused(a, PREC_F32, s);
        }
        if (check) {
            const int nb = pdr ? pdr_plain_blocks(g) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g));
            launch_reduce_check(partials, nb, &misc->res_check, rows, params->tol, &misc->done, &misc->iters, 10, s);
        }
    }
    if (pingpong && (iters & 1)) {
        // after an odd number of iterations the result sits in the scratch buffer; an early stop
        // (always after an even count) leaves it in the caller's planes.  Copy back unless stopped.
        Fields from = bufs[1], to = bufs[0];
        for (int q = 0; q < NFIELDS; ++q)
            if (!uf[q]) from.f[q] = to.f[q] = nullptr;
        launch_parity_fix(from, to, g, PREC_F32, params->tol > 0.0 ? &misc->done : nullptr, 0, s);
    }
    if (res2) {
        const int nb = pdr ? pdr_plain_blocks(g) : (plain ? admm_plain_blocks(g) : admm_fused_blocks(g));
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
    return iterate_common(f, Ix, Iy, It, H, W, pitch, a_tilde, params, iters, scratch, res2, stream, false);
}

of_status of_pdr_iterate(of_fields f, const float *Ix, const float *Iy, const float *It, int H, int W, int pitch,
                         const of_params *params, int iters, void *scratch, double *res2, void *stream) {
    return iterate_common(f, Ix, Iy, It, H, W, pitch, 1.f, params, iters, scratch, res2, stream, true);
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
    launch_energy(f, Ix, Iy, It, g, beta, lambda, PREC_F32, buf, buf + nb, st);
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
