// tvl1_step.cu -- stage-by-stage solves for the serving loop's continuous batching.
//
// A whole solve (tvl1_api.cu) runs one pair, or one fixed batch, through the coarse-to-fine
// schedule of Sec. 4 in a captured CUDA graph.  The serving loop instead keeps a changing set of
// requests in flight: each step advances every active pair by one stage -- one warp (one
// linearisation) of its current pyramid level -- and the inner iterations of all of them run in
// shared launches over a work-list rebuilt for the step: the streaming ADMM kernel's tiles (or,
// for pDR and ALG1, one grid slice per pair) of every pair at its own level and size.  A request
// that arrives joins at the next step; one that finishes its last stage leaves.  Per pair the
// kernels and their order are those of the whole solve, so a request's flow does not depend on
// the others in the step (the streaming kernel computes every pixel alike for any strip height
// and work-list, and it equals the level-resident engine bitwise).
//
// Each pair's descriptor lists its current state buffer first, so pairs whose ping-pong
// parities differ share one launch.  Pairs in the finest level's last warp with FP32 storage
// (16-bit storage with fp32_last_warp) run in a second group of launches with the FP32 kernels.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tvl1_plan.h"
#include "tvl1_step.h"

namespace tvl1 {

namespace {

cudaError_t grow_device(char **p, size_t *cap, size_t need, cudaStream_t s) {
    if (need <= *cap) return cudaSuccess;
    if (*p) cudaFreeAsync(*p, s);  // stream-ordered: work queued before still reads the old block
    *p = nullptr;
    *cap = 0;
    const size_t n = std::max(need, (size_t)1 << 20) * 3 / 2;
    cudaError_t e = cudaMallocAsync((void **)p, n, s);
    if (e == cudaSuccess) *cap = n;
    return e;
}

struct Bufs {
    Fields st[2];
    const void *dat[3];
};

Bufs bufs_of(const StepPair &q) {
    Bufs b;
    char *A = q.A;
    const Plan &pl = q.pl;
    if (q.in32) {
        b.st[0] = fields_at(A + pl.stA32, pl.plane32);
        b.st[1] = fields_at(A + pl.stB32, pl.plane32);
        for (int d = 0; d < 3; ++d) b.dat[d] = A + pl.data32 + d * pl.plane32;
    } else {
        b.st[0] = fields_at(A + pl.stA, pl.planeS);
        b.st[1] = fields_at(A + pl.stB, pl.planeS);
        for (int d = 0; d < 3; ++d) b.dat[d] = A + pl.data + d * pl.planeT;
    }
    return b;
}

Misc *misc_of(const StepPair &q) { return (Misc *)(q.A + q.pl.misc); }

}  // namespace

size_t step_pair_bytes(int H, int W, const of_params *p) { return make_plan(H, W, p).total; }

void step_pair_init(StepPair &q, char *region, int H, int W, const of_params *p) {
    q = StepPair();
    q.A = region;
    q.pl = make_plan(H, W, p);
    q.H = H;
    q.W = W;
    q.l = p->levels - 1;
    q.prec = q.pl.prec;
    q.pflow = q.pl.pflow;
}

void step_pair_start(StepPair &q, const float *I0, const float *I1, const of_params *p, cudaStream_t s) {
    const Plan &pl = q.pl;
    cudaMemcpy2DAsync(q.A + pl.img0[0], (size_t)pl.P[0] * 4, I0, (size_t)q.W * 4, (size_t)q.W * 4, q.H,
                      cudaMemcpyHostToDevice, s);
    cudaMemcpy2DAsync(q.A + pl.img1[0], (size_t)pl.P[0] * 4, I1, (size_t)q.W * 4, (size_t)q.W * 4, q.H,
                      cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(misc_of(q), 0, sizeof(Misc), s);
    const GaussTaps taps = gauss_taps(p->eta);
    for (int l = 1; l < pl.L; ++l) {
        launch_pyr_down((float *)(q.A + pl.img0[l - 1]), geom_of(pl, l - 1), (float *)(q.A + pl.img0[l]),
                        geom_of(pl, l), taps, (float *)(q.A + pl.blur), s);
        launch_pyr_down((float *)(q.A + pl.img1[l - 1]), geom_of(pl, l - 1), (float *)(q.A + pl.img1[l]),
                        geom_of(pl, l), taps, (float *)(q.A + pl.blur), s);
    }
}

void step_pair_finish(const StepPair &q, float *u, float *v, Misc *misc, cudaStream_t s) {
    const Plan &pl = q.pl;
    const int lo = pl.out_level;
    const size_t on = (size_t)pl.H[lo] * pl.P[lo];
    const float *out = (const float *)(q.A + pl.out);
    cudaMemcpy2DAsync(u, (size_t)pl.W[lo] * 4, out, (size_t)pl.P[lo] * 4, (size_t)pl.W[lo] * 4, pl.H[lo],
                      cudaMemcpyDeviceToHost, s);
    cudaMemcpy2DAsync(v, (size_t)pl.W[lo] * 4, out + on, (size_t)pl.P[lo] * 4, (size_t)pl.W[lo] * 4, pl.H[lo],
                      cudaMemcpyDeviceToHost, s);
    if (misc) cudaMemcpyAsync(misc, misc_of(q), sizeof(Misc), cudaMemcpyDeviceToHost, s);
}

StepTables::~StepTables() {
    for (int b = 0; b < NSTAGE; ++b) {
        if (ev[b]) cudaEventDestroy(ev[b]);
        if (host[b]) cudaFreeHost(host[b]);
    }
    if (dev) cudaFree(dev);
}

namespace {

// One group of pairs (same storage types) through `iters` inner iterations in shared launches.
cudaError_t run_group(std::vector<StepPair *> &G, const of_params *p, StepTables &T, int prec, int pflow,
                      cudaStream_t s) {
    const int n = (int)G.size();
    const bool pdr = p->method == OF_PDR, cp = p->method == OF_CP;
    const bool pingpong = !pdr;
    const bool has_w = p->beta != 0.f;
    const int SWD = admm_fused_strip_w(), WARPS = admm_fused_warps();
    // strip height: the built-in rule on the step's total strip rows, or the parameters' height
    long strip_rows = 0;
    Geom gmax{0, 0, 0};
    for (StepPair *q : G) {
        const Geom g = geom_of(q->pl, q->l);
        strip_rows += (long)((g.W + SWD - 1) / SWD) * g.H;
        gmax.H = std::max(gmax.H, g.H);
        gmax.W = std::max(gmax.W, g.W);
    }
    gmax.pitch = pitch_of(gmax.W);
    const int ty = p->rows_per_warp > 0 ? p->rows_per_warp : admm_fused_rows_per_warp(strip_rows, prec != PREC_F32);
    const int rows = ty * WARPS;
    int ntiles = 0;
    for (StepPair *q : G) {
        const Geom g = geom_of(q->pl, q->l);
        ntiles += ((g.W + SWD - 1) / SWD) * ((g.H + rows - 1) / rows);
    }
    const int Gb = cp ? cp_blocks(gmax) : pdr_plain_blocks(gmax);
    const size_t nparts = (pdr || cp) ? (size_t)n * Gb : (size_t)std::max(ntiles, 1);
    // table layout: PairIter[n] | PairScalars[n] | plist[n] | TileRef[ntiles] | partials
    const size_t o_pi = 0, o_ps = align_up(sizeof(PairIter) * n, 256);
    const size_t o_pl = o_ps + align_up(sizeof(PairScalars) * n, 256);
    const size_t o_tr = o_pl + align_up(sizeof(int) * n, 256);
    const size_t o_pa = o_tr + align_up(sizeof(TileRef) * (size_t)std::max(ntiles, 1), 256);
    const size_t tab = o_pa, total = o_pa + align_up(sizeof(double) * nparts, 256);
    cudaError_t e = grow_device(&T.dev, &T.dev_bytes, total, s);
    if (e != cudaSuccess) return e;
    // host staging: a ring of pinned buffers, each reused only after its last copy has run
    const int b = T.next;
    T.next = (T.next + 1) % StepTables::NSTAGE;
    if (T.ev[b]) cudaEventSynchronize(T.ev[b]);
    else if ((e = cudaEventCreateWithFlags(&T.ev[b], cudaEventDisableTiming)) != cudaSuccess) return e;
    if (tab > T.host_bytes[b]) {
        if (T.host[b]) cudaFreeHost(T.host[b]);
        T.host[b] = nullptr;
        T.host_bytes[b] = 0;
        if ((e = cudaHostAlloc((void **)&T.host[b], tab * 3 / 2, cudaHostAllocDefault)) != cudaSuccess) return e;
        T.host_bytes[b] = tab * 3 / 2;
    }
    char *h = T.host[b];
    memset(h, 0, tab);
    PairIter *pi = (PairIter *)(h + o_pi);
    PairScalars *ps = (PairScalars *)(h + o_ps);
    int *pl = (int *)(h + o_pl);
    TileRef *tr = (TileRef *)(h + o_tr);
    int t = 0;
    for (int k = 0; k < n; ++k) {
        StepPair &q = *G[k];
        const Geom g = geom_of(q.pl, q.l);
        const Bufs bf = bufs_of(q);
        Misc *m = misc_of(q);
        PairIter &P = pi[k];
        P.g = g;
        P.buf[0] = bf.st[q.cur];          // the current state first: parity 0 for every pair
        P.buf[1] = bf.st[q.cur ^ 1];
        P.Ix = bf.dat[0];
        P.Iy = bf.dat[1];
        P.It = bf.dat[2];
        P.ms_max = &m->ms_max;
        P.done = p->tol > 0.0 ? &m->done : nullptr;
        P.tmp = (float *)(q.A + q.pl.tmp);
        pl[k] = k;
        const int t0 = t;
        if (!(pdr || cp))
            for (int y = 0; y < (g.H + rows - 1) / rows; ++y)
                for (int x = 0; x < (g.W + SWD - 1) / SWD; ++x) tr[t++] = TileRef{k, x, y, 0};
        ps[k].res_check = &m->res_check;
        ps[k].res_final = &m->res_final;
        ps[k].done = &m->done;
        ps[k].iters = &m->iters;
        ps[k].rows = (double)g.H * g.W * (has_w ? 3.0 : 2.0);
        ps[k].part_begin = (pdr || cp) ? k * Gb : t0;
        ps[k].part_end = (pdr || cp) ? (k + 1) * Gb : t;
        ps[k].timeout = &m->timeout;
    }
    if ((e = cudaMemcpyAsync(T.dev, h, tab, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(T.ev[b], s)) != cudaSuccess) return e;
    const PairIter *dpi = (const PairIter *)(T.dev + o_pi);
    const PairScalars *dps = (const PairScalars *)(T.dev + o_ps);
    const int *dpl = (const int *)(T.dev + o_pl);
    const TileRef *dtr = (const TileRef *)(T.dev + o_tr);
    double *part = (double *)(T.dev + o_pa);
    const Coefs k = coefs_of(p);
    for (int it = 0; it < p->iters; ++it) {
        const bool check = p->tol > 0.0 && (it + 1) % 10 == 0;
        IterArgs a{};
        a.k = k;
        a.pairs = dpi;
        a.partials = (check || it == p->iters - 1) ? part : nullptr;
        if (pdr) {
            a.g = gmax;
            a.ntiles = n;
            a.plist = dpl;
            a.parity = 0;
            launch_pdr_fused(a, prec, pflow, s);
        } else if (cp) {
            a.g = gmax;
            a.ntiles = n;
            a.plist = dpl;
            a.parity = it & 1;
            launch_cp(a, prec, pflow, s);
        } else {
            a.tiles = dtr;
            a.ntiles = ntiles;
            a.tile_h = ty;
            a.parity = it & 1;
            launch_admm_fused(a, prec, pflow, s);
        }
        if (check) launch_reduce_check_batched(part, dps, n, p->tol, 10, 0, s);
    }
    if (p->iters > 0) {
        launch_count_iters_batched(dps, n, p->tol > 0.0 ? p->iters % 10 : p->iters, p->tol > 0.0, s);
        launch_reduce_check_batched(part, dps, n, 0.0, 0, 1, s);  // residual of the stage's last iteration
    }
    // the state after the stage: buffer cur ^ (iters & 1) for the ping-pong engines, unless the pair
    // stopped (always after an even count), which leaves it in buffer cur: copy it over then
    for (StepPair *q : G) {
        if (!pingpong || !(p->iters & 1)) continue;
        const Bufs bf = bufs_of(*q);
        if (p->tol > 0.0)
            launch_parity_fix(bf.st[q->cur], bf.st[q->cur ^ 1], geom_of(q->pl, q->l), cp ? pflow : prec, pflow,
                              &misc_of(*q)->done, 1, s);
        q->cur ^= 1;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t step_run(std::vector<StepPair *> &act, const of_params *p, StepTables &T, cudaStream_t s) {
    const bool pdr = p->method == OF_PDR, cp = p->method == OF_CP;
    const bool has_w = p->beta != 0.f;
    std::vector<StepPair *> g16, g32;
    // stage set-up of every pair: level transfer at a level's first warp, then the warping
    for (StepPair *qp : act) {
        StepPair &q = *qp;
        const Plan &pl = q.pl;
        const Geom g = geom_of(pl, q.l);
        Bufs bf = bufs_of(q);
        if (q.wp == 0) {
            if (q.l == pl.L - 1) {
                launch_fill(bf.st[q.cur].f + F_W, q.pflow, 3, g, 0.f, s);
            } else {
                const Geom gc = geom_of(pl, q.l + 1);
                const int nxt = q.cur ^ 1;
                launch_upsample(bf.st[q.cur].f[F_W], gc, bf.st[nxt].f[F_W], g, 1.f, q.pflow, s);
                launch_upsample(bf.st[q.cur].f[F_U], gc, bf.st[nxt].f[F_U], g, (float)g.W / (float)gc.W, q.pflow, s);
                launch_upsample(bf.st[q.cur].f[F_V], gc, bf.st[nxt].f[F_V], g, (float)g.H / (float)gc.H, q.pflow, s);
                q.cur = nxt;
            }
            // duals restart at 0 (ALG1 keeps its dual in the flow fields' type)
            launch_fill(bf.st[q.cur].f + F_P1, cp ? q.pflow : q.prec, F_S - F_P1 + 1, g, 0.f, s);
            if (!has_w) launch_fill(bf.st[q.cur].f + F_W, q.pflow, 1, g, 0.f, s);
            if (pdr || cp) {
                const void *src[3] = {bf.st[q.cur].f[F_W], bf.st[q.cur].f[F_U], bf.st[q.cur].f[F_V]};
                void *dst[3] = {bf.st[q.cur].f[F_WB], bf.st[q.cur].f[F_UB], bf.st[q.cur].f[F_VB]};
                launch_copy_planes(src, dst, 3, g, q.pflow, s);
            }
            launch_derivatives((float *)(q.A + pl.img1[q.l]), g, (float *)(q.A + pl.I1x), (float *)(q.A + pl.I1y), s);
        }
        if (pl.use32_last && q.l == 0 && q.wp == p->warps - 1 && !q.in32) {
            // precision policy: the finest level's last warp runs with FP32 storage
            const Fields to = fields_at(q.A + pl.stA32, pl.plane32);
            launch_convert(bf.st[q.cur].f + F_W, q.pflow, to.f + F_W, PREC_F32, 3, g, s);
            launch_convert(bf.st[q.cur].f + F_P1, cp ? q.pflow : q.prec, to.f + F_P1, PREC_F32, F_S - F_P1 + 1, g, s);
            launch_convert(bf.st[q.cur].f + F_WB, q.pflow, to.f + F_WB, PREC_F32, 3, g, s);
            q.in32 = true;
            q.cur = 0;
            q.prec = q.pflow = PREC_F32;
            bf = bufs_of(q);
        }
        Misc *m = misc_of(q);
        cudaMemsetAsync(&m->ms_max, 0, sizeof(float) + sizeof(int), s);  // ms_max and the stop flag
        launch_warp((float *)(q.A + pl.img0[q.l]), (float *)(q.A + pl.img1[q.l]), (float *)(q.A + pl.I1x),
                    (float *)(q.A + pl.I1y), bf.st[q.cur].f[F_U], bf.st[q.cur].f[F_V], g, p->beta, (void *)bf.dat[0],
                    (void *)bf.dat[1], (void *)bf.dat[2], &m->ms_max, q.prec, q.pflow, s);
        (q.in32 && pl.prec != PREC_F32 ? g32 : g16).push_back(qp);
    }
    cudaError_t e = cudaSuccess;
    if (!g16.empty()) e = run_group(g16, p, T, g16[0]->prec, g16[0]->pflow, s);
    if (e == cudaSuccess && !g32.empty()) e = run_group(g32, p, T, PREC_F32, PREC_F32, s);
    if (e != cudaSuccess) return e;
    // advance; a pair done with its output level writes its energy and flow
    for (StepPair *qp : act) {
        StepPair &q = *qp;
        if (++q.wp < p->warps) continue;
        if (q.l > q.pl.out_level) {
            --q.l;
            q.wp = 0;
            continue;
        }
        const Plan &pl = q.pl;
        const Geom g = geom_of(pl, q.l);
        const Bufs bf = bufs_of(q);
        Misc *m = misc_of(q);
        const int mb = pl.max_blocks;
        double *pe = (double *)(q.A + pl.partials) + mb, *pd = (double *)(q.A + pl.partials) + 2 * mb;
        Fields fe = bf.st[q.cur];
        if (pdr || cp) fe.f[F_S] = nullptr;
        if (!has_w) fe.f[F_W] = nullptr;
        launch_energy(fe, bf.dat[0], bf.dat[1], bf.dat[2], g, p->beta, p->lambda, q.prec, q.pflow, pe, pd, s);
        launch_sum(pe, energy_blocks(g), &m->energy, s);
        launch_sum(pd, energy_blocks(g), &m->dual, s);
        float *out = (float *)(q.A + pl.out);
        const size_t on = (size_t)pl.H[pl.out_level] * pl.P[pl.out_level];
        const void *src[3] = {bf.st[q.cur].f[F_U], bf.st[q.cur].f[F_V], bf.st[q.cur].f[F_W]};
        void *dst[3] = {out, out + on, out + 2 * on};
        launch_convert(src, q.pflow, dst, PREC_F32, 3, g, s);
        q.finished = true;
    }
    return cudaGetLastError();
}

}  // namespace tvl1
