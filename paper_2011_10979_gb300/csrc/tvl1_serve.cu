// tvl1_serve.cu -- the serving loop of the C ABI (include/tvl1flow.h).
//
// The paper solves one pair at a time; serving is this library's addition.  The loop runs on its
// own host thread and CUDA stream and batches continuously across image sizes:
//  - requests wait in a FIFO queue and are admitted while at most `max_active` are in flight and
//    the device bytes of all admitted requests stay within the HBM budget (a request's bytes are
//    those of its solve's arena, taken from a memory pool of the server's own; a request larger
//    than the whole budget is rejected with OF_ENOMEM);
//  - an admitted request's images go to the device and its pyramid is built at once;
//  - each step (tvl1_step.cu) advances every admitted request by one warp of its current pyramid
//    level, and the inner iterations of all of them run in shared launches over one work-list of
//    every request's current level: requests of different sizes and at different levels share
//    each launch, a request that arrives joins at the next step, one that finishes leaves;
//  - a finished request's flow goes back to pinned host memory and the request retires when that
//    copy completes; its device bytes return to the pool for the next admission.
// Requests run in lanes by size -- up to 100,000 pixels, up to 500,000, and larger -- each with its
// own stream, step loop and launches, so that a small request's steps are not as long as those of
// the largest images in the mix (a step takes as long as one warp of all its requests); the lanes
// run concurrently on the device.  At most two steps per lane are queued ahead of the device, so a
// new request waits at most that long to join.  A request's flow does not depend on the other
// requests in its steps: alone and in the mix it is bitwise the same (and equal to of_solve's).
#include <time.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tvl1flow.h"
#include "tvl1_internal.h"
#include "tvl1_plan.h"
#include "tvl1_step.h"

using namespace tvl1;

namespace {

double now_s() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

struct Request {
    uint64_t id = 0;
    int H = 0, W = 0, h = 0, w = 0;  // input and output sizes
    std::vector<float> I0, I1, u, v;
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = OF_OK;
    std::string err;
    bool done = false;
    // in flight
    StepPair q;
    int lane = 0;
    char *dev = nullptr;
    size_t dev_bytes = 0;
    float *pin = nullptr;  // pinned: I0 | I1 | u | v
    size_t pin_elems = 0;
    Misc misc{};
    cudaEvent_t ev = nullptr;  // the result's copy to the host
};

constexpr int NLANES = 3;
constexpr long LANE_MAX_PX[NLANES - 1] = {100000L, 500000L};  // the largest images of each lane but the last

int lane_of(int H, int W) {
    int k = 0;
    while (k < NLANES - 1 && (long)H * W > LANE_MAX_PX[k]) ++k;
    return k;
}

// One lane: its stream, launch tables, the requests it advances and its last two steps' events.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t step_ev[2] = {};
    long long steps = 0;
    StepTables tables;
    std::vector<Request *> active;
};

struct Server {
    of_params params;
    size_t budget = 0, held = 0;
    int device = 0, max_active = 1;
    cudaMemPool_t pool = nullptr;
    Lane lanes[NLANES];
    std::deque<Request *> queue;
    std::vector<Request *> downloading;
    std::map<uint64_t, Request *> reqs;
    std::multimap<size_t, float *> pins;  // pinned staging buffers not in use, by size
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    std::atomic<bool> stopping{false};
    uint64_t next_id = 1;
};

std::mutex g_servers_mu;
std::map<of_ctx *, Server *> g_servers;

Server *server_of(of_ctx *ctx) {
    std::lock_guard<std::mutex> g(g_servers_mu);
    auto it = g_servers.find(ctx);
    return it == g_servers.end() ? nullptr : it->second;
}

void out_size(const of_params &p, int H, int W, int *h, int *w) {
    *h = H;
    *w = W;
    for (int l = 0; l < p.out_level; ++l) {
        *h = level_size(*h, p.eta);
        *w = level_size(*w, p.eta);
    }
}

float *take_pin(Server *S, size_t elems, size_t *got) {
    auto it = S->pins.lower_bound(elems);
    if (it != S->pins.end()) {
        float *p = it->second;
        *got = it->first;
        S->pins.erase(it);
        return p;
    }
    float *p = nullptr;
    if (cudaHostAlloc((void **)&p, elems * sizeof(float), cudaHostAllocDefault) != cudaSuccess) return nullptr;
    *got = elems;
    return p;
}

void finish_request(Server *S, Request *r, int status, const std::string &err) {
    r->status = status;
    r->err = err;
    r->t_done = now_s();
    r->done = true;
    r->I0.clear();
    r->I0.shrink_to_fit();
    r->I1.clear();
    r->I1.shrink_to_fit();
    if (r->dev) {
        cudaFreeAsync(r->dev, S->lanes[r->lane].stream);
        S->held -= r->dev_bytes;
        r->dev = nullptr;
    }
    if (r->pin) S->pins.insert({r->pin_elems, r->pin});
    r->pin = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
}

// Retires requests whose result has reached the host; called with the lock held.
void retire(Server *S) {
    for (size_t k = 0; k < S->downloading.size();) {
        Request *r = S->downloading[k];
        const cudaError_t e = cudaEventQuery(r->ev);
        if (e == cudaErrorNotReady) {
            ++k;
            continue;
        }
        if (e == cudaSuccess) {
            const size_t nin = (size_t)r->H * r->W, n = (size_t)r->h * r->w;
            r->u.assign(r->pin + 2 * nin, r->pin + 2 * nin + n);
            r->v.assign(r->pin + 2 * nin + n, r->pin + 2 * nin + 2 * n);
            const bool finite = std::isfinite(r->misc.res_final) && std::isfinite(r->misc.energy);
            finish_request(S, r, finite ? OF_OK : OF_ENUMERIC,
                           finite ? "" : "non-finite residual or energy (NaN/Inf in the inputs?)");
        } else {
            finish_request(S, r, OF_ECUDA, std::string("request failed on the device: ") + cudaGetErrorString(e));
        }
        S->downloading[k] = S->downloading.back();
        S->downloading.pop_back();
    }
}

// Admits queued requests within the budget and the in-flight limit and starts their solves
// (device memory, copy in, pyramid) on their lane's stream; called with the lock held.
void admit(Server *S) {
    auto in_flight = [S] {
        size_t n = S->downloading.size();
        for (const Lane &L : S->lanes) n += L.active.size();
        return n;
    };
    while (!S->queue.empty() && (int)in_flight() < S->max_active) {
        Request *r = S->queue.front();
        const size_t need = step_pair_bytes(r->H, r->W, &S->params);
        if (need > S->budget) {
            S->queue.pop_front();
            finish_request(S, r, OF_ENOMEM, "request needs more device memory than the serving budget");
            continue;
        }
        if (S->held + need > S->budget) return;  // wait until memory frees up
        r->lane = lane_of(r->H, r->W);
        Lane &L = S->lanes[r->lane];
        const size_t nin = (size_t)r->H * r->W, nout = (size_t)r->h * r->w;
        r->pin = take_pin(S, 2 * nin + 2 * nout, &r->pin_elems);
        if (!r->pin) {
            S->queue.pop_front();
            finish_request(S, r, OF_ENOMEM, "cudaHostAlloc failed");
            continue;
        }
        if (cudaMallocFromPoolAsync((void **)&r->dev, need, S->pool, L.stream) != cudaSuccess) {
            cudaGetLastError();
            S->pins.insert({r->pin_elems, r->pin});
            r->pin = nullptr;
            r->dev = nullptr;
            if (in_flight() == 0) {  // nothing in flight will free memory
                S->queue.pop_front();
                finish_request(S, r, OF_ENOMEM, "the device has no room for the request's arena");
                continue;
            }
            return;  // the pool is short of device memory now: retry after retirements
        }
        S->queue.pop_front();
        r->dev_bytes = need;
        S->held += need;
        std::copy(r->I0.begin(), r->I0.end(), r->pin);
        std::copy(r->I1.begin(), r->I1.end(), r->pin + nin);
        step_pair_init(r->q, r->dev, r->H, r->W, &S->params);
        step_pair_start(r->q, r->pin, r->pin + nin, &S->params, L.stream);
        r->t_start = now_s();
        L.active.push_back(r);
    }
}

// One step of a lane; false when the lane had nothing to run or two steps already in flight.
bool run_lane(Server *S, Lane &L) {
    if (L.active.empty()) return false;
    cudaEvent_t ev = L.step_ev[L.steps & 1];
    if (L.steps >= 2 && cudaEventQuery(ev) == cudaErrorNotReady) return false;
    std::vector<StepPair *> batch;
    for (Request *r : L.active) batch.push_back(&r->q);
    const cudaError_t e = step_run(batch, &S->params, L.tables, L.stream);
    cudaEventRecord(ev, L.stream);
    ++L.steps;
    std::lock_guard<std::mutex> g(S->mu);
    if (e != cudaSuccess) {
        for (Request *r : L.active) finish_request(S, r, OF_ECUDA, std::string("serving step failed: ") + cudaGetErrorString(e));
        L.active.clear();
        return true;
    }
    for (size_t k = 0; k < L.active.size();) {
        Request *r = L.active[k];
        if (!r->q.finished) {
            ++k;
            continue;
        }
        const size_t nin = (size_t)r->H * r->W, n = (size_t)r->h * r->w;
        step_pair_finish(r->q, r->pin + 2 * nin, r->pin + 2 * nin + n, &r->misc, L.stream);
        cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
        cudaEventRecord(r->ev, L.stream);
        S->downloading.push_back(r);
        L.active[k] = L.active.back();
        L.active.pop_back();
    }
    return true;
}

void loop(Server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            retire(S);
            if (!S->stopping) admit(S);
            bool any = false;
            for (const Lane &L : S->lanes) any |= !L.active.empty();
            if (S->stopping && !any && S->downloading.empty()) break;
            if (!any) {
                if (S->downloading.empty() && S->queue.empty()) S->cv.wait_for(lk, std::chrono::milliseconds(2));
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(50));
                }
                continue;
            }
        }
        bool ran = false;
        for (Lane &L : S->lanes) ran |= run_lane(S, L);
        if (!ran) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

void destroy_server(Server *S) {
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stopping = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    for (Lane &L : S->lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    for (auto &kv : S->reqs) {
        Request *r = kv.second;
        if (r->dev) cudaFreeAsync(r->dev, S->lanes[r->lane].stream);
        if (r->pin) cudaFreeHost(r->pin);
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
    }
    for (Lane &L : S->lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    for (auto &kv : S->pins) cudaFreeHost(kv.second);
    for (Lane &L : S->lanes) {
        for (cudaEvent_t e : L.step_ev)
            if (e) cudaEventDestroy(e);
        if (L.stream) cudaStreamDestroy(L.stream);
        L.stream = nullptr;
    }
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
}

}  // namespace

extern "C" {

void tvl1_server_destroy(of_ctx *ctx) {
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> g(g_servers_mu);
        auto it = g_servers.find(ctx);
        if (it != g_servers.end()) {
            S = it->second;
            g_servers.erase(it);
        }
    }
    if (S) destroy_server(S);
}

of_status of_server_start(of_ctx *ctx, const of_params *params, size_t hbm_budget, int max_active) {
    if (!ctx || !params || max_active < 1 || max_active > 256) {
        tvl1_set_error("of_server_start: bad arguments (max_active in [1, 256])");
        return OF_EINVAL;
    }
    if (of_arena_bytes(16, 16, params) == 0) return OF_EINVAL;  // validates the parameters
    if (params->c_adapt_iters != 0) {
        tvl1_set_error("of_server_start: c_adapt_iters is supported for single-pair solves only");
        return OF_EINVAL;
    }
    if (params->engine == OF_ENGINE_PLAIN) {
        tvl1_set_error("of_server_start: the serving loop batches on the fused kernels (not OF_ENGINE_PLAIN)");
        return OF_EINVAL;
    }
    if (server_of(ctx)) {
        tvl1_set_error("of_server_start: a serving loop already runs on this context");
        return OF_EBUSY;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    Server *S = new Server();
    S->params = *params;
    S->device = dev;
    S->max_active = max_active;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->budget = hbm_budget ? hbm_budget : (size_t)(0.6 * (double)tot);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    uint64_t keep = UINT64_MAX;  // the pool keeps freed blocks for the next admissions
    bool ok = cudaMemPoolCreate(&S->pool, &props) == cudaSuccess &&
              cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess;
    for (Lane &L : S->lanes)
        ok = ok && cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&L.step_ev[0], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&L.step_ev[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy_server(S);
        tvl1_set_error("of_server_start: could not create the loop's streams, memory pool or events");
        return OF_ECUDA;
    }
    {
        std::lock_guard<std::mutex> g(g_servers_mu);
        g_servers[ctx] = S;
    }
    S->th = std::thread(loop, S);
    return OF_OK;
}

of_status of_server_submit(of_ctx *ctx, const float *I0, const float *I1, int H, int W, uint64_t *req_id) {
    Server *S = server_of(ctx);
    if (!S) {
        tvl1_set_error("of_server_submit: no serving loop on this context");
        return OF_EBUSY;
    }
    if (!I0 || !I1 || !req_id || H < 1 || W < 1 || H > OF_MAX_SIDE || W > OF_MAX_SIDE) {
        tvl1_set_error("of_server_submit: bad arguments (NULL pointer, or a side outside [1, OF_MAX_SIDE])");
        return OF_EINVAL;
    }
    Request *r = new Request();
    r->H = H;
    r->W = W;
    out_size(S->params, H, W, &r->h, &r->w);
    r->I0.assign(I0, I0 + (size_t)H * W);
    r->I1.assign(I1, I1 + (size_t)H * W);
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stopping) {
            delete r;
            tvl1_set_error("of_server_submit: the loop is stopping");
            return OF_EBUSY;
        }
        r->id = S->next_id++;
        S->reqs[r->id] = r;
        S->queue.push_back(r);
    }
    S->cv.notify_all();
    *req_id = r->id;
    return OF_OK;
}

of_status of_server_poll(of_ctx *ctx, uint64_t req_id, float *u, float *v, of_stats *stats, int *done) {
    Server *S = server_of(ctx);
    if (!S) {
        tvl1_set_error("of_server_poll: no serving loop on this context");
        return OF_EBUSY;
    }
    if (!done) return OF_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) {
        tvl1_set_error("of_server_poll: unknown request id");
        return OF_EINVAL;
    }
    Request *r = it->second;
    *done = r->done ? 1 : 0;
    if (!r->done) return OF_OK;
    of_status st = (of_status)r->status;
    if (st == OF_OK) {
        if (u) std::copy(r->u.begin(), r->u.end(), u);
        if (v) std::copy(r->v.begin(), r->v.end(), v);
    } else {
        tvl1_set_error(r->err.c_str());
    }
    if (stats) {
        const double rows = (double)r->h * r->w * (S->params.beta != 0.f ? 3.0 : 2.0);
        stats->iters_run = r->misc.iters;
        stats->residual = S->params.iters > 0 ? sqrt(r->misc.res_final / rows) : 0.0;
        stats->energy = r->misc.energy;
        stats->dual_value = (S->params.method == OF_PDR || S->params.method == OF_CP) ? NAN : r->misc.dual;
        stats->ms = (float)(1e3 * (r->t_done - r->t_submit));
    }
    S->reqs.erase(it);
    delete r;
    return st;
}

of_status of_server_stop(of_ctx *ctx) {
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> g(g_servers_mu);
        auto it = g_servers.find(ctx);
        if (it == g_servers.end()) {
            tvl1_set_error("of_server_stop: no serving loop on this context");
            return OF_EBUSY;
        }
        S = it->second;
        g_servers.erase(it);
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        for (Request *r : S->queue) {
            S->reqs.erase(r->id);
            delete r;
        }
        S->queue.clear();
    }
    destroy_server(S);
    return OF_OK;
}

}  // extern "C"
