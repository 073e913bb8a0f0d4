// tvl1_serve.cu -- batched solves and the serving loop of the C ABI (include/tvl1flow.h).
//
// The paper solves one pair at a time; serving is this library's addition.  The loop runs on
// its own host thread.  Requests wait in a FIFO queue and are admitted into one of
// `max_active` slots as soon as a slot is free and the device bytes of all slot arenas stay
// within the HBM budget.  Each slot owns a context (arena + cached CUDA graphs per image size),
// a CUDA stream and pinned staging buffers, so admitted requests of different sizes run
// concurrently on the device: their kernels interleave as the streams progress, and a request
// that arrives while others are in flight starts as soon as it is admitted (continuous
// batching).  Every request's arithmetic is the same graph it would run alone, so its result is
// bitwise identical alone and in the mix.
#include <time.h>

#include <algorithm>
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
};

struct Slot {
    of_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    float *pin = nullptr;  // pinned staging: I0 | I1 | u | v
    size_t pin_elems = 0;
    Request *req = nullptr;
};

struct Server {
    of_params params;
    size_t budget = 0;
    int device = 0;
    std::vector<Slot> slots;
    std::deque<Request *> queue;
    std::map<uint64_t, Request *> reqs;
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
        int a = (int)((double)*h * p.eta + 0.5), b = (int)((double)*w * p.eta + 0.5);
        *h = a < 1 ? 1 : a;
        *w = b < 1 ? 1 : b;
    }
}

size_t slot_bytes(const Slot &s) { return tvl1_ctx_bytes(s.ctx); }

// Retires finished requests; called with the lock held.
void retire(Server *S) {
    for (auto &sl : S->slots) {
        if (!sl.req) continue;
        cudaError_t e = cudaEventQuery(sl.ev);
        if (e == cudaErrorNotReady) continue;
        Request *r = sl.req;
        if (e != cudaSuccess) {
            r->status = OF_ECUDA;
            r->err = std::string("request failed on the device: ") + cudaGetErrorString(e);
        } else {
            const size_t n = (size_t)r->h * r->w, nin = (size_t)r->H * r->W;
            r->u.assign(sl.pin + 2 * nin, sl.pin + 2 * nin + n);
            r->v.assign(sl.pin + 2 * nin + n, sl.pin + 2 * nin + 2 * n);
        }
        r->t_done = now_s();
        r->done = true;
        r->I0.clear();
        r->I0.shrink_to_fit();
        r->I1.clear();
        r->I1.shrink_to_fit();
        sl.req = nullptr;
    }
}

// Admits queued requests into free slots within the budget; called with the lock held.
void admit(Server *S) {
    while (!S->queue.empty()) {
        Request *r = S->queue.front();
        const size_t need = of_arena_bytes(r->H, r->W, &S->params);
        if (need == 0 || need > S->budget) {
            S->queue.pop_front();
            r->status = need == 0 ? OF_EINVAL : OF_ENOMEM;
            r->err = need == 0 ? "invalid request" : "request needs more device memory than the serving budget";
            r->done = true;
            r->t_done = now_s();
            continue;
        }
        size_t held = 0;
        for (auto &sl : S->slots) held += slot_bytes(sl);
        // a free slot whose arena already fits, else the free slot whose growth costs least
        int best = -1;
        size_t best_cost = (size_t)-1;
        for (size_t k = 0; k < S->slots.size(); ++k) {
            Slot &sl = S->slots[k];
            if (sl.req) continue;
            const size_t have = slot_bytes(sl);
            const size_t cost = need > have ? need - have : 0;
            if (cost < best_cost) {
                best_cost = cost;
                best = (int)k;
            }
        }
        if (best < 0) return;                          // no free slot
        if (held + best_cost > S->budget) return;      // wait until memory frees up
        Slot &sl = S->slots[best];
        const size_t nin = (size_t)r->H * r->W, nout = (size_t)r->h * r->w;
        const size_t elems = 2 * nin + 2 * nout;
        if (elems > sl.pin_elems) {
            if (sl.pin) cudaFreeHost(sl.pin);
            sl.pin = nullptr;
            sl.pin_elems = 0;
            if (cudaHostAlloc((void **)&sl.pin, elems * sizeof(float), cudaHostAllocDefault) != cudaSuccess) {
                S->queue.pop_front();
                r->status = OF_ENOMEM;
                r->err = "cudaHostAlloc failed";
                r->done = true;
                continue;
            }
            sl.pin_elems = elems;
        }
        S->queue.pop_front();
        std::copy(r->I0.begin(), r->I0.end(), sl.pin);
        std::copy(r->I1.begin(), r->I1.end(), sl.pin + nin);
        r->t_start = now_s();
        int st = tvl1_solve_async(sl.ctx, sl.pin, sl.pin + nin, r->H, r->W, &S->params, sl.pin + 2 * nin,
                                  sl.pin + 2 * nin + nout, sl.stream);
        if (st != OF_OK) {
            r->status = st;
            r->err = of_last_error(nullptr);
            r->done = true;
            r->t_done = now_s();
            continue;
        }
        cudaEventRecord(sl.ev, sl.stream);
        sl.req = r;
    }
}

void loop(Server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::unique_lock<std::mutex> lk(S->mu);
        retire(S);
        if (!S->stopping) admit(S);
        bool active = false;
        for (auto &sl : S->slots) active |= sl.req != nullptr;
        if (S->stopping && !active) break;
        if (!active && S->queue.empty()) {
            S->cv.wait_for(lk, std::chrono::milliseconds(2));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
}

void destroy_server(Server *S) {
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stopping = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        of_destroy(sl.ctx);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.pin) cudaFreeHost(sl.pin);
    }
    for (auto &kv : S->reqs) delete kv.second;
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
    if (server_of(ctx)) {
        tvl1_set_error("of_server_start: a serving loop already runs on this context");
        return OF_EBUSY;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    Server *S = new Server();
    S->params = *params;
    // slots run on concurrent streams: a persistent launch needs the whole GPU to itself (its
    // warps wait on each other), so the slots take the per-iteration engines instead
    if (S->params.engine == OF_ENGINE_PERSISTENT) S->params.engine = OF_ENGINE_FUSED;
    S->device = dev;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->budget = hbm_budget ? hbm_budget : (size_t)(0.6 * (double)tot);
    S->slots.resize(max_active);
    for (auto &sl : S->slots) {
        if (of_create(&sl.ctx, dev, S->budget) != OF_OK ||
            cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            destroy_server(S);
            tvl1_set_error("of_server_start: could not create slot resources");
            return OF_ECUDA;
        }
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
    if (!I0 || !I1 || !req_id || H < 1 || W < 1) {
        tvl1_set_error("of_server_submit: bad arguments");
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
        stats->iters_run = 0;
        stats->residual = stats->energy = stats->dual_value = 0.0;
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
