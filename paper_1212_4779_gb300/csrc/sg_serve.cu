// sg_serve.cu -- many queries at once: batches (concurrent streams, or one
// captured CUDA graph replayed with a single launch) and a serving loop with
// continuous batching (a worker thread that admits queued requests into
// free device slots as soon as memory allows).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sg_internal.cuh"

using namespace sgi;

namespace {

// --------------------------------------------------------------- streams

// Non-blocking streams for batches, per device, created on first use and
// kept for the life of the process.
struct StreamPool {
    std::mutex mu;
    std::vector<cudaStream_t> streams;
};
StreamPool g_pools[64];

sg_status pool_streams(int count, std::vector<cudaStream_t> &out)
{
    int dev = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d is beyond 64", dev);
        return SG_EINVAL;
    }
    StreamPool &p = g_pools[dev];
    std::lock_guard<std::mutex> lock(p.mu);
    while ((int)p.streams.size() < count) {
        cudaStream_t s;
        SG_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        p.streams.push_back(s);
    }
    out.assign(p.streams.begin(), p.streams.begin() + count);
    return SG_OK;
}

sg_workspace *query_ws(const sg_query &q) { return q.ws ? q.ws : &q.graph->ws; }

sg_status check_batch(int32_t nq, sg_query *q, int32_t concurrency)
{
    if (nq < 0 || (nq > 0 && !q) || concurrency < 1) {
        set_error("batch: need nq >= 0, queries, concurrency >= 1");
        return SG_EINVAL;
    }
    std::vector<const sg_workspace *> used;
    for (int32_t i = 0; i < nq; ++i) {
        q[i].status = SG_OK;
        if (check_query_tuning(q[i].tuning) != SG_OK) {
            q[i].status = SG_EINVAL;
            return SG_EINVAL;
        }
        if (!q[i].graph || !q[i].out_seeds || !q[i].out_gains) {
            q[i].status = SG_EINVAL;
            set_error("batch: query %d has a NULL graph or output", i);
            return SG_EINVAL;
        }
        if (q[i].ws && (q[i].ws->owner_n != q[i].graph->n || q[i].ws->device != q[i].graph->device)) {
            q[i].status = SG_EINVAL;
            set_error("batch: query %d has a workspace of another graph", i);
            return SG_EINVAL;
        }
        used.push_back(query_ws(q[i]));
    }
    std::sort(used.begin(), used.end());
    if (std::adjacent_find(used.begin(), used.end()) != used.end()) {
        set_error("batch: two queries share one workspace");
        return SG_EINVAL;
    }
    return SG_OK;
}

// Fork the pool streams from `origin`, run every query on its stream, join.
// prepare: size every workspace first (allocations) so that the launch pass
// allocates nothing (needed under stream capture).
sg_status run_batch(int32_t nq, sg_query *q, const std::vector<cudaStream_t> &ps, cudaStream_t origin)
{
    sg_status first = SG_OK;
    for (int32_t i = 0; i < nq; ++i) {
        KnobScope ks(q[i].tuning);
        const sg_status rc = select_impl(q[i].graph, *query_ws(q[i]), q[i].R, q[i].k, q[i].cascade, q[i].seed,
                                         origin, q[i].out_seeds, q[i].out_gains, nullptr, true);
        q[i].status = rc;
        if (rc != SG_OK && first == SG_OK) first = rc;
    }
    if (first != SG_OK) return first;
    cudaEvent_t fork;
    SG_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    SG_CUDA_TRY(cudaEventRecord(fork, origin));
    for (cudaStream_t s : ps) SG_CUDA_TRY(cudaStreamWaitEvent(s, fork, 0));
    for (int32_t i = 0; i < nq; ++i) {
        cudaStream_t s = ps[(size_t)i % ps.size()];
        KnobScope ks(q[i].tuning);
        const sg_status rc = select_impl(q[i].graph, *query_ws(q[i]), q[i].R, q[i].k, q[i].cascade, q[i].seed, s,
                                         q[i].out_seeds, q[i].out_gains, nullptr, false);
        q[i].status = rc;
        if (rc != SG_OK && first == SG_OK) first = rc;
    }
    std::vector<cudaEvent_t> joins(ps.size());
    for (size_t j = 0; j < ps.size(); ++j) {
        SG_CUDA_TRY(cudaEventCreateWithFlags(&joins[j], cudaEventDisableTiming));
        SG_CUDA_TRY(cudaEventRecord(joins[j], ps[j]));
        SG_CUDA_TRY(cudaStreamWaitEvent(origin, joins[j], 0));
    }
    cudaEventDestroy(fork);
    for (auto e : joins) cudaEventDestroy(e);
    return first;
}

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct sg_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

// ---------------------------------------------------------------- server

namespace {

struct SrvRequest {
    int64_t id;
    sg_graph *g;
    int32_t R, k;
    sg_cascade c;
    uint64_t seed;
    double t_submit = 0, t_done = 0;
    sg_status status = SG_OK;
    int state = 0;  // 0 queued, 1 running, 2 finished
    std::vector<int32_t> seeds;
    std::vector<int64_t> gains;
};

struct SrvWs {
    sg_graph *g;
    sg_workspace *ws;
    int32_t W;
    size_t bytes;
    bool busy;
    uint64_t last_use;
};

struct SrvSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t *h_seeds = nullptr;
    int64_t *h_gains = nullptr;
    SrvRequest *req = nullptr;
    int ws_index = -1;
};

}  // namespace

struct sg_server {
    sg_server_cfg cfg;
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SrvRequest *> queue;
    std::unordered_map<int64_t, SrvRequest *> reqs;
    std::vector<SrvSlot> slots;
    std::vector<SrvWs> pool;
    // workspaces are built and released on a stream of their own, so that
    // admission never waits for a running request; a slot's stream waits
    // on setup_ev before using a fresh workspace
    cudaStream_t setup_st = nullptr;
    cudaEvent_t setup_ev = nullptr;
    std::thread worker;
    bool stopping = false;
    int64_t next_id = 1;
    uint64_t tick = 0;
    int64_t running = 0, finished = 0;
};

namespace {

// Worker: retire finished slots, then admit queued requests in arrival
// order while a slot and memory are free.  Called with the lock held.
void srv_retire(sg_server *s)
{
    for (auto &sl : s->slots) {
        if (!sl.req) continue;
        const cudaError_t e = cudaEventQuery(sl.ev);
        if (e == cudaErrorNotReady) continue;
        SrvRequest *r = sl.req;
        if (e != cudaSuccess) {
            r->status = SG_ECUDA;
        } else {
            r->seeds.assign(sl.h_seeds, sl.h_seeds + r->k);
            r->gains.assign(sl.h_gains, sl.h_gains + r->k);
            // a failed device step leaves seeds of -1 and gains of -flags
            if (r->k > 0 && sl.h_seeds[0] == -1 && sl.h_gains[0] < 0)
                r->status = flags_status((int32_t)(-sl.h_gains[0]));
        }
        r->t_done = now_ms();
        r->state = 2;
        s->pool[(size_t)sl.ws_index].busy = false;
        s->pool[(size_t)sl.ws_index].last_use = ++s->tick;
        sl.req = nullptr;
        sl.ws_index = -1;
        --s->running;
        ++s->finished;
    }
}

// An idle workspace for (g, W), creating one within the memory budget
// (releasing least recently used idle ones if needed).  -1: none now.
// *fresh: the workspace was created now; its set-up (allocations and
// clears) is queued on the setup stream and marked by setup_ev.  Nothing
// here waits on the host.
int srv_workspace(sg_server *s, sg_graph *g, int32_t W, bool *impossible, bool *fresh)
{
    *impossible = false;
    *fresh = false;
    for (size_t i = 0; i < s->pool.size(); ++i)
        if (!s->pool[i].busy && s->pool[i].g == g && s->pool[i].W >= W) return (int)i;
    const size_t need = workspace_bytes(g, W, s->cfg.k_cap);
    while (s->used + need > s->budget) {
        int lru = -1;
        for (size_t i = 0; i < s->pool.size(); ++i)
            if (!s->pool[i].busy && (lru < 0 || s->pool[i].last_use < s->pool[(size_t)lru].last_use)) lru = (int)i;
        if (lru < 0) break;
        // idle: its last request has finished (its slot event completed), so
        // the release is queued in stream order without waiting
        sg_workspace *w = s->pool[(size_t)lru].ws;
        free_workspace(*w, s->setup_st);
        delete w;
        s->used -= s->pool[(size_t)lru].bytes;
        s->pool.erase(s->pool.begin() + lru);
        // running slots index the pool: entries after the erased one moved
        // down (the erased entry was idle, so no slot held it)
        for (auto &sl : s->slots)
            if (sl.req && sl.ws_index > lru) --sl.ws_index;
    }
    if (s->used + need > s->budget) {
        *impossible = s->running == 0;  // nothing will ever free memory
        return -1;
    }
    sg_workspace *w = new (std::nothrow) sg_workspace();
    if (!w) return -1;
    cudaStream_t st = s->setup_st;
    if (ensure_workspace(g, *w, W, s->cfg.k_cap, st) != SG_OK ||
        (heavy_index_enabled(g, W) && ensure_heavy_index(g, *w, W, st) != SG_OK) ||
        cudaEventRecord(s->setup_ev, st) != cudaSuccess) {
        free_workspace(*w, st);
        delete w;
        *impossible = s->running == 0;
        return -1;
    }
    *fresh = true;
    w->owner_n = g->n;
    w->device = g->device;
    s->pool.push_back(SrvWs{g, w, W, need, false, ++s->tick});
    s->used += need;
    return (int)s->pool.size() - 1;
}

// Admits queued requests in arrival order while a slot and memory allow.
// Called with the lock held; the lock is released while a request's
// kernels are enqueued (submit and poll never wait behind a launch
// sequence).  Only the worker touches slots and the workspace pool.
void srv_admit(sg_server *s, std::unique_lock<std::mutex> &lock)
{
    while (!s->queue.empty()) {
        SrvSlot *free_slot = nullptr;
        for (auto &sl : s->slots)
            if (!sl.req) {
                free_slot = &sl;
                break;
            }
        if (!free_slot) return;
        SrvRequest *r = s->queue.front();
        const int32_t W = (r->R + 63) / 64;
        bool impossible = false, fresh = false;
        const int wi = srv_workspace(s, r->g, W, &impossible, &fresh);
        if (wi < 0) {
            if (!impossible) return;  // wait for memory
            s->queue.pop_front();
            r->status = SG_ENOMEM;
            r->t_done = now_ms();
            r->state = 2;
            ++s->finished;
            continue;
        }
        s->queue.pop_front();
        s->pool[(size_t)wi].busy = true;
        r->state = 1;
        free_slot->req = r;
        free_slot->ws_index = wi;
        ++s->running;
        sg_workspace *ws = s->pool[(size_t)wi].ws;
        lock.unlock();
        sg_status rc = SG_OK;
        if (fresh && cudaStreamWaitEvent(free_slot->st, s->setup_ev, 0) != cudaSuccess) rc = SG_ECUDA;
        if (rc == SG_OK)
            rc = select_impl(r->g, *ws, r->R, r->k, r->c, r->seed, free_slot->st, free_slot->h_seeds,
                             free_slot->h_gains, nullptr, false);
        if (rc == SG_OK && cudaEventRecord(free_slot->ev, free_slot->st) != cudaSuccess) rc = SG_ECUDA;
        lock.lock();
        if (rc != SG_OK) {
            s->pool[(size_t)free_slot->ws_index].busy = false;
            free_slot->req = nullptr;
            free_slot->ws_index = -1;
            --s->running;
            r->status = rc;
            r->t_done = now_ms();
            r->state = 2;
            ++s->finished;
        }
    }
}

void srv_loop(sg_server *s)
{
    cudaSetDevice(s->device);
    g_builtin_alloc = 1;
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        srv_retire(s);
        srv_admit(s, lock);
        if (s->stopping && s->queue.empty() && s->running == 0) break;
        // wake on a submission, or poll the running slots every 50 us
        s->cv.wait_for(lock, std::chrono::microseconds(s->running ? 50 : 2000));
    }
}

}  // namespace

extern "C" {

sg_status sg_select_batch(int32_t nq, sg_query *q, int32_t concurrency, void *stream)
{
    clear_error();
    SG_TRY(check_batch(nq, q, concurrency));
    if (nq == 0) return SG_OK;
    std::vector<cudaStream_t> ps;
    SG_TRY(pool_streams(std::min(concurrency, nq), ps));
    return run_batch(nq, q, ps, (cudaStream_t)stream);
}

sg_status sg_batch_capture(int32_t nq, sg_query *q, int32_t concurrency, void *stream, sg_batch **out)
{
    clear_error();
    if (!out) {
        set_error("sg_batch_capture: NULL out");
        return SG_EINVAL;
    }
    SG_TRY(check_batch(nq, q, concurrency));
    if (!stream) {
        set_error("sg_batch_capture: needs a non-default stream");
        return SG_EINVAL;
    }
    for (int32_t i = 0; i < nq; ++i) {
        cudaPointerAttributes a1, a2;
        if (cudaPointerGetAttributes(&a1, q[i].out_seeds) != cudaSuccess ||
            cudaPointerGetAttributes(&a2, q[i].out_gains) != cudaSuccess ||
            a1.type == cudaMemoryTypeUnregistered || a2.type == cudaMemoryTypeUnregistered) {
            cudaGetLastError();
            q[i].status = SG_EINVAL;
            set_error("sg_batch_capture: query %d outputs must be device or pinned host memory", i);
            return SG_EINVAL;
        }
    }
    cudaStream_t origin = (cudaStream_t)stream;
    std::vector<cudaStream_t> ps;
    SG_TRY(pool_streams(std::max(1, std::min(concurrency, nq)), ps));
    // size every workspace (allocations) before recording
    for (int32_t i = 0; i < nq; ++i) {
        KnobScope ks(q[i].tuning);
        const sg_status rc = select_impl(q[i].graph, *query_ws(q[i]), q[i].R, q[i].k, q[i].cascade, q[i].seed,
                                         origin, q[i].out_seeds, q[i].out_gains, nullptr, true);
        q[i].status = rc;
        if (rc != SG_OK) return rc;
    }
    SG_CUDA_TRY(cudaStreamSynchronize(origin));
    sg_batch *b = new (std::nothrow) sg_batch();
    if (!b) {
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    SG_CUDA_TRY(cudaGetDevice(&b->device));
    SG_CUDA_TRY(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
    const sg_status rc = run_batch(nq, q, ps, origin);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(origin, &graph);
    if (rc != SG_OK || ce != cudaSuccess) {
        if (ce != cudaSuccess) set_error("sg_batch_capture: capture failed: %s", cudaGetErrorString(ce));
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        delete b;
        return rc != SG_OK ? rc : SG_ECUDA;
    }
    b->graph = graph;
    const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
    if (ie != cudaSuccess) {
        set_error("sg_batch_capture: instantiate failed: %s", cudaGetErrorString(ie));
        cudaGraphDestroy(graph);
        delete b;
        return SG_ECUDA;
    }
    *out = b;
    return SG_OK;
}

sg_status sg_batch_launch(sg_batch *b, void *stream)
{
    clear_error();
    if (!b) {
        set_error("sg_batch_launch: NULL batch");
        return SG_EINVAL;
    }
    SG_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return SG_OK;
}

void sg_batch_free(sg_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

sg_status sg_server_create(const sg_server_cfg *cfg, sg_server **out)
{
    clear_error();
    if (!cfg || !out || cfg->max_running < 1 || cfg->k_cap < 1) {
        set_error("sg_server_create: need max_running >= 1 and k_cap >= 1");
        return SG_EINVAL;
    }
    sg_server *s = new (std::nothrow) sg_server();
    if (!s) {
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    s->cfg = *cfg;
    SG_CUDA_TRY(cudaGetDevice(&s->device));
    size_t fr = 0, tot = 0;
    SG_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    s->budget = cfg->memory_budget ? cfg->memory_budget : (size_t)(0.8 * (double)fr);
    s->slots.resize((size_t)cfg->max_running);
    if (cudaStreamCreateWithFlags(&s->setup_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->setup_ev, cudaEventDisableTiming) != cudaSuccess) {
        set_error("sg_server_create: stream/event creation failed");
        cudaGetLastError();
        sg_server_destroy(s);
        return SG_ECUDA;
    }
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_seeds, sizeof(int32_t) * (size_t)cfg->k_cap) != cudaSuccess ||
            cudaMallocHost(&sl.h_gains, sizeof(int64_t) * (size_t)cfg->k_cap) != cudaSuccess) {
            set_error("sg_server_create: stream/event/pinned allocation failed");
            cudaGetLastError();
            sg_server_destroy(s);
            return SG_ECUDA;
        }
    }
    s->worker = std::thread(srv_loop, s);
    *out = s;
    return SG_OK;
}

sg_status sg_server_submit(sg_server *s, sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed,
                           int64_t *request_id)
{
    clear_error();
    if (!s || !g || !request_id) {
        set_error("sg_server_submit: NULL argument");
        return SG_EINVAL;
    }
    SG_TRY(check_query(g, R, k));
    Coins co;
    SG_TRY(make_coins(c, seed, R, &co));
    if (k > s->cfg.k_cap) {
        set_error("sg_server_submit: k = %d exceeds the server's k_cap %d", k, s->cfg.k_cap);
        return SG_EINVAL;
    }
    if (g->device != s->device) {
        set_error("sg_server_submit: graph lives on another device");
        return SG_EINVAL;
    }
    SrvRequest *r = new (std::nothrow) SrvRequest();
    if (!r) {
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    r->g = g;
    r->R = R;
    r->k = k;
    r->c = c;
    r->seed = seed;
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) {
            delete r;
            set_error("sg_server_submit: server is shutting down");
            return SG_EBUSY;
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        *request_id = r->id;
    }
    s->cv.notify_one();
    return SG_OK;
}

sg_status sg_server_poll(sg_server *s, int64_t request_id, int32_t *done, int32_t *out_seeds, int64_t *out_gains,
                         double *latency_ms)
{
    clear_error();
    if (!s || !done) {
        set_error("sg_server_poll: NULL argument");
        return SG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) {
        set_error("sg_server_poll: unknown request %lld", (long long)request_id);
        return SG_EINVAL;
    }
    SrvRequest *r = it->second;
    if (r->state != 2) {
        *done = 0;
        return SG_OK;
    }
    *done = 1;
    const sg_status st = r->status;
    if (st == SG_OK) {
        if (out_seeds) memcpy(out_seeds, r->seeds.data(), sizeof(int32_t) * (size_t)r->k);
        if (out_gains) memcpy(out_gains, r->gains.data(), sizeof(int64_t) * (size_t)r->k);
    }
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    s->reqs.erase(it);
    --s->finished;
    delete r;
    if (st != SG_OK) set_error("request %lld failed with status %d", (long long)request_id, (int)st);
    return st;
}

sg_status sg_server_counts(sg_server *s, int64_t *queued, int64_t *running, int64_t *finished)
{
    if (!s) {
        set_error("sg_server_counts: NULL server");
        return SG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = s->running;
    if (finished) *finished = s->finished;
    return SG_OK;
}

void sg_server_destroy(sg_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv.notify_one();
    if (s->worker.joinable()) s->worker.join();
    DeviceGuard dg(s->device);
    cudaDeviceSynchronize();
    {
        const int prev = g_builtin_alloc;
        g_builtin_alloc = 1;  // the workspaces came from the built-in allocator
        for (auto &w : s->pool) {
            free_workspace(*w.ws, (cudaStream_t)0);
            delete w.ws;
        }
        g_builtin_alloc = prev;
    }
    cudaDeviceSynchronize();
    for (auto &sl : s->slots) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.h_seeds) cudaFreeHost(sl.h_seeds);
        if (sl.h_gains) cudaFreeHost(sl.h_gains);
    }
    if (s->setup_ev) cudaEventDestroy(s->setup_ev);
    if (s->setup_st) cudaStreamDestroy(s->setup_st);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
