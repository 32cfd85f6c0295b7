// A search service with continuous batching, in the library (no paper
// counterpart: the serving pattern of a request stream over a device-resident
// index).  Host threads submit requests of a few queries, each with its own k,
// eps and e_s; one worker thread forms batches and keeps up to `slots` of them in
// flight, each on its own CUDA stream with its own device and pinned host buffers.
//
// Scheduling: one launch runs one (k, eps, e_s) class, so pending requests are
// kept in arrival order and a batch takes the class of the oldest pending request
// and, in order, every pending request of that class while the batch holds at most
// max_queries queries.  A launch copies the batch's queries to the device, runs
// the pivot seeds and the search on the slot's stream, copies ids and distances
// back and records an event; the worker polls the events, hands each request its
// rows and frees the slot.  A request's result depends only on its queries and
// class, never on its batch (the seeds and the search are per query).
//
// A launch that has not completed within timeout_ms fails its requests with
// ONNG_E_LIMIT and stops the server (every later submit and poll fails): its
// stream may still hold work, so its buffers are not reused.
//
// Memory: the server allocates its buffers at create (device: queries, seeds,
// results and a search workspace per slot; pinned host: queries and results per
// slot) and frees them at destroy; it is the one part of the library that
// allocates.  The index arrays stay owned by the caller and must outlive the
// server.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace onng {
namespace {

struct Req {
    uint64_t ticket = 0;
    std::vector<float> q;  // nq x d
    int32_t nq = 0, k = 0, es = 0;
    float eps = 0.f;
    int status = -1;  // -1 pending or running, else the final onng_status
    std::vector<int32_t> ids;
    std::vector<float> dist;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    float *q_dev = nullptr;
    int32_t *seeds = nullptr, *ids_dev = nullptr;
    float *dist_dev = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    float *q_host = nullptr;
    int32_t *ids_host = nullptr;
    float *dist_host = nullptr;
    std::vector<Req *> reqs;
    int32_t k = 0, nq = 0;
    bool busy = false;
    std::chrono::steady_clock::time_point t0;
};

bool same_class(const Req *a, const Req *b)
{
    return a->k == b->k && a->es == b->es && std::memcmp(&a->eps, &b->eps, sizeof(float)) == 0;
}

}  // namespace
}  // namespace onng

struct onng_server {
    onng_index idx{};
    onng_serve_config cfg{};
    int device = 0;
    std::vector<onng::Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<onng::Req *> pending;
    std::unordered_map<uint64_t, onng::Req *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int failed = ONNG_OK;  // set once a launch failed or timed out
    std::thread worker;
};

namespace onng {
namespace {

void free_slot_buffers(Slot &s)
{
    if (s.st)
        cudaStreamSynchronize(s.st);
    cudaFree(s.q_dev);
    cudaFree(s.seeds);
    cudaFree(s.ids_dev);
    cudaFree(s.dist_dev);
    cudaFree(s.ws);
    cudaFreeHost(s.q_host);
    cudaFreeHost(s.ids_host);
    cudaFreeHost(s.dist_host);
    if (s.done)
        cudaEventDestroy(s.done);
    if (s.st)
        cudaStreamDestroy(s.st);
    s = Slot{};
}

// Forms a batch from the pending requests (caller holds the lock) and launches it
// on slot s; returns the status of the launch.
int launch(onng_server *srv, Slot &s)
{
    const onng_serve_config &c = srv->cfg;
    const int d = srv->idx.d;
    Req *first = srv->pending.front();
    int nq = 0;
    for (auto it = srv->pending.begin(); it != srv->pending.end();) {
        Req *r = *it;
        if (same_class(r, first) && nq + r->nq <= c.max_queries) {
            std::memcpy(s.q_host + (size_t)nq * d, r->q.data(), sizeof(float) * (size_t)r->nq * d);
            nq += r->nq;
            s.reqs.push_back(r);
            it = srv->pending.erase(it);
        } else {
            ++it;
        }
    }
    s.k = first->k;
    s.nq = nq;
    onng_search_params p{};
    p.k = first->k;
    p.e_s = first->es;
    p.eps = first->eps;
    p.precision = c.precision;
    p.k_rerank = std::max(c.k_rerank, first->k);
    onng_stream_t st = reinterpret_cast<onng_stream_t>(s.st);
    ONNG_CUDA_TRY(cudaMemcpyAsync(s.q_dev, s.q_host, sizeof(float) * (size_t)nq * d, cudaMemcpyHostToDevice, s.st),
                  "onng_serve: query copy");
    int status = onng_seeds_pivot(srv->idx.X, srv->idx.n, d, s.q_dev, nq, c.n_pivot, c.n_seed, s.seeds, nullptr, 0,
                                  st);
    if (!status)
        status = onng_search(&srv->idx, s.q_dev, nq, &p, s.seeds, c.n_seed, nullptr, nullptr, s.ids_dev, s.dist_dev,
                             nullptr, s.ws, s.ws_bytes, st);
    if (status)
        return status;
    ONNG_CUDA_TRY(cudaMemcpyAsync(s.ids_host, s.ids_dev, sizeof(int32_t) * (size_t)nq * s.k, cudaMemcpyDeviceToHost,
                                  s.st),
                  "onng_serve: result copy");
    ONNG_CUDA_TRY(cudaMemcpyAsync(s.dist_host, s.dist_dev, sizeof(float) * (size_t)nq * s.k,
                                  cudaMemcpyDeviceToHost, s.st),
                  "onng_serve: result copy");
    ONNG_CUDA_TRY(cudaEventRecord(s.done, s.st), "onng_serve: event");
    s.busy = true;
    s.t0 = std::chrono::steady_clock::now();
    return ONNG_OK;
}

// Hands a completed slot's rows to its requests (caller holds the lock).
void complete(Slot &s, int status)
{
    int row = 0;
    for (Req *r : s.reqs) {
        if (status == ONNG_OK) {
            r->ids.assign(s.ids_host + (size_t)row * s.k, s.ids_host + (size_t)(row + r->nq) * s.k);
            r->dist.assign(s.dist_host + (size_t)row * s.k, s.dist_host + (size_t)(row + r->nq) * s.k);
        }
        r->status = status;
        row += r->nq;
    }
    s.reqs.clear();
    s.busy = false;
}

void fail_all(onng_server *srv, int status)
{
    srv->failed = status;
    for (Req *r : srv->pending)
        r->status = status;
    srv->pending.clear();
}

void worker_loop(onng_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lock(srv->mu);
    const auto limit = std::chrono::milliseconds(srv->cfg.timeout_ms);
    while (!srv->stop) {
        bool any_busy = false;
        for (Slot &s : srv->slots) {
            if (!s.busy)
                continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) {
                complete(s, ONNG_OK);
                srv->cv_done.notify_all();
            } else if (e != cudaErrorNotReady) {
                set_error(ONNG_E_CUDA, "onng_serve: %s", cudaGetErrorString(e));
                complete(s, ONNG_E_CUDA);
                fail_all(srv, ONNG_E_CUDA);
                srv->cv_done.notify_all();
            } else if (std::chrono::steady_clock::now() - s.t0 > limit) {
                // the watchdog: this launch's stream may still run, so the server stops
                complete(s, ONNG_E_LIMIT);
                s.busy = true;  // never reused
                fail_all(srv, ONNG_E_LIMIT);
                srv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        if (srv->failed) {
            srv->cv_work.wait(lock, [srv] { return srv->stop; });
            break;
        }
        bool launched = false;
        for (Slot &s : srv->slots) {
            if (s.busy || srv->pending.empty())
                continue;
            const int st = launch(srv, s);
            if (st) {
                complete(s, st);
                fail_all(srv, st);
                srv->cv_done.notify_all();
                break;
            }
            launched = true;
            any_busy = true;
        }
        if (launched || srv->failed)
            continue;
        if (any_busy)
            srv->cv_work.wait_for(lock, std::chrono::microseconds(50));
        else
            srv->cv_work.wait(lock, [srv] { return srv->stop || !srv->pending.empty(); });
    }
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" int onng_serve_create(const onng_index *idx, const onng_serve_config *cfg, onng_server **out)
{
    ONNG_RANGE("onng_serve_create");
    ONNG_REQUIRE(idx && cfg && out, ONNG_E_INVAL, "onng_serve_create: NULL argument");
    *out = nullptr;
    ONNG_REQUIRE(idx->n > 0 && idx->d > 0 && idx->X, ONNG_E_INVAL, "onng_serve_create: empty index");
    ONNG_REQUIRE(cfg->slots >= 1 && cfg->slots <= 64 && cfg->max_queries >= 1 && cfg->k_max >= 1 &&
                     cfg->n_pivot >= 1 && cfg->n_seed >= 1 && cfg->timeout_ms >= 1,
                 ONNG_E_INVAL, "onng_serve_create: bad configuration");
    onng_server *srv = new onng_server();
    srv->idx = *idx;
    srv->cfg = *cfg;
    cudaGetDevice(&srv->device);
    srv->slots.resize((size_t)cfg->slots);
    onng_search_params p{};
    p.k = cfg->k_max;
    p.precision = cfg->precision;
    p.k_rerank = std::max(cfg->k_rerank, cfg->k_max);
    const size_t ws = onng_search_workspace_bytes(cfg->max_queries, idx, &p);
    const size_t nqd = (size_t)cfg->max_queries * idx->d, nqk = (size_t)cfg->max_queries * cfg->k_max;
    for (Slot &s : srv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaMalloc(&s.q_dev, sizeof(float) * nqd);
        if (e == cudaSuccess)
            e = cudaMalloc(&s.seeds, sizeof(int32_t) * (size_t)cfg->max_queries * cfg->n_seed);
        if (e == cudaSuccess)
            e = cudaMalloc(&s.ids_dev, sizeof(int32_t) * nqk);
        if (e == cudaSuccess)
            e = cudaMalloc(&s.dist_dev, sizeof(float) * nqk);
        if (e == cudaSuccess)
            e = cudaMalloc(&s.ws, ws);
        if (e == cudaSuccess)
            e = cudaMallocHost(&s.q_host, sizeof(float) * nqd);
        if (e == cudaSuccess)
            e = cudaMallocHost(&s.ids_host, sizeof(int32_t) * nqk);
        if (e == cudaSuccess)
            e = cudaMallocHost(&s.dist_host, sizeof(float) * nqk);
        if (e != cudaSuccess) {
            for (Slot &t : srv->slots)
                free_slot_buffers(t);
            delete srv;
            return set_error(ONNG_E_CUDA, "onng_serve_create: %s", cudaGetErrorString(e));
        }
        s.ws_bytes = ws;
    }
    srv->worker = std::thread(worker_loop, srv);
    *out = srv;
    return ONNG_OK;
}

extern "C" int onng_serve_submit(onng_server *srv, const float *Q, int32_t nq, int32_t k, float eps, int32_t e_s,
                                 uint64_t *ticket)
{
    ONNG_REQUIRE(srv && Q && ticket, ONNG_E_INVAL, "onng_serve_submit: NULL argument");
    ONNG_REQUIRE(nq >= 1 && nq <= srv->cfg.max_queries, ONNG_E_INVAL, "onng_serve_submit: nq must be in [1, %d]",
                 srv->cfg.max_queries);
    ONNG_REQUIRE(k >= 1 && k <= srv->cfg.k_max, ONNG_E_INVAL, "onng_serve_submit: k must be in [1, %d]",
                 srv->cfg.k_max);
    ONNG_REQUIRE(eps >= 0.f, ONNG_E_INVAL, "onng_serve_submit: eps must be >= 0");
    Req *r = new Req();
    r->q.assign(Q, Q + (size_t)nq * srv->idx.d);
    r->nq = nq;
    r->k = k;
    r->eps = eps;
    r->es = e_s;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (srv->failed) {
            delete r;
            return set_error(srv->failed, "onng_serve_submit: the server stopped after a failed launch");
        }
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        srv->pending.push_back(r);
        *ticket = r->ticket;
    }
    srv->cv_work.notify_one();
    return ONNG_OK;
}

extern "C" int onng_serve_poll(onng_server *srv, uint64_t ticket, int32_t *ids, float *dist, int32_t timeout_ms)
{
    ONNG_REQUIRE(srv && ids && dist, ONNG_E_INVAL, "onng_serve_poll: NULL argument");
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    ONNG_REQUIRE(it != srv->reqs.end(), ONNG_E_INVAL, "onng_serve_poll: unknown ticket %llu",
                 (unsigned long long)ticket);
    Req *r = it->second;
    if (!srv->cv_done.wait_for(lock, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                               [r] { return r->status >= 0; }))
        return set_error(ONNG_E_AGAIN, "onng_serve_poll: request %llu not done yet", (unsigned long long)ticket);
    const int status = r->status;
    if (status == ONNG_OK) {
        std::memcpy(ids, r->ids.data(), sizeof(int32_t) * r->ids.size());
        std::memcpy(dist, r->dist.data(), sizeof(float) * r->dist.size());
    }
    srv->reqs.erase(it);
    delete r;
    if (status)
        return set_error(status, "onng_serve_poll: request %llu failed (status %d)", (unsigned long long)ticket,
                         status);
    return ONNG_OK;
}

extern "C" int onng_serve_destroy(onng_server *srv)
{
    if (!srv)
        return ONNG_OK;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable())
        srv->worker.join();
    for (Slot &s : srv->slots)
        free_slot_buffers(s);
    for (auto &kv : srv->reqs)
        delete kv.second;
    delete srv;
    return ONNG_OK;
}
