// Serving: local-community queries (graph, seed set, scale) answered as they
// arrive, with continuous batching.
//
// A query is a set of seeds on one resident graph at one scale; its answer is
// the community each seed grows to (Alg. 1 repeated while it adds, as in a
// run).  Queries wait in one FIFO.  A pool of workers, each with its own CUDA
// stream and growth pipeline (slot arenas, retry lists, output buffer), takes
// batches: the oldest waiting query and every later one on the same graph that
// fits the batch's unit limit and the memory budget.  A batch is one
// persistent growth launch over all its units (each unit carries its own
// scale), plus the larger slot classes for the units that outgrow the first.
// While one worker's batch is on the device, the next worker stages and
// launches another: queries that arrive meanwhile are admitted as soon as a
// worker and memory are free, and the batches overlap on the GPU (the SMs a
// finishing batch releases take the next batch's CTAs).  Results are copied
// to host memory; every unit is grown independently and exactly, so a query's
// result does not depend on what it was batched with.
//
// Admission by memory: a query reserves its units' per-unit records plus its
// expected member lists (the mean list length seen on its graph so far, with
// a margin) until its batch completes; a batch waits while the reservations in
// flight would exceed the budget (a query larger than the budget alone still
// runs, alone).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "grow.cuh"
#include "ladder.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Query {
    u64 id = 0;
    int32_t graph_id = -1;
    DevGraph G;
    i64 max_part_n = 0;
    double alpha = 0.0;
    std::vector<i32> seeds;
    int32_t state = MSCD_Q_QUEUED;
    int status = MSCD_OK;
    i64 reserved = 0;  // bytes held against the budget while running
    Clock::time_point t_submit, t_start, t_done;
    std::vector<i64> ptr;  // results
    std::vector<i32> nodes;
    std::vector<double> fitness;
};

// Per-unit device records of a batch: offset, length, hash, fitness,
// statistics, status, seed, scale.
constexpr i64 UNIT_BYTES = 8 + 4 + 8 + 8 + 8 * MSCD_NSTATS + 4 + 4 + 8;

struct Worker {
    GrowPipe pipe;
    i64 cap = 0;  // units the per-unit buffers hold
    i64 *uoff = nullptr;
    i32 *ulen = nullptr;
    u64 *uhash = nullptr;
    double *uf = nullptr;
    i64 *ustat = nullptr;
    i32 *ustatus = nullptr;
    i32 *seeds = nullptr;
    double *alpha = nullptr;
    // pinned host staging
    i32 *h_seeds = nullptr;
    double *h_alpha = nullptr;
    i64 *h_uoff = nullptr;
    i32 *h_ulen = nullptr;
    double *h_uf = nullptr;
    i32 *h_status = nullptr;
    i32 *h_nodes = nullptr;
    i64 h_nodes_cap = 0;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // device interval of the batch in flight
    std::thread th;
};

void free_worker(Worker &w) {
    cudaFree(w.uoff);
    cudaFree(w.ulen);
    cudaFree(w.uhash);
    cudaFree(w.uf);
    cudaFree(w.ustat);
    cudaFree(w.ustatus);
    cudaFree(w.seeds);
    cudaFree(w.alpha);
    cudaFreeHost(w.h_seeds);
    cudaFreeHost(w.h_alpha);
    cudaFreeHost(w.h_uoff);
    cudaFreeHost(w.h_ulen);
    cudaFreeHost(w.h_uf);
    cudaFreeHost(w.h_status);
    cudaFreeHost(w.h_nodes);
    if (w.ev_start) cudaEventDestroy(w.ev_start);
    if (w.ev_end) cudaEventDestroy(w.ev_end);
    w.ev_start = w.ev_end = nullptr;
    pipe_free(w.pipe);
    if (w.pipe.st) cudaStreamDestroy(w.pipe.st);
    w.pipe.st = nullptr;
}

int alloc_worker(Worker &w, i64 cap) {
    w.cap = cap;
    MSCD_CUDA(cudaMalloc((void **)&w.uoff, cap * sizeof(i64)));
    MSCD_CUDA(cudaMalloc((void **)&w.ulen, cap * sizeof(i32)));
    MSCD_CUDA(cudaMalloc((void **)&w.uhash, cap * sizeof(u64)));
    MSCD_CUDA(cudaMalloc((void **)&w.uf, cap * sizeof(double)));
    MSCD_CUDA(cudaMalloc((void **)&w.ustat, cap * MSCD_NSTATS * sizeof(i64)));
    MSCD_CUDA(cudaMalloc((void **)&w.ustatus, cap * sizeof(i32)));
    MSCD_CUDA(cudaMalloc((void **)&w.seeds, cap * sizeof(i32)));
    MSCD_CUDA(cudaMalloc((void **)&w.alpha, cap * sizeof(double)));
    MSCD_CUDA(cudaMallocHost((void **)&w.h_seeds, cap * sizeof(i32)));
    MSCD_CUDA(cudaMallocHost((void **)&w.h_alpha, cap * sizeof(double)));
    MSCD_CUDA(cudaMallocHost((void **)&w.h_uoff, cap * sizeof(i64)));
    MSCD_CUDA(cudaMallocHost((void **)&w.h_ulen, cap * sizeof(i32)));
    MSCD_CUDA(cudaMallocHost((void **)&w.h_uf, cap * sizeof(double)));
    MSCD_CUDA(cudaMallocHost((void **)&w.h_status, cap * sizeof(i32)));
    MSCD_CUDA(cudaStreamCreateWithFlags(&w.pipe.st, cudaStreamNonBlocking));
    MSCD_CUDA(cudaEventCreate(&w.ev_start));
    MSCD_CUDA(cudaEventCreate(&w.ev_end));
    return pipe_reserve(w.pipe, cap);
}

}  // namespace

struct Server {
    int device = 0;
    mscd_serve_params sp{};
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Query *> pending;
    std::map<u64, std::unique_ptr<Query>> queries;
    std::map<int32_t, int> busy;           // queries not yet done, per graph
    std::map<int32_t, double> mean_len;    // observed member-list length, per graph
    u64 next_id = 1;
    i64 budget = 0, in_use = 0;
    bool stopping = false;
    std::vector<std::unique_ptr<Worker>> workers;
    mscd_serve_stats stats{};
    // Device intervals of completed batches, in milliseconds after `ref`, an
    // event recorded when the server started: [start, end) from the batch's
    // first copy to its last, as the GPU timed them on the worker's stream.
    cudaEvent_t ref = nullptr;
    std::vector<std::pair<double, double>> intervals;

    // expected bytes of a query while it runs
    i64 estimate(const Query &q) {
        auto it = mean_len.find(q.graph_id);
        const double len = it != mean_len.end() ? it->second : std::min<double>(256.0, (double)q.max_part_n);
        return (i64)q.seeds.size() * (UNIT_BYTES + (i64)std::ceil(4.0 * 1.5 * len));
    }

    void run_worker(Worker *w);
    int grow_batch(Worker *w, std::vector<Query *> &batch);
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

int Server::grow_batch(Worker *w, std::vector<Query *> &batch) {
    const DevGraph &G = batch[0]->G;
    i64 n = 0;
    for (Query *q : batch) {
        std::memcpy(w->h_seeds + n, q->seeds.data(), q->seeds.size() * sizeof(i32));
        std::fill(w->h_alpha + n, w->h_alpha + n + (i64)q->seeds.size(), q->alpha);
        n += (i64)q->seeds.size();
    }
    cudaStream_t st = w->pipe.st;
    MSCD_CUDA(cudaEventRecord(w->ev_start, st));
    MSCD_CUDA(cudaMemcpyAsync(w->seeds, w->h_seeds, n * sizeof(i32), cudaMemcpyHostToDevice, st));
    MSCD_CUDA(cudaMemcpyAsync(w->alpha, w->h_alpha, n * sizeof(double), cudaMemcpyHostToDevice, st));
    std::vector<int> ladder;
    std::vector<bool> in_smem;
    int rc = make_ladder(G, batch[0]->max_part_n, w->pipe.p, &ladder, &in_smem);
    if (rc) return rc;
    GrowArgs proto{};
    proto.G = G;
    proto.seeds = w->seeds;
    proto.unit_alpha = w->alpha;
    proto.n_seeds = n;
    proto.max_rounds = w->pipe.p.max_rounds;
    proto.uoff = w->uoff;
    proto.ulen = w->ulen;
    proto.uhash = w->uhash;
    proto.uf = w->uf;
    proto.ustat = w->ustat;
    proto.ustatus = w->ustatus;
    proto.log_kmax = G.kmax > 1 ? (float)std::log((double)G.kmax) : 0.0f;
    unsigned long long cursor = 0;
    const i64 out_budget = std::max<i64>(n * 64, (i64)(sp.memory_budget / (4 * (i64)sizeof(i32))));
    if ((rc = grow_units(w->pipe, proto, n, ladder, in_smem, false, out_budget, batch[0]->max_part_n, &cursor)))
        return rc;
    const i64 total = (i64)cursor;
    if (total > w->h_nodes_cap) {
        cudaFreeHost(w->h_nodes);
        w->h_nodes = nullptr;
        w->h_nodes_cap = 0;
        const i64 cap = std::max<i64>(total + total / 4, 1 << 20);
        MSCD_CUDA(cudaMallocHost((void **)&w->h_nodes, cap * sizeof(i32)));
        w->h_nodes_cap = cap;
    }
    MSCD_CUDA(cudaMemcpyAsync(w->h_uoff, w->uoff, n * sizeof(i64), cudaMemcpyDeviceToHost, st));
    MSCD_CUDA(cudaMemcpyAsync(w->h_ulen, w->ulen, n * sizeof(i32), cudaMemcpyDeviceToHost, st));
    MSCD_CUDA(cudaMemcpyAsync(w->h_uf, w->uf, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSCD_CUDA(cudaMemcpyAsync(w->h_status, w->ustatus, n * sizeof(i32), cudaMemcpyDeviceToHost, st));
    if (total > 0)
        MSCD_CUDA(cudaMemcpyAsync(w->h_nodes, w->pipe.out_nodes, total * sizeof(i32), cudaMemcpyDeviceToHost, st));
    MSCD_CUDA(cudaEventRecord(w->ev_end, st));
    MSCD_CUDA(cudaStreamSynchronize(st));
    {
        float t0 = 0.0f, t1 = 0.0f;
        if (cudaEventElapsedTime(&t0, ref, w->ev_start) == cudaSuccess &&
            cudaEventElapsedTime(&t1, ref, w->ev_end) == cudaSuccess) {
            std::lock_guard<std::mutex> lk(m);
            intervals.push_back({(double)t0, (double)t1});
        }
    }
    // split per query: lists in seed order
    i64 u = 0;
    for (Query *q : batch) {
        const i64 m = (i64)q->seeds.size();
        q->ptr.assign(m + 1, 0);
        for (i64 j = 0; j < m; ++j) q->ptr[j + 1] = q->ptr[j] + w->h_ulen[u + j];
        q->nodes.resize(q->ptr[m]);
        q->fitness.assign(w->h_uf + u, w->h_uf + u + m);
        int st_q = MSCD_OK;
        for (i64 j = 0; j < m; ++j) {
            std::memcpy(q->nodes.data() + q->ptr[j], w->h_nodes + w->h_uoff[u + j],
                        (size_t)w->h_ulen[u + j] * sizeof(i32));
            if (w->h_status[u + j] != MSCD_OK && st_q == MSCD_OK) st_q = w->h_status[u + j];
        }
        q->status = st_q;
        u += m;
    }
    return MSCD_OK;
}

void Server::run_worker(Worker *w) {
    cudaSetDevice(device);
    for (;;) {
        std::vector<Query *> batch;
        i64 reserve = 0;
        {
            std::unique_lock<std::mutex> lk(m);
            for (;;) {
                if (stopping && pending.empty()) return;
                if (!pending.empty()) {
                    Query *q0 = pending.front();
                    const i64 e0 = estimate(*q0);
                    // the oldest query runs when it fits what is free, or alone
                    if (in_use == 0 || in_use + e0 <= budget) break;
                }
                cv_work.wait(lk);
            }
            // the oldest query, then later ones on its graph while they fit
            i64 units = 0;
            const int32_t gid = pending.front()->graph_id;
            for (auto it = pending.begin(); it != pending.end();) {
                Query *q = *it;
                const i64 e = estimate(*q);
                const bool first = batch.empty();
                if (q->graph_id == gid && units + (i64)q->seeds.size() <= w->cap &&
                    (first || in_use + reserve + e <= budget)) {
                    batch.push_back(q);
                    units += (i64)q->seeds.size();
                    reserve += e;
                    q->state = MSCD_Q_RUNNING;
                    q->t_start = Clock::now();
                    it = pending.erase(it);
                    if (units >= w->cap) break;
                } else {
                    ++it;
                }
            }
            in_use += reserve;
            stats.batches++;
            stats.max_in_flight_bytes = std::max<i64>(stats.max_in_flight_bytes, in_use);
        }
        const int rc = grow_batch(w, batch);
        {
            std::lock_guard<std::mutex> lk(m);
            const Clock::time_point now = Clock::now();
            i64 entries = 0, units = 0;
            for (Query *q : batch) {
                if (rc != MSCD_OK) q->status = rc;
                q->state = MSCD_Q_DONE;
                q->t_done = now;
                if (--busy[q->graph_id] == 0) busy.erase(q->graph_id);
                if (rc == MSCD_OK) {
                    entries += (i64)q->nodes.size();
                    units += (i64)q->seeds.size();
                }
                stats.queries_done++;
                stats.units_done += (i64)q->seeds.size();
            }
            if (units > 0) {
                double &ml = mean_len[batch[0]->graph_id];
                const double obs = (double)entries / (double)units;
                ml = ml > 0.0 ? 0.75 * ml + 0.25 * obs : obs;
            }
            in_use -= reserve;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

// ---- context hooks (defined with the context) ----
Server **ctx_server(mscd_ctx *c);
bool ctx_graph_part(mscd_ctx *c, int32_t id, DevGraph *g, i64 *max_part_n);
int ctx_device_of(mscd_ctx *c);
int ctx_sm_count_of(mscd_ctx *c);
mscd_params ctx_params_of(mscd_ctx *c);

void serve_destroy(Server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &w : s->workers)
        if (w->th.joinable()) w->th.join();
    cudaSetDevice(s->device);
    for (auto &w : s->workers) free_worker(*w);
    if (s->ref) cudaEventDestroy(s->ref);
    delete s;
}

bool serve_graph_busy(Server *s, int32_t graph_id) {
    if (!s) return false;
    std::lock_guard<std::mutex> lk(s->m);
    return s->busy.count(graph_id) > 0;
}

extern "C" {

int mscd_serve_start(mscd_ctx *c, const mscd_serve_params *params) {
    if (!c) return MSCD_EINVAL;
    Server **slot = ctx_server(c);
    if (*slot) return MSCD_EBUSY;
    mscd_serve_params sp{};
    sp.struct_size = (int32_t)sizeof(mscd_serve_params);
    if (params) {
        if (params->struct_size != (int32_t)sizeof(mscd_serve_params)) return MSCD_EINVAL;
        sp = *params;
    }
    if (sp.workers <= 0) sp.workers = 4;
    if (sp.max_batch_units <= 0) sp.max_batch_units = 1 << 16;
    if (sp.workers > 64 || sp.max_batch_units > ((i64)1 << 26)) return MSCD_EINVAL;
    const int dev = ctx_device_of(c);
    MSCD_CUDA(cudaSetDevice(dev));
    if (sp.memory_budget <= 0) {
        size_t fr = 0, tot = 0;
        MSCD_CUDA(cudaMemGetInfo(&fr, &tot));
        sp.memory_budget = (i64)(fr / 4);
    }
    Server *s = new (std::nothrow) Server();
    if (!s) return MSCD_ENOMEM;
    s->device = dev;
    s->sp = sp;
    s->budget = sp.memory_budget;
    int rc = MSCD_OK;
    for (int i = 0; i < sp.workers && rc == MSCD_OK; ++i) {
        s->workers.push_back(std::make_unique<Worker>());
        Worker &w = *s->workers.back();
        w.pipe.sm_count = ctx_sm_count_of(c);
        w.pipe.p = ctx_params_of(c);
        w.pipe.p.schedule = MSCD_SCHED_PERSISTENT;
        rc = alloc_worker(w, sp.max_batch_units);
    }
    if (rc) {
        for (auto &w : s->workers) free_worker(*w);
        delete s;
        return rc;
    }
    if (rc == MSCD_OK) rc = cuda_status(cudaEventCreate(&s->ref));
    if (rc == MSCD_OK) rc = cuda_status(cudaEventRecord(s->ref, s->workers[0]->pipe.st));
    if (rc == MSCD_OK) rc = cuda_status(cudaEventSynchronize(s->ref));
    if (rc) {
        for (auto &w : s->workers) free_worker(*w);
        if (s->ref) cudaEventDestroy(s->ref);
        delete s;
        return rc;
    }
    for (auto &w : s->workers) {
        Worker *wp = w.get();
        wp->th = std::thread([s, wp] { s->run_worker(wp); });
    }
    *slot = s;
    return MSCD_OK;
}

int mscd_serve_stop(mscd_ctx *c) {
    if (!c) return MSCD_EINVAL;
    Server **slot = ctx_server(c);
    if (!*slot) return MSCD_EINVAL;
    serve_destroy(*slot);
    *slot = nullptr;
    return MSCD_OK;
}

int mscd_query_submit(mscd_ctx *c, int32_t graph_id, const int32_t *seeds, int32_t n_seeds, double alpha,
                      uint64_t *qid) {
    if (!c || !qid || n_seeds < 1 || !seeds) return MSCD_EINVAL;
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return MSCD_EINVAL;
    Server *s = *ctx_server(c);
    if (!s) return MSCD_EINVAL;
    auto q = std::make_unique<Query>();
    if (!ctx_graph_part(c, graph_id, &q->G, &q->max_part_n)) return MSCD_EINVAL;
    if ((i64)n_seeds > s->sp.max_batch_units) return MSCD_ERANGE;
    for (int32_t i = 0; i < n_seeds; ++i)
        if (seeds[i] < 0 || (i64)seeds[i] >= q->G.n) return MSCD_EINVAL;
    q->graph_id = graph_id;
    q->alpha = alpha;
    q->seeds.assign(seeds, seeds + n_seeds);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->m);
        if (s->stopping) return MSCD_EINVAL;
        q->id = s->next_id++;
        *qid = q->id;
        s->busy[graph_id]++;
        s->pending.push_back(q.get());
        s->queries[q->id] = std::move(q);
        s->stats.queries_submitted++;
    }
    s->cv_work.notify_one();
    return MSCD_OK;
}

int mscd_query_poll(mscd_ctx *c, uint64_t qid, int32_t *state) {
    if (!c || !state) return MSCD_EINVAL;
    Server *s = *ctx_server(c);
    if (!s) return MSCD_EINVAL;
    std::lock_guard<std::mutex> lk(s->m);
    auto it = s->queries.find(qid);
    if (it == s->queries.end()) return MSCD_EINVAL;
    *state = it->second->state;
    return MSCD_OK;
}

int mscd_query_wait(mscd_ctx *c, uint64_t qid, int64_t timeout_us, int32_t *state) {
    if (!c || !state) return MSCD_EINVAL;
    Server *s = *ctx_server(c);
    if (!s) return MSCD_EINVAL;
    std::unique_lock<std::mutex> lk(s->m);
    auto it = s->queries.find(qid);
    if (it == s->queries.end()) return MSCD_EINVAL;
    Query *q = it->second.get();
    const auto until = Clock::now() + std::chrono::microseconds(std::max<int64_t>(timeout_us, 0));
    while (q->state != MSCD_Q_DONE)
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout) break;
    *state = q->state;
    return MSCD_OK;
}

int mscd_query_result(mscd_ctx *c, uint64_t qid, int64_t *ptr, int32_t *nodes, int64_t nodes_cap, double *fitness,
                      int64_t *n_nodes, double *times_ms) {
    if (!c || !n_nodes) return MSCD_EINVAL;
    Server *s = *ctx_server(c);
    if (!s) return MSCD_EINVAL;
    std::unique_ptr<Query> done;
    {
        std::lock_guard<std::mutex> lk(s->m);
        auto it = s->queries.find(qid);
        if (it == s->queries.end()) return MSCD_EINVAL;
        Query *q = it->second.get();
        if (q->state != MSCD_Q_DONE) return MSCD_ENORESULT;
        if (times_ms) {
            times_ms[0] = ms_between(q->t_submit, q->t_start);
            times_ms[1] = ms_between(q->t_start, q->t_done);
            times_ms[2] = ms_between(q->t_submit, q->t_done);
        }
        if (q->status != MSCD_OK && q->status != MSCD_ETIMEOUT && q->status != MSCD_EUNDECIDED) {
            const int st = q->status;
            s->queries.erase(it);
            return st;
        }
        *n_nodes = (i64)q->nodes.size();
        if (nodes_cap < (i64)q->nodes.size() || (!q->nodes.empty() && !nodes) || !ptr) return MSCD_ESMALL;
        done = std::move(it->second);
        s->queries.erase(it);
    }
    std::copy(done->ptr.begin(), done->ptr.end(), ptr);
    std::copy(done->nodes.begin(), done->nodes.end(), nodes);
    if (fitness) std::copy(done->fitness.begin(), done->fitness.end(), fitness);
    return done->status;
}

int mscd_serve_get_stats(mscd_ctx *c, mscd_serve_stats *out) {
    if (!c || !out) return MSCD_EINVAL;
    Server *s = *ctx_server(c);
    if (!s) return MSCD_EINVAL;
    std::lock_guard<std::mutex> lk(s->m);
    *out = s->stats;
    out->queued = (i64)s->pending.size();
    out->in_flight_bytes = s->in_use;
    out->budget_bytes = s->budget;
    // sweep over the batches' device intervals: ends before starts at equal times
    std::vector<std::pair<double, int>> ev;
    ev.reserve(2 * s->intervals.size());
    for (const auto &iv : s->intervals) {
        ev.push_back({iv.first, +1});
        ev.push_back({iv.second, -1});
    }
    std::sort(ev.begin(), ev.end());
    i64 cur = 0, best = 0;
    double overlap = 0.0, last = 0.0;
    for (const auto &e : ev) {
        if (cur >= 2) overlap += e.first - last;
        cur += e.second;
        last = e.first;
        best = std::max(best, cur);
    }
    out->max_concurrent_batches = best;
    out->overlap_us = (i64)(overlap * 1000.0);
    return MSCD_OK;
}

int mscd_serve_batch_intervals(mscd_ctx *c, double *start_ms, double *end_ms, int64_t cap, int64_t *n) {
    if (!c || !n) return MSCD_EINVAL;
    Server *s = *ctx_server(c);
    if (!s) return MSCD_EINVAL;
    std::lock_guard<std::mutex> lk(s->m);
    *n = (i64)s->intervals.size();
    if (cap < *n || (*n > 0 && (!start_ms || !end_ms))) return MSCD_ESMALL;
    for (i64 i = 0; i < *n; ++i) {
        start_ms[i] = s->intervals[i].first;
        end_ms[i] = s->intervals[i].second;
    }
    return MSCD_OK;
}

}  // extern "C"
