// Request-serving loop with continuous batching (bt_server_*).
//
// Requests (one graph each) are queued by bt_server_submit.  Worker threads,
// each with its own handle (stream, memory pool, device-resident index), take
// every admissible waiting request when they become free, decompose them as
// one batch (bt_decompose_batch: one disjoint-union pipeline), and complete
// them.  Requests that arrive while a batch is on the GPU wait for the next
// free worker; with two or more workers the batches overlap on the device.
// A large request runs alone; one worker serves small requests first and
// the others large ones first (see the admission code), so small requests do
// not wait behind a large graph.
// The peel of each batch is one persistent cooperative kernel, so each
// worker's peel spans only its share of the SMs: the peels of all workers can
// then be resident together instead of queuing for the whole GPU.
// Admission: a request's device footprint is bounded from its degrees in O(m)
// (priority-obeyed wedges W <= sum over edges of min(d(u), d(v)), Lemma 6;
// BE-Index bytes grow with W) and the sum over in-flight requests must stay
// under the configured budget.  A request whose bound alone exceeds the
// budget is rejected with BT_ERR_NOMEM.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bt_internal.cuh"

namespace {

struct Request {
    uint64_t id;
    bt_graph g;
    uint64_t bytes;      // admission bound, without the counting kernels' per-block counters
    uint64_t cnt_bytes;  // those counters for this graph (a batch needs them once, for its largest graph)
    int status = -1; // -1 pending
    double t_submit = 0, t_start = 0, t_done = 0;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Per-block counters of the counting kernels: two u32 arrays per resident
// block, one entry per vertex of the largest graph of a batch; at most
// (SMs x resident threads per SM) / 256-thread blocks are resident.
uint64_t counter_bound(const bt_graph &g, uint64_t resident_blocks) {
    return ((uint64_t)g.nU + g.nL) * 8ull * resident_blocks;
}

// Upper bound on the device bytes a decomposition of g needs (host, O(m)),
// apart from the counters above.
uint64_t footprint_bound(const bt_graph &g, uint32_t flags, bool device_ptrs) {
    const uint64_t m = g.m;
    const uint64_t n = (uint64_t)g.nU + g.nL;
    uint64_t W = 0;
    if (!device_ptrs && m) {
        std::vector<uint32_t> du(g.nU, 0), dl(g.nL, 0);
        for (uint64_t i = 0; i < m; ++i) {
            int32_t u = g.edges[2 * i], v = g.edges[2 * i + 1];
            if (u >= 0 && v >= 0 && (uint32_t)u < g.nU && (uint32_t)v < g.nL) {
                du[u]++;
                dl[v]++;
            }
        }
        for (uint64_t i = 0; i < m; ++i) {
            int32_t u = g.edges[2 * i], v = g.edges[2 * i + 1];
            if (u >= 0 && v >= 0 && (uint32_t)u < g.nU && (uint32_t)v < g.nL)
                W += std::min(du[u], dl[v]);
        }
    } else {
        W = m * m;  // no host view of the edges: the trivial bound
    }
    (void)flags;
    // CSR and sort scratch, per-edge peel state, index (pairs, bloom ids,
    // links, death stamps, blooms) and per-SM counters
    return (n + 1) * 32 + m * 160 + W * 32 + (64ull << 20);
}

}  // namespace

struct bt_server {
    int device = 0;
    bt_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    std::vector<std::thread> workers;
    bool stop = false;
    uint64_t next_id = 1;
    uint64_t in_flight_bytes = 0;
    uint64_t resident_blocks = 0;  // 256-thread blocks the device holds at once
    bt_server_stats stats{};
    std::vector<bt_handle *> handles;

    void worker_main(int wi) {
        bt_handle *h = handles[wi];
        int rc = BT_OK;
        std::vector<Request *> batch;
        std::vector<bt_graph> graphs;
        std::vector<int> status;
        for (;;) {
            batch.clear();
            uint64_t bytes = 0, cmax = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
                if (queue.empty() && stop) break;
                // requests that can never fit are rejected first
                for (auto it = queue.begin(); it != queue.end();) {
                    Request *r = *it;
                    if (r->bytes + r->cnt_bytes <= cfg.memory_budget_bytes) {
                        ++it;
                        continue;
                    }
                    it = queue.erase(it);
                    r->status = BT_ERR_NOMEM;
                    r->t_done = now_s();
                    stats.rejected++;
                    stats.completed++;
                    cv_done.notify_all();
                }
                // A large request (>= large_edges edges) runs alone.  One
                // worker: queue order.  Several: worker 0 takes the oldest
                // large request first, the last worker the small ones first
                // (passing large ones), the others as worker 0; each falls
                // back to the other kind when its own has none waiting (the
                // last worker only when two or more large requests wait).
                const auto is_large = [&](const Request *r) { return r->g.m >= cfg.large_edges; };
                const auto fits = [&](const Request *r) {
                    return in_flight_bytes + bytes + r->bytes + std::max(cmax, r->cnt_bytes) <=
                           cfg.memory_budget_bytes;
                };
                // the oldest waiting large requests, up to large_batch of them
                const auto take_large = [&]() {
                    const uint32_t cap = cfg.large_batch ? cfg.large_batch : 1u;
                    for (auto it = queue.begin(); it != queue.end() && batch.size() < cap;) {
                        if (!is_large(*it)) {
                            ++it;
                            continue;
                        }
                        if (!fits(*it)) break;  // the oldest large one waits for memory
                        bytes += (*it)->bytes;
                        cmax = std::max(cmax, (*it)->cnt_bytes);
                        batch.push_back(*it);
                        it = queue.erase(it);
                    }
                    return !batch.empty();
                };
                const auto take_small = [&](bool stop_at_large) {
                    for (auto it = queue.begin(); it != queue.end();) {
                        Request *r = *it;
                        if (is_large(r)) {
                            if (stop_at_large) break;
                            ++it;
                            continue;
                        }
                        if (!fits(r)) break;
                        if (cfg.max_batch_graphs && batch.size() >= cfg.max_batch_graphs) break;
                        it = queue.erase(it);
                        bytes += r->bytes;
                        cmax = std::max(cmax, r->cnt_bytes);
                        batch.push_back(r);
                    }
                    return !batch.empty();
                };
                if (cfg.workers == 1) {
                    if (!queue.empty() && is_large(queue.front())) take_large();
                    else take_small(true);
                } else if (wi == (int)cfg.workers - 1) {
                    // it helps with large requests only when two or more
                    // wait, so that one worker usually stays free for small ones
                    if (!take_small(false)) {
                        int waiting = 0;
                        for (const Request *r : queue) waiting += is_large(r) ? 1 : 0;
                        if (waiting >= 2) take_large();
                    }
                } else {
                    if (!take_large()) take_small(false);
                }
                if (batch.empty()) {
                    // the head waits for memory held by other workers
                    cv_work.wait_for(lk, std::chrono::milliseconds(1));
                    continue;
                }
                bytes += cmax;  // one set of counters for the whole batch
                in_flight_bytes += bytes;
                stats.peak_in_flight_bytes = std::max(stats.peak_in_flight_bytes, in_flight_bytes);
                stats.batches++;
                const double t0 = now_s();
                for (Request *r : batch) r->t_start = t0;
            }
            graphs.clear();
            const double t0 = now_s();
            for (Request *r : batch) graphs.push_back(r->g);
            // fixed schedules: the batch autotuner would time candidates on
            // the request path whenever a new batch shape appears
            bt_tune tune{};
            const bool large = batch[0]->g.m >= cfg.large_edges;  // batches are all large or all small
            tune.count_threads = large ? 1024 : 256;
            tune.peel_item = 32;
            bt_batch_stats bs{};
            rc = bt_decompose_batch(h, graphs.data(), (uint32_t)graphs.size(), &tune, &bs,
                                    cfg.flags & BT_TIE_LOWER_FIRST);
            // results are published under the lock only: a poll that sees a
            // status may free the request at once
            status.assign(batch.size(), rc);
            if (rc != BT_OK && graphs.size() > 1) {
                // isolate the failing request(s): retry one by one
                for (size_t i = 0; i < batch.size(); ++i)
                    status[i] = bt_decompose_batch(h, &graphs[i], 1, &tune, nullptr,
                                                   cfg.flags & BT_TIE_LOWER_FIRST);
            }
            const double t1 = now_s();
            {
                std::lock_guard<std::mutex> lk(mu);
                stats.max_batch_graphs = std::max<uint64_t>(stats.max_batch_graphs, batch.size());
                in_flight_bytes -= bytes;
                stats.busy_seconds += t1 - t0;
                stats.edges += bs.edges;
                for (size_t i = 0; i < batch.size(); ++i) {
                    batch[i]->t_done = t1;
                    batch[i]->status = status[i];
                    stats.completed++;
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

extern "C" {

int bt_server_create(bt_server **out, int device, const bt_server_config *cfg) {
    if (!out) return BT_ERR_ARG;
    *out = nullptr;
    bt_server *s = new (std::nothrow) bt_server();
    if (!s) return BT_ERR_NOMEM;
    s->device = device;
    if (cfg) s->cfg = *cfg;
    if (!s->cfg.memory_budget_bytes) s->cfg.memory_budget_bytes = 120ull << 30;
    if (!s->cfg.workers) s->cfg.workers = 2;
    if (!s->cfg.large_edges) s->cfg.large_edges = 1u << 20;
    if (!s->cfg.large_batch) s->cfg.large_batch = 2;
    if (s->cfg.flags & ~(uint32_t)BT_TIE_LOWER_FIRST) {
        delete s;
        return BT_ERR_ARG;
    }
    int sms = 0, tpm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&tpm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess) {
        delete s;
        return BT_ERR_CUDA;
    }
    s->resident_blocks = (uint64_t)sms * (uint64_t)tpm / 256;
    for (uint32_t i = 0; i < s->cfg.workers; ++i) {
        bt_handle *h = nullptr;
        int rc = bt_create(&h, device, nullptr);
        if (rc != BT_OK) {
            for (bt_handle *x : s->handles) bt_destroy(x);
            delete s;
            return rc;
        }
        bt::share_peel_sms(h, (int)s->cfg.workers);  // peels of all workers fit on the GPU at once
        s->handles.push_back(h);
    }
    for (uint32_t i = 0; i < s->cfg.workers; ++i)
        s->workers.emplace_back(&bt_server::worker_main, s, (int)i);
    *out = s;
    return BT_OK;
}

int bt_server_destroy(bt_server *s) {
    if (!s) return BT_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (bt_handle *h : s->handles) bt_destroy(h);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return BT_OK;
}

int bt_server_cancel_queued(bt_server *s, uint64_t *cancelled_out) {
    if (!s) return BT_ERR_ARG;
    uint64_t n = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_s();
        for (Request *r : s->queue) {
            r->t_done = t;
            r->status = BT_ERR_CANCELLED;
            s->stats.completed++;
            ++n;
        }
        s->queue.clear();
    }
    s->cv_done.notify_all();
    if (cancelled_out) *cancelled_out = n;
    return BT_OK;
}

int bt_server_submit(bt_server *s, const bt_graph *g, uint64_t *request_id) {
    if (!s || !g || !request_id) return BT_ERR_ARG;
    if (g->m && (!g->edges || !g->phi_out)) return BT_ERR_ARG;
    Request *r = new (std::nothrow) Request();
    if (!r) return BT_ERR_NOMEM;
    r->g = *g;
    r->bytes = footprint_bound(*g, s->cfg.flags, false);
    r->cnt_bytes = counter_bound(*g, s->resident_blocks);
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        s->stats.submitted++;
    }
    s->cv_work.notify_one();
    *request_id = r->id;
    return BT_OK;
}

int bt_server_poll(bt_server *s, uint64_t request_id, int wait, bt_request_info *info) {
    if (!s || !info) return BT_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return BT_ERR_STATE;
    Request *r = it->second;
    if (wait) s->cv_done.wait(lk, [&] { return r->status != -1; });
    info->done = r->status != -1;
    info->status = r->status == -1 ? BT_OK : r->status;
    info->queue_seconds = (r->t_start > 0 ? r->t_start : now_s()) - r->t_submit;
    info->latency_seconds = (info->done ? r->t_done : now_s()) - r->t_submit;
    info->admitted_bytes = r->bytes + r->cnt_bytes;
    if (info->done) {  // results delivered: forget the request
        s->reqs.erase(it);
        delete r;
    }
    return BT_OK;
}

int bt_server_stats_read(bt_server *s, bt_server_stats *out) {
    if (!s || !out) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = s->queue.size();
    out->in_flight_bytes = s->in_flight_bytes;
    return BT_OK;
}

}  // extern "C"
