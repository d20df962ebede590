// Serving: s-line queries over resident hypergraphs, admitted by predicted
// output memory and executed concurrently.
//
// Ensembles over s are the paper's motivation for computing many s-line graphs
// of one hypergraph (Algorithm 3, Section III-D; the ensemble analyses of
// Section V). Here each query (graph, s) runs on a worker that owns a CUDA
// stream and a streaming window; the worker uses a view of the registered
// graph (shared device arrays, private plan), so queries on the same or on
// different graphs overlap on the device. Admission reserves the predicted
// bytes of a result that is kept on the device: 12 * floor(W_s / s), since
// every s-incident pair accounts for at least s wedges (Section III-E); W_s is
// computed for every graph and s <= max_s at registration. Results larger
// than max_result_pairs are streamed through the worker's window and return
// their counts and digest only. Queries are taken in arrival order, skipping a
// query whose reservation does not fit until memory is released. Small queries
// may be run several at a time as one batch (the disjoint union with per-row s,
// slg_batch_load), which shares one plan, counting pass and fill among them.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "handle.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// a query this small (predicted wedges) may join any batch of small queries
constexpr int64_t BATCH_TINY_WEDGES = (int64_t)1 << 26;

struct ServeQuery {
    int32_t graph = 0, s = 0;
    int64_t reserved = 0;  // bytes held against the budget
    int64_t work = 0;      // predicted W_s
    Clock::time_point t_submit, t_start, t_done;
    slg_status status = SLG_OK;
    bool started = false, done = false, materialized = false;
    int64_t pairs = 0, wedges = 0;
    uint64_t digest = 0;
    int32_t batch_size = 1;  // queries of the batch this one ran in (1: alone)
    int32_t *I = nullptr, *J = nullptr, *O = nullptr;
    std::string error;
};

struct Worker {
    cudaStream_t st = nullptr;
    int32_t *wI = nullptr, *wJ = nullptr, *wO = nullptr;  // streaming window
    std::thread th;
};

double us_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

}  // namespace

struct slg_server {
    slg_serve_cfg cfg{};
    int device = 0;
    std::vector<slg_graph*> graphs;
    std::vector<std::vector<int64_t>> wedges;  // [graph][s-1], s = 1..max_s
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, ServeQuery> q;
    uint64_t next_ticket = 1;
    int64_t mem_in_use = 0, mem_peak = 0, window_bytes = 0;
    int busy = 0;
    bool stop = false;
    std::vector<Worker> workers;
    // statistics since the last reset
    std::vector<double> lat_us;
    int64_t done_pairs = 0, done_wedges = 0, completed = 0;
    int64_t batched = 0, batches = 0, batch_overflows = 0, batch_failures = 0;
    std::string batch_error;  // the last batch failure's message
    Clock::time_point first_submit, last_done;
    bool any_submit = false;
};

namespace {

int64_t predicted_wedges(const slg_server* S, int32_t graph, int32_t s) {
    const std::vector<int64_t>& w = S->wedges[(size_t)graph];
    const int32_t k = std::min<int32_t>(s, (int32_t)w.size());
    return w[(size_t)k - 1];  // W_s is non-increasing in s
}

int64_t predicted_pairs(const slg_server* S, int32_t graph, int32_t s) {
    return predicted_wedges(S, graph, s) / s;
}

// The reservation a query needs: its kept result, or nothing when it streams.
int64_t reservation(const slg_server* S, int32_t graph, int32_t s) {
    const int64_t p = predicted_pairs(S, graph, s);
    return p <= S->cfg.max_result_pairs ? 12 * std::max<int64_t>(p, 1) : 0;
}

void run_query(slg_server* S, Worker& W, ServeQuery& Q) {
    slg_graph* view = slg::make_view(S->graphs[(size_t)Q.graph], W.st);
    struct Free {
        slg_graph* v;
        ~Free() { slg_free(v); }
    } guard{view};
    int64_t pairs = 0, wedges = 0;
    slg_status rc = slg_count(view, Q.s, &pairs, &wedges);
    if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
    Q.pairs = pairs;
    Q.wedges = wedges;
    uint64_t* dig = S->cfg.digest ? &Q.digest : nullptr;
    // kept only when admission reserved it (the prediction bounds the pairs)
    if (Q.reserved > 0 && pairs <= S->cfg.max_result_pairs) {
        const size_t n = (size_t)std::max<int64_t>(pairs, 1);
        SLG_CUDA_TRY(cudaMallocAsync((void**)&Q.I, sizeof(int32_t) * n, W.st));
        SLG_CUDA_TRY(cudaMallocAsync((void**)&Q.J, sizeof(int32_t) * n, W.st));
        SLG_CUDA_TRY(cudaMallocAsync((void**)&Q.O, sizeof(int32_t) * n, W.st));
        Q.materialized = true;
        int64_t P = 0;
        rc = slg_build_window(view, Q.s, 0, view->g.m, Q.I, Q.J, Q.O, pairs, &P, dig, nullptr);
        if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
    } else {
        const int64_t cap = S->cfg.window_pairs;
        std::vector<int32_t> splits((size_t)view->g.m + 2);
        int32_t nw = 0;
        rc = slg_plan_windows(view, Q.s, cap, splits.data(), view->g.m + 1, &nw);
        if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
        uint64_t total = 0;
        for (int32_t w = 0; w < nw; ++w) {
            int64_t P = 0;
            uint64_t d = 0;
            rc = slg_build_window(view, Q.s, splits[(size_t)w], splits[(size_t)w + 1], W.wI, W.wJ,
                                  W.wO, cap, &P, dig ? &d : nullptr, nullptr);
            if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
            total += d;
        }
        Q.digest = total;
    }
    SLG_CUDA_TRY(cudaStreamSynchronize(W.st));
}

// Several small queries as one batch on the worker: the batch's list (every
// member's list in member order, member-local ids) is filled into the
// worker's window in one pass; each member's pairs, digest (the sum of its
// rows' digests) and, when kept, its slice of the window are taken from there.
// Returns false, leaving the queries untouched, when the lists together do
// not fit the window.
bool run_batch(slg_server* S, Worker& W, std::vector<ServeQuery>& Qs) {
    const int32_t k = (int32_t)Qs.size();
    std::vector<slg_graph*> gs((size_t)k);
    std::vector<int32_t> ss((size_t)k);
    for (int32_t b = 0; b < k; ++b) {
        gs[(size_t)b] = S->graphs[(size_t)Qs[(size_t)b].graph];
        ss[(size_t)b] = Qs[(size_t)b].s;
    }
    slg_graph* bh = nullptr;
    slg_status rc = slg_batch_load(gs.data(), ss.data(), k, W.st, &bh);
    if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
    struct Free {
        slg_graph* v;
        ~Free() { slg_free(v); }
    } guard{bh};
    bh->stage_max_bytes = 0;  // workers share the device: no staging pool
    int64_t total = 0;
    rc = slg_count(bh, 0, &total, nullptr);
    if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
    if (total > S->cfg.window_pairs) return false;
    std::vector<int64_t> pbase((size_t)k + 1);
    std::vector<int32_t> rbase((size_t)k + 1);
    int32_t kk = 0;
    if ((rc = slg_batch_pair_offsets(bh, pbase.data())) != SLG_OK ||
        (rc = slg_batch_info(bh, &kk, rbase.data())) != SLG_OK)
        throw slg::Error{rc, slg_last_error()};
    const int32_t M = bh->g.m;
    uint64_t* rowdig = nullptr;
    if (S->cfg.digest) SLG_CUDA_TRY(cudaMallocAsync((void**)&rowdig, sizeof(uint64_t) * ((size_t)M + 1), W.st));
    struct FreeDev {
        uint64_t* p;
        cudaStream_t st;
        ~FreeDev() { if (p) cudaFreeAsync(p, st); }
    } guard2{rowdig, W.st};
    if (rowdig) SLG_CUDA_TRY(cudaMemsetAsync(rowdig, 0, sizeof(uint64_t) * ((size_t)M + 1), W.st));
    int64_t P = 0;
    rc = slg_build_window(bh, 0, 0, M, W.wI, W.wJ, W.wO, S->cfg.window_pairs, &P, nullptr, rowdig);
    if (rc != SLG_OK) throw slg::Error{rc, slg_last_error()};
    std::vector<uint64_t> dig(rowdig ? (size_t)M : 0);
    if (rowdig)
        SLG_CUDA_TRY(cudaMemcpyAsync(dig.data(), rowdig, sizeof(uint64_t) * (size_t)M,
                                     cudaMemcpyDeviceToHost, W.st));
    for (int32_t b = 0; b < k; ++b) {
        ServeQuery& Q = Qs[(size_t)b];
        Q.pairs = pbase[(size_t)b + 1] - pbase[(size_t)b];
        Q.wedges = predicted_wedges(S, Q.graph, Q.s);  // exact: s <= max_s
        if (Q.reserved > 0 && Q.pairs <= S->cfg.max_result_pairs) {
            const size_t n = (size_t)std::max<int64_t>(Q.pairs, 1);
            SLG_CUDA_TRY(cudaMallocAsync((void**)&Q.I, sizeof(int32_t) * n, W.st));
            SLG_CUDA_TRY(cudaMallocAsync((void**)&Q.J, sizeof(int32_t) * n, W.st));
            SLG_CUDA_TRY(cudaMallocAsync((void**)&Q.O, sizeof(int32_t) * n, W.st));
            Q.materialized = true;
            const size_t bytes = sizeof(int32_t) * (size_t)Q.pairs;
            if (bytes) {
                const int64_t at = pbase[(size_t)b];
                SLG_CUDA_TRY(cudaMemcpyAsync(Q.I, W.wI + at, bytes, cudaMemcpyDeviceToDevice, W.st));
                SLG_CUDA_TRY(cudaMemcpyAsync(Q.J, W.wJ + at, bytes, cudaMemcpyDeviceToDevice, W.st));
                SLG_CUDA_TRY(cudaMemcpyAsync(Q.O, W.wO + at, bytes, cudaMemcpyDeviceToDevice, W.st));
            }
        }
    }
    SLG_CUDA_TRY(cudaStreamSynchronize(W.st));
    for (int32_t b = 0; b < k && rowdig; ++b) {
        uint64_t d = 0;
        for (int32_t r = rbase[(size_t)b]; r < rbase[(size_t)b + 1]; ++r) d += dig[(size_t)r];
        Qs[(size_t)b].digest = d;
    }
    return true;
}

void free_result(ServeQuery& Q, cudaStream_t st) {
    if (Q.I) cudaFreeAsync(Q.I, st);
    if (Q.J) cudaFreeAsync(Q.J, st);
    if (Q.O) cudaFreeAsync(Q.O, st);
    Q.I = Q.J = Q.O = nullptr;
}

void worker_loop(slg_server* S, size_t wi) {
    Worker& W = S->workers[wi];
    cudaSetDevice(S->device);
    std::vector<uint64_t> tickets;
    for (;;) {
        uint64_t ticket = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) return;
                // a pending query whose reservation fits: the first one, or the
                // one with the least predicted work; small-query workers skip
                // the large ones
                const bool small_only = (int32_t)wi < S->cfg.small_workers;
                auto pick = S->pending.end();
                for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
                    const ServeQuery& Q = S->q[*it];
                    if (S->mem_in_use + Q.reserved > S->cfg.memory_budget) continue;
                    if (small_only && Q.work > S->cfg.small_wedges) continue;
                    if (pick == S->pending.end() || S->q[*pick].work > Q.work) pick = it;
                    if (S->cfg.policy == 0) break;
                }
                if (pick != S->pending.end()) {
                    ticket = *pick;
                    S->pending.erase(pick);
                    break;
                }
                S->cv_work.wait(lk);
            }
            tickets.assign(1, ticket);
            int64_t held = S->q[ticket].reserved;
            // a small query takes other pending small queries along (any graph, any s)
            auto small = [&](const ServeQuery& X) {
                return X.work <= S->cfg.small_wedges && X.s <= S->cfg.max_s;
            };
            if (S->cfg.batch_max > 1 && small(S->q[ticket])) {
                // members of similar size: a batch finishes as a whole, so the
                // smallest pending queries go first, each predicted at most four
                // times the first query's work (or tiny outright)
                const int64_t cap = std::max<int64_t>(4 * S->q[ticket].work, BATCH_TINY_WEDGES);
                std::vector<std::pair<int64_t, uint64_t>> cand;
                for (uint64_t t : S->pending) {
                    const ServeQuery& X = S->q[t];
                    if (small(X) && X.work <= cap) cand.emplace_back(X.work, t);
                }
                std::sort(cand.begin(), cand.end());
                for (const auto& c : cand) {
                    if ((int32_t)tickets.size() >= S->cfg.batch_max) break;
                    const ServeQuery& X = S->q[c.second];
                    if (S->mem_in_use + held + X.reserved > S->cfg.memory_budget) continue;
                    held += X.reserved;
                    tickets.push_back(c.second);
                    S->pending.erase(std::find(S->pending.begin(), S->pending.end(), c.second));
                }
            }
            const Clock::time_point now = Clock::now();
            for (uint64_t t : tickets) {
                ServeQuery& Q = S->q[t];
                S->mem_in_use += Q.reserved;
                Q.started = true;
                Q.t_start = now;
            }
            S->mem_peak = std::max(S->mem_peak, S->mem_in_use);
            S->busy += (int)tickets.size();
        }
        std::vector<ServeQuery> local(tickets.size());
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t x = 0; x < tickets.size(); ++x) local[x] = S->q[tickets[x]];
        }
        bool batched = false, failed = false;
        std::string why;
        if (local.size() > 1) {
            try {
                batched = run_batch(S, W, local);
                for (ServeQuery& Q : local) {
                    Q.status = SLG_OK;
                    Q.batch_size = batched ? (int32_t)local.size() : 1;
                }
            } catch (const slg::Error& e) {
                for (ServeQuery& Q : local) {  // run them one by one instead
                    free_result(Q, W.st);
                    Q.materialized = false;
                    Q.digest = 0;
                    Q.batch_size = 1;
                }
                batched = false;
                failed = true;
                why = e.msg;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (batched) {
                S->batches += 1;
                S->batched += (int64_t)local.size();
            } else if (failed) {
                S->batch_failures += 1;
                S->batch_error = why;
            } else {
                S->batch_overflows += 1;  // the lists together exceeded the window
            }
        }
        if (!batched) {
            for (ServeQuery& Q : local) {
                try {
                    run_query(S, W, Q);
                    Q.status = SLG_OK;
                } catch (const slg::Error& e) {
                    Q.status = e.code;
                    Q.error = e.msg;
                    free_result(Q, W.st);
                    Q.materialized = false;
                }
            }
        }
        for (size_t x = 0; x < tickets.size(); ++x) {
            const uint64_t ticket_x = tickets[x];
            ServeQuery& local_x = local[x];
            std::lock_guard<std::mutex> lk(S->mu);
            ServeQuery& Q = S->q[ticket_x];
            Q.status = local_x.status;
            Q.error = local_x.error;
            Q.pairs = local_x.pairs;
            Q.wedges = local_x.wedges;
            Q.digest = local_x.digest;
            Q.batch_size = local_x.batch_size;
            Q.I = local_x.I;
            Q.J = local_x.J;
            Q.O = local_x.O;
            Q.materialized = local_x.materialized;
            Q.t_done = Clock::now();
            Q.done = true;
            // a kept result holds its exact size until released; the rest returns
            const int64_t keep = Q.materialized ? 12 * std::max<int64_t>(Q.pairs, 1) : 0;
            S->mem_in_use -= Q.reserved - keep;
            Q.reserved = keep;
            S->busy -= 1;
            S->completed += 1;
            S->lat_us.push_back(us_between(Q.t_submit, Q.t_done));
            S->done_pairs += Q.pairs;
            S->done_wedges += Q.wedges;
            S->last_done = Q.t_done;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

slg_status sfail(slg_status code, const std::string& msg) {
    slg::set_error(code, msg);
    return code;
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    const double x = p * (double)(v.size() - 1);
    const size_t a = (size_t)x;
    const size_t b = std::min(a + 1, v.size() - 1);
    return v[a] + (v[b] - v[a]) * (x - (double)a);
}

}  // namespace

extern "C" {

slg_status slg_serve_create(const slg_serve_cfg* cfg, slg_server** out) {
    if (!out || !cfg) return sfail(SLG_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->workers < 1 || cfg->window_pairs < 1 || cfg->max_s < 1 || cfg->memory_budget < 0 ||
        cfg->max_result_pairs < 0 || cfg->policy < 0 || cfg->policy > 1 ||
        cfg->small_workers < 0 || cfg->small_workers >= cfg->workers)
        return sfail(SLG_EINVAL, "bad server configuration");
    slg_server* S = new slg_server();
    S->cfg = *cfg;
    try {
        SLG_CUDA_TRY(cudaGetDevice(&S->device));
        S->workers.resize((size_t)cfg->workers);
        S->window_bytes = 12 * cfg->window_pairs;
        for (Worker& W : S->workers) {
            SLG_CUDA_TRY(cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking));
            SLG_CUDA_TRY(cudaMalloc((void**)&W.wI, sizeof(int32_t) * cfg->window_pairs));
            SLG_CUDA_TRY(cudaMalloc((void**)&W.wJ, sizeof(int32_t) * cfg->window_pairs));
            SLG_CUDA_TRY(cudaMalloc((void**)&W.wO, sizeof(int32_t) * cfg->window_pairs));
        }
        for (size_t i = 0; i < S->workers.size(); ++i)
            S->workers[i].th = std::thread(worker_loop, S, i);
    } catch (const slg::Error& e) {
        slg_serve_destroy(S);
        return sfail(e.code, e.msg);
    }
    *out = S;
    return SLG_OK;
}

void slg_serve_destroy(slg_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (Worker& W : S->workers)
        if (W.th.joinable()) W.th.join();
    for (auto& kv : S->q) free_result(kv.second, nullptr);
    for (Worker& W : S->workers) {
        if (W.wI) cudaFree(W.wI);
        if (W.wJ) cudaFree(W.wJ);
        if (W.wO) cudaFree(W.wO);
        if (W.st) {
            cudaStreamSynchronize(W.st);
            cudaStreamDestroy(W.st);
        }
    }
    cudaDeviceSynchronize();
    delete S;
}

slg_status slg_serve_register(slg_server* S, slg_graph* g, int32_t* graph_id) {
    if (!S || !g || !graph_id) return sfail(SLG_EINVAL, "NULL argument");
    if (g->g.srow) return sfail(SLG_EINVAL, "register single graphs, not batches");
    try {
        cudaStream_t st;
        SLG_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        slg_graph* view = slg::make_view(g, st);
        std::vector<int64_t> w((size_t)S->cfg.max_s);
        try {
            for (int32_t s = 1; s <= S->cfg.max_s; ++s) {
                slg::plan_build(view->g, s, view->bp, view->plan, st);
                w[(size_t)s - 1] = view->plan.wedges;
            }
        } catch (...) {
            slg_free(view);
            cudaStreamDestroy(st);
            throw;
        }
        slg_free(view);
        SLG_CUDA_TRY(cudaStreamSynchronize(st));
        SLG_CUDA_TRY(cudaStreamDestroy(st));
        std::lock_guard<std::mutex> lk(S->mu);
        *graph_id = (int32_t)S->graphs.size();
        S->graphs.push_back(g);
        S->wedges.push_back(std::move(w));
    } catch (const slg::Error& e) {
        return sfail(e.code, e.msg);
    }
    return SLG_OK;
}

slg_status slg_serve_submit(slg_server* S, int32_t graph_id, int32_t s, uint64_t* ticket) {
    if (!S || !ticket) return sfail(SLG_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    if (graph_id < 0 || graph_id >= (int32_t)S->graphs.size())
        return sfail(SLG_EINVAL, "unknown graph id");
    if (s < 1) return sfail(SLG_EINVAL, "s must be >= 1");
    const int64_t need = reservation(S, graph_id, s);
    if (need > S->cfg.memory_budget)
        return sfail(SLG_ECAPACITY, "the query's result can never fit the memory budget");
    const uint64_t t = S->next_ticket++;
    ServeQuery& Q = S->q[t];
    Q.graph = graph_id;
    Q.s = s;
    Q.reserved = need;
    Q.work = predicted_wedges(S, graph_id, s);
    Q.t_submit = Clock::now();
    if (!S->any_submit) {
        S->first_submit = Q.t_submit;
        S->any_submit = true;
    }
    S->pending.push_back(t);
    *ticket = t;
    lk.unlock();
    // every worker re-examines the queue: a worker restricted to small
    // queries may not take this one, so waking a single waiter could stall it
    S->cv_work.notify_all();
    return SLG_OK;
}

slg_status slg_serve_poll(slg_server* S, uint64_t ticket, int32_t timeout_ms,
                          slg_serve_result* out) {
    if (!S || !out) return sfail(SLG_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->q.find(ticket);
    if (it == S->q.end()) return sfail(SLG_EINVAL, "unknown ticket");
    if (!it->second.done) {
        const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
        while (!S->q[ticket].done)
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
    }
    const ServeQuery& Q = S->q[ticket];
    if (!Q.done) return sfail(SLG_ETIMEOUT, "query not finished within the timeout");
    out->status = Q.status;
    out->materialized = Q.materialized ? 1 : 0;
    out->pairs = Q.pairs;
    out->wedges = Q.wedges;
    out->digest = Q.digest;
    out->latency_us = us_between(Q.t_submit, Q.t_done);
    out->queue_us = us_between(Q.t_submit, Q.t_start);
    out->batch_size = Q.batch_size;
    if (Q.status != SLG_OK) return sfail(Q.status, Q.error);
    return SLG_OK;
}

slg_status slg_serve_fetch(slg_server* S, uint64_t ticket, int32_t* I, int32_t* J, int32_t* O,
                           int64_t cap) {
    if (!S) return sfail(SLG_EINVAL, "NULL argument");
    int32_t *sI, *sJ, *sO;
    int64_t n;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->q.find(ticket);
        if (it == S->q.end() || !it->second.done) return sfail(SLG_EINVAL, "no finished query");
        if (!it->second.materialized) return sfail(SLG_EINVAL, "result was streamed, not kept");
        n = it->second.pairs;
        sI = it->second.I;
        sJ = it->second.J;
        sO = it->second.O;
    }
    if (n > cap) return sfail(SLG_ECAPACITY, "buffer too small");
    if (n > 0 && (!I || !J || !O)) return sfail(SLG_EINVAL, "NULL output");
    try {
        if (n > 0) {
            SLG_CUDA_TRY(cudaMemcpy(I, sI, sizeof(int32_t) * n, cudaMemcpyDefault));
            SLG_CUDA_TRY(cudaMemcpy(J, sJ, sizeof(int32_t) * n, cudaMemcpyDefault));
            SLG_CUDA_TRY(cudaMemcpy(O, sO, sizeof(int32_t) * n, cudaMemcpyDefault));
        }
    } catch (const slg::Error& e) {
        return sfail(e.code, e.msg);
    }
    return SLG_OK;
}

slg_status slg_serve_release(slg_server* S, uint64_t ticket) {
    if (!S) return sfail(SLG_EINVAL, "NULL argument");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->q.find(ticket);
        if (it == S->q.end()) return sfail(SLG_EINVAL, "unknown ticket");
        if (!it->second.done) return sfail(SLG_EBUSY, "query still running");
        ServeQuery& Q = it->second;
        free_result(Q, nullptr);  // its producing stream was synchronised when it finished
        S->mem_in_use -= Q.reserved;
        S->q.erase(it);
    }
    S->cv_work.notify_all();
    return SLG_OK;
}

slg_status slg_serve_stats(slg_server* S, int32_t reset, slg_serve_stats_t* out) {
    if (!S || !out) return sfail(SLG_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->completed = S->completed;
    out->p50_us = percentile(S->lat_us, 0.50);
    out->p99_us = percentile(S->lat_us, 0.99);
    out->max_us = S->lat_us.empty() ? 0 : *std::max_element(S->lat_us.begin(), S->lat_us.end());
    double sum = 0;
    for (double x : S->lat_us) sum += x;
    out->mean_us = S->lat_us.empty() ? 0 : sum / (double)S->lat_us.size();
    const double span = S->any_submit && S->completed
                            ? us_between(S->first_submit, S->last_done) * 1e-6 : 0;
    out->span_s = span;
    out->queries_per_s = span > 0 ? (double)S->completed / span : 0;
    out->pairs_per_s = span > 0 ? (double)S->done_pairs / span : 0;
    out->wedges_per_s = span > 0 ? (double)S->done_wedges / span : 0;
    out->peak_memory = S->mem_peak;
    out->pending = (int64_t)S->pending.size();
    out->running = S->busy;
    out->batched = S->batched;
    out->batches = S->batches;
    out->batch_overflows = S->batch_overflows;
    out->batch_failures = S->batch_failures;
    if (S->batch_failures) slg::set_error(SLG_OK, "last batch failure: " + S->batch_error);
    if (reset) {
        S->lat_us.clear();
        S->completed = S->done_pairs = S->done_wedges = 0;
        S->batched = S->batches = S->batch_overflows = S->batch_failures = 0;
        S->any_submit = false;
        S->mem_peak = S->mem_in_use;
    }
    return SLG_OK;
}

}  // extern "C"
