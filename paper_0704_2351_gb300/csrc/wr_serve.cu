// Batched rank jobs and the rank server.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "wr_internal.cuh"

namespace wr {
wr_status rank_one(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params, wr_result **out);
}

using namespace wr;

extern "C" wr_status wr_rank_batch(wr_ctx *ctx, size_t njobs, const wr_matrix *const *mats,
                                   const wr_params *params, wr_result **outs) {
    if (!ctx || (njobs && (!mats || !params || !outs))) return fail(WR_EINVAL, "null argument");
    wr_status first = WR_OK;
    for (size_t j = 0; j < njobs; j++) {
        outs[j] = nullptr;
        wr_status st = rank_one(ctx, mats[j], &params[j], &outs[j]);
        if (st != WR_OK && first == WR_OK) first = st;
    }
    return first;
}

// ------------------------------------------------------------------ server

struct wr_server {
    wr_ctx *ctx = nullptr;  // own stream on the caller's device
    wr_server_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    struct Req {
        uint64_t ticket;
        const wr_matrix *mat;
        wr_params prm;
        std::chrono::steady_clock::time_point t_submit;
    };
    std::deque<Req> queue;
    struct Done {
        wr_status st;
        wr_result *res;
    };
    std::map<uint64_t, Done> done;
    std::vector<double> lat_ms;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0;
    int32_t max_resident = 0;
    std::chrono::steady_clock::time_point t_first, t_last;
    bool have_first = false, stop = false;
    std::thread worker;
};

static void server_loop(wr_server *s) {
    cudaSetDevice(s->ctx->device);
    for (;;) {
        wr_server::Req rq;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop && s->queue.empty()) return;
            rq = s->queue.front();
            s->queue.pop_front();
            s->max_resident = std::max(s->max_resident, 1);
        }
        wr_result *res = nullptr;
        wr_status st = rank_one(s->ctx, rq.mat, &rq.prm, &res);
        auto now = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->done[rq.ticket] = wr_server::Done{st, res};
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - rq.t_submit).count());
            if (st == WR_OK) s->completed++;
            else s->failed++;
            s->t_last = now;
        }
        s->cv_done.notify_all();
    }
}

extern "C" wr_status wr_server_start(wr_ctx *ctx, const wr_server_cfg *cfg, wr_server **out) {
    if (!ctx || !cfg || !out) return fail(WR_EINVAL, "null argument");
    *out = nullptr;
    wr_server *s = new wr_server();
    s->cfg = *cfg;
    if (s->cfg.max_slots < 1) s->cfg.max_slots = 1;
    if (s->cfg.queue_cap < 1) s->cfg.queue_cap = 1 << 20;
    wr_status st = wr_create(&s->ctx, ctx->device, nullptr);
    if (st != WR_OK) {
        delete s;
        return st;
    }
    s->worker = std::thread(server_loop, s);
    *out = s;
    return WR_OK;
}

extern "C" wr_status wr_submit(wr_server *srv, const wr_matrix *mat, const wr_params *params, uint64_t *ticket) {
    if (!srv || !mat || !params || !ticket) return fail(WR_EINVAL, "null argument");
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    std::lock_guard<std::mutex> lk(srv->mu);
    if ((int64_t)srv->queue.size() >= srv->cfg.queue_cap) return fail(WR_EBUSY, "server queue full");
    auto now = std::chrono::steady_clock::now();
    if (!srv->have_first) {
        srv->t_first = now;
        srv->have_first = true;
    }
    *ticket = srv->next_ticket++;
    srv->queue.push_back(wr_server::Req{*ticket, mat, *params, now});
    srv->submitted++;
    srv->cv_work.notify_one();
    return WR_OK;
}

extern "C" wr_status wr_wait(wr_server *srv, uint64_t ticket, uint32_t timeout_ms, wr_result **out) {
    if (!srv || !out) return fail(WR_EINVAL, "null argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(srv->mu);
    bool ok = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                    [&] { return srv->done.count(ticket) > 0; });
    if (!ok) return fail(WR_ETIMEDOUT, "result not ready");
    auto d = srv->done[ticket];
    srv->done.erase(ticket);
    *out = d.res;
    return d.st;
}

extern "C" wr_status wr_server_stats(wr_server *srv, wr_stats *out) {
    if (!srv || !out) return fail(WR_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    std::vector<double> v = srv->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, q * v.size() - 1e-9));
        return v[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double span = srv->have_first ? std::chrono::duration<double>(srv->t_last - srv->t_first).count() : 0.0;
    out->throughput_rps = span > 0 ? (double)srv->completed / span : 0.0;
    out->max_resident = srv->max_resident;
    return WR_OK;
}

extern "C" void wr_server_stop(wr_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (auto &kv : srv->done) wr_result_free(kv.second.res);
    wr_destroy(srv->ctx);
    delete srv;
}
