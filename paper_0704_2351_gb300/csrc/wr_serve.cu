// Batched rank jobs and the continuous-batching rank server.
//
// Both run every job through the same single-job path (rank_one), each job on
// one of several slots.  A slot is a context of its own (its own non-blocking
// stream on the caller's device) driven by one host thread, so the captured
// sequence loops and the sigma-basis kernels of different jobs are in flight
// on the device at the same time: small matrices that cannot fill 152 SMs on
// their own share the GPU, and the single-block M-Basis chunks of several jobs
// run side by side.  A job's kernels, launch shapes and arithmetic do not
// depend on what runs beside it, so its result is bit-identical to the same
// job run alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "wr_internal.cuh"

namespace wr {
wr_status rank_one(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params, wr_result **out);
wr_status rank_multi(wr_ctx *ctx, const wr_matrix *mat, const wr_params *const *params, int G, wr_result **outs);

// Upper bound of the device memory one rank_one call allocates besides the
// loaded matrix: the kept sequence and basis, the sequence state (blocks,
// diagonals, split accumulators, exact term sums) beside the sigma-basis
// state (the sigma-basis trails the sequence while it runs), then the
// readout (after both are released).
size_t rank_device_bytes(const wr_ctx *ctx, const wr_matrix *mat, const Resolved &r, int num_sms) {
    // the paired generic block (m = n) runs the SpMM at twice the width
    const bool pairable = !r.symmetric && r.m == r.n && 2 * r.nv <= 64;
    const size_t L = (size_t)r.L, m = (size_t)r.m, n = (size_t)r.n, q = m + n,
                 nv = (size_t)r.nv * (pairable ? 2 : 1);
    const size_t N = (size_t)r.N, M = (size_t)r.M;
    const size_t nsplit = (size_t)(mat->a.nsplit + mat->at.nsplit);
    const size_t seq = 4 * N * nv + 4 * M * nv + 4 * (3 * N + 2 * M) + 4 * N * m + 8 * nv * nsplit + 8 * L * m * n;
    const size_t keep = 4 * L * m * n + 4 * (L + 2) * n * q + 4 * q;
    size_t sigma = 4 * (L + 2) * n * q + 4 * (size_t)(2 * num_sms) * 64 * m * q + 4 * 65 * q * q + 4 * (m * q + 4 * q);
    if (sigma_uses_pm(ctx, (int64_t)L, (int)m, (int)n)) {
        // PM-Basis: the residual F, three bases of up to L/2 + 2 coefficients
        // (the basis so far, a segment's or half's, their product), one
        // product's transform buffers (operands and three outputs of Lz
        // points, Lz <= the power of two >= L) and the twiddle tables
        size_t Lz = 1;
        while (Lz < L) Lz <<= 1;
        sigma += 4 * L * m * q + 3 * 4 * (L / 2 + 2) * q * q + 4 * 5 * q * q * Lz + 4 * 6 * (Lz / 2);
    }
    const size_t readout = 4 * 2 * (L + 2) * n * n + 64;
    return keep + std::max(seq + sigma, readout) + (1u << 20);
}

}  // namespace wr

using namespace wr;

extern "C" wr_status wr_rank_device_bytes(const wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                          uint64_t *bytes) {
    if (!ctx || !mat || !params || !bytes) return fail(WR_EINVAL, "null argument");
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    *bytes = r.N == 0 ? 0 : (uint64_t)rank_device_bytes(ctx, mat, r, ctx->num_sms);
    return WR_OK;
}

extern "C" wr_status wr_set_batch_slots(wr_ctx *ctx, int32_t slots) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if (slots < 1 || slots > 64) return fail(WR_EINVAL, "batch slots must be in 1..64");
    ctx->batch_slots = slots;
    return WR_OK;
}

extern "C" wr_status wr_set_batch_fusion(wr_ctx *ctx, int32_t on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->batch_fuse = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_rank_batch(wr_ctx *ctx, size_t njobs, const wr_matrix *const *mats,
                                   const wr_params *params, wr_result **outs) {
    if (!ctx || (njobs && (!mats || !params || !outs))) return fail(WR_EINVAL, "null argument");
    for (size_t j = 0; j < njobs; j++) outs[j] = nullptr;
    if (njobs == 0) return WR_OK;
    auto t0 = std::chrono::steady_clock::now();
    // Work items: single jobs, or groups of up to 4 jobs on the same matrix
    // with the same m = n, side, length and outputs (any primes and seeds)
    // that share one sequence loop (fusion on, early termination off).
    std::vector<double> cost(njobs, 0.0);
    std::vector<Resolved> rs(njobs);
    std::vector<char> ok(njobs, 0);
    for (size_t j = 0; j < njobs; j++) {
        if (mats[j] && resolve(mats[j], &params[j], rs[j]) == WR_OK) {
            ok[j] = 1;
            cost[j] = (double)rs[j].L * (double)(mats[j]->nnz + 1) * rs[j].nv;
        }
    }
    std::vector<std::vector<size_t>> items;
    {
        std::vector<char> used(njobs, 0);
        for (size_t j = 0; j < njobs; j++) {
            if (used[j]) continue;
            used[j] = 1;
            std::vector<size_t> it{j};
            const bool fusable = ctx->batch_fuse && ctx->early_term == 0 && ok[j] && rs[j].N > 0 &&
                                 multi_eligible(ctx, rs[j]);
            if (fusable) {
                const int gmax = multi_max_jobs(rs[j]);
                for (size_t k = j + 1; k < njobs && (int)it.size() < gmax; k++) {
                    if (used[k] || !ok[k] || mats[k] != mats[j]) continue;
                    const Resolved &a = rs[j], &b = rs[k];
                    if (b.m != a.m || b.n != a.n || b.side != a.side || b.L != a.L || b.symmetric != a.symmetric ||
                        params[k].want != params[j].want)
                        continue;
                    used[k] = 1;
                    it.push_back(k);
                }
            }
            items.push_back(std::move(it));
        }
    }
    // largest items first (longest-processing-time order balances the slots)
    std::vector<double> icost(items.size(), 0.0);
    for (size_t i = 0; i < items.size(); i++)
        for (size_t j : items[i]) icost[i] += cost[j];
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return icost[a] > icost[b]; });

    const int nslots = (int)std::min<size_t>(items.size(), (size_t)std::max(1, ctx->batch_slots));
    std::vector<wr_ctx *> slots(nslots, nullptr);
    for (int k = 0; k < nslots; k++) {
        wr_status st = make_child(ctx, &slots[k]);
        if (st != WR_OK) {
            for (auto *c : slots) wr_destroy(c);
            return st;
        }
    }
    std::vector<wr_status> status(njobs, WR_OK);
    std::vector<std::string> msg(njobs);
    std::atomic<size_t> next{0};
    auto worker = [&](int k) {
        cudaSetDevice(ctx->device);
        for (;;) {
            const size_t i = next.fetch_add(1);
            if (i >= items.size()) return;
            const std::vector<size_t> &it = items[order[i]];
            if (it.size() == 1) {
                const size_t j = it[0];
                status[j] = rank_one(slots[k], mats[j], &params[j], &outs[j]);
                if (status[j] != WR_OK) msg[j] = wr_last_error();
                continue;
            }
            std::vector<const wr_params *> ps;
            std::vector<wr_result *> rr(it.size(), nullptr);
            for (size_t j : it) ps.push_back(&params[j]);
            const wr_status st = rank_multi(slots[k], mats[it[0]], ps.data(), (int)it.size(), rr.data());
            const std::string m = st != WR_OK ? wr_last_error() : std::string();
            for (size_t g = 0; g < it.size(); g++) {
                outs[it[g]] = rr[g];
                status[it[g]] = st;
                msg[it[g]] = m;
            }
        }
    };
    std::vector<std::thread> th;
    for (int k = 1; k < nslots; k++) th.emplace_back(worker, k);
    worker(0);
    for (auto &t : th) t.join();
    for (auto *c : slots) {
        ctx->launches += c->launches;
        wr_destroy(c);
    }
    ctx->last = wr_timings{};
    ctx->last.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (size_t j = 0; j < njobs; j++)
        if (status[j] != WR_OK) return fail(status[j], "batch job " + std::to_string(j) + ": " + msg[j]);
    return WR_OK;
}

// ------------------------------------------------------------------ server

struct wr_server {
    int device = 0;
    wr_server_cfg cfg{};
    std::vector<wr_ctx *> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    struct Req {
        uint64_t ticket;
        const wr_matrix *mat;
        wr_params prm;
        uint64_t bytes;  // admission estimate
        std::chrono::steady_clock::time_point t_submit;
    };
    std::deque<Req> queue;
    struct Done {
        wr_status st;
        wr_result *res;
        std::string msg;
    };
    std::map<uint64_t, Done> done;
    std::vector<double> lat_ms;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0;
    uint64_t resident_bytes = 0;
    int32_t resident = 0, max_resident = 0;
    std::chrono::steady_clock::time_point t_first, t_last;
    bool have_first = false, stop = false;
    std::vector<std::thread> workers;
};

// The head of the queue is admitted when a slot is idle (this worker) and
// its memory estimate fits beside the requests already resident.  Strict
// arrival order: a large request at the head waits for memory rather than
// being overtaken indefinitely.
static bool admissible(const wr_server *s) {
    if (s->queue.empty()) return false;
    if (s->cfg.hbm_budget == 0 || s->resident == 0) return true;
    return s->resident_bytes + s->queue.front().bytes <= s->cfg.hbm_budget;
}

static void server_loop(wr_server *s, int k) {
    cudaSetDevice(s->device);
    wr_ctx *ctx = s->slots[k];
    for (;;) {
        wr_server::Req rq;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return (s->stop && s->queue.empty()) || admissible(s); });
            if (s->queue.empty()) return;  // stopping
            rq = s->queue.front();
            s->queue.pop_front();
            s->resident++;
            s->resident_bytes += rq.bytes;
            s->max_resident = std::max(s->max_resident, s->resident);
        }
        s->cv_work.notify_all();  // the next head may fit as well
        wr_result *res = nullptr;
        wr_status st = rank_one(ctx, rq.mat, &rq.prm, &res);
        std::string msg = st == WR_OK ? std::string() : std::string(wr_last_error());
        auto now = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->resident--;
            s->resident_bytes -= rq.bytes;
            s->done[rq.ticket] = wr_server::Done{st, res, msg};
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - rq.t_submit).count());
            if (st == WR_OK) s->completed++;
            else s->failed++;
            s->t_last = now;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

extern "C" wr_status wr_server_start(wr_ctx *ctx, const wr_server_cfg *cfg, wr_server **out) {
    if (!ctx || !cfg || !out) return fail(WR_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->max_slots > 64) return fail(WR_EINVAL, "max_slots must be at most 64");
    wr_server *s = new wr_server();
    s->device = ctx->device;
    s->cfg = *cfg;
    if (s->cfg.max_slots < 1) s->cfg.max_slots = 1;
    if (s->cfg.queue_cap < 1) s->cfg.queue_cap = 1 << 20;
    for (int k = 0; k < s->cfg.max_slots; k++) {
        wr_ctx *c = nullptr;
        wr_status st = make_child(ctx, &c);
        if (st != WR_OK) {
            for (auto *x : s->slots) wr_destroy(x);
            delete s;
            return st;
        }
        s->slots.push_back(c);
    }
    for (int k = 0; k < s->cfg.max_slots; k++) s->workers.emplace_back(server_loop, s, k);
    *out = s;
    return WR_OK;
}

extern "C" wr_status wr_submit(wr_server *srv, const wr_matrix *mat, const wr_params *params, uint64_t *ticket) {
    if (!srv || !mat || !params || !ticket) return fail(WR_EINVAL, "null argument");
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    const uint64_t bytes = r.N == 0 ? 0 : (uint64_t)rank_device_bytes(srv->slots[0], mat, r, srv->slots[0]->num_sms);
    if (srv->cfg.hbm_budget && bytes > srv->cfg.hbm_budget)
        return fail(WR_EINVAL, "request needs up to " + std::to_string(bytes) + " bytes of device memory, above the "
                               "server's budget of " + std::to_string(srv->cfg.hbm_budget));
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return fail(WR_EBUSY, "server stopping");
        if ((int64_t)srv->queue.size() >= srv->cfg.queue_cap) return fail(WR_EBUSY, "server queue full");
        auto now = std::chrono::steady_clock::now();
        if (!srv->have_first) {
            srv->t_first = now;
            srv->have_first = true;
        }
        *ticket = srv->next_ticket++;
        srv->queue.push_back(wr_server::Req{*ticket, mat, *params, bytes, now});
        srv->submitted++;
    }
    srv->cv_work.notify_all();
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
    if (d.st != WR_OK) return fail(d.st, d.msg);
    return WR_OK;
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
    out->kernel_launches = 0;
    for (auto *c : srv->slots) out->kernel_launches += c->launches;
    return WR_OK;
}

extern "C" void wr_server_stop(wr_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers)
        if (t.joinable()) t.join();
    for (auto &kv : srv->done) wr_result_free(kv.second.res);
    for (auto *c : srv->slots) wr_destroy(c);
    delete srv;
}
