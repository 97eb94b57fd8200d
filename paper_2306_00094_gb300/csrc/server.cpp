// Serving loop: requests (problem, right-hand sides) arrive at any time; a bounded set of
// slots runs them concurrently, each slot on its own CUDA stream with a stream-ordered
// workspace, so the kernels of requests in flight overlap on the device.  A request is
// admitted when a slot is free and its predicted device footprint fits the HBM budget;
// otherwise it waits in the queue.  Factorizations stay resident on the device in their
// problems (setup is paid once per problem and amortized over the requests).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

#include "solve.hpp"

using namespace nlf;

namespace {

struct Request {
    nlfeti_ticket id = 0;
    nlfeti_problem *prob = nullptr;
    int R = 0, kind = 0;
    std::vector<double> rhs, g, out;
    bool has_g = false;
    size_t bytes = 0;
    nlfeti_status status = NLFETI_OK;
    std::string err;
    nlfeti_stats stats{};
    bool done = false;
    std::chrono::steady_clock::time_point t_submit, t_start, t_done;
};

size_t predict_bytes(const nlfeti_problem *p, int R) {
    const size_t nl = (size_t)std::max<int64_t>(p->n_lambda, 1), nu = (size_t)std::max<int64_t>(p->n_u, 1),
                 nv = (size_t)std::max<int64_t>(p->sum_nk, 1), nd = (size_t)std::max<int64_t>(p->n_dofs_total, 1);
    return sizeof(double) * (size_t)R * (10 * nl + 4 * nu + 4 * nv + 4 * nd) + (1 << 20);
}

// Right-hand-side counts are rounded up to a few bucket sizes (the extra columns are zero and
// converge at once), so that a slot meets the same (problem, count) pairs again and reuses
// their workspaces and captured PCG graphs.
int rhs_bucket(int R) {
    static const int b[] = {1, 2, 4, 8, 12, 16, 24, 32};
    for (int v : b)
        if (R <= v) return v;
    return (R + 15) / 16 * 16;
}

// Recently used workspaces of one slot, keyed by (problem, right-hand-side count), bounded
// in bytes (least recently used first out).
struct WsCache {
    struct Entry {
        uint64_t uid = 0;
        int R = 0;
        size_t bytes = 0;
        uint64_t stamp = 0;
        std::unique_ptr<SolveWS> ws;
    };
    std::vector<Entry> entries;
    size_t bytes = 0, cap = 0;
    uint64_t clock = 0;
    SolveWS &get(nlfeti_problem *p, int R, cudaStream_t st) {
        for (auto &e : entries)
            if (e.uid == p->uid && e.R == R) {
                e.stamp = ++clock;
                return *e.ws;
            }
        const size_t need = predict_bytes(p, R);
        while (!entries.empty() && bytes + need > cap) {
            auto lru = std::min_element(entries.begin(), entries.end(),
                                        [](const Entry &a, const Entry &b) { return a.stamp < b.stamp; });
            bytes -= lru->bytes;
            entries.erase(lru);
        }
        Entry e;
        e.uid = p->uid;
        e.R = R;
        e.bytes = need;
        e.stamp = ++clock;
        e.ws.reset(new SolveWS());
        e.ws->async_stream = st;
        bytes += need;
        entries.push_back(std::move(e));
        return *entries.back().ws;
    }
};

}  // namespace

struct nlfeti_server {
    nlfeti_ctx *ctx = nullptr;
    size_t budget = 0, in_use = 0;
    int slots = 1, active = 0;
    bool stop = false;
    nlfeti_ticket next = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<nlfeti_ticket, std::shared_ptr<Request>> all;
    std::vector<std::thread> workers;

    void worker() {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return; }
        // each slot keeps recently used workspaces besides the admission budget: a share of
        // the budget (half of it over all slots), or 2 GiB without a budget
        WsCache cache;
        cache.cap = budget ? std::max<size_t>(size_t(256) << 20, budget / (2 * (size_t)slots)) : size_t(2) << 30;
        for (;;) {
            std::shared_ptr<Request> rq;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    if (stop) return true;
                    if (queue.empty()) return false;
                    const auto &h = queue.front();
                    return budget == 0 || in_use + h->bytes <= budget || active == 0;
                });
                if (stop && queue.empty()) break;
                if (queue.empty()) continue;
                rq = queue.front();
                queue.pop_front();
                in_use += rq->bytes;
                active++;
            }
            rq->t_start = std::chrono::steady_clock::now();
            nlfeti_status st_code = NLFETI_OK;
            std::string msg;
            try {
                nlfeti_problem *p = rq->prob;
                const int Rb = rhs_bucket(rq->R);
                SolveWS &ws = cache.get(p, Rb, st);
                const size_t bytes = sizeof(double) * (size_t)p->n_dofs_total * rq->R;
                const size_t bytes_b = sizeof(double) * (size_t)p->n_dofs_total * Rb;
                if (ws.in_rhs.bytes < bytes_b) ws.in_rhs.alloc_async(st, bytes_b);
                if (ws.out_u.bytes < bytes_b) ws.out_u.alloc_async(st, bytes_b);
                if (rq->has_g && ws.in_g.bytes < bytes_b) ws.in_g.alloc_async(st, bytes_b);
                NLF_CUDA(cudaMemcpyAsync(ws.in_rhs.p, rq->rhs.data(), bytes, cudaMemcpyHostToDevice, st));
                if (bytes_b > bytes)
                    NLF_CUDA(cudaMemsetAsync(ws.in_rhs.as<unsigned char>() + bytes, 0, bytes_b - bytes, st));
                if (rq->has_g) {
                    NLF_CUDA(cudaMemcpyAsync(ws.in_g.p, rq->g.data(), bytes, cudaMemcpyHostToDevice, st));
                    if (bytes_b > bytes)
                        NLF_CUDA(cudaMemsetAsync(ws.in_g.as<unsigned char>() + bytes, 0, bytes_b - bytes, st));
                }
                rq->out.resize((size_t)p->n_dofs_total * rq->R);
                try {
                    solve_device(p, ws, st, Rb, rq->kind, ws.in_rhs.as<double>(),
                                 rq->has_g ? ws.in_g.as<double>() : nullptr, ws.out_u.as<double>(), &rq->stats);
                } catch (const Error &e) {
                    if (e.st != NLFETI_E_NOT_CONVERGED) throw;
                    st_code = e.st;
                    msg = e.msg;
                }
                NLF_CUDA(cudaMemcpyAsync(rq->out.data(), ws.out_u.p, bytes, cudaMemcpyDeviceToHost, st));
                NLF_CUDA(cudaStreamSynchronize(st));
            } catch (const Error &e) {
                st_code = e.st;
                msg = e.msg;
                cudaStreamSynchronize(st);
            }
            rq->t_done = std::chrono::steady_clock::now();
            rq->stats.ms_solve = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_start).count();
            {
                std::lock_guard<std::mutex> lk(mu);
                rq->status = st_code;
                rq->err = msg;
                rq->done = true;
                in_use -= rq->bytes;
                active--;
                rq->rhs.clear();
                rq->rhs.shrink_to_fit();
                rq->g.clear();
                rq->g.shrink_to_fit();
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        cache.entries.clear();
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
};

extern "C" {

nlfeti_status nlfeti_server_create(nlfeti_ctx *ctx, size_t hbm_budget, int max_slots, nlfeti_server **out) {
    if (!ctx || !out || max_slots < 1 || max_slots > 64) return NLFETI_E_INVALID;
    nlfeti_server *s = new (std::nothrow) nlfeti_server();
    if (!s) return NLFETI_E_NOMEM;
    s->ctx = ctx;
    s->budget = hbm_budget;
    s->slots = max_slots;
    try {
        for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s] { s->worker(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->workers) t.join();
        delete s;
        return NLFETI_E_INVALID;
    }
    ctx_attach(ctx);
    *out = s;
    return NLFETI_OK;
}

nlfeti_status nlfeti_submit(nlfeti_server *s, nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs,
                            const double *g, nlfeti_ticket *out) {
    if (!s || !p || !rhs || !out || nrhs < 1 || (rhs_kind != 0 && rhs_kind != 1)) return NLFETI_E_INVALID;
    if ((p->opt.precision == 0 && !p->op64.ready) || (p->opt.precision == 1 && !p->op32.ready)) {
        set_error(s->ctx, "problem not factored for its precision");
        return NLFETI_E_INVALID;
    }
    auto rq = std::make_shared<Request>();
    rq->prob = p;
    rq->R = nrhs;
    rq->kind = rhs_kind;
    const size_t n = (size_t)p->n_dofs_total * nrhs;
    try {
        rq->rhs.assign(rhs, rhs + n);
        if (g) { rq->g.assign(g, g + n); rq->has_g = true; }
    } catch (...) {
        return NLFETI_E_NOMEM;
    }
    rq->bytes = predict_bytes(p, nrhs) + (g ? 3 : 2) * sizeof(double) * n;
    if (s->budget && rq->bytes > s->budget) {
        set_error(s->ctx, "request footprint exceeds the server HBM budget");
        return NLFETI_E_NOMEM;
    }
    rq->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        rq->id = s->next++;
        s->queue.push_back(rq);
        s->all[rq->id] = rq;
    }
    s->cv_work.notify_one();
    *out = rq->id;
    return NLFETI_OK;
}

nlfeti_status nlfeti_wait(nlfeti_server *s, nlfeti_ticket t, int timeout_ms, double *u_out, nlfeti_stats *stats) {
    if (!s) return NLFETI_E_INVALID;
    std::shared_ptr<Request> rq;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->all.find(t);
        if (it == s->all.end()) return NLFETI_E_INVALID;
        rq = it->second;
        auto pred = [&] { return rq->done; };
        if (timeout_ms < 0) s->cv_done.wait(lk, pred);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return NLFETI_E_TIMEOUT;
        s->all.erase(t);
    }
    if (u_out && !rq->out.empty()) std::copy(rq->out.begin(), rq->out.end(), u_out);
    if (stats) {
        *stats = rq->stats;
        stats->ms_queue = std::chrono::duration<double, std::milli>(rq->t_start - rq->t_submit).count();
    }
    if (rq->status != NLFETI_OK) set_error(s->ctx, rq->err);
    return rq->status;
}

void nlfeti_server_destroy(nlfeti_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    nlfeti_ctx *c = s->ctx;
    delete s;
    ctx_detach(c);
}

}  // extern "C"
