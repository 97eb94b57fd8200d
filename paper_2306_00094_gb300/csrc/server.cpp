// Serving loop with continuous batching.
//
// Requests (a problem and its right-hand sides) arrive at any time.  A bounded set of slots
// (worker threads, each with its own CUDA stream) runs them, so the kernels of the batches in
// flight overlap on the device.  When a slot takes the request at the head of the queue it
// also takes the other queued requests on the same problem with the same kind of load, up to
// kMergeCols right-hand sides: they run as one batched solve whose launches serve all of them
// (every column of a batched solve is computed in an order that does not depend on the other
// columns, so each request gets bitwise the result it would get alone).  A request that
// arrives while a batch of its problem runs joins the next batch.
//
// Memory: the server counts the device bytes it holds -- the solve workspaces it keeps (per
// problem and right-hand-side bucket; a workspace in use by a slot or cached for reuse) and
// the problems it created itself for requests given by their inputs (nlfeti_submit_mesh) --
// against its HBM budget.  A batch is admitted when a slot is free and its workspace (and, for
// a problem not yet created, the problem's predicted footprint) fits the budget after evicting
// idle cached workspaces and problems, least recently used first; otherwise it waits.
// Problems the caller created and passes to nlfeti_submit are the caller's memory.
//
// Factorization cache: a request given by its inputs (mesh, kernel, decomposition, options) is
// keyed by a hash of their contents; the first request of a key creates, assembles and factors
// the problem in its slot (ms_setup / ms_factor in its stats), later ones reuse it while it
// stays cached (setup amortized over repeated solves, as in the paper's timings).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <thread>

#include "solve.hpp"

using namespace nlf;

namespace {

constexpr int kMergeCols = 64;   // right-hand sides of one batch, at most

// a problem given by its inputs (copied at submission)
struct Inputs {
    int dim = 2;
    int64_t n_nodes = 0, n_elems = 0;
    std::vector<double> xy;
    std::vector<int32_t> elems, labels;
    std::vector<int8_t> node_dir, elem_dir;
    nlfeti_kernel kern{};
    int32_t K = 0;
    nlfeti_options opt{};
    nlfeti_mesh mesh() const {
        return nlfeti_mesh{dim, n_nodes, xy.data(), n_elems, elems.data(), node_dir.data(), elem_dir.data()};
    }
    nlfeti_decomp decomp() const { return nlfeti_decomp{K, labels.data()}; }
};

struct Request {
    nlfeti_ticket id = 0;
    nlfeti_problem *prob = nullptr;       // the caller's, or the cached one (set by the slot)
    uint64_t key = 0;                     // requests by inputs: the cache key
    std::shared_ptr<Inputs> inputs;
    int R = 0, kind = 0;
    std::vector<double> rhs, g, out;
    bool has_g = false;
    nlfeti_status status = NLFETI_OK;
    std::string err;
    nlfeti_stats stats{};
    bool done = false;
    std::chrono::steady_clock::time_point t_submit, t_start, t_done;
};

uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

size_t predict_ws_bytes(const nlfeti_problem *p, int R) {
    const size_t nl = (size_t)std::max<int64_t>(p->n_lambda, 1), nu = (size_t)std::max<int64_t>(p->n_u, 1),
                 nv = (size_t)std::max<int64_t>(p->sum_nk, 1), nd = (size_t)std::max<int64_t>(p->n_dofs_total, 1),
                 nup = (size_t)std::max<int64_t>(p->n_up, 1), nvp = (size_t)std::max<int64_t>(p->n_vp, 1);
    // Lambda (10), U (3) and subdomain (4) vectors, the apply and residual inputs, the forcing
    // right-hand sides, the load vector, and the input / output / Dirichlet staging (3 n_dofs);
    // in FP32: the 7 Lambda vectors of the FP32 PCG iterations and the paired apply input
    const size_t nxp = (size_t)std::max<int64_t>(p->n_xp, 1), R2 = (size_t)(R + 1) / 2 * 2;
    return sizeof(double) * (size_t)R * (10 * nl + 3 * nu + nup + 4 * nv + 2 * nvp + 4 * nd) +
           sizeof(float) * (7 * nl * (size_t)R + nxp * R2) + (size_t(2) << 20);
}

// Right-hand-side counts are rounded up to a few bucket sizes (the extra columns are zero and
// converge at once), so that a slot meets the same (problem, count) pairs again and reuses
// their workspaces and captured PCG graphs.
int rhs_bucket(int R) {
    static const int b[] = {1, 2, 4, 8, 12, 16, 24, 32, 48, 64};
    for (int v : b)
        if (R <= v) return v;
    return (R + 15) / 16 * 16;
}

struct WsEntry {
    uint64_t uid = 0;
    int R = 0;
    size_t bytes = 0;
    uint64_t stamp = 0;
    bool in_use = false;
    std::unique_ptr<SolveWS> ws;
};

struct CachedProblem {
    uint64_t key = 0;
    nlfeti_problem *p = nullptr;
    size_t bytes = 0;
    int inflight = 0;
    uint64_t stamp = 0;
    bool ready = false;    // created and factored (or failed: p == nullptr)
};

}  // namespace

struct nlfeti_server {
    nlfeti_ctx *ctx = nullptr;
    size_t budget = 0, bytes = 0, peak_bytes = 0;
    int slots = 1, active = 0, peak_active = 0;
    bool stop = false;
    nlfeti_ticket next = 1;
    uint64_t clock = 0;
    int64_t n_done = 0, n_batches = 0, n_merged = 0, n_hits = 0, n_misses = 0, n_evicted = 0;
    std::mutex mu, create_mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<nlfeti_ticket, std::shared_ptr<Request>> all;
    std::list<WsEntry> wss;                 // list: entries stay put while others come and go
    std::list<CachedProblem> probs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;      // one per slot, alive until the server is destroyed
    cudaStream_t alloc_stream = nullptr;    // allocations and frees of the workspaces (never captured)

    void charge(size_t b) {
        bytes += b;
        peak_bytes = std::max(peak_bytes, bytes);
    }

    // the cached problem of a key (nullptr if none)
    CachedProblem *find_problem(uint64_t key) {
        for (auto &c : probs)
            if (c.key == key) return &c;
        return nullptr;
    }

    // free idle entries, least recently used first, until need more bytes fit (mu held);
    // returns whether they fit
    bool make_room(size_t need) {
        if (budget == 0) return true;
        while (bytes + need > budget) {
            // the least recently used idle workspace or idle problem
            auto w = wss.end();
            for (auto it = wss.begin(); it != wss.end(); ++it)
                if (!it->in_use && (w == wss.end() || it->stamp < w->stamp)) w = it;
            auto c = probs.end();
            for (auto it = probs.begin(); it != probs.end(); ++it)
                if (it->ready && it->p && it->inflight == 0 && (c == probs.end() || it->stamp < c->stamp)) c = it;
            if (w == wss.end() && c == probs.end()) return false;
            if (w != wss.end() && (c == probs.end() || w->stamp <= c->stamp)) {
                bytes -= w->bytes;
                wss.erase(w);
            } else {
                evict_problem(c);
            }
        }
        return true;
    }

    void evict_problem(std::list<CachedProblem>::iterator c) {
        const uint64_t uid = c->p->uid;
        for (auto it = wss.begin(); it != wss.end();) {
            if (it->uid == uid && !it->in_use) {
                bytes -= it->bytes;
                it = wss.erase(it);
            } else {
                ++it;
            }
        }
        nlfeti_problem_destroy(c->p);
        bytes -= c->bytes;
        ++n_evicted;
        probs.erase(c);
    }

    // the batch a request starts (mu held): it and the later queued requests on the same
    // problem with the same kind of load, while the columns fit kMergeCols
    std::vector<std::shared_ptr<Request>> take_batch(const std::shared_ptr<Request> &head) {
        std::vector<std::shared_ptr<Request>> b;
        b.push_back(head);
        int cols = head->R;
        bool after = false;
        for (auto &q : queue) {
            if (q == head) { after = true; continue; }
            if (!after) continue;
            const bool same = head->inputs ? (q->inputs && q->key == head->key) : (!q->inputs && q->prob == head->prob);
            if (same && q->kind == head->kind && cols + q->R <= kMergeCols) {
                b.push_back(q);
                cols += q->R;
            }
        }
        return b;
    }

    void worker(cudaStream_t st) {
        for (;;) {
            std::vector<std::shared_ptr<Request>> batch;
            WsEntry *wsent = nullptr;
            CachedProblem *cp = nullptr;
            bool create = false;
            size_t create_bytes = 0;
            nlfeti_problem *p = nullptr;
            int Rb = 0, cols = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop && queue.empty()) break;
                    if (!queue.empty() && admit(batch, wsent, cp, create, create_bytes, p, Rb, cols)) break;
                    cv_work.wait(lk);
                }
                if (batch.empty()) break;
            }
            run_batch(st, batch, wsent, cp, create, create_bytes, p, Rb, cols);
        }
        cudaStreamSynchronize(st);
    }

    // admission (mu held): the first queued request that is not waiting for another slot to
    // create its problem starts a batch; on success the batch is out of the queue, its workspace
    // entry reserved and counted, and its problem pinned.  A batch that does not fit the budget
    // yet waits (and holds back the requests behind it, first come first served).
    bool admit(std::vector<std::shared_ptr<Request>> &batch, WsEntry *&wsent, CachedProblem *&cp, bool &create,
               size_t &create_bytes, nlfeti_problem *&p, int &Rb, int &cols) {
        std::shared_ptr<Request> head;
        for (;;) {
            head = nullptr;
            cp = nullptr;
            create = false;
            for (auto &q : queue) {
                if (!q->inputs) { head = q; break; }
                CachedProblem *c = find_problem(q->key);
                if (c && !c->ready) continue;               // being created by another slot
                head = q;
                cp = c;
                break;
            }
            if (!head) return false;
            if (head->inputs && cp && !cp->p) {             // its creation failed just now
                queue.erase(std::find(queue.begin(), queue.end(), head));
                finish_locked(head, NLFETI_E_INVALID, "the problem of this request could not be created");
                continue;
            }
            if (head->inputs && !cp) {
                create = true;
                create_bytes = predict_bytes_of(*head->inputs);
                if (create_bytes == 0) {                    // invalid inputs: refused
                    queue.erase(std::find(queue.begin(), queue.end(), head));
                    finish_locked(head, NLFETI_E_INVALID, "invalid problem inputs");
                    continue;
                }
            }
            break;
        }
        p = head->inputs ? (cp ? cp->p : nullptr) : head->prob;
        batch = take_batch(head);
        cols = 0;
        for (auto &r : batch) cols += r->R;
        Rb = rhs_bucket(cols);
        // workspace: a free cached one of this (problem, bucket), or a new one
        wsent = nullptr;
        if (!create)
            for (auto &e : wss)
                if (!e.in_use && e.uid == p->uid && e.R == Rb) wsent = &e;
        size_t need = 0, ws_bytes = 0;
        if (!wsent) {
            // a new problem's workspace is sized once the problem exists: reserve a share of
            // the problem's footprint meanwhile (settled after the creation)
            ws_bytes = create ? std::max<size_t>(create_bytes / 8, size_t(64) << 20) : predict_ws_bytes(p, Rb);
            need += ws_bytes;
        }
        if (create) need += create_bytes;
        if (budget && need > budget) {
            for (auto &r : batch) {
                queue.erase(std::find(queue.begin(), queue.end(), r));
                finish_locked(r, NLFETI_E_NOMEM, "request footprint exceeds the server HBM budget");
            }
            batch.clear();
            return false;
        }
        // pin the entries that must survive the eviction below
        if (wsent) wsent->in_use = true;
        if (cp) cp->inflight++;
        if (!make_room(need)) {
            if (wsent) wsent->in_use = false;
            if (cp) cp->inflight--;
            batch.clear();
            return false;
        }
        for (auto &r : batch) queue.erase(std::find(queue.begin(), queue.end(), r));
        if (!wsent) {
            WsEntry e;
            e.uid = create ? 0 : p->uid;
            e.R = Rb;
            e.bytes = ws_bytes;
            e.in_use = true;
            e.ws.reset(new SolveWS());
            e.ws->alloc_stream = alloc_stream;
            wss.push_back(std::move(e));
            wsent = &wss.back();
            charge(ws_bytes);
        }
        wsent->stamp = ++clock;
        if (create) {
            CachedProblem c;
            c.key = head->key;
            c.bytes = create_bytes;
            c.inflight = 1;
            c.stamp = ++clock;
            probs.push_back(c);
            cp = &probs.back();
            charge(create_bytes);
            ++n_misses;
        } else if (cp) {
            cp->stamp = ++clock;
            ++n_hits;
        }
        active++;
        peak_active = std::max(peak_active, active);
        ++n_batches;
        if (batch.size() > 1) n_merged += (int64_t)batch.size();
        for (auto &r : batch) r->t_start = std::chrono::steady_clock::now();
        return true;
    }

    size_t predict_bytes_of(const Inputs &in) {
        try {
            const nlfeti_mesh m = in.mesh();
            const nlfeti_decomp d = in.decomp();
            return predict_problem_bytes(&m, &in.kern, &d, in.opt.precision == 1 ? 2 : 1);
        } catch (...) {
            return 0;
        }
    }

    void finish_locked(const std::shared_ptr<Request> &r, nlfeti_status st, const std::string &msg) {
        r->status = st;
        r->err = msg;
        r->done = true;
        r->t_done = std::chrono::steady_clock::now();
        r->rhs.clear();
        r->g.clear();
        cv_done.notify_all();
    }

    // pointers into wss / probs are re-found by identity after the lock is released
    void run_batch(cudaStream_t st, std::vector<std::shared_ptr<Request>> &batch, WsEntry *wsent, CachedProblem *cp,
                   bool create, size_t create_bytes, nlfeti_problem *p, int Rb, int cols) {
        SolveWS *ws = wsent->ws.get();
        const uint64_t key = cp ? cp->key : 0;
        nlfeti_status code = NLFETI_OK;
        std::string msg;
        double ms_setup = 0, ms_factor = 0;
        auto &head = batch.front();
        if (create) {
            // create, assemble and factor the problem (the context is not thread-safe: one
            // creation at a time, on the context's stream)
            std::lock_guard<std::mutex> g(create_mu);
            const nlfeti_mesh m = head->inputs->mesh();
            const nlfeti_decomp d = head->inputs->decomp();
            nlfeti_problem *np = nullptr;
            code = nlfeti_problem_create(ctx, &m, &head->inputs->kern, &d, &np);
            if (code == NLFETI_OK) {
                nlfeti_problem_set_options(np, &head->inputs->opt);
                code = nlfeti_factor(np, head->inputs->opt.precision == 1 ? 2 : 1);
                if (code != NLFETI_OK) {
                    nlfeti_problem_destroy(np);
                    np = nullptr;
                }
            }
            if (code != NLFETI_OK) msg = nlfeti_last_error(ctx);
            else {
                ms_setup = np->ms_setup;
                ms_factor = np->ms_factor;
            }
            p = np;
            std::lock_guard<std::mutex> lk(mu);
            CachedProblem *c = find_problem(key);
            c->p = np;
            c->ready = true;
            if (np) {
                wsent = find_ws(ws);
                wsent->uid = np->uid;
            }
            cv_work.notify_all();
        }
        if (code == NLFETI_OK) {
            try {
                ws->async_stream = st;      // the slot's stream (the workspace may have served another)
                const int64_t nd = p->n_dofs_total;
                const size_t bytes_b = sizeof(double) * (size_t)nd * Rb;
                if (ws->in_rhs.bytes < bytes_b) ws->in_rhs.alloc_async(alloc_stream, bytes_b);
                if (ws->out_u.bytes < bytes_b) ws->out_u.alloc_async(alloc_stream, bytes_b);
                bool any_g = false;
                for (auto &r : batch) any_g |= r->has_g;
                if (any_g && ws->in_g.bytes < bytes_b) ws->in_g.alloc_async(alloc_stream, bytes_b);
                NLF_CUDA(cudaStreamSynchronize(alloc_stream));
                // the columns of the batch, then zero columns up to the bucket
                size_t col = 0;
                for (auto &r : batch) {
                    const size_t n = sizeof(double) * (size_t)nd * r->R;
                    NLF_CUDA(cudaMemcpyAsync(ws->in_rhs.as<unsigned char>() + col, r->rhs.data(), n,
                                             cudaMemcpyHostToDevice, st));
                    if (any_g) {
                        if (r->has_g)
                            NLF_CUDA(cudaMemcpyAsync(ws->in_g.as<unsigned char>() + col, r->g.data(), n,
                                                     cudaMemcpyHostToDevice, st));
                        else
                            NLF_CUDA(cudaMemsetAsync(ws->in_g.as<unsigned char>() + col, 0, n, st));
                    }
                    col += n;
                }
                if (bytes_b > col) {
                    NLF_CUDA(cudaMemsetAsync(ws->in_rhs.as<unsigned char>() + col, 0, bytes_b - col, st));
                    if (any_g) NLF_CUDA(cudaMemsetAsync(ws->in_g.as<unsigned char>() + col, 0, bytes_b - col, st));
                }
                nlfeti_stats s{};
                try {
                    solve_device(p, *ws, st, Rb, head->kind, ws->in_rhs.as<double>(),
                                 any_g ? ws->in_g.as<double>() : nullptr, ws->out_u.as<double>(), &s);
                } catch (const Error &e) {
                    if (e.st != NLFETI_E_NOT_CONVERGED) throw;
                    code = e.st;
                    msg = e.msg;
                }
                col = 0;
                for (auto &r : batch) {
                    const size_t n = sizeof(double) * (size_t)nd * r->R;
                    r->out.resize((size_t)nd * r->R);
                    NLF_CUDA(cudaMemcpyAsync(r->out.data(), ws->out_u.as<unsigned char>() + col, n,
                                             cudaMemcpyDeviceToHost, st));
                    r->stats = s;
                    col += n;
                }
                NLF_CUDA(cudaStreamSynchronize(st));
            } catch (const Error &e) {
                code = e.st;
                msg = e.msg;
                cudaStreamSynchronize(st);
            }
        }
        const auto t_done = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(mu);
            auto wit = std::find_if(wss.begin(), wss.end(), [&](const WsEntry &e) { return e.ws.get() == ws; });
            WsEntry *w = &*wit;
            if (!p) {                                   // failed creation: drop its workspace
                bytes -= w->bytes;
                wss.erase(wit);
            } else {
                w->in_use = false;
                w->stamp = ++clock;
                if (create && w->bytes < predict_ws_bytes(p, Rb)) {
                    // the workspace's own size, now that the problem exists
                    const size_t real = predict_ws_bytes(p, Rb);
                    charge(real - w->bytes);
                    w->bytes = real;
                }
            }
            if (key) {
                auto cit = std::find_if(probs.begin(), probs.end(), [&](const CachedProblem &c) { return c.key == key; });
                if (cit != probs.end()) {
                    cit->inflight--;
                    if (!cit->p) {                      // failed creation: forget the key
                        bytes -= cit->bytes;
                        probs.erase(cit);
                    }
                }
            }
            (void)create_bytes;
            for (auto &r : batch) {
                r->t_done = t_done;
                r->stats.ms_solve = std::chrono::duration<double, std::milli>(t_done - r->t_start).count();
                r->stats.ms_setup = create ? ms_setup : 0.0;
                r->stats.ms_factor = create ? ms_factor : 0.0;
                r->status = code;
                r->err = msg;
                r->done = true;
                r->rhs.clear();
                r->rhs.shrink_to_fit();
                r->g.clear();
                r->g.shrink_to_fit();
                ++n_done;
            }
            active--;
            (void)cols;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }

    WsEntry *find_ws(SolveWS *ws) {
        for (auto &e : wss)
            if (e.ws.get() == ws) return &e;
        return nullptr;
    }

    nlfeti_status enqueue(std::shared_ptr<Request> rq, nlfeti_ticket *out) {
        rq->t_submit = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(mu);
            if (stop) return NLFETI_E_INVALID;
            rq->id = next++;
            queue.push_back(rq);
            all[rq->id] = rq;
        }
        cv_work.notify_all();
        *out = rq->id;
        return NLFETI_OK;
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
    if (cudaStreamCreateWithFlags(&s->alloc_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return NLFETI_E_CUDA;
    }
    for (int i = 0; i < max_slots; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto x : s->streams) cudaStreamDestroy(x);
            cudaStreamDestroy(s->alloc_stream);
            delete s;
            return NLFETI_E_CUDA;
        }
        s->streams.push_back(st);
    }
    try {
        for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s, i] { s->worker(s->streams[i]); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->workers) t.join();
        for (auto x : s->streams) cudaStreamDestroy(x);
        cudaStreamDestroy(s->alloc_stream);
        delete s;
        return NLFETI_E_INVALID;
    }
    ctx_attach(ctx);
    *out = s;
    return NLFETI_OK;
}

nlfeti_status nlfeti_submit(nlfeti_server *s, nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs,
                            const double *g, nlfeti_ticket *out) {
    if (!s || !p || !rhs || !out || nrhs < 1 || nrhs > kMergeCols || (rhs_kind != 0 && rhs_kind != 1))
        return NLFETI_E_INVALID;
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
    if (s->budget && predict_ws_bytes(p, rhs_bucket(nrhs)) > s->budget) {
        set_error(s->ctx, "request footprint exceeds the server HBM budget");
        return NLFETI_E_NOMEM;
    }
    return s->enqueue(rq, out);
}

nlfeti_status nlfeti_submit_mesh(nlfeti_server *s, const nlfeti_mesh *mesh, const nlfeti_kernel *kernel,
                                 const nlfeti_decomp *decomp, const nlfeti_options *opt, int nrhs, int rhs_kind,
                                 const double *rhs, const double *g, nlfeti_ticket *out) {
    if (!s || !mesh || !kernel || !decomp || !rhs || !out || nrhs < 1 || nrhs > kMergeCols ||
        (rhs_kind != 0 && rhs_kind != 1) || !mesh->xy || !mesh->elems || !mesh->node_is_dirichlet ||
        !mesh->elem_is_dirichlet || !decomp->elem_subdomain || mesh->n_nodes < 1 || mesh->n_elems < 1 ||
        (mesh->dim != 1 && mesh->dim != 2))
        return NLFETI_E_INVALID;
    auto in = std::make_shared<Inputs>();
    nlfeti_options o;
    nlfeti_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != 0 && o.precision != 1) return NLFETI_E_INVALID;
    try {
        in->dim = mesh->dim;
        in->n_nodes = mesh->n_nodes;
        in->n_elems = mesh->n_elems;
        in->xy.assign(mesh->xy, mesh->xy + mesh->n_nodes * mesh->dim);
        in->elems.assign(mesh->elems, mesh->elems + mesh->n_elems * (mesh->dim + 1));
        in->node_dir.assign(mesh->node_is_dirichlet, mesh->node_is_dirichlet + mesh->n_nodes);
        in->elem_dir.assign(mesh->elem_is_dirichlet, mesh->elem_is_dirichlet + mesh->n_elems);
        in->labels.assign(decomp->elem_subdomain, decomp->elem_subdomain + mesh->n_elems);
    } catch (...) {
        return NLFETI_E_NOMEM;
    }
    in->kern = *kernel;
    in->K = decomp->K;
    in->opt = o;
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &in->dim, sizeof(in->dim));
    h = fnv(h, in->xy.data(), sizeof(double) * in->xy.size());
    h = fnv(h, in->elems.data(), sizeof(int32_t) * in->elems.size());
    h = fnv(h, in->node_dir.data(), in->node_dir.size());
    h = fnv(h, in->elem_dir.data(), in->elem_dir.size());
    h = fnv(h, in->labels.data(), sizeof(int32_t) * in->labels.size());
    h = fnv(h, &in->K, sizeof(in->K));
    const double kf[3] = {kernel->delta, kernel->s, kernel->scale};
    const int ki[2] = {kernel->type, kernel->ball};
    h = fnv(h, kf, sizeof(kf));
    h = fnv(h, ki, sizeof(ki));
    const double of[3] = {o.tol, o.inner_tol, o.refine_tol};
    const int64_t oi[9] = {o.precision, o.max_it, o.max_refine, o.batched, o.graph_loop, o.precond_fp16,
                           (int64_t)o.hbm_budget, o.factor_tc, o.residual_format};
    h = fnv(h, of, sizeof(of));
    h = fnv(h, oi, sizeof(oi));
    if (h == 0) h = 1;
    const int nc = kernel->type == NLFETI_K_PERIDYNAMIC ? 2 : 1;
    auto rq = std::make_shared<Request>();
    rq->key = h;
    rq->inputs = in;
    rq->R = nrhs;
    rq->kind = rhs_kind;
    const size_t n = (size_t)mesh->n_nodes * nc * nrhs;
    try {
        rq->rhs.assign(rhs, rhs + n);
        if (g) { rq->g.assign(g, g + n); rq->has_g = true; }
    } catch (...) {
        return NLFETI_E_NOMEM;
    }
    return s->enqueue(rq, out);
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
        if (rq->t_start < rq->t_submit) stats->ms_queue = 0.0;
    }
    if (rq->status != NLFETI_OK) set_error(s->ctx, rq->err);
    return rq->status;
}

nlfeti_status nlfeti_server_get_info(nlfeti_server *s, nlfeti_server_info *out) {
    if (!s || !out) return NLFETI_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out->requests_done = s->n_done;
    out->batches = s->n_batches;
    out->merged_requests = s->n_merged;
    out->problem_hits = s->n_hits;
    out->problem_misses = s->n_misses;
    out->problems_evicted = s->n_evicted;
    out->problems_cached = 0;
    for (auto &c : s->probs) out->problems_cached += c.p ? 1 : 0;
    out->peak_active = s->peak_active;
    out->queued = (int32_t)s->queue.size();
    out->bytes_in_use = s->bytes;
    out->peak_bytes = s->peak_bytes;
    return NLFETI_OK;
}

void nlfeti_server_destroy(nlfeti_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto x : s->streams) cudaStreamSynchronize(x);
    s->wss.clear();                         // stream-ordered frees on the allocation stream
    cudaStreamSynchronize(s->alloc_stream);
    for (auto &c : s->probs)
        if (c.p) nlfeti_problem_destroy(c.p);
    s->probs.clear();
    for (auto x : s->streams) cudaStreamDestroy(x);
    cudaStreamDestroy(s->alloc_stream);
    nlfeti_ctx *c = s->ctx;
    delete s;
    ctx_detach(c);
}

}  // extern "C"
