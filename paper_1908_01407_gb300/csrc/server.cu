// Serving loop: BFS / SSSP / PageRank requests against resident graphs,
// with continuous batching. Each of max_inflight worker slots owns a
// context (its own stream, pool and traversal workspaces) and takes the
// next job as soon as it is free: the oldest pending request, and, for BFS,
// every other pending BFS on the same graph up to 64, packed into one
// multi-source bit-frontier launch. A job is admitted only while its memory
// estimate fits the HBM budget. Persistent kernels of concurrent slots are
// given grids that split the GPU between the jobs running or waiting when
// they start, so their work overlaps; a job that starts while no other job
// runs or waits gets the whole GPU.
// Results stay on the device until fetched. Latency is measured from submit
// to the moment the slot sees the job finish on the GPU.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

using namespace gbx;

namespace gbx {
gb_info msbfs_launch(gb_context *ctx, const gb_matrix *A, const uint32_t *d_srcs, uint32_t k, int32_t *levels,
                     const gb_desc *desc, struct BfsResult *res_out);
}

namespace {

using Clock = std::chrono::steady_clock;

double now_us() {
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Result {
    gb_context *owner = nullptr;   // context whose pool holds the buffer
    void *dev = nullptr;           // device buffer
    size_t bytes = 0;
    uint32_t n = 0;
    int refs = 0;                  // tickets not yet fetched
};

enum TicketState { QUEUED, RUNNING, DONE };

struct Ticket {
    gb_request req;
    TicketState state = QUEUED;
    gb_info status = GB_SUCCESS;
    double t_submit = 0, t_done = 0;
    std::shared_ptr<Result> result;
    uint32_t row = 0;              // row of a batched BFS result
    uint32_t batch = 1;
};

}  // namespace

struct gb_server_t {
    gb_context *ctx = nullptr;
    gb_server_cfg cfg;
    std::vector<const gb_matrix *> graphs;
    std::vector<gb_context *> wctx;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    uint64_t budget = 0, in_use = 0, peak = 0;
    uint64_t held = 0;             // bytes of finished, unfetched results (part of in_use)
    int running = 0;
    int share = 0;                 // blocks of a persistent kernel when slots run together
    // statistics
    std::vector<double> lat;
    uint64_t submitted = 0, completed = 0, batches = 0, batched_bfs = 0;
    double t_first = -1, t_last = 0;
};

namespace {

size_t work_bytes(uint32_t n) { return (size_t)n * 64 + (1u << 20); }

// Below SINGLE_BFS_MAX_K sources on a graph of at least SINGLE_BFS_MIN_N
// vertices, k single-source traversals (direction-optimised, with early exit
// per vertex) beat one 64-bit bit-frontier launch, whose pulls scan until
// every source is covered.
constexpr uint32_t SINGLE_BFS_MIN_N = 1u << 21;
constexpr uint32_t SINGLE_BFS_MAX_K = 24;

void worker_loop(gb_server *S, int w) {
    gb_context *ctx = S->wctx[w];
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        if (S->stop) break;
        // ---- form a job from the oldest request
        uint64_t head = S->pending.front();
        Ticket &H = S->tickets[head];
        const gb_request req = H.req;
        const gb_matrix *A = S->graphs[req.graph_id];
        std::vector<uint64_t> job;
        auto gather = [&]() {
            job.clear();
            for (uint64_t t : S->pending) {
                Ticket &T = S->tickets[t];
                if (T.req.kind == GB_REQ_BFS && T.req.graph_id == req.graph_id) job.push_back(t);
                if (job.size() == 64) break;
            }
        };
        if (req.kind == GB_REQ_BFS) {
            gather();
            double age = now_us() - H.t_submit;
            if (job.size() < 64 && S->cfg.batch_window_us > 0 && age < S->cfg.batch_window_us &&
                S->running + 1 >= (int)S->cfg.max_inflight) {
                // every other slot is busy: give concurrent requests on the same
                // graph a short window to join (an idle GPU starts at once)
                S->cv_work.wait_for(lk, std::chrono::microseconds((int64_t)(S->cfg.batch_window_us - age)));
                if (S->stop) break;
                if (S->pending.empty() || S->pending.front() != head) continue;   // another slot took it
                gather();
            }
        } else {
            job.push_back(head);
        }
        const uint32_t n = A->nrows;
        const uint32_t k = (uint32_t)job.size();
        size_t rbytes = (req.kind == GB_REQ_BFS ? (size_t)k : 1) * n * 4 + 16;
        size_t need = rbytes + work_bytes(n);
        // ---- admission by free HBM budget
        // wait while running jobs or unfetched results still hold memory
        while (S->in_use + need > S->budget && (S->running > 0 || S->held > 0) && !S->stop) S->cv_done.wait(lk);
        if (S->stop) break;
        if (S->pending.empty() || S->pending.front() != head) continue;          // taken meanwhile
        for (uint64_t t : job) {
            auto it = std::find(S->pending.begin(), S->pending.end(), t);
            if (it != S->pending.end()) S->pending.erase(it);
            S->tickets[t].state = RUNNING;
        }
        if (S->in_use + need > S->budget) {
            for (uint64_t t : job) {
                Ticket &T = S->tickets[t];
                T.state = DONE;
                T.status = GB_OUT_OF_MEMORY;
                T.t_done = now_us();
            }
            S->cv_done.notify_all();
            continue;
        }
        S->in_use += need;
        S->peak = std::max(S->peak, S->in_use);
        S->running++;
        // a job that starts with nothing else running or waiting takes the whole
        // GPU; otherwise its persistent kernels get an equal part of it for the
        // jobs running or waiting now (4 blocks per SM split between them), never
        // less than the share that lets every slot run at once. A long job that
        // overlaps one other thus keeps half the GPU, not an eighth of it.
        {
            const int conc = std::min(S->running + (int)S->pending.size(), (int)S->cfg.max_inflight);
            ctx->grid_limit = conc <= 1 ? 0 : std::max(S->share, 4 * S->ctx->num_sms / conc);
        }
        std::vector<uint32_t> srcs;
        for (uint64_t t : job) srcs.push_back(S->tickets[t].req.src);
        lk.unlock();
        // ---- run on this slot's stream
        auto res = std::make_shared<Result>();
        res->owner = ctx;
        res->n = n;
        res->bytes = rbytes;
        res->refs = (int)k;
        gb_info st = dalloc(ctx, &res->dev, rbytes);
        if (st == GB_SUCCESS) {
            if (req.kind == GB_REQ_BFS && (k == 1 || (n >= SINGLE_BFS_MIN_N && k < SINGLE_BFS_MAX_K))) {
                // one request, or a few on a large graph: the single-source
                // kernel, one launch per source, each into its own row
                for (uint32_t q = 0; q < k && st == GB_SUCCESS; ++q)
                    st = gb_bfs(ctx, A, srcs[q], (int32_t *)res->dev + (size_t)q * n, nullptr, GB_DEVICE, nullptr,
                                nullptr);
                if (st == GB_SUCCESS) st = sync(ctx);
            } else if (req.kind == GB_REQ_BFS) {
                Scratch ds(ctx);
                st = ds.alloc(64 * 4);
                if (st == GB_SUCCESS) st = copy_in(ctx, ds.p, srcs.data(), (size_t)k * 4, GB_HOST);
                if (st == GB_SUCCESS) st = msbfs_launch(ctx, A, ds.as<uint32_t>(), k, (int32_t *)res->dev, nullptr, nullptr);
                if (st == GB_SUCCESS) st = sync(ctx);
            } else if (req.kind == GB_REQ_SSSP) {
                uint32_t it = 0;
                st = gb_sssp(ctx, A, req.src, (uint32_t *)res->dev, GB_DEVICE, nullptr, &it, nullptr);
            } else {
                st = gb_pagerank(ctx, A, S->cfg.pagerank_damping, S->cfg.pagerank_iters, (float *)res->dev, nullptr,
                                 GB_DEVICE);
                if (st == GB_SUCCESS) st = sync(ctx);
            }
        }
        double t_done = now_us();
        lk.lock();
        S->running--;
        S->in_use -= work_bytes(n);
        if (st != GB_SUCCESS) {
            if (res->dev) dfree(ctx, res->dev);
            res->dev = nullptr;
            S->in_use -= rbytes;
        } else {
            S->held += rbytes;
        }
        S->batches++;
        if (req.kind == GB_REQ_BFS) S->batched_bfs += k;
        for (uint32_t q = 0; q < k; ++q) {
            Ticket &T = S->tickets[job[q]];
            T.state = DONE;
            T.status = st;
            T.t_done = t_done;
            T.result = st == GB_SUCCESS ? res : nullptr;
            T.row = q;
            T.batch = k;
            S->lat.push_back(t_done - T.t_submit);
            S->completed++;
        }
        S->t_last = std::max(S->t_last, t_done);
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

gb_info gb_server_create(gb_server **s, gb_context *ctx, const gb_server_cfg *cfg) {
    if (!s || !ctx) return fail(GB_NULL_POINTER, "gb_server_create: NULL argument");
    GB_CUDA(cudaSetDevice(ctx->device));
    gb_server *S = new gb_server();
    S->ctx = ctx;
    gb_server_cfg c = {8, 200, 0, 50, 0.85f};
    if (cfg) {
        c = *cfg;
        if (!c.max_inflight) c.max_inflight = 8;
        if (!c.pagerank_iters) c.pagerank_iters = 50;
        if (c.pagerank_damping <= 0.f) c.pagerank_damping = 0.85f;
    }
    if (c.max_inflight > 64) c.max_inflight = 64;
    S->cfg = c;
    size_t fr = 0, tot = 0;
    GB_CUDA(cudaMemGetInfo(&fr, &tot));
    S->budget = c.hbm_budget_bytes ? c.hbm_budget_bytes : (uint64_t)(fr * 0.8);
    // slots: own contexts; persistent grids sized so all slots fit at once
    int grid_limit = std::max(1, (int)(3 * ctx->num_sms / c.max_inflight));
    for (uint32_t w = 0; w < c.max_inflight; ++w) {
        gb_context *wc = nullptr;
        gb_info r = gb_init(ctx->device, &wc);
        if (r != GB_SUCCESS) {
            for (auto x : S->wctx) gb_finalize(x);
            delete S;
            return r;
        }
        wc->grid_limit = c.max_inflight > 1 ? grid_limit : 0;
        S->wctx.push_back(wc);
    }
    S->share = c.max_inflight > 1 ? grid_limit : 0;
    for (uint32_t w = 0; w < c.max_inflight; ++w) S->workers.emplace_back(worker_loop, S, (int)w);
    *s = S;
    return GB_SUCCESS;
}

gb_info gb_server_add_graph(gb_server *S, const gb_matrix *A, uint32_t *graph_id) {
    if (!S || !A || !graph_id) return fail(GB_NULL_POINTER, "gb_server_add_graph: NULL argument");
    if (!A->built) return fail(GB_INVALID_VALUE, "gb_server_add_graph: matrix not built");
    if (A->nrows != A->ncols) return fail(GB_DIMENSION_MISMATCH, "gb_server_add_graph: matrix must be square");
    std::lock_guard<std::mutex> g(S->mu);
    S->graphs.push_back(A);
    *graph_id = (uint32_t)S->graphs.size() - 1;
    return GB_SUCCESS;
}

gb_info gb_server_submit(gb_server *S, const gb_request *req, uint64_t *ticket) {
    if (!S || !req || !ticket) return fail(GB_NULL_POINTER, "gb_server_submit: NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    if (req->graph_id >= S->graphs.size()) return fail(GB_INVALID_INDEX, "gb_server_submit: unknown graph");
    const gb_matrix *A = S->graphs[req->graph_id];
    if (req->kind < GB_REQ_BFS || req->kind > GB_REQ_PAGERANK) return fail(GB_INVALID_VALUE, "gb_server_submit: kind");
    if (req->kind != GB_REQ_PAGERANK && req->src >= A->nrows)
        return fail(GB_INVALID_INDEX, "gb_server_submit: source out of range");
    if (req->kind == GB_REQ_SSSP && (!A->has_vals || A->type != GB_UINT32))
        return fail(GB_DOMAIN_MISMATCH, "gb_server_submit: SSSP needs uint32 edge weights");
    uint64_t t = S->next_ticket++;
    Ticket T;
    T.req = *req;
    T.t_submit = now_us();
    if (S->t_first < 0) S->t_first = T.t_submit;
    S->tickets[t] = T;
    S->pending.push_back(t);
    S->submitted++;
    *ticket = t;
    S->cv_work.notify_one();
    return GB_SUCCESS;
}

gb_info gb_server_wait(gb_server *S, uint64_t ticket, uint32_t timeout_ms, gb_result *res) {
    if (!S || !res) return fail(GB_NULL_POINTER, "gb_server_wait: NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail(GB_INVALID_INDEX, "gb_server_wait: unknown ticket");
    bool done = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                    [&] { return S->tickets[ticket].state == DONE; });
    if (!done) return fail(GB_TIMEOUT, "gb_server_wait: ticket %llu not done", (unsigned long long)ticket);
    Ticket &T = S->tickets[ticket];
    res->status = T.status;
    res->n = S->graphs[T.req.graph_id]->nrows;
    res->latency_us = T.t_done - T.t_submit;
    res->batch_size = T.batch;
    return GB_SUCCESS;
}

gb_info gb_server_fetch(gb_server *S, uint64_t ticket, void *out, gb_mem mem) {
    if (!S || !out) return fail(GB_NULL_POINTER, "gb_server_fetch: NULL argument");
    std::shared_ptr<Result> r;
    uint32_t row = 0;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return fail(GB_INVALID_INDEX, "gb_server_fetch: unknown ticket");
        if (it->second.state != DONE) return fail(GB_INVALID_VALUE, "gb_server_fetch: ticket not done");
        if (it->second.status != GB_SUCCESS) return fail(it->second.status, "gb_server_fetch: the request failed");
        r = it->second.result;
        row = it->second.row;
        if (!r) return fail(GB_NO_VALUE, "gb_server_fetch: result already fetched");
        it->second.result.reset();
    }
    gb_context *oc = r->owner;
    GB_CUDA(cudaSetDevice(oc->device));
    gb_info st = copy_out(oc, out, (const char *)r->dev + (size_t)row * r->n * 4, (size_t)r->n * 4, mem);
    if (st == GB_SUCCESS && mem == GB_DEVICE) st = sync(oc);
    std::lock_guard<std::mutex> g(S->mu);
    if (--r->refs == 0) {
        dfree(oc, r->dev);
        r->dev = nullptr;
        S->in_use -= r->bytes;
        S->held -= r->bytes;
        S->cv_done.notify_all();
    }
    S->tickets.erase(ticket);
    return st;
}

gb_info gb_server_stats_get(gb_server *S, gb_server_stats *st) {
    if (!S || !st) return fail(GB_NULL_POINTER, "gb_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->batches = S->batches;
    st->batched_bfs = S->batched_bfs;
    st->hbm_in_use = S->in_use;
    st->hbm_peak = S->peak;
    if (!S->lat.empty()) {
        std::vector<double> v = S->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        st->p50_us = pct(0.50);
        st->p99_us = pct(0.99);
        double s = 0;
        for (double x : v) s += x;
        st->mean_us = s / v.size();
        double span = S->t_last - S->t_first;
        st->qps = span > 0 ? S->completed / (span * 1e-6) : 0;
    }
    return GB_SUCCESS;
}

gb_info gb_server_destroy(gb_server **s) {
    if (!s) return fail(GB_NULL_POINTER, "gb_server_destroy: NULL");
    gb_server *S = *s;
    if (!S) return GB_SUCCESS;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->tickets)
        if (kv.second.result && kv.second.result->dev) {
            dfree(kv.second.result->owner, kv.second.result->dev);
            kv.second.result->dev = nullptr;
        }
    for (auto c : S->wctx) gb_finalize(c);
    delete S;
    *s = nullptr;
    return GB_SUCCESS;
}

}  // extern "C"
