// Serving loop: one worker thread per context with continuous batching.
//
// Requests (rank, order statistic, sort on one ciphertext; their blocked forms on a
// stack of blocks) are queued by any thread.  Whenever the worker is free it takes the oldest
// request together with every queued request of the same operation, arguments and
// ciphertext shape, stacks them into one ciphertext (one launch per kernel for the
// stack), runs the circuit once and splits the result.  The stack is capped so that
// its working set stays inside the context's memory budget.  A stacked member's
// result is bit-identical to the result of its request alone, since every kernel
// treats the members independently.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rk_internal.cuh"

rk_ct* circuit_rank(rk_ctx* c, const rk_ct* in, uint32_t flags);
rk_ct* circuit_order_stat(rk_ctx* c, const rk_ct* in, uint32_t k, uint32_t flags);
rk_ct* circuit_sort(rk_ctx* c, const rk_ct* in, uint32_t flags);
void circuit_rank_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
void circuit_rank_blocked_tc(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
void circuit_order_stat_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, uint32_t k, rk_ct** outs);
void circuit_sort_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    uint32_t op, arg, flags;
    const rk_ct* in;
    double t_submit;
};

struct Result {
    rk_ct* out = nullptr;
    rk_status status = RK_OK;
    std::string error;
};

bool same_batch(const Request& a, const Request& b) {
    return a.op == b.op && a.arg == b.arg && a.flags == b.flags && a.op < RK_OP_RANK_BLOCKED && a.in->level == b.in->level &&
           a.in->N == b.in->N && a.in->Q == b.in->Q && a.in->n_real == b.in->n_real && a.in->layout == b.in->layout &&
           a.in->B == 1 && b.in->B == 1;
}

}  // namespace

struct rk_server {
    rk_ctx* ctx = nullptr;
    size_t budget = 0;
    int max_stack = 1;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    uint64_t next_ticket = 1;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_map<uint64_t, bool> pending;   // submitted, not yet collected
    std::vector<double> latency;                  // seconds, submit to result ready
    uint64_t batches = 0, members = 0;
    size_t used0 = 0, used_max = 0;               // device memory in use at start / at most
};

namespace {

size_t device_used() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    return total_b - free_b;
}

// Working set of one stacked member at `level`: its share of the key-switching
// scratch plus the circuit's live ciphertexts (at most 24 at once in these circuits).
size_t member_bytes(const rk_ctx* c, int level) {
    const size_t n = c->n, L1 = c->L + 1, QP = c->L + 1 + c->alpha;
    const size_t scratch = (L1 + (size_t)c->beta(c->L) * QP + 2 * QP + 2 * L1 + 3 * L1 + 2 * L1) * n * 8;
    return scratch + 24 * 2 * (size_t)(level + 1) * n * 8;
}

void run_batch(rk_server* s, std::vector<Request>& batch, std::vector<Result>& res) {
    rk_ctx* c = s->ctx;
    const Request& r0 = batch[0];
    if (r0.op >= RK_OP_RANK_BLOCKED) {
        const int L = r0.in->B;
        std::vector<rk_ct*> views(L), outs(L, nullptr);
        for (int i = 0; i < L; i++) views[i] = ct_view(r0.in, i);
        try {
            if (r0.op == RK_OP_RANK_BLOCKED && (r0.flags & RK_TIES_CORRECT))
                circuit_rank_blocked_tc(c, views.data(), L, outs.data());
            else if (r0.op == RK_OP_RANK_BLOCKED)
                circuit_rank_blocked(c, views.data(), L, outs.data());
            else if (r0.op == RK_OP_ORDER_STAT_BLOCKED)
                circuit_order_stat_blocked(c, views.data(), L, r0.arg, outs.data());
            else
                circuit_sort_blocked(c, views.data(), L, outs.data());
        } catch (...) {
            for (auto* v : views) ct_free(v);
            for (auto* o : outs) ct_free(o);
            throw;
        }
        for (auto* v : views) ct_free(v);
        res[0].out = ct_stack(c, outs.data(), L);
        for (auto* o : outs) ct_free(o);
        return;
    }
    std::vector<const rk_ct*> ins;
    for (auto& r : batch) ins.push_back(r.in);
    rk_ct* st = batch.size() > 1 ? ct_stack(c, ins.data(), (int)ins.size()) : nullptr;
    const rk_ct* x = st ? st : r0.in;
    rk_ct* y = nullptr;
    try {
        switch (r0.op) {
            case RK_OP_RANK: y = circuit_rank(c, x, r0.flags); break;
            case RK_OP_ORDER_STAT: y = circuit_order_stat(c, x, r0.arg, r0.flags); break;
            case RK_OP_SORT: y = circuit_sort(c, x, r0.flags); break;
            default: throw rk_error(RK_EINVAL, "unknown server operation");
        }
    } catch (...) {
        ct_free(st);
        throw;
    }
    ct_free(st);
    if (batch.size() == 1) {
        res[0].out = y;
        return;
    }
    std::vector<rk_ct*> parts(batch.size(), nullptr);
    ct_unstack(c, y, parts.data());
    ct_free(y);
    for (size_t i = 0; i < batch.size(); i++) res[i].out = parts[i];
}

void worker_loop(rk_server* s) {
    rk_ctx* c = s->ctx;
    cudaSetDevice(c->device);
    for (;;) {
        std::vector<Request> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
            if (s->queue.empty()) return;   // stopping and drained
            batch.push_back(s->queue.front());
            s->queue.pop_front();
            const Request& r0 = batch[0];
            const int cap = std::max<int>(1, std::min<size_t>(s->max_stack, s->budget / member_bytes(c, r0.in->level)));
            for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < cap;) {
                if (same_batch(*it, r0)) {
                    batch.push_back(*it);
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        std::vector<Result> res(batch.size());
        try {
            run_batch(s, batch, res);
            RK_CUDA(cudaStreamSynchronize(c->stream));
        } catch (const rk_error& e) {
            for (auto& r : res) {
                ct_free(r.out);
                r.out = nullptr;
                r.status = e.code;
                r.error = e.what();
            }
        } catch (const std::exception& e) {
            for (auto& r : res) {
                ct_free(r.out);
                r.out = nullptr;
                r.status = RK_EINVAL;
                r.error = e.what();
            }
        }
        const double t = now_s();
        const size_t used = device_used();
        std::lock_guard<std::mutex> lk(s->mu);
        s->used_max = std::max(s->used_max, used);
        s->batches++;
        s->members += batch.size();
        for (size_t i = 0; i < batch.size(); i++) {
            s->latency.push_back(t - batch[i].t_submit);
            s->done[batch[i].ticket] = std::move(res[i]);
        }
        s->cv_done.notify_all();
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

rk_server* server_start(rk_ctx* c, size_t budget, int max_stack) {
    RK_REQUIRE(!c->server, RK_EINVAL, "a server is already running on this context");
    RK_REQUIRE(budget > 0 && max_stack >= 1, RK_EINVAL, "server: budget and stack cap must be positive");
    RK_CUDA(cudaStreamSynchronize(c->stream));
    rk_server* s = new rk_server();
    s->ctx = c;
    s->budget = budget;
    s->max_stack = max_stack;
    s->used0 = s->used_max = device_used();
    s->worker = std::thread(worker_loop, s);
    c->server = s;
    return s;
}

uint64_t server_submit(rk_ctx* c, uint32_t op, uint32_t arg, uint32_t flags, const rk_ct* in) {
    rk_server* s = c->server;
    RK_REQUIRE(s, RK_EINVAL, "no server running on this context");
    RK_REQUIRE(op >= RK_OP_RANK && op <= RK_OP_SORT_BLOCKED, RK_EINVAL, "unknown server operation");
    RK_REQUIRE(op >= RK_OP_RANK_BLOCKED ? in->B >= 1 : in->B == 1, RK_EINVAL,
               "server requests take one ciphertext (blocked rank: a stack of blocks)");
    std::lock_guard<std::mutex> lk(s->mu);
    RK_REQUIRE(!s->stopping, RK_EINVAL, "server is stopping");
    const uint64_t t = s->next_ticket++;
    s->queue.push_back(Request{t, op, arg, flags, in, now_s()});
    s->pending[t] = true;
    s->cv_work.notify_one();
    return t;
}

// Collects the result of `ticket` once it is ready (waiting at most timeout_s; a
// negative timeout waits without limit, zero only polls).  Returns nullptr while pending.
rk_ct* server_collect(rk_ctx* c, uint64_t ticket, double timeout_s) {
    rk_server* s = c->server;
    RK_REQUIRE(s, RK_EINVAL, "no server running on this context");
    std::unique_lock<std::mutex> lk(s->mu);
    RK_REQUIRE(s->pending.count(ticket), RK_EINVAL, "unknown or already collected ticket");
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_s < 0)
            s->cv_done.wait(lk, ready);
        else if (timeout_s > 0)
            s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    }
    if (!ready()) return nullptr;
    Result r = std::move(s->done[ticket]);
    s->done.erase(ticket);
    s->pending.erase(ticket);
    if (r.status != RK_OK) throw rk_error(r.status, "request failed: " + r.error);
    return r.out;
}

void server_stats(rk_ctx* c, double out[8]) {
    rk_server* s = c->server;
    RK_REQUIRE(s, RK_EINVAL, "no server running on this context");
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = (double)s->latency.size();
    out[1] = percentile(s->latency, 0.5);
    out[2] = percentile(s->latency, 0.99);
    out[3] = s->latency.empty() ? 0.0 : *std::max_element(s->latency.begin(), s->latency.end());
    out[4] = (double)s->batches;
    out[5] = s->batches ? (double)s->members / (double)s->batches : 0.0;
    out[6] = (double)(s->used_max > s->used0 ? s->used_max - s->used0 : 0);
    out[7] = (double)s->queue.size();
}

size_t server_latencies(rk_ctx* c, double* out, size_t cap) {
    rk_server* s = c->server;
    RK_REQUIRE(s, RK_EINVAL, "no server running on this context");
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t m = std::min(cap, s->latency.size());
    for (size_t i = 0; i < m; i++) out[i] = s->latency[i];
    return s->latency.size();
}

// Drains the queue, joins the worker and frees every result nobody collected.
void server_stop(rk_ctx* c) {
    rk_server* s = c->server;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->done) ct_free(kv.second.out);
    c->server = nullptr;
    delete s;
}
