// Serving loop: continuous batching over concurrent execution lanes.
//
// Requests (rank, order statistic, sort on one ciphertext; their blocked forms on a
// stack of blocks) are queued by any thread.  The server runs one worker thread per
// execution lane; a lane has a stream, a scratch area and plaintext caches of its own
// over the context's keys and tables (ctx_lane_create), so batches on different
// lanes run concurrently on the device.  Whenever a lane is free and the memory
// budget admits the oldest queued request, the lane takes it together with every
// queued request of the same operation, arguments and ciphertext shape (up to the
// stack cap and to what the budget still admits) and runs them as one batch:
// requests that arrive while other batches run are admitted as soon as a lane and
// memory are free, without waiting for the running batches.
//
// Slot packing (Sec. 2.3 layout, Q queries a ciphertext): a batch of single-ciphertext
// requests whose padded length N leaves room for Q = (n/2)/N^2 >= 2 queries is packed
// when the packing rotations' keys exist.  Request q of a group of up to Q moves to
// slots q N^2 + [0, N^2) by a tree of stacked rotations (level k adds member i + 2^k,
// rotated right by N^2 2^k, to member i), the circuit runs once on the stack of packed
// ciphertexts, and each result comes back to slot 0 by the mirrored tree (left
// rotations by N^2 2^k).  The packing's key switches add their noise, so a packed
// request's decryption equals its result alone within the circuit's tolerance; an
// unpacked batch member is bit-identical to its request alone, since every kernel
// treats stacked members independently.
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
rk_ctx* ctx_lane_create(rk_ctx* parent);
void ctx_lane_release(rk_ctx* c);

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
    std::vector<rk_ctx*> lanes;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    uint64_t next_ticket = 1;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_map<uint64_t, bool> pending;   // submitted, not yet collected
    std::vector<double> latency;                  // seconds, submit to result ready
    uint64_t batches = 0, members = 0, packed = 0;
    size_t used0 = 0, used_max = 0;               // device memory in use at start / at most
    size_t in_flight = 0;                         // working set admitted for running batches
    int running = 0;                              // lanes running a batch
    double busy_lane_s = 0.0;                     // sum over batches of their run time
    double t_first = 0.0, t_last = 0.0;           // first batch start, last batch end
    int max_running = 0;
};

namespace {

size_t device_used() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    return total_b - free_b;
}

// Live ciphertexts a batch member holds at once in these circuits (at most 24 of the
// input's level); the key-switching scratch is the lane's own, sized at start.
size_t member_bytes(const rk_ctx* c, int level) { return (size_t)24 * 2 * (size_t)(level + 1) * c->n * 8; }

// Queries of padded length N one ciphertext holds (a power of two).
int pack_slots(const rk_ctx* c, const rk_ct* in) {
    if (in->B != 1 || in->Q != 1 || in->layout != RK_LAYOUT_ROW) return 1;
    return (int)std::min<size_t>((size_t)c->n / 2 / ((size_t)in->N * in->N), 1u << 20);
}

// The packing tree's rotations (right by N^2 2^k to pack, left to unpack) need keys.
bool pack_keys_exist(const rk_ctx* c, uint32_t N, int Q) {
    const int64_t N2 = (int64_t)N * N;
    for (int s = 1; s < Q; s <<= 1)
        for (int64_t r : {-N2 * s, N2 * s})
            if (!c->gal.count(galois_left(c, (int)r))) return false;
    return true;
}

// Queries a packed ciphertext of this request's shape takes: its whole slot capacity
// when the packing keys exist, else 1 (no packing).
int pack_capacity(const rk_ctx* c, const Request& r) {
    if (r.op >= RK_OP_RANK_BLOCKED) return 1;
    const int q = pack_slots(c, r.in);
    return q >= 2 && pack_keys_exist(c, r.in->N, q) ? q : 1;
}

// Stack (lane-owned copy) of the given handles.
rk_ct* stack_copy(rk_ctx* lane, const std::vector<const rk_ct*>& xs) { return ct_stack(lane, xs.data(), (int)xs.size()); }

void free_all(std::vector<rk_ct*>& v) {
    for (auto*& p : v) {
        ct_free(p);
        p = nullptr;
    }
}

// Pack `m` inputs (lane-owned single ciphertexts) into groups of Q queries: returns the
// G = ceil(m / Q) packed ciphertexts (Q in their metadata), member j of group g holding
// request g Q + j at slots j N^2 + [0, N^2).
std::vector<rk_ct*> pack(rk_ctx* lane, std::vector<rk_ct*>& xs, int Q) {
    const int m = (int)xs.size(), N2 = (int)(xs[0]->N * xs[0]->N);
    for (int s = 1; s < Q; s <<= 1) {
        // pairs (i, i + s) inside a group, i a multiple of 2s: x_i += x_(i+s) >>> N^2 s
        std::vector<int> lo, hi;
        for (int i = 0; i < m; i++)
            if ((i % Q) % (2 * s) == 0 && (i % Q) + s < Q && i + s < m) {
                lo.push_back(i);
                hi.push_back(i + s);
            }
        if (lo.empty()) continue;
        std::vector<const rk_ct*> src;
        for (int j : hi) src.push_back(xs[j]);
        rk_ct* st = stack_copy(lane, src);
        rk_ct* rot = ct_alloc_like(st, st->level, st->B);
        try {
            const int r = -N2 * s;
            rk_ct* outs[1] = {rot};
            ev_rotate_many(lane, st, &r, 1, outs);
            for (size_t p = 0; p < lo.size(); p++) {
                rk_ct* v = ct_view(rot, (int)p);
                ev_add(lane, xs[lo[p]], v, xs[lo[p]]);
                ct_free(v);
            }
        } catch (...) {
            ct_free(st);
            ct_free(rot);
            throw;
        }
        ct_free(st);
        ct_free(rot);
    }
    std::vector<rk_ct*> groups;
    for (int g = 0; g * Q < m; g++) {
        rk_ct* x = xs[g * Q];
        xs[g * Q] = nullptr;
        x->Q = (uint32_t)Q;
        groups.push_back(x);
    }
    free_all(xs);
    return groups;
}

// Results of `counts[g]` packed requests per group of the stacked result `y`: request j
// of group g is y_g rotated left by j N^2 (a tree over j), returned with Q = 1.
std::vector<rk_ct*> unpack(rk_ctx* lane, const rk_ct* y, const std::vector<int>& counts, uint32_t N) {
    const int G = (int)counts.size(), N2 = (int)(N * N);
    std::vector<std::vector<rk_ct*>> part(G);
    std::vector<rk_ct*> all;
    try {
        for (int g = 0; g < G; g++) {
            part[g].assign(counts[g], nullptr);
            rk_ct* v = ct_view(y, g);
            const rk_ct* one[1] = {v};
            part[g][0] = ct_stack(lane, one, 1);
            ct_free(v);
        }
        int Qmax = 1;
        for (int c : counts) Qmax = std::max(Qmax, c);
        for (int s = 1; s < Qmax; s <<= 1) {
            std::vector<std::pair<int, int>> src;   // (group, j): j + s gets rot(j, N^2 s)
            for (int g = 0; g < G; g++)
                for (int j = 0; j < s && j + s < counts[g]; j++) src.push_back({g, j});
            if (src.empty()) continue;
            std::vector<const rk_ct*> xs;
            for (auto& p : src) xs.push_back(part[p.first][p.second]);
            rk_ct* st = stack_copy(lane, xs);
            rk_ct* rot = ct_alloc_like(st, st->level, st->B);
            try {
                const int r = N2 * s;
                rk_ct* outs[1] = {rot};
                ev_rotate_many(lane, st, &r, 1, outs);
                std::vector<rk_ct*> singles(src.size(), nullptr);
                ct_unstack(lane, rot, singles.data());
                for (size_t p = 0; p < src.size(); p++) part[src[p].first][src[p].second + s] = singles[p];
            } catch (...) {
                ct_free(st);
                ct_free(rot);
                throw;
            }
            ct_free(st);
            ct_free(rot);
        }
        for (auto& pg : part)
            for (auto* x : pg) {
                x->Q = 1;
                all.push_back(x);
            }
    } catch (...) {
        for (auto& pg : part) free_all(pg);
        throw;
    }
    return all;
}

rk_ct* run_single(rk_ctx* lane, const Request& r0, const rk_ct* x) {
    switch (r0.op) {
        case RK_OP_RANK: return circuit_rank(lane, x, r0.flags);
        case RK_OP_ORDER_STAT: return circuit_order_stat(lane, x, r0.arg, r0.flags);
        case RK_OP_SORT: return circuit_sort(lane, x, r0.flags);
        default: throw rk_error(RK_EINVAL, "unknown server operation");
    }
}

// Runs one batch on `lane`; res[i] receives request i's result (lane-owned until the
// caller hands it over).  Returns whether the batch was slot-packed.
bool run_batch(rk_server* s, rk_ctx* lane, std::vector<Request>& batch, std::vector<Result>& res) {
    const Request& r0 = batch[0];
    if (r0.op >= RK_OP_RANK_BLOCKED) {
        const int L = r0.in->B;
        const rk_ct* one[1] = {r0.in};
        rk_ct* own = ct_stack(lane, one, 1);   // the lane's copy: every temporary is the lane's
        std::vector<rk_ct*> views(L, nullptr), outs(L, nullptr);
        try {
            for (int i = 0; i < L; i++) views[i] = ct_view(own, i);
            if (r0.op == RK_OP_RANK_BLOCKED && (r0.flags & RK_TIES_CORRECT))
                circuit_rank_blocked_tc(lane, views.data(), L, outs.data());
            else if (r0.op == RK_OP_RANK_BLOCKED)
                circuit_rank_blocked(lane, views.data(), L, outs.data());
            else if (r0.op == RK_OP_ORDER_STAT_BLOCKED)
                circuit_order_stat_blocked(lane, views.data(), L, r0.arg, outs.data());
            else
                circuit_sort_blocked(lane, views.data(), L, outs.data());
            res[0].out = ct_stack(lane, outs.data(), L);
        } catch (...) {
            free_all(views);
            free_all(outs);
            ct_free(own);
            throw;
        }
        free_all(views);
        free_all(outs);
        ct_free(own);
        return false;
    }
    const int m = (int)batch.size();
    // queries a packed ciphertext takes: a power of two, so that masks are cached for
    // few distinct Q
    int Q = 1;
    const int qcap = pack_capacity(lane, r0);
    while (Q < m && Q < qcap) Q <<= 1;
    if (Q >= 2) {
        std::vector<rk_ct*> xs(m, nullptr), groups;
        rk_ct *st = nullptr, *y = nullptr;
        try {
            for (int i = 0; i < m; i++) {
                const rk_ct* one[1] = {batch[i].in};
                xs[i] = ct_stack(lane, one, 1);
            }
            groups = pack(lane, xs, Q);
            std::vector<int> counts;
            for (int g = 0; g < (int)groups.size(); g++) counts.push_back(std::min(Q, m - g * Q));
            std::vector<const rk_ct*> gp(groups.begin(), groups.end());
            st = gp.size() > 1 ? stack_copy(lane, gp) : nullptr;
            y = run_single(lane, r0, st ? st : groups[0]);
            std::vector<rk_ct*> outs = unpack(lane, y, counts, r0.in->N);
            for (int i = 0; i < m; i++) res[i].out = outs[i];
        } catch (...) {
            free_all(xs);
            free_all(groups);
            ct_free(st);
            ct_free(y);
            throw;
        }
        free_all(groups);
        ct_free(st);
        ct_free(y);
        return true;
    }
    std::vector<const rk_ct*> ins;
    for (auto& r : batch) ins.push_back(r.in);
    rk_ct* st = stack_copy(lane, ins);
    rk_ct* y = nullptr;
    try {
        y = run_single(lane, r0, st);
    } catch (...) {
        ct_free(st);
        throw;
    }
    ct_free(st);
    if (m == 1) {
        res[0].out = y;
        return false;
    }
    std::vector<rk_ct*> parts(m, nullptr);
    try {
        ct_unstack(lane, y, parts.data());
    } catch (...) {
        ct_free(y);
        free_all(parts);
        throw;
    }
    ct_free(y);
    for (int i = 0; i < m; i++) res[i].out = parts[i];
    return false;
}

// Requests the oldest queued request can be batched with: same shape, up to the stack
// cap (times the packing capacity) and to the memory still free in the budget.
bool form_batch(rk_server* s, std::vector<Request>& batch, size_t& bytes) {
    rk_ctx* c = s->ctx;
    const Request& r0 = s->queue.front();
    const size_t per = member_bytes(c, r0.in->level) * (size_t)std::max(1, r0.in->B);
    const size_t room = s->budget > s->in_flight ? s->budget - s->in_flight : 0;
    if (s->running > 0 && per > room) return false;   // wait for memory: a running batch frees it
    const int qcap = pack_capacity(c, r0);
    const int stacks = std::max<int>(1, std::min<size_t>(s->max_stack, std::max<size_t>(room, per) / per));
    const int cap = r0.op < RK_OP_RANK_BLOCKED ? stacks * qcap : 1;
    batch.push_back(r0);
    s->queue.pop_front();
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < cap;) {
        if (same_batch(*it, batch[0])) {
            batch.push_back(*it);
            it = s->queue.erase(it);
        } else {
            ++it;
        }
    }
    const int members = (int)((batch.size() + qcap - 1) / qcap);
    bytes = per * (size_t)members;
    return true;
}

void worker_loop(rk_server* s, rk_ctx* lane) {
    cudaSetDevice(lane->device);
    for (;;) {
        std::vector<Request> batch;
        size_t bytes = 0;
        double t0 = 0.0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->queue.empty()) {
                    if (s->stopping) return;   // stopping and drained
                    s->cv_work.wait(lk);
                    continue;
                }
                if (form_batch(s, batch, bytes)) break;
                s->cv_work.wait(lk);
            }
            s->in_flight += bytes;
            s->running++;
            s->max_running = std::max(s->max_running, s->running);
            t0 = now_s();
            if (s->t_first == 0.0) s->t_first = t0;
        }
        std::vector<Result> res(batch.size());
        bool was_packed = false;
        try {
            was_packed = run_batch(s, lane, batch, res);
            RK_CUDA(cudaStreamSynchronize(lane->stream));
        } catch (const rk_error& e) {
            cudaStreamSynchronize(lane->stream);
            for (auto& r : res) {
                ct_free(r.out);
                r.out = nullptr;
                r.status = e.code;
                r.error = e.what();
            }
        } catch (const std::exception& e) {
            cudaStreamSynchronize(lane->stream);
            for (auto& r : res) {
                ct_free(r.out);
                r.out = nullptr;
                r.status = RK_EINVAL;
                r.error = e.what();
            }
        }
        for (auto& r : res)   // hand the results to the server's context (its stream frees them)
            if (r.out) r.out->ctx = s->ctx;
        const double t = now_s();
        const size_t used = device_used();
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_flight -= bytes;
        s->running--;
        s->busy_lane_s += t - t0;
        s->t_last = std::max(s->t_last, t);
        s->used_max = std::max(s->used_max, used);
        s->batches++;
        s->members += batch.size();
        if (was_packed) s->packed += batch.size();
        for (size_t i = 0; i < batch.size(); i++) {
            s->latency.push_back(t - batch[i].t_submit);
            s->done[batch[i].ticket] = std::move(res[i]);
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
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
    RK_REQUIRE(!c->lane_of, RK_EINVAL, "a serving lane cannot run a server");
    RK_REQUIRE(budget > 0 && max_stack >= 1, RK_EINVAL, "server: budget and stack cap must be positive");
    RK_REQUIRE(c->server_lanes >= 1 && c->server_lanes <= 16, RK_EINVAL, "server: 1 to 16 lanes");
    RK_CUDA(cudaStreamSynchronize(c->stream));
    rk_server* s = new rk_server();
    s->ctx = c;
    s->budget = budget;
    s->max_stack = max_stack;
    try {
        for (int i = 0; i < c->server_lanes; i++) {
            rk_ctx* lane = ctx_lane_create(c);
            s->lanes.push_back(lane);
            // the scratch of stacks of up to 16 members, allocated now (growing it later
            // frees the old area, which waits for the whole device)
            ensure_batch(lane, 16);
        }
        RK_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        for (auto* l : s->lanes) ctx_lane_release(l);
        delete s;
        throw;
    }
    s->used0 = s->used_max = device_used();
    for (auto* lane : s->lanes) s->workers.emplace_back(worker_loop, s, lane);
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
    s->cv_work.notify_all();
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

// [lanes, most lanes busy at once, mean lanes busy over the serving time (sum of batch
// run times / first batch start to last batch end), requests served slot-packed,
// scratch bytes of the lanes]
void server_stats_lanes(rk_ctx* c, double out[5]) {
    rk_server* s = c->server;
    RK_REQUIRE(s, RK_EINVAL, "no server running on this context");
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = (double)s->lanes.size();
    out[1] = (double)s->max_running;
    const double span = s->t_last - s->t_first;
    out[2] = span > 0 ? s->busy_lane_s / span : 0.0;
    out[3] = (double)s->packed;
    size_t sb = 0;
    for (auto* l : s->lanes) sb += l->scratch_words * 8;
    out[4] = (double)sb;
}

size_t server_latencies(rk_ctx* c, double* out, size_t cap) {
    rk_server* s = c->server;
    RK_REQUIRE(s, RK_EINVAL, "no server running on this context");
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t m = std::min(cap, s->latency.size());
    for (size_t i = 0; i < m; i++) out[i] = s->latency[i];
    return s->latency.size();
}

// Drains the queue, joins the workers, releases the lanes and frees every result
// nobody collected.
void server_stop(rk_ctx* c) {
    rk_server* s = c->server;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& w : s->workers)
        if (w.joinable()) w.join();
    for (auto* l : s->lanes) ctx_lane_release(l);
    for (auto& kv : s->done) ct_free(kv.second.out);
    c->server = nullptr;
    delete s;
}
